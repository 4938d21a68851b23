"""Writes the stored oracle results of the low-SNR frame's crops.

Calls only the CPU oracle (oracle/) on inputs from the seeded generators
(paper_2411_00991_gb300.synth); nothing here touches the CUDA library.  Two
files are written next to this script:

lowsnr256_fp64_chain.txt
    The oracle's chain on the 256 x 256 crop of the 2048 x 2048 low-SNR
    recipe (PSF sigma 4 px on 31 x 31, peak 5 / background 1 photons per
    pixel, sCMOS maps, gain 2.1; ``synth.lowsnr_2048(crop=256)``) with a
    refresh every 10 sweeps and burn-in 10, for chains 0 and 3 over sweeps
    1..20: per sweep the log posterior (Eq. 9), the accepted-update count
    and a SHA-256 of the accept decisions; after sweep 20 the sums of the
    object, its square, the expected image and the posterior mean, and
    their values at seeded sample positions.  A SHA-256 of the inputs is
    stored so that a test can tell that it sees the same frame.

lowsnr32_oracle_means.txt
    Posterior means of 40 independent oracle chains (chain ids 100..139) on
    the 32 x 32 crop of the same recipe, 250 sweeps, burn-in 50, refresh
    every 50: per camera pixel the average of the chain means and their
    sample variance (the Monte Carlo standard error of the pooled mean is
    sqrt(var / 40)).

Run:  python tests/golden/make_lowsnr_goldens.py [--jobs N]
(about 20 minutes for the chains and 50 for the means on 6 cores).
"""
from __future__ import annotations

import argparse
import hashlib
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

CHAIN_CROP, CHAIN_T, CHAIN_REFRESH, CHAIN_BURN, CHAIN_IDS = 256, 20, 10, 10, (0, 3)
N_RHO_SAMPLES, N_MU_SAMPLES = 384, 192
MEANS_CROP, MEANS_T, MEANS_BURN, MEANS_REFRESH = 32, 250, 50, 50
MEANS_CHAINS = tuple(range(100, 140))


def chain_problem():
    from paper_2411_00991_gb300 import synth
    p = synth.lowsnr_2048(crop=CHAIN_CROP)
    p.refresh_every, p.burn_in = CHAIN_REFRESH, CHAIN_BURN
    return p


def means_problem():
    from paper_2411_00991_gb300 import synth
    p = synth.lowsnr_2048(crop=MEANS_CROP)
    p.refresh_every, p.burn_in = MEANS_REFRESH, MEANS_BURN
    return p


def input_hash(p) -> str:
    h = hashlib.sha256()
    for a in (p.image, p.offset, p.var):
        h.update(np.ascontiguousarray(a, dtype=np.float32).tobytes())
    h.update(np.ascontiguousarray(p.psf, dtype=np.float64).tobytes())
    h.update(repr((float(p.gain), p.S, p.seed, p.step)).encode())
    return h.hexdigest()


def accept_hash(acc) -> str:
    return hashlib.sha256(np.packbits(np.asarray(acc, dtype=np.uint8).ravel()).tobytes()).hexdigest()


def sample_positions(n_obj: int, n_mu: int):
    rng = np.random.default_rng(20411)
    return (np.sort(rng.choice(n_obj, N_RHO_SAMPLES, replace=False)),
            np.sort(rng.choice(n_mu, N_MU_SAMPLES, replace=False)))


def run_chain(chain: int):
    from oracle import oracle as O
    p = chain_problem()
    t0 = time.time()
    r = O.Oracle(p, chain=chain).run(CHAIN_T, want_acc_log=True)
    return chain, r, time.time() - t0


def run_mean(chain: int):
    from oracle import oracle as O
    p = means_problem()
    r = O.Oracle(p, chain=chain).run(MEANS_T)
    R = p.R
    return (r["sum"] / r["n_sum"])[R:-R, R:-R]


def write_chains(results):
    p = chain_problem()
    Ho, Wo = p.object_shape()
    pos_rho, pos_mu = sample_positions(Ho * Wo, p.H * p.W)
    lines = ["# oracle chain, synth.lowsnr_2048(crop=256), refresh_every 10, burn_in 10, sweeps 1..20",
             "# written by tests/golden/make_lowsnr_goldens.py (CPU oracle only)",
             f"input_sha256 {input_hash(p)}",
             f"sweeps {CHAIN_T} refresh_every {CHAIN_REFRESH} burn_in {CHAIN_BURN}"]
    for chain, r, dt in sorted(results, key=lambda x: x[0]):
        lines.append(f"chain {chain}")
        for t in range(CHAIN_T):
            lines.append(f"sweep {t + 1} trace {float(r['trace'][t])!r} n_acc {int(r['n_acc'][t])} "
                         f"acc_sha256 {accept_hash(r['acc_log'][t])}")
        rho, mu = r["rho"].ravel(), r["mu"].ravel()
        mean = (r["sum"] / r["n_sum"]).ravel()
        lines.append(f"rho_sum {float(rho.sum())!r} rho_sq_sum {float((rho * rho).sum())!r}")
        lines.append(f"mu_sum {float(mu.sum())!r} mean_sum {float(mean.sum())!r} n_mean {int(r['n_sum'])}")
        lines.append("rho_samples " + " ".join(f"{int(k)}:{float(rho[k])!r}" for k in pos_rho))
        lines.append("mean_samples " + " ".join(f"{int(k)}:{float(mean[k])!r}" for k in pos_rho))
        lines.append("mu_samples " + " ".join(f"{int(k)}:{float(mu[k])!r}" for k in pos_mu))
        lines.append(f"end_chain {chain}")
    with open(os.path.join(HERE, "lowsnr256_fp64_chain.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


def write_means(means):
    p = means_problem()
    m = np.stack(means)
    avg, var = m.mean(0), m.var(0, ddof=1)
    lines = ["# oracle posterior means, synth.lowsnr_2048(crop=32), 250 sweeps, burn_in 50, refresh_every 50",
             f"# chains {MEANS_CHAINS[0]}..{MEANS_CHAINS[-1]}; per camera pixel (row-major): mean of the chain "
             "means, their sample variance (ddof 1)",
             "# written by tests/golden/make_lowsnr_goldens.py (CPU oracle only)",
             f"input_sha256 {input_hash(p)}",
             f"n_chains {m.shape[0]} shape {avg.shape[0]} {avg.shape[1]}"]
    for a, v in zip(avg.ravel(), var.ravel()):
        lines.append(f"{a:.12e} {v:.6e}")
    with open(os.path.join(HERE, "lowsnr32_oracle_means.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--jobs", type=int, default=6)
    ap.add_argument("--only", choices=["chains", "means"], default=None)
    a = ap.parse_args()
    from oracle import oracle as O
    O.build()
    with mp.get_context("spawn").Pool(a.jobs) as pool:
        rc = pool.map_async(run_chain, CHAIN_IDS) if a.only in (None, "chains") else None
        rm = pool.map_async(run_mean, MEANS_CHAINS) if a.only in (None, "means") else None
        if rc is not None:
            res = rc.get()
            write_chains(res)
            print("chains written:", [round(dt) for _, _, dt in res], "s", flush=True)
        if rm is not None:
            write_means(rm.get())
            print("means written", flush=True)


if __name__ == "__main__":
    main()
