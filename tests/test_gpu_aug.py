"""The photon-count augmented sampler on the GPU (BDECON_FLAG_AUGMENTED).

Double precision: the chain equals the oracle's augmented chain -- the
photon counts drawn at every sweep, the accept decisions, the object, the
expected image and the trace (log joint density p(w, phi, rho)) -- for
small problems with ragged patches, sCMOS maps, a stride wider than the
PSF, two chains and a refresh inside the run.  Any launch plan, a batch, a
CUDA graph give bit-identical chains.  Single precision: the augmented float
sampler targets the posterior of Eq. 9 -- its posterior means agree with
independent chains of the marginal double oracle within 3 Monte Carlo
standard errors on at least 99% of the pixels.
"""
import functools
import multiprocessing as mp

import numpy as np
import pytest

import oracle_jobs
from oracle import oracle as O
from paper_2411_00991_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2411_00991_gb300 import bdecon  # noqa: E402

RTOL = 1e-12


def _aug(**kw):
    p = synth.small_problem(**kw)
    p.augmented = True
    return p


@pytest.mark.parametrize("kw,plan", [
    (dict(H=20, W=24, L=5, seed=111, refresh_every=4), None),
    (dict(H=17, W=13, L=3, seed=112, maps=True, refresh_every=0), None),
    (dict(H=16, W=19, L=5, stride=7, seed=113, maps=True), None),
    (dict(H=12, W=12, L=7, seed=114, n_chains=2, burn_in=3), None),
    # two one-warp update teams per block, several rounds per class step
    (dict(H=30, W=27, L=5, seed=115, maps=True, refresh_every=4), (3, 3, 2)),
])
def test_fp64_augmented_chain_matches_oracle(kw, plan):
    p = _aug(**kw)
    T = 12
    s = bdecon.Sampler(p, precision=bdecon.BDECON_FP64, max_sweeps=T + 4, flags=bdecon.FLAG_ACCEPT_LOG)
    if plan is not None:
        s.set_plan(*plan)
        pl = s.get_plan(0)
        assert (pl["tile_i"], pl["tile_j"], pl["warps"]) == plan
    s.sweep(T)
    for c in range(p.n_chains):
        ref = O.Oracle(p, chain=c).run(T, want_acc_log=True)
        np.testing.assert_array_equal(s.get_phi(0, c), ref["phi"])
        mism = np.argwhere(s.accept_log(0, c) != ref["acc_log"])
        assert mism.size == 0, f"{len(mism)} accept decisions differ, first {mism[:3]}"
        np.testing.assert_allclose(s.get_state(0, c)[0], ref["rho"], rtol=RTOL)
        np.testing.assert_allclose(s.get_mu(0, c), ref["mu"], rtol=RTOL)
        np.testing.assert_allclose(s.trace(0, c), ref["trace"], rtol=RTOL)
    if T > p.burn_in:
        s.posterior_mean()
    s.close()


@pytest.mark.parametrize("precision", [bdecon.BDECON_FP64, bdecon.BDECON_FP32])
def test_augmented_plans_batches_and_graphs_are_bit_identical(precision):
    probs = [_aug(H=20, W=24, L=5, seed=115, refresh_every=4, burn_in=2),
             synth.small_problem(H=17, W=13, L=3, maps=True, seed=116, n_chains=2, refresh_every=4, burn_in=2),
             _aug(H=26, W=22, L=11, sigma=1.8, seed=117, refresh_every=4, burn_in=2)]
    T = 9

    def collect(s, k, pr):
        return [s.get_state(k, 0)[0], s.trace(k, 0), s.posterior_mean(k)] + \
            ([s.get_phi(k, 0)] if pr.augmented else [])

    ref = []
    for k, pr in enumerate(probs):
        a = bdecon.Sampler(pr, precision=precision, max_sweeps=T + 4)
        a.sweep(T)
        ref.append(collect(a, 0, pr))
        a.close()
    for mode in ("batch", "plan", "graph", "one_launch"):
        b = bdecon.Sampler(probs, precision=precision, max_sweeps=T + 4)
        if mode == "plan":
            b.set_plan(2, 3, 4, p=0)
        elif mode == "graph":
            b.set_graph(True)
        elif mode == "one_launch":
            b.set_grouping(True)
        b.sweep(4)
        b.sweep(T - 4)
        for k in range(len(probs)):
            for x, y in zip(collect(b, k, probs[k]), ref[k]):
                np.testing.assert_array_equal(x, y, err_msg=f"{mode} problem {k}")
        b.close()


def test_delta_is_refused_for_augmented_problems():
    s = bdecon.Sampler(_aug(H=9, W=9, L=3, seed=118), precision=bdecon.BDECON_FP32, max_sweeps=4)
    with pytest.raises(bdecon.BdeconError, match="augmented"):
        s.delta(5, 1.0)
    s.close()


# ------------------------------------------------ float, against the oracle
H = W = 30
LPSF = 3
SEED = 21
T = 600
BURN = 100
N_ORACLE = 48
N_GPU = 64


@pytest.fixture(scope="module")
def marginal_oracle_means():
    with mp.get_context("spawn").Pool(min(16, mp.cpu_count())) as pool:
        job = functools.partial(oracle_jobs.small_chain_mean, H, W, LPSF, SEED, BURN, 50, T)
        return np.stack(pool.map(job, range(N_ORACLE)))


def test_fp32_augmented_means_within_3_mcse_of_marginal_oracle(marginal_oracle_means):
    probs = []
    for k in range(N_GPU):
        p = synth.small_problem(H=H, W=W, L=LPSF, seed=SEED, burn_in=BURN, refresh_every=50)
        p.seed = 20_000 + k
        p.augmented = True
        probs.append(p)
    s = bdecon.Sampler(probs, precision=bdecon.BDECON_FP32, max_sweeps=T)
    s.sweep(T)
    g = np.stack([s.posterior_mean(k) for k in range(N_GPU)])
    s.close()
    a = marginal_oracle_means
    d = g.mean(0) - a.mean(0)
    se = np.sqrt(g.var(0, ddof=1) / g.shape[0] + a.var(0, ddof=1) / a.shape[0])
    frac = float(np.mean(np.abs(d) <= 3 * se))
    print(f"augmented float vs marginal oracle: {frac:.4f} of pixels within 3 MCSE")
    assert frac >= 0.99
