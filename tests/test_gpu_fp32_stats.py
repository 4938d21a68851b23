"""Single-precision sampler against the double-precision oracle.

The float sweep takes its own accept decisions (a log acceptance ratio a few
1e-6 away from the double one flips a decision now and then), so its chain
is not the oracle's chain; what must agree is (a) the log-posterior trace it
reports -- a double running sum of float per-update changes, rebased at each
double refresh -- with the oracle's Eq. 9 evaluated at the float chain's own
state, within 1e-5 relative, and (b) the law of the chain: posterior means
of independent float chains and of independent oracle chains agree within
3 Monte Carlo standard errors on at least 99% of the pixels.  A likelihood
with the wrong detector gain must fail (b), so the test has the power to
see a wrong target.
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

TRACE_RTOL = 1e-5


@pytest.mark.parametrize("refresh_every", [50, 0])
def test_fp32_trace_matches_oracle_posterior_of_its_state(refresh_every):
    # the 64x64 widefield frame of 12 blobs and 3 lines, 9x9 PSF; with a
    # refresh every 50 sweeps and without any (the running sum alone)
    prob = synth.widefield_64()
    prob.refresh_every = refresh_every
    orc = O.Oracle(prob)
    s = bdecon.Sampler(prob, precision=bdecon.BDECON_FP32, max_sweeps=200)
    done = 0
    for t in (1, 49, 50, 120, 200):
        s.sweep(t - done)
        done = t
        rho, tt = s.get_state()
        assert tt == t
        tr = s.trace()                      # values after sweeps 1..t
        assert tr.size == t
        ref = orc.log_posterior(rho)
        assert abs(tr[t - 1] - ref) <= TRACE_RTOL * abs(ref), (t, tr[t - 1], ref)
    assert s.accept_counts().sum() > 1000
    s.close()


@pytest.mark.parametrize("plan", [None, (6, 6, 0)])
def test_widefield512_fp32_trace_matches_oracle_over_200_sweeps(plan):
    # the 512x512 widefield frame (L = 17, 1 chain) at full size over many
    # sweeps, in the plan a user gets -- one patch per block, one update team,
    # the one-team kernel form -- and in a streamed multi-round plan (tiles of
    # 6 x 6 patches, tile state in global memory, several rounds per class
    # step); the trace at sweeps 50 (a refresh), 100 and 200 equals the
    # oracle's Eq. 9 of the chain's state within 1e-5
    prob = synth.widefield_512()
    orc = O.Oracle(prob)
    s = bdecon.Sampler(prob, precision=bdecon.BDECON_FP32, max_sweeps=200)
    if plan is not None:
        s.set_plan(*plan)
    pl = s.get_plan(0)
    if plan is None:
        assert (pl["tile_i"], pl["tile_j"]) == (1, 1)
    else:
        assert (pl["tile_i"], pl["tile_j"]) == (6, 6)
    done = 0
    for t in (50, 100, 200):
        s.sweep(t - done)
        done = t
        s.sync()
        rho, tt = s.get_state()
        assert tt == t
        tr = s.trace()
        assert np.isfinite(tr).all()
        ref = orc.log_posterior_fft(rho)
        print("plan %s sweep %d: trace %.10g oracle %.10g rel %.2e" % (pl, t, tr[t - 1], ref,
                                                                       abs(tr[t - 1] - ref) / abs(ref)))
        assert abs(tr[t - 1] - ref) <= TRACE_RTOL * abs(ref), (t, tr[t - 1], ref)
    assert s.accept_counts().sum() > 10000
    s.close()


# ---------------------------------------------------------------- means
H = W = 30
LPSF = 3
SEED = 21
T = 600
BURN = 100
N_ORACLE = 48
N_GPU = 64


def _problem(gain_scale=1.0):
    p = synth.small_problem(H=H, W=W, L=LPSF, seed=SEED, burn_in=BURN, refresh_every=50)
    p.gain = p.gain * gain_scale
    return p


def _gpu_chain_means(precision, gain_scale=1.0):
    # independent chains: one problem per chain, with its own seed (the
    # oracle uses seed SEED, chains 0..N_ORACLE-1)
    probs = []
    for k in range(N_GPU):
        p = _problem(gain_scale)
        p.seed = 10_000 + k
        probs.append(p)
    s = bdecon.Sampler(probs, precision=precision, max_sweeps=T)
    s.sweep(T)
    out = np.stack([s.posterior_mean(k) for k in range(N_GPU)])
    s.close()
    return out


@pytest.fixture(scope="module")
def oracle_means():
    with mp.get_context("spawn").Pool(min(16, mp.cpu_count())) as pool:
        job = functools.partial(oracle_jobs.small_chain_mean, H, W, LPSF, SEED, BURN, 50, T)
        return np.stack(pool.map(job, range(N_ORACLE)))


def _within_3_mcse(a, b):
    d = a.mean(0) - b.mean(0)
    se = np.sqrt(a.var(0, ddof=1) / a.shape[0] + b.var(0, ddof=1) / b.shape[0])
    return float(np.mean(np.abs(d) <= 3 * se))


def test_fp32_posterior_means_within_3_mcse_of_oracle(oracle_means):
    g = _gpu_chain_means(bdecon.BDECON_FP32)
    frac = _within_3_mcse(g, oracle_means)
    print(f"fraction of pixels within 3 MCSE: {frac:.4f}")
    assert frac >= 0.99


def test_mcse_check_rejects_wrong_gain(oracle_means):
    g = _gpu_chain_means(bdecon.BDECON_FP64, gain_scale=1.5)
    frac = _within_3_mcse(g, oracle_means)
    print(f"wrong gain: fraction within 3 MCSE {frac:.4f}")
    assert frac < 0.9
