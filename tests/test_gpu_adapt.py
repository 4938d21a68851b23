"""Burn-in adaptation of the per-pixel proposal scale on the GPU.

Double precision: the chain, including every pixel's adapted scale, equals
the oracle's (identical accept decisions; scales and objects within 1e-12),
through burn-in and after it, where the scales freeze.  Single precision:
adaptation raises the acceptance rate as it does in the oracle.  Batched:
an adapting problem gives the same chain alone and next to non-adapting
ones.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2411_00991_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2411_00991_gb300 import bdecon  # noqa: E402

RTOL = 1e-12


def _adapting(seed=91, **kw):
    p = synth.small_problem(H=20, W=24, L=5, maps=True, seed=seed, burn_in=12, refresh_every=5, **kw)
    p.adapt_target = 0.3
    return p


def test_fp64_adapted_chain_matches_oracle():
    p = _adapting(n_chains=2)
    T = 20
    s = bdecon.Sampler(p, precision=bdecon.BDECON_FP64, max_sweeps=T + 4, flags=bdecon.FLAG_ACCEPT_LOG)
    s.sweep(T)
    for c in range(2):
        ref = O.Oracle(p, chain=c).run(T, want_acc_log=True)
        assert np.array_equal(s.accept_log(0, c), ref["acc_log"])
        np.testing.assert_allclose(s.get_steps(0, c), ref["steps"], rtol=RTOL)
        np.testing.assert_allclose(s.get_state(0, c)[0], ref["rho"], rtol=RTOL)
        np.testing.assert_allclose(s.trace(0, c), ref["trace"], rtol=RTOL)
    steps = s.get_steps(0, 0)
    assert np.unique(steps).size > 10
    s.sweep(3)                                       # past burn-in: frozen
    np.testing.assert_array_equal(s.get_steps(0, 0), steps)
    s.close()


def test_unadapted_problem_reports_its_step():
    p = synth.small_problem(H=9, W=11, L=3, seed=92)
    s = bdecon.Sampler(p, precision=bdecon.BDECON_FP32, max_sweeps=4)
    assert np.all(s.get_steps() == p.step)
    s.close()


def test_fp32_adaptation_moves_acceptance_like_the_oracle():
    # On this model the acceptance rate falls slowly with the scale (the
    # Dirichlet prior with sum(alpha) = 1 is singular where spectrum
    # coefficients vanish), so within a 300-sweep burn-in the scales are still
    # shrinking toward the target.  The float chain's acceptance in the last
    # 100 burn-in sweeps must match the double oracle's (statistically) and be
    # well above the unadapted chain's.
    def prob(target):
        p = synth.small_problem(H=40, W=44, L=5, seed=93, burn_in=300, refresh_every=50)
        p.adapt_target = target
        return p
    Ho, Wo = prob(0.0).object_shape()
    rates = []
    for target in (0.25, 0.0):
        s = bdecon.Sampler(prob(target), precision=bdecon.BDECON_FP32, max_sweeps=310)
        s.sweep(300)
        rates.append(s.accept_counts()[200:300].sum() / (100 * Ho * Wo))
        s.close()
    ref = O.Oracle(prob(0.25)).run(300)["n_acc"][200:300].sum() / (100 * Ho * Wo)
    assert abs(rates[0] - ref) < 0.15 * ref, (rates[0], ref)
    assert rates[0] > 2 * rates[1], rates


@pytest.mark.parametrize("precision", [bdecon.BDECON_FP64, bdecon.BDECON_FP32])
def test_adapting_problem_same_alone_and_in_batch(precision):
    probs = [_adapting(seed=94), synth.small_problem(H=17, W=13, L=3, seed=95, burn_in=2),
             _adapting(seed=96, n_chains=2)]
    T = 16
    b = bdecon.Sampler(probs, precision=precision, max_sweeps=T)
    b.sweep(T)
    got = [(b.get_state(k, 0)[0], b.get_steps(k, 0), b.posterior_mean(k)) for k in range(3)]
    b.close()
    for k, pr in enumerate(probs):
        a = bdecon.Sampler(pr, precision=precision, max_sweeps=T)
        a.sweep(T)
        want = (a.get_state(0, 0)[0], a.get_steps(0, 0), a.posterior_mean(0))
        a.close()
        for x, y in zip(got[k], want):
            np.testing.assert_array_equal(x, y)
