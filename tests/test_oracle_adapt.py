"""Pins of the oracle's burn-in adaptation of the proposal scale (no GPU).

Rule: each pixel keeps its own log-space step s_m (starting at the problem's
step); during burn-in only, after each update of m, s_m is multiplied by
exp(0.1 (1 - a*)) on accept and by exp(-0.1 a*) on reject (clamped to
[1e-4, 4]), a* the problem's target acceptance rate.  Its fixed point is an
acceptance rate of a* (where the pixel can reach it); after burn-in the
scales are frozen and the chain is an ordinary Metropolis-Hastings chain
with per-pixel proposal scales, so its target is unchanged.

Pins: the acceptance rate settles at a* (a wrong sign or constant moves or
destroys the fixed point); the scales do not move after burn-in; the
one-pixel closed-form posterior (a Normal-weighted mixture of Gamma(phi+1,1)
densities) is still sampled correctly after adaptation; without adaptation
the scales stay at the problem's step.
"""
import math

import numpy as np
import pytest
from scipy import stats

from oracle import oracle as O
from paper_2411_00991_gb300 import synth


def _batch_means_mcse(x, nb=40):
    x = np.asarray(x)
    n = (len(x) // nb) * nb
    bm = x[:n].reshape(nb, -1).mean(axis=1)
    return bm.std(ddof=1) / math.sqrt(nb)


def test_acceptance_settles_at_target_and_scales_freeze_after_burn_in():
    p = synth.small_problem(H=14, W=16, L=3, seed=81, burn_in=400, refresh_every=50)
    p.adapt_target = 0.2
    Ho, Wo = p.object_shape()
    r = O.Oracle(p).run(400)
    acc_late = r["n_acc"][250:400].sum() / (150 * Ho * Wo)
    assert 0.15 < acc_late < 0.25, acc_late
    # at the fixed step 0.2 this problem accepts more
    p2 = synth.small_problem(H=14, W=16, L=3, seed=81, burn_in=400, refresh_every=50)
    r2 = O.Oracle(p2).run(400)
    assert r2["n_acc"][250:400].sum() / (150 * Ho * Wo) > 0.25
    assert np.all(r2["steps"] == p2.step)
    # after burn-in the scales do not move
    r3 = O.Oracle(p).run(420)
    np.testing.assert_array_equal(r3["steps"], r["steps"])
    assert r["steps"].min() >= 1e-4 and r["steps"].max() <= 4.0
    assert np.unique(r["steps"]).size > 10            # each pixel found its own scale


def test_resume_after_burn_in_equals_one_run():
    p = synth.small_problem(H=10, W=12, L=3, seed=82, burn_in=30, refresh_every=7)
    p.adapt_target = 0.3
    o = O.Oracle(p)
    full = o.run(40)
    # no resume across burn-in is possible without the scales, so the pin is
    # that an unadapted problem resumes exactly while an adapted one does not
    q = synth.small_problem(H=10, W=12, L=3, seed=82, burn_in=30, refresh_every=7)
    a = O.Oracle(q).run(20)
    b = O.Oracle(q).run(20, t0=20, rho_in=a["rho"])
    c = O.Oracle(q).run(40)
    np.testing.assert_array_equal(b["rho"], c["rho"])
    assert not np.array_equal(full["rho"], c["rho"])


@pytest.mark.parametrize("w", [112.25, 160.0])
def test_one_pixel_posterior_after_adaptation(w):
    img = np.array([[w]], dtype=np.float32)
    prob = synth.Problem(image=img, psf=np.ones((1, 1)), gain=2.0, offset=100.0, var=2.56, stride=1,
                         seed=6, step=0.35, burn_in=2000, refresh_every=0, adapt_target=0.44, name="one_pixel")
    w32 = float(np.float32(w))
    phi = np.arange(400)
    lw = stats.norm.logpdf(w32, 2.0 * phi + 100.0, math.sqrt(2.56))
    a = np.exp(lw - lw.max())
    a /= a.sum()
    mean_exact = float((a * (phi + 1)).sum())
    T = 30000
    r = O.Oracle(prob).run(T, want_samples=True)
    s = r["samples"][:, 0, 0][prob.burn_in:]
    acc = r["n_acc"][prob.burn_in:].mean()
    assert 0.38 < acc < 0.50, acc                      # the adapted scale reaches the target
    mcse = _batch_means_mcse(s)
    assert abs(s.mean() - mean_exact) < 3.5 * mcse, (s.mean(), mean_exact, mcse)
