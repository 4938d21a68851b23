"""Pins of the oracle's photon-count augmented sampler (no GPU).

The paper writes the completed likelihood (Eq. 5) with the photon counts as
variables; summing them out gives Eq. 6.  The augmented sampler draws every
phi_n from p(phi | w_n, mu_n) at the start of a sweep, then updates rho
against sum_n phi_n log mu_n - mu_n.  Pins:
  * the photon-count draw, applied to a fine grid of uniforms, reproduces
    the normalised product Normal(w; G phi + o, var) Poisson(phi; mu)
    computed with scipy, count by count;
  * the per-pixel completed log likelihood, summed over phi, is Eq. 6;
  * the one-pixel closed-form posterior of rho (a Normal-weighted mixture
    of Gamma(phi + 1, 1)) is sampled correctly by the augmented chain;
  * the chain's state is rho alone (the counts are redrawn every sweep), so
    resuming from rho is exact.
"""
import math

import numpy as np
import pytest
from scipy import stats
from scipy.special import logsumexp

from oracle import oracle as O
from paper_2411_00991_gb300 import synth


@pytest.mark.parametrize("w,mu,G,var", [(112.25, 7.3, 2.0, 2.56), (100.4, 0.2, 2.1, 5.0),
                                        (420.0, 150.0, 2.0, 1.0), (99.0, 3.0, 1.0, 0.3)])
def test_phi_draw_reproduces_the_conditional_pmf(w, mu, G, var):
    o = 100.0
    N = 20000
    draws = np.array([O.sample_phi(w, o, G, var, mu, (k + 0.5) / N) for k in range(N)])
    phi = np.arange(0, int(draws.max()) + 50)
    lp = stats.norm.logpdf(w, G * phi + o, math.sqrt(var)) + stats.poisson.logpmf(phi, mu)
    p = np.exp(lp - logsumexp(lp))
    counts = np.bincount(draws, minlength=phi.size)[:phi.size]
    # a grid of uniforms puts N p_phi +- 1 points in each count's interval
    assert np.all(np.abs(counts - N * p) <= 1.0 + 1e-9 * N), np.max(np.abs(counts - N * p))


@pytest.mark.parametrize("w,mu", [(112.25, 7.3), (100.4, 0.2), (150.0, 40.0)])
def test_completed_likelihood_sums_to_eq6(w, mu):
    o, G, var = 100.0, 2.0, 2.56
    terms = [O.logjoint_pixel(w, o, G, var, mu, k) for k in range(400)]
    assert logsumexp(terms) == pytest.approx(O.loglik(w, o, G, var, mu), rel=1e-12, abs=1e-12)


def _batch_means_mcse(x, nb=40):
    x = np.asarray(x)
    n = (len(x) // nb) * nb
    bm = x[:n].reshape(nb, -1).mean(axis=1)
    return bm.std(ddof=1) / math.sqrt(nb)


@pytest.mark.parametrize("w", [112.25, 101.5, 160.0])
def test_one_pixel_posterior_with_augmented_sampler(w):
    img = np.array([[w]], dtype=np.float32)
    prob = synth.Problem(image=img, psf=np.ones((1, 1)), gain=2.0, offset=100.0, var=2.56, stride=1,
                         seed=8, step=0.35, burn_in=500, refresh_every=0, augmented=True, name="one_pixel")
    w32 = float(np.float32(w))
    phi = np.arange(400)
    lw = stats.norm.logpdf(w32, 2.0 * phi + 100.0, math.sqrt(2.56))
    a = np.exp(lw - lw.max())
    a /= a.sum()
    mean_exact = float((a * (phi + 1)).sum())
    cdf = lambda x: (a[None, :] * stats.gamma.cdf(np.asarray(x)[:, None], phi[None, :] + 1)).sum(axis=1)
    T = 30000
    r = O.Oracle(prob).run(T, want_samples=True)
    s = r["samples"][:, 0, 0][prob.burn_in:]
    mcse = _batch_means_mcse(s)
    assert abs(s.mean() - mean_exact) < 3.5 * mcse, (s.mean(), mean_exact, mcse)
    assert stats.kstest(s[::30], cdf).pvalue > 1e-3


def test_augmented_chain_resumes_exactly_from_rho():
    p = synth.small_problem(H=12, W=13, L=3, seed=83, refresh_every=4)
    p.augmented = True
    full = O.Oracle(p).run(14)
    a = O.Oracle(p).run(6)
    b = O.Oracle(p).run(8, t0=6, rho_in=a["rho"])
    np.testing.assert_array_equal(b["rho"], full["rho"])
    np.testing.assert_array_equal(b["phi"], full["phi"])
    o = O.Oracle(p)
    assert full["trace"][-1] == pytest.approx(o.log_joint(full["rho"], full["phi"]), rel=1e-12)
    # a differently seeded chain differs (the counts are drawn, not fixed)
    q = synth.small_problem(H=12, W=13, L=3, seed=83, refresh_every=4)
    q.augmented = True
    q.seed = 84
    assert not np.array_equal(O.Oracle(q).run(14)["rho"], full["rho"])
