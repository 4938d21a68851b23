"""Pins of the oracle's sampler (no GPU).

The single-site Metropolis-within-Gibbs chain is checked against posteriors
known independently of the oracle:
  * one pixel, delta PSF, flat prior: the posterior of rho is a Normal-
    weighted mixture of Gamma(phi+1, 1) densities (closed form);
  * two pixels, delta PSF, one 1x2 Dirichlet patch: posterior means by
    nested quadrature (scipy) of the density written from Eq. 6-9;
and against invariants of the sub-lattice schedule (conditional
independence of a class; exact resume from a checkpoint).
"""
import math

import numpy as np
import pytest
from scipy import integrate, stats

from oracle import oracle as O
from paper_2411_00991_gb300 import synth


def _batch_means_mcse(x, nb=40):
    x = np.asarray(x)
    n = (len(x) // nb) * nb
    bm = x[:n].reshape(nb, -1).mean(axis=1)
    return bm.std(ddof=1) / math.sqrt(nb)


def _phi_weights(w, o, G, var, phimax=400):
    phi = np.arange(phimax)
    lw = stats.norm.logpdf(w, G * phi + o, math.sqrt(var))
    a = np.exp(lw - lw.max())
    return phi, a / a.sum()


def _one_pixel_problem(w, o=100.0, G=2.0, var=2.56, seed=5):
    img = np.array([[w]], dtype=np.float32)
    return synth.Problem(image=img, psf=np.ones((1, 1)), gain=G, offset=o, var=var,
                         stride=1, n_chains=1, seed=seed, step=0.35, burn_in=500,
                         refresh_every=0, name="one_pixel")


@pytest.mark.parametrize("w", [112.25, 101.5, 160.0])
def test_one_pixel_posterior_closed_form(w):
    # p(rho | w) ∝ sum_phi Normal(w; G phi + o, var) Poisson(phi; rho) on rho > 0;
    # each Poisson term integrates over rho to a Gamma(phi + 1, 1) density.
    prob = _one_pixel_problem(w)
    w32 = float(np.float32(w))
    phi, a = _phi_weights(w32, 100.0, 2.0, 2.56)
    mean_exact = float((a * (phi + 1)).sum())
    cdf = lambda x: (a[None, :] * stats.gamma.cdf(np.asarray(x)[:, None], phi[None, :] + 1)).sum(axis=1)
    T = 30000
    r = O.Oracle(prob).run(T, want_samples=True)
    s = r["samples"][:, 0, 0][prob.burn_in:]
    assert r["n_sum"] == T - prob.burn_in
    assert r["mean"][0, 0] == pytest.approx(s.mean(), rel=1e-12)
    mcse = _batch_means_mcse(s)
    assert abs(s.mean() - mean_exact) < 3.5 * mcse, (s.mean(), mean_exact, mcse)
    thin = s[::30]
    assert stats.kstest(thin, cdf).pvalue > 1e-3
    # the Hastings term matters: without it the chain would target exp(l)/rho,
    # whose mean is one lower
    assert abs(s.mean() - (mean_exact - 1.0)) > 10 * mcse


def test_two_pixel_dirichlet_posterior_quadrature():
    # 1x2 object, delta PSF, stride 2: one patch holds both pixels, so the
    # Dirichlet prior of Eq. 8 couples them; alpha = (1/2, 1/2) for a delta PSF.
    w = (108.0, 116.0)
    o, G, var = 100.0, 2.0, 2.56
    img = np.array([w], dtype=np.float32)
    prob = synth.Problem(image=img, psf=np.ones((1, 1)), gain=G, offset=o, var=var, stride=2,
                         seed=11, step=0.35, burn_in=1000, refresh_every=0, name="two_pixel")
    phis = [_phi_weights(float(np.float32(x)), o, G, var) for x in w]

    def lik(k, rho):
        phi, a = phis[k]
        return float((a * stats.poisson.pmf(phi, rho)).sum())

    def prior(x, y):   # (x+y)^(-1/2) |x-y|^(-1/2) (|x+y| + |x-y|), the |x-y|^(-1/2) left to quad
        return (x + y) ** -0.5 * ((x + y) + abs(x - y))

    # integrate over b in (0, B) and d = |a - b| in (0, D) on both sides of a = b
    B, D = 45.0, 45.0

    def moments():
        out = np.zeros(3)
        for sgn in (+1, -1):
            def inner(b, f):
                g = lambda d: (lambda aa: 0.0 if aa <= 0 else f(aa, b) * lik(0, aa) * lik(1, b) * prior(aa, b))(b + sgn * d)
                hi = D if sgn > 0 else b
                v, _ = integrate.quad(g, 0.0, hi, weight="alg", wvar=(-0.5, 0.0), limit=200)
                return v
            for k, f in enumerate((lambda aa, bb: 1.0, lambda aa, bb: aa, lambda aa, bb: bb)):
                v, _ = integrate.quad(lambda b: inner(b, f), 0.0, B, limit=200, epsrel=1e-7)
                out[k] += v
        return out

    Z, Ea, Eb = moments()
    Ea, Eb = Ea / Z, Eb / Z
    T = 40000
    r = O.Oracle(prob).run(T, want_samples=True)
    s = r["samples"][prob.burn_in:, 0, :]
    for k, ex in ((0, Ea), (1, Eb)):
        mcse = _batch_means_mcse(s[:, k])
        assert abs(s[:, k].mean() - ex) < 3.5 * mcse, (k, s[:, k].mean(), ex, mcse)
    # without the prior the two means would be the independent one-pixel means
    ind = [float((a * (phi + 1)).sum()) for phi, a in phis]
    assert max(abs(Ea - ind[0]), abs(Eb - ind[1])) > 0.3


def _box_problem(stride):
    # a flat 5x5 PSF makes neighbouring windows interact strongly
    prob = synth.small_problem(H=14, W=15, L=5, stride=stride, seed=21, refresh_every=0, step=0.8)
    prob.psf = np.ones((5, 5))
    return prob


def test_class_updates_are_conditionally_independent():
    # S >= L: windows of one class are disjoint and each patch holds one
    # pixel of the class, so the order inside a class cannot matter.
    for prob in (_box_problem(5), synth.small_problem(H=14, W=15, L=5, seed=21, refresh_every=4)):
        orc = O.Oracle(prob)
        a = orc.run(20, order=0, want_acc_log=True)
        b = orc.run(20, order=1, want_acc_log=True)
        np.testing.assert_array_equal(a["acc_log"], b["acc_log"])
        np.testing.assert_array_equal(a["rho"], b["rho"])
        np.testing.assert_array_equal(a["mu"], b["mu"])
        np.testing.assert_array_equal(a["trace"], b["trace"])
        assert 0 < a["n_acc"].sum() < 20 * a["rho"].size


def test_dependence_is_detected_when_stride_below_support():
    # negative control: with S < L windows of one class overlap and the
    # order inside the class changes the chain
    orc = O.Oracle(_box_problem(3))
    a = orc.run(20, order=0, want_acc_log=True)
    b = orc.run(20, order=1, want_acc_log=True)
    assert (a["acc_log"] != b["acc_log"]).any()
    assert not np.array_equal(a["mu"], b["mu"])


def test_incremental_mu_tracks_convolution():
    prob = synth.small_problem(H=16, W=12, L=5, seed=3, refresh_every=0)
    orc = O.Oracle(prob)
    r = orc.run(12)
    K = prob.psf / prob.psf.sum()
    np.testing.assert_allclose(r["mu"], O.convolve(r["rho"], K), rtol=1e-12)


def test_resume_is_exact():
    prob = synth.small_problem(H=12, W=13, L=5, seed=8, refresh_every=3, burn_in=2)
    orc = O.Oracle(prob)
    full = orc.run(6, want_acc_log=True)
    first = orc.run(3, want_acc_log=True)
    second = orc.run(3, t0=3, rho_in=first["rho"], want_acc_log=True)
    np.testing.assert_array_equal(full["acc_log"][3:], second["acc_log"])
    np.testing.assert_array_equal(full["rho"], second["rho"])
    np.testing.assert_array_equal(full["trace"][3:], second["trace"])
    assert full["n_sum"] == 4 and second["n_sum"] == 3
    np.testing.assert_allclose(full["sum"], first["sum"] + second["sum"], rtol=1e-15)


def test_trace_is_log_posterior_of_state():
    prob = synth.small_problem(H=10, W=9, L=3, seed=4)
    orc = O.Oracle(prob)
    r = orc.run(3, want_samples=True)
    for t in range(3):
        assert r["trace"][t] == orc.log_posterior(r["samples"][t])


def test_single_update_matches_first_class_of_a_sweep():
    # the local evaluation reproduces the chain's first-class decisions
    prob = synth.small_problem(H=15, W=17, L=5, maps=True, seed=13)
    orc = O.Oracle(prob)
    rho0 = orc.init()
    r = orc.run(1, want_acc_log=True, want_samples=True)
    S = prob.S
    Ho, Wo = prob.object_shape()
    for i in range(0, Ho, S):
        for j in range(0, Wo, S):
            m = i * Wo + j
            acc, rn, dl, dp = orc.single_update(rho0, m, 1)
            ok, dl2, dp2 = orc.delta(rho0, m, rn)
            assert acc == bool(r["acc_log"][0, i, j])
            assert r["samples"][0, i, j] == (rn if acc else rho0[i, j])
            assert dl == pytest.approx(dl2, abs=1e-10) and dp == pytest.approx(dp2, abs=1e-10)
