"""Pins of the oracle's model functions (no GPU).

Every function of the oracle is checked against something other than
itself: library routines (FFT convolution, numpy FFT, scipy Dirichlet and
Poisson/Normal densities), explicit brute-force sums, closed-form limits and
invariants of the paper's model (Eq. 1-9).
"""
import math

import numpy as np
import pytest
from scipy import integrate, signal, special, stats

from oracle import oracle as O
from paper_2411_00991_gb300 import synth


# ------------------------------------------------------------ Eq. 1-2 ----

@pytest.mark.parametrize("L,H,W", [(1, 5, 7), (3, 6, 5), (5, 11, 9), (9, 20, 17)])
def test_convolution_matches_library(L, H, W):
    rng = np.random.default_rng(L * 100 + H)
    K = rng.uniform(0, 1, size=(L, L))        # asymmetric kernel: orientation matters
    rho = rng.uniform(0.1, 5, size=(H + L - 1, W + L - 1))
    mu = O.convolve(rho, K)
    ref1 = signal.convolve2d(rho, K, mode="valid")
    ref2 = signal.fftconvolve(rho, K, mode="valid")
    assert mu.shape == (H, W)
    np.testing.assert_allclose(mu, ref1, rtol=1e-13)
    np.testing.assert_allclose(mu, ref2, rtol=1e-11)


def test_delta_psf_is_identity():
    rng = np.random.default_rng(3)
    rho = rng.uniform(0.1, 5, size=(9, 8))
    K = np.zeros((3, 3)); K[1, 1] = 1.0
    np.testing.assert_array_equal(O.convolve(rho, K), rho[1:-1, 1:-1])


# ------------------------------------------------------------ Eq. 3-6 ----

def _loglik_explicit(w, o, G, var, mu, phimax):
    phi = np.arange(phimax + 1)
    t = stats.norm.logpdf(w, loc=G * phi + o, scale=math.sqrt(var)) + stats.poisson.logpmf(phi, mu)
    return special.logsumexp(t)


CASES = [
    # w, o, G, var, mu
    (110.0, 100.0, 2.0, 2.56, 5.0),
    (100.0, 100.0, 2.0, 2.56, 0.3),
    (97.0, 100.0, 2.0, 2.56, 1.0),        # negative photon estimate
    (200.0, 100.0, 2.0, 2.56, 50.0),
    (200.0, 100.0, 2.0, 2.56, 3.0),       # data far above mu
    (102.0, 100.0, 2.0, 2.56, 80.0),      # data far below mu
    (141.7, 99.1, 2.1, 0.05, 20.0),       # tiny read noise
    (141.7, 99.1, 2.1, 40.0, 20.0),       # read noise dominates
    (1100.0, 100.0, 2.0, 2.56, 480.0),    # bright
    (104.0, 100.0, 1.0, 9.0, 0.01),
    # the extremes of the 2048x2048 low-SNR frame (read-noise variance down to
    # 1e-3 ADU^2, i.e. 1/s^2 up to 4410, photon estimates -5.8 .. 10.6)
    (100.0 + 2.1 * 0.0226, 100.0, 2.1, 0.001, 1.1),
    (100.0 + 2.1 * 1.984, 100.0, 2.1, 0.001, 1.3),
    (100.0 + 2.1 * 1.5, 100.0, 2.1, 0.001, 1.3),     # two photon counts equally likely
    (100.0 - 2.1 * 5.79, 100.0, 2.1, 0.001, 1.1),    # far below the offset
    (100.0 + 2.1 * 10.55, 100.0, 2.1, 0.001, 2.0),
]


@pytest.mark.parametrize("w,o,G,var,mu", CASES)
def test_loglik_explicit_sum(w, o, G, var, mu):
    phimax = int(max((w - o) / G, mu) + 60 * math.sqrt(max(mu, 1.0)) + 80 * math.sqrt(var) / G + 100)
    ref = _loglik_explicit(w, o, G, var, mu, phimax)
    got = O.loglik(w, o, G, var, mu)
    assert got == pytest.approx(ref, rel=1e-12, abs=1e-12)


@pytest.mark.parametrize("k,mu", [(0, 0.7), (3, 2.5), (17, 11.0), (60, 75.0)])
def test_loglik_poisson_limit(k, mu):
    # sigma -> 0 with an integer photon count: the Normal picks phi = k
    G, o, var = 2.0, 100.0, 1e-6
    w = o + G * k
    got = O.loglik(w, o, G, var, mu)
    ref = -0.5 * math.log(2 * math.pi * var) + stats.poisson.logpmf(k, mu)
    assert got == pytest.approx(ref, rel=1e-12, abs=1e-10)


@pytest.mark.parametrize("w", [95.0, 100.0, 103.3])
def test_loglik_normal_limit(w):
    # mu -> 0: only phi = 0 survives, Normal(w; o, var) e^{-mu}
    o, G, var, mu = 100.0, 2.0, 2.56, 1e-14
    ref = stats.norm.logpdf(w, o, math.sqrt(var)) - mu
    assert O.loglik(w, o, G, var, mu) == pytest.approx(ref, rel=1e-12, abs=1e-12)


@pytest.mark.parametrize("mu,var", [(0.5, 2.56), (4.0, 2.56), (12.0, 0.3)])
def test_loglik_normalised_over_w(mu, var):
    o, G = 100.0, 2.0
    f = lambda w: math.exp(O.loglik(w, o, G, var, mu))
    hi = o + G * (mu + 12 * math.sqrt(mu) + 12) + 12 * math.sqrt(var)
    lo = o - 12 * math.sqrt(var)
    pts = [o + G * k for k in range(0, int(mu + 12 * math.sqrt(mu) + 12))][:50]
    val, err = integrate.quad(f, lo, hi, points=pts, limit=400, epsabs=1e-12, epsrel=1e-12)
    assert val == pytest.approx(1.0, abs=1e-8)


# ------------------------------------------------------------ Eq. 7-8 ----

@pytest.mark.parametrize("ph,pw", [(9, 9), (4, 6), (1, 5), (7, 1), (2, 2), (1, 1)])
def test_patch_dft_matches_fft(ph, pw):
    rng = np.random.default_rng(ph * 10 + pw)
    x = rng.uniform(0.1, 3, size=(ph, pw))
    np.testing.assert_allclose(O.patch_dft(x), np.fft.fft2(x), rtol=0, atol=1e-12 * x.sum())


@pytest.mark.parametrize("L,ph,pw", [(9, 9, 9), (9, 4, 9), (9, 1, 9), (5, 3, 2), (5, 7, 7), (17, 17, 1), (3, 1, 1)])
def test_alpha_is_sampled_otf(L, ph, pw):
    # alpha_k is |OTF| at frequency (k/ph, l/pw): the DTFT of the centred
    # PSF evaluated on the patch's frequency grid, normalised to sum 1.
    rng = np.random.default_rng(L + ph + pw)
    K = rng.uniform(0.01, 1, size=(L, L)); K /= K.sum()
    R = L // 2
    x = np.arange(L) - R
    Ey = np.exp(-2j * np.pi * np.outer(np.arange(ph), x) / ph)     # (ph, L)
    Ex = np.exp(-2j * np.pi * np.outer(np.arange(pw), x) / pw)     # (pw, L)
    otf = Ey @ K @ Ex.T
    ref = np.abs(otf) / np.abs(otf).sum()
    np.testing.assert_allclose(O.alpha(K, ph, pw), ref, rtol=1e-12, atol=1e-15)


def test_alpha_gaussian_properties():
    K = synth.gaussian_psf(1.5, 9)
    a = O.alpha(K, 9, 9)
    assert a.sum() == pytest.approx(1.0, abs=1e-14)
    assert a[0, 0] == a.max()                       # DC carries the most weight
    # Hermitian symmetry of a real PSF: |OTF(-k)| = |OTF(k)|
    idx = (-np.arange(9)) % 9
    np.testing.assert_allclose(a, a[np.ix_(idx, idx)], rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("ph,pw", [(9, 9), (3, 5), (2, 2), (1, 4)])
def test_log_prior_matches_scipy_dirichlet(ph, pw):
    rng = np.random.default_rng(ph * 7 + pw)
    K = synth.gaussian_psf(1.0, 5)
    a = O.alpha(K, ph, pw)
    x = rng.uniform(0.2, 4, size=(ph, pw))
    spec = np.fft.fft2(x)
    mod = np.abs(spec).ravel()
    xs = mod / mod.sum()
    av = a.ravel()
    lB = special.gammaln(av).sum() - special.gammaln(av.sum())
    ref = stats.dirichlet.logpdf(xs, av) + lB
    assert O.log_prior_patch(spec, a) == pytest.approx(ref, rel=1e-11, abs=1e-9)


def test_log_prior_scale_invariant():
    # property (3) of the prior (Methods, "Prior"): degenerate under rho -> c rho
    rng = np.random.default_rng(5)
    K = synth.gaussian_psf(1.3, 7)
    a = O.alpha(K, 7, 7)
    spec = np.fft.fft2(rng.uniform(0.2, 4, size=(7, 7)))
    base = O.log_prior_patch(spec, a)
    for c in (1e-3, 0.5, 7.0, 1e4):
        assert O.log_prior_patch(c * spec, a) == pytest.approx(base, rel=1e-11, abs=1e-9)


def test_single_pixel_patch_prior_is_flat():
    a = O.alpha(np.ones((1, 1)), 1, 1)
    assert a[0, 0] == 1.0
    for v in (0.1, 3.0, 77.0):
        assert O.log_prior_patch(np.array([[v + 0j]]), a) == 0.0


# --------------------------------------------------------------- Eq. 9 ---

def _logpost_independent(prob, rho):
    """Log posterior assembled from library pieces only (scipy/numpy)."""
    g, o, v = prob.maps()
    K = prob.psf / prob.psf.sum()
    mu = signal.convolve2d(rho, K, mode="valid")
    w = prob.image.astype(np.float64)
    ll = 0.0
    for n in range(w.size):
        wn, on, gn, vn, mn = w.flat[n], o.flat[n], g.flat[n], v.flat[n], mu.flat[n]
        phimax = int(max((wn - on) / gn, mn) + 40 + 20 * math.sqrt(mn + 1))
        ll += _loglik_explicit(wn, on, gn, vn, mn, phimax)
    S = prob.S
    Ho, Wo = rho.shape
    R = prob.L // 2
    x = np.arange(prob.L) - R
    lp = 0.0
    for i0 in range(0, Ho, S):
        for j0 in range(0, Wo, S):
            patch = rho[i0:i0 + S, j0:j0 + S]
            ph, pw = patch.shape
            Ey = np.exp(-2j * np.pi * np.outer(np.arange(ph), x) / ph)
            Ex = np.exp(-2j * np.pi * np.outer(np.arange(pw), x) / pw)
            al = np.abs(Ey @ K @ Ex.T); al /= al.sum()
            mod = np.abs(np.fft.fft2(patch))
            lp += ((al - 1) * np.log(mod)).sum() + (ph * pw - 1) * np.log(mod.sum())
    return ll + lp


def test_log_posterior_assembly():
    prob = synth.small_problem(H=9, W=11, L=5, maps=True, seed=11)
    rho = synth.random_state(prob, 3)
    orc = O.Oracle(prob)
    assert orc.log_posterior(rho) == pytest.approx(_logpost_independent(prob, rho), rel=1e-11)


@pytest.mark.parametrize("L,S,maps", [(5, 5, False), (5, 7, True), (3, 3, True), (7, 7, False)])
def test_incremental_delta_equals_posterior_difference(L, S, maps):
    # dL + dP of one single-site change equals the change of the full log
    # posterior: pins the window indexing, PSF orientation, patch location
    # and the twiddle sign of the incremental spectrum update.
    prob = synth.small_problem(H=13, W=10, L=L, stride=S, maps=maps, seed=L + S)
    orc = O.Oracle(prob)
    rho = synth.random_state(prob, 9)
    Ho, Wo = prob.object_shape()
    rng = np.random.default_rng(1)
    ms = [0, Wo - 1, (Ho - 1) * Wo, Ho * Wo - 1] + list(rng.integers(0, Ho * Wo, size=10))
    base = orc.log_posterior(rho)
    for m in ms:
        new = rho.flat[m] * math.exp(rng.normal(0, 0.3))
        ok, dl, dp = orc.delta(rho, m, new)
        assert ok
        r2 = rho.copy(); r2.flat[m] = new
        assert dl + dp == pytest.approx(orc.log_posterior(r2) - base, abs=1e-9)


def test_init_rule():
    prob = synth.small_problem(H=6, W=5, L=3, seed=2)
    orc = O.Oracle(prob)
    rho = orc.init()
    g, o, v = prob.maps()
    b0 = max(0.1, float(np.mean((prob.image.astype(np.float64) - o) / g)))
    Ho, Wo = prob.object_shape()
    for m in range(Ho * Wo):
        z, _ = O.draw(prob.seed, m, 0, 0)
        assert rho.flat[m] == pytest.approx(b0 * math.exp(0.1 * z), rel=1e-15)


@pytest.mark.parametrize("kw", [
    dict(H=20, W=24, L=5, seed=7, maps=True),              # ragged patch tail, sCMOS maps
    dict(H=16, W=19, L=5, stride=7, seed=9),               # stride > L, partial patches
    dict(H=14, W=13, L=3, subpixel=2, seed=3),             # lattice finer than the camera
])
def test_fft_evaluator_equals_definitional_log_posterior(kw):
    # the large-frame evaluator takes the patch spectra from numpy's FFT instead
    # of the DFT written out by its definition; Eq. 9 must not change
    prob = synth.small_problem(**kw)
    orc = O.Oracle(prob)
    rho = synth.random_state(prob, 11)
    a, b = orc.log_posterior(rho), orc.log_posterior_fft(rho)
    assert b == pytest.approx(a, rel=1e-12)
    # and its likelihood part is Eq. 6 summed at the convolution of rho
    mu = O.expected(rho, prob.H, prob.W, prob.psf / prob.psf.sum(), prob.subpixel)
    g, o, v = prob.maps()
    ll = sum(O.loglik(float(w), float(oo), float(gg), float(vv), float(m))
             for w, oo, gg, vv, m in zip(prob.image.ravel(), o.ravel(), g.ravel(), v.ravel(), mu.ravel()))
    assert orc.log_likelihood(rho) == pytest.approx(ll, rel=1e-12)
