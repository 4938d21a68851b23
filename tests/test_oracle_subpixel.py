"""Pins of the oracle on an object lattice finer than the camera (no GPU).

With f lattice cells per camera pixel side, Eq. 1's pixel integral sums the
f x f cells of each camera pixel: mu = bin_f(K (x) rho) (the paper's Nyquist
object lattice).  Pins:
  * the oracle's expected image equals scipy's valid convolution on the
    lattice followed by f x f binning (asymmetric kernels, f = 2, 3);
  * dL + dP of a single-site change equals the change of the full log
    posterior (window rows and kernel phase of every sub-cell position);
  * with the default stride (L + f - 1, the camera window of one update) the
    order inside a class does not matter; with a narrower stride it does;
  * the sampler's running expected image tracks the convolution;
  * the local single-update evaluation reproduces the first class.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2411_00991_gb300 import synth


@pytest.mark.parametrize("f,L,H,W", [(2, 3, 7, 9), (3, 5, 6, 5), (2, 5, 8, 6), (1, 5, 6, 7)])
def test_expected_image_is_lattice_blur_then_binning(f, L, H, W):
    rng = np.random.default_rng(f * 10 + L)
    K = rng.random((L, L))
    K /= K.sum()
    rho = rng.random((f * H + L - 1, f * W + L - 1)) + 0.1
    np.testing.assert_allclose(O.expected(rho, H, W, K, f), synth.expected_image(rho, K, f), rtol=1e-10)


@pytest.mark.parametrize("f,L,maps", [(2, 3, False), (2, 5, True), (3, 3, True)])
def test_incremental_delta_equals_posterior_difference_on_fine_lattice(f, L, maps):
    prob = synth.small_problem(H=9, W=8, L=L, maps=maps, seed=40 + f + L, subpixel=f)
    orc = O.Oracle(prob)
    rho = synth.random_state(prob, 9)
    Ho, Wo = prob.object_shape()
    assert (Ho, Wo) == (f * 9 + L - 1, f * 8 + L - 1)
    rng = np.random.default_rng(2)
    ms = [0, Wo - 1, (Ho - 1) * Wo, Ho * Wo - 1] + list(rng.integers(0, Ho * Wo, size=12))
    base = orc.log_posterior(rho)
    for m in ms:
        new = rho.flat[m] * math.exp(rng.normal(0, 0.3))
        ok, dl, dp = orc.delta(rho, m, new)
        assert ok
        r2 = rho.copy()
        r2.flat[m] = new
        assert dl + dp == pytest.approx(orc.log_posterior(r2) - base, abs=1e-9)


def _box(f, stride):
    prob = synth.small_problem(H=10, W=11, L=3, seed=23, refresh_every=0, step=0.8, subpixel=f, stride=stride)
    prob.psf = np.ones((3, 3))
    return prob


def test_class_independence_at_default_stride_and_dependence_below():
    good = _box(2, 0)                       # stride L + f - 1 = 4
    assert good.S == 4
    orc = O.Oracle(good)
    a = orc.run(15, order=0, want_acc_log=True)
    b = orc.run(15, order=1, want_acc_log=True)
    np.testing.assert_array_equal(a["acc_log"], b["acc_log"])
    np.testing.assert_array_equal(a["rho"], b["rho"])
    assert 0 < a["n_acc"].sum()
    bad = _box(2, 3)                        # windows of one class overlap
    orc = O.Oracle(bad)
    a = orc.run(15, order=0, want_acc_log=True)
    b = orc.run(15, order=1, want_acc_log=True)
    assert not np.array_equal(a["mu"], b["mu"])


def test_running_expected_image_tracks_convolution_and_single_update():
    prob = synth.small_problem(H=10, W=9, L=3, seed=24, refresh_every=0, subpixel=2)
    orc = O.Oracle(prob)
    r = orc.run(10)
    K = prob.psf / prob.psf.sum()
    np.testing.assert_allclose(r["mu"], O.expected(r["rho"], prob.H, prob.W, K, 2), rtol=1e-12)
    rho0 = orc.init()
    r1 = orc.run(1, want_acc_log=True, want_samples=True)
    S = prob.S
    Ho, Wo = prob.object_shape()
    for i in range(0, Ho, S):
        for j in range(0, Wo, S):
            m = i * Wo + j
            acc, rn, dl, dp = orc.single_update(rho0, m, 1)
            assert acc == bool(r1["acc_log"][0, i, j])
            assert r1["samples"][0, i, j] == (rn if acc else rho0[i, j])
