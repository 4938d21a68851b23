"""The Airy PSF input generator (the paper's widefield PSF, Methods), with
pins from the closed form of the Airy pattern: the fraction of the energy
inside the first dark ring (radius 0.61 lambda / NA) is
1 - J0(x0)^2 - J1(x0)^2 at x0 = 3.8317 (0.838), and the encircled energy
inside radius r is 1 - J0(x)^2 - J1(x)^2 with x = 2 pi NA r / lambda
(Rayleigh)."""
import math

import numpy as np
from scipy.special import j0, j1, jn_zeros

from paper_2411_00991_gb300 import synth


def _encircled(na, lam, r):
    x = 2 * math.pi * na * r / lam
    return 1.0 - j0(x) ** 2 - j1(x) ** 2


def test_airy_encircled_energy_matches_closed_form():
    na, lam, px, L = 1.4, 520.0, 8.0, 241
    k = synth.airy_psf(na, lam, px, L, sub=4)
    R = L // 2
    y, x = np.mgrid[-R:R + 1, -R:R + 1] * px
    r = np.hypot(y, x)
    x0 = jn_zeros(1, 1)[0]
    r0 = x0 * lam / (2 * math.pi * na)
    half = R * px                       # the support holds the disc of radius half
    frac_num = k[r <= r0].sum() / k[r <= half].sum()
    frac_ref = _encircled(na, lam, r0) / _encircled(na, lam, half)
    assert abs(frac_num - frac_ref) < 4e-3, (frac_num, frac_ref)
    assert abs(_encircled(na, lam, r0) - 0.8378) < 1e-3


def test_airy_is_normalised_symmetric_and_near_its_gaussian_approximation():
    k = synth.airy_psf(1.4, 520.0, 65.0, 17)
    assert abs(k.sum() - 1.0) < 1e-12 and (k > 0).all()
    np.testing.assert_allclose(k, k.T, atol=1e-15)
    np.testing.assert_allclose(k, k[::-1, ::-1], atol=1e-15)
    g = synth.gaussian_psf(synth.psf_sigma_from_optics(1.4, 520.0, 65.0), 17)
    assert abs(k[8, 8] / g[8, 8] - 1.0) < 0.1
