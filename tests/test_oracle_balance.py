"""Detailed balance of the oracle's single-site updates on a tiny object (no GPU).

A 4 x 4 object under a 2 x 2 camera with an asymmetric 3 x 3 PSF (Eq. 1-2:
every camera pixel sees every one of the four central object pixels, so the
window terms couple them), sCMOS-style per-pixel offsets and variances
(Eq. 4-6), and stride 4: one 4 x 4 patch, i.e. the literal global prior of
Eq. 7-8 with two-dimensional twiddles.  The four central object pixels move
on a log-spaced grid rho = b exp(h k), k = -3..3 (7^4 = 2401 states); the
twelve outer pixels stay fixed.

Each single-site kernel T_m is built from what the oracle's sampler itself
computes for an update -- the local likelihood change over the PSF window
and the local patch-prior change (Oracle.delta, the function the sampler
calls) -- with the proposal rho' = rho exp(+-h), probability 1/2 each, and
the sampler's decision rule  log u < dL + dP + log(rho'/rho)  (the last
term is the Hastings term of the log-space walk).  The grid's stationary
weights are taken from the oracle's full evaluation of Eq. 9 (Oracle.
log_posterior) times the Jacobian prod rho_m of the log grid.  Then
  * every pair of neighbouring states satisfies p_i T_ij = p_j T_ji to 1e-12;
  * p is invariant under a whole sweep T_sweep = T_1 T_2 T_3 T_4 in the
    sampler's class order.
Negative controls: the Hastings term with the wrong sign, and the window
terms taken with the PSF transposed, both break detailed balance by many
orders of magnitude more than the tolerance.
"""
import itertools
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2411_00991_gb300 import synth

K_GRID = 3           # grid index k = -K_GRID .. K_GRID per free site
H_STEP = 0.25        # log spacing of the grid
FREE = [(1, 1), (1, 2), (2, 1), (2, 2)]   # class (raster) order of the free sites at stride 4
TOL = 1e-12


def _problem(psf):
    rng = np.random.default_rng(2411)
    img = (100.0 + 2.0 * np.array([[13.0, 7.0], [9.0, 16.0]]) + rng.normal(0, 1.0, (2, 2))).astype(np.float32)
    off = rng.normal(100.0, 1.0, (2, 2)).astype(np.float32)
    var = rng.gamma(2.0, 1.0, (2, 2)).astype(np.float32) + np.float32(0.5)
    return synth.Problem(image=img, psf=psf, gain=2.0, offset=off, var=var, stride=4, n_chains=1,
                         seed=3, step=H_STEP, burn_in=0, refresh_every=0, name="balance4x4")


PSF = np.array([[0.05, 0.10, 0.02],
                [0.08, 0.40, 0.15],
                [0.03, 0.12, 0.05]])


def _grid():
    rng = np.random.default_rng(7)
    base = rng.uniform(3.0, 9.0, (4, 4))
    states = list(itertools.product(range(-K_GRID, K_GRID + 1), repeat=4))
    index = {s: n for n, s in enumerate(states)}
    rhos = []
    for s in states:
        r = base.copy()
        for (i, j), k in zip(FREE, s):
            r[i, j] = base[i, j] * math.exp(H_STEP * k)
        rhos.append(r)
    return states, index, rhos


def _log_weights(orc, rhos):
    lp = np.array([orc.log_posterior(r) for r in rhos])
    jac = np.array([sum(math.log(r[i, j]) for i, j in FREE) for r in rhos])
    return lp + jac


def _kernels(local, states, index, rhos, hastings_sign=1.0):
    """T[m][(n, n')] = probability of the single-site move n -> n' at free site m."""
    Wo = 4
    T = []
    for m, (i, j) in enumerate(FREE):
        Tm = {}
        for n, s in enumerate(states):
            for step in (-1, 1):
                k = s[m] + step
                if abs(k) > K_GRID:
                    continue            # off the grid: rejected, the chain stays
                s2 = list(s)
                s2[m] = k
                n2 = index[tuple(s2)]
                rho, rho2 = rhos[n], rhos[n2]
                ok, dl, dp = local.delta(rho, i * Wo + j, float(rho2[i, j]))
                assert ok
                la = dl + dp + hastings_sign * math.log(rho2[i, j] / rho[i, j])
                Tm[(n, n2)] = 0.5 * min(1.0, math.exp(la))
        T.append(Tm)
    return T


def _balance_error(T, logw):
    w = np.exp(logw - logw.max())
    worst = 0.0
    for Tm in T:
        for (n, n2), t in Tm.items():
            a, b = w[n] * t, w[n2] * Tm[(n2, n)]
            worst = max(worst, abs(a - b) / max(a, b))
    return worst


def _apply(Tm, p):
    q = p.copy()
    for (n, n2), t in Tm.items():
        q[n] -= p[n] * t
        q[n2] += p[n] * t
    return q


@pytest.fixture(scope="module")
def setup():
    prob = _problem(PSF)
    orc = O.Oracle(prob)
    states, index, rhos = _grid()
    assert prob.object_shape() == (4, 4) and prob.S == 4
    logw = _log_weights(orc, rhos)
    return prob, orc, states, index, rhos, logw


def test_single_site_kernels_satisfy_detailed_balance(setup):
    prob, orc, states, index, rhos, logw = setup
    T = _kernels(orc, states, index, rhos)
    err = _balance_error(T, logw)
    print("max relative detailed-balance error %.3g" % err)
    assert err <= TOL


def test_sweep_leaves_the_posterior_invariant(setup):
    prob, orc, states, index, rhos, logw = setup
    T = _kernels(orc, states, index, rhos)
    p = np.exp(logw - logw.max())
    p /= p.sum()
    q = p
    for Tm in T:                      # one sweep: the free sites in class order
        q = _apply(Tm, q)
    err = np.max(np.abs(q - p)) / p.max()
    print("max |p T_sweep - p| / max p = %.3g" % err)
    assert err <= TOL
    # the sweep mixes: it is not the identity on this grid
    assert sum(t for Tm in T for t in Tm.values()) > 100


def test_wrong_hastings_sign_breaks_balance(setup):
    prob, orc, states, index, rhos, logw = setup
    err = _balance_error(_kernels(orc, states, index, rhos, hastings_sign=-1.0), logw)
    assert err > 1e-3


def test_transposed_psf_in_the_window_breaks_balance(setup):
    prob, orc, states, index, rhos, logw = setup
    wrong = O.Oracle(_problem(PSF.T.copy()))
    err = _balance_error(_kernels(wrong, states, index, rhos), logw)
    assert err > 1e-3
