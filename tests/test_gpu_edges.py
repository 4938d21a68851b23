"""Edge cases of the GPU sampler against the oracle: the largest PSF side and
stride the library accepts (L = 63, S = 64, ragged 4-pixel edge patches), a
one-pixel frame with a delta PSF (a single patch of one pixel: a sweep is one
update, so no proposal can be drawn ahead), and a one-row frame."""
import math

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


def _max_problem():
    p = synth.small_problem(H=6, W=6, L=63, sigma=6.0, stride=64, seed=91, maps=True, refresh_every=2)
    assert p.object_shape() == (68, 68)
    return p


def test_largest_psf_and_stride_first_class_exact():
    # after one sweep the first-class pixels (one per patch: four patches of
    # 64 x 64, 64 x 4, 4 x 64, 4 x 4) hold the result of their single update
    # from the initial object, which the oracle evaluates one by one
    prob = _max_problem()
    s = bdecon.Sampler(prob, precision=bdecon.BDECON_FP64, max_sweeps=4, flags=bdecon.FLAG_ACCEPT_LOG)
    orc = O.Oracle(prob)
    rho0 = orc.init()
    np.testing.assert_allclose(s.get_state()[0], rho0, rtol=RTOL)
    s.sweep(1)
    rho1, _ = s.get_state()
    acc = s.accept_log()[0]
    Wo = prob.object_shape()[1]
    for i, j in ((0, 0), (0, 64), (64, 0), (64, 64)):
        a_o, rn, dl, dp = orc.single_update(rho0, i * Wo + j, 1)
        assert bool(acc[i, j]) == a_o
        np.testing.assert_allclose(rho1[i, j], rn if a_o else rho0[i, j], rtol=RTOL)
    s.close()


@pytest.mark.parametrize("precision,tol", [(bdecon.BDECON_FP64, 1e-12), (bdecon.BDECON_FP32, 1e-5)])
def test_largest_psf_trace_matches_oracle(precision, tol):
    prob = _max_problem()
    orc = O.Oracle(prob)
    s = bdecon.Sampler(prob, precision=precision, max_sweeps=8)
    for t in (1, 2, 3):
        s.sweep(1)
        s.sync()
        rho, tt = s.get_state()
        assert tt == t
        tr = s.trace()
        ref = orc.log_posterior(rho)
        assert abs(tr[-1] - ref) <= tol * abs(ref), (t, tr[-1], ref)
    s.close()


@pytest.mark.parametrize("kw,T", [
    (dict(H=1, W=1, L=1), 40),                 # one pixel, delta PSF: one update per sweep
    (dict(H=1, W=40, L=3), 12),                # one camera row
])
def test_degenerate_frames_exact_chain(kw, T):
    prob = synth.small_problem(seed=92, refresh_every=5, burn_in=2, **kw)
    s = bdecon.Sampler(prob, precision=bdecon.BDECON_FP64, max_sweeps=T + 4, flags=bdecon.FLAG_ACCEPT_LOG)
    s.sweep(T)
    s.sync()
    ref = O.Oracle(prob).run(T, want_acc_log=True)
    np.testing.assert_array_equal(s.accept_log(), ref["acc_log"])
    rho, t = s.get_state()
    assert t == T
    np.testing.assert_allclose(rho, ref["rho"], rtol=RTOL)
    np.testing.assert_allclose(s.trace(), ref["trace"], rtol=RTOL)
    np.testing.assert_allclose(s.posterior_mean(), ref["mean"], rtol=RTOL)
    assert math.isfinite(s.log_posterior())
    s.close()


def test_one_patch_plan_without_room_for_the_one_team_form():
    # the 512x512 frame with a 4-warp update team: one patch per block fits
    # the general kernel forms (lean: 8 blocks of 128 threads per SM) but not
    # the one-team form (80 registers: 6 per SM, fewer than 1024 blocks), so
    # the plan keeps one patch per block in the general form; every block is
    # co-resident, and the chain equals that of a plan of 2 x 2-patch tiles
    p = synth.widefield_512()
    p.truth = None
    p.team_warps = 4
    T = 3
    out = []
    for plan in (None, (2, 2, 0)):
        s = bdecon.Sampler(p, precision=bdecon.BDECON_FP32, max_sweeps=T + 4)
        if plan is not None:
            s.set_plan(*plan)
        pl = s.get_plan(0)
        if plan is None:
            assert (pl["tile_i"], pl["tile_j"], pl["warps"]) == (1, 1, 4)
        s.sweep(T)
        s.sync()
        rho, t = s.get_state(0, 0)
        tr = s.trace(0, 0)
        assert t == T and np.isfinite(tr).all()
        out.append((rho, tr, s.get_mu(0, 0)))
        s.close()
    for x, y in zip(out[0], out[1]):
        np.testing.assert_array_equal(x, y)
