"""GPU parity of libbdecon against the CPU oracle, through the C ABI.

Double precision: the GPU chain must reproduce the oracle's chain exactly
(identical accept decisions; object, expected image, trace and posterior
mean within 1e-12 relative).  Single precision: the per-update arithmetic
(dL, dP) is compared with the oracle's double values; the double evaluator
of Eq. 9 is compared at 1e-12.  Plan invariance: every launch plan gives
bit-identical results.
"""
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


def _run_gpu(prob, T, precision=bdecon.BDECON_FP64, flags=bdecon.FLAG_ACCEPT_LOG, plan=None):
    s = bdecon.Sampler(prob, precision=precision, max_sweeps=max(T, 1) + 8, flags=flags)
    if plan is not None:
        s.set_plan(*plan)
    s.sweep(T)
    s.sync()
    out = {}
    for c in range(prob.n_chains):
        rho, t = s.get_state(0, c)
        assert t == T
        d = dict(rho=rho, mu=s.get_mu(0, c), trace=s.trace(0, c), acc=s.accept_counts(0, c))
        if flags & bdecon.FLAG_ACCEPT_LOG:
            d["acc_log"] = s.accept_log(0, c)
        out[c] = d
    out["mean"] = s.posterior_mean(0) if T > prob.burn_in else None
    out["plan"] = s.get_plan(0)
    s.close()
    return out


def _compare_exact(prob, T, plan=None):
    g = _run_gpu(prob, T, plan=plan)
    if plan is not None:
        assert (g["plan"]["tile_i"], g["plan"]["tile_j"], g["plan"]["warps"]) == tuple(plan)
    sums = []
    for c in range(prob.n_chains):
        ref = O.Oracle(prob, chain=c).run(T, want_acc_log=True)
        gc = g[c]
        mism = np.argwhere(gc["acc_log"] != ref["acc_log"])
        assert mism.size == 0, f"chain {c}: {len(mism)} accept decisions differ, first {mism[:3]}"
        np.testing.assert_array_equal(gc["acc"], ref["n_acc"])
        np.testing.assert_allclose(gc["rho"], ref["rho"], rtol=RTOL)
        np.testing.assert_allclose(gc["mu"], ref["mu"], rtol=RTOL)
        np.testing.assert_allclose(gc["trace"], ref["trace"], rtol=RTOL)
        sums.append(ref["sum"])
        n_sum = ref["n_sum"]
    if g["mean"] is not None:
        np.testing.assert_allclose(g["mean"], sum(sums) / (n_sum * prob.n_chains), rtol=RTOL)


@pytest.mark.parametrize("kw", [
    dict(H=20, W=24, L=5, seed=7),                                   # ragged patch tail
    dict(H=17, W=13, L=3, seed=8, maps=True),                        # sCMOS maps
    dict(H=16, W=19, L=5, stride=7, seed=9, maps=True),              # stride > L, partial patches
    dict(H=12, W=12, L=7, seed=10, n_chains=2, burn_in=3),           # two chains, burn-in
    dict(H=9, W=30, L=1, seed=11),                                   # delta PSF
])
def test_fp64_exact_chain_small(kw):
    prob = synth.small_problem(refresh_every=5, **kw)
    _compare_exact(prob, 12)


def test_fp64_exact_chain_widefield64_50_sweeps():
    prob = synth.widefield_64()
    prob.burn_in = 25
    _compare_exact(prob, 50)


@pytest.mark.parametrize("precision", [bdecon.BDECON_FP64, bdecon.BDECON_FP32])
def test_plan_invariance(precision):
    prob = synth.small_problem(H=30, W=27, L=5, seed=12, maps=True, n_chains=2, refresh_every=4)
    runs = [_run_gpu(prob, 9, precision=precision, plan=pl)
            for pl in (None, (2, 3, 1), (3, 3, 4), (1, 2, 2), (4, 5, 8), (3, 4, 2), (2, 2, 2))]
    base = runs[0]
    for r in runs[1:]:
        for c in range(prob.n_chains):
            np.testing.assert_array_equal(r[c]["acc_log"], base[c]["acc_log"])
            np.testing.assert_array_equal(r[c]["rho"], base[c]["rho"])
            np.testing.assert_array_equal(r[c]["mu"], base[c]["mu"])
            np.testing.assert_array_equal(r[c]["trace"], base[c]["trace"])
        np.testing.assert_array_equal(r["mean"], base["mean"])


@pytest.mark.parametrize("precision,tol", [(bdecon.BDECON_FP64, 1e-9), (bdecon.BDECON_FP32, None)])
def test_delta_matches_oracle(precision, tol):
    prob = synth.small_problem(H=22, W=19, L=7, seed=14, maps=True)
    rho = synth.random_state(prob, 5, lo=0.5, hi=25.0)
    s = bdecon.Sampler(prob, precision=precision, max_sweeps=8)
    s.set_state(rho, 0)
    if precision == bdecon.BDECON_FP32:
        rho = rho.astype(np.float32).astype(np.float64)   # the state the float sampler holds
    orc = O.Oracle(prob)
    Ho, Wo = prob.object_shape()
    rng = np.random.default_rng(2)
    ms = [0, Wo - 1, Ho * Wo - 1, (Ho // 2) * Wo + Wo // 2] + list(rng.integers(0, Ho * Wo, 24))
    errs = []
    for m in ms:
        new = float(rho.flat[m] * math.exp(rng.normal(0, 0.3)))
        if precision == bdecon.BDECON_FP32:
            new = float(np.float32(new))
        ok_g, dl_g, dp_g = s.delta(m, new)
        ok_o, dl_o, dp_o = orc.delta(rho, m, new)
        assert ok_g == ok_o
        if tol is not None:
            assert dl_g == pytest.approx(dl_o, abs=tol, rel=1e-9)
            assert dp_g == pytest.approx(dp_o, abs=tol, rel=1e-9)
        else:
            errs.append((abs(dl_g - dl_o), abs(dp_g - dp_o), abs(dl_o) + abs(dp_o)))
    if errs:
        e = np.array(errs)
        # float arithmetic: errors a few ulps of the magnitudes involved
        assert (e[:, 0] <= 2e-4 + 1e-5 * e[:, 2]).all(), e[:, 0].max()
        assert (e[:, 1] <= 2e-4 + 1e-5 * e[:, 2]).all(), e[:, 1].max()
    s.close()


@pytest.mark.parametrize("precision", [bdecon.BDECON_FP64, bdecon.BDECON_FP32])
def test_log_posterior_evaluator(precision):
    prob = synth.small_problem(H=25, W=23, L=5, seed=15, maps=True, stride=6)
    rho = synth.random_state(prob, 6)
    s = bdecon.Sampler(prob, precision=precision, max_sweeps=8)
    s.set_state(rho, 0)
    if precision == bdecon.BDECON_FP32:
        rho = rho.astype(np.float32).astype(np.float64)
    ref = O.Oracle(prob).log_posterior(rho)
    assert s.log_posterior() == pytest.approx(ref, rel=RTOL)
    assert s.trace().size == 0
    s.close()


def test_resume_from_checkpoint_is_exact():
    prob = synth.small_problem(H=14, W=16, L=5, seed=16, refresh_every=3)
    a = bdecon.Sampler(prob, precision=bdecon.BDECON_FP64, max_sweeps=16)
    a.sweep(6)
    rho_a, _ = a.get_state()
    tr_a = a.trace()
    b = bdecon.Sampler(prob, precision=bdecon.BDECON_FP64, max_sweeps=16)
    b.sweep(3)
    rho3, t3 = b.get_state()
    c = bdecon.Sampler(prob, precision=bdecon.BDECON_FP64, max_sweeps=16)
    c.set_state(rho3, t3)
    c.sweep(3)
    rho_c, t = c.get_state()
    assert t == 6
    np.testing.assert_array_equal(rho_c, rho_a)
    np.testing.assert_array_equal(c.trace()[3:6], tr_a[3:6])
    for x in (a, b, c):
        x.close()


@pytest.mark.parametrize("frame,chains,precision", [
    ("widefield_512", (0,), bdecon.BDECON_FP64),
    ("widefield_512", (0,), bdecon.BDECON_FP32),
    ("lowsnr_2048", (0, 3), bdecon.BDECON_FP64),
])
def test_full_frame_first_class_sampled(frame, chains, precision):
    # full-size frames in the launch plan a user gets: the 512x512 widefield
    # frame (L = 17, 1 chain) and the 2048x2048 low-SNR frame (L = 31, sCMOS
    # maps, 4 chains).  After one sweep the first-class pixels hold exactly
    # the result of their single update from the initial object, which the
    # oracle evaluates one by one
    prob = getattr(synth, frame)()
    s = bdecon.Sampler(prob, precision=precision, max_sweeps=4, flags=bdecon.FLAG_ACCEPT_LOG)
    refs = {}
    for c in chains:
        orc = O.Oracle(prob, chain=c)
        refs[c] = (orc, orc.init())
        if precision == bdecon.BDECON_FP64:
            np.testing.assert_allclose(s.get_state(0, c)[0], refs[c][1], rtol=RTOL)
    s.sweep(1)
    S = prob.S
    Ho, Wo = prob.object_shape()
    for c in chains:
        orc, ref0 = refs[c]
        rho1, _ = s.get_state(0, c)
        acc = s.accept_log(0, c)[0]
        rng = np.random.default_rng(3 + c)
        picks = [(0, 0), (Ho - 1 - (Ho - 1) % S, Wo - 1 - (Wo - 1) % S)] + \
            [(int(a) * S, int(b) * S) for a, b in zip(rng.integers(0, (Ho - 1) // S + 1, 14),
                                                       rng.integers(0, (Wo - 1) // S + 1, 14))]
        near = 0
        for i, j in picks:
            m = i * Wo + j
            a_o, rn, dl, dp = orc.single_update(ref0, m, 1)
            if precision == bdecon.BDECON_FP64:
                assert bool(acc[i, j]) == a_o
                np.testing.assert_allclose(rho1[i, j], rn if a_o else ref0[i, j], rtol=1e-12)
            else:
                z, u = O.draw(prob.seed, m, 1, c)
                margin = abs(math.log(u) - (dl + dp + prob.step * z))
                if margin > 1e-3:
                    assert bool(acc[i, j]) == a_o
                    np.testing.assert_allclose(rho1[i, j], rn if a_o else ref0[i, j], rtol=2e-6)
                else:
                    near += 1
        assert near <= 2
        assert np.isfinite(s.trace(0, c)).all()
    s.close()


def test_accumulated_mean_and_variance():
    prob = synth.small_problem(H=12, W=14, L=3, seed=17, burn_in=2, n_chains=2)
    s = bdecon.Sampler(prob, precision=bdecon.BDECON_FP64, max_sweeps=16, flags=bdecon.FLAG_SECOND_MOMENT)
    s.sweep(7)
    mean, var = s.posterior_mean(), s.posterior_var()
    crop = s.posterior_mean(crop=True)
    s.close()
    samples = []
    for c in range(2):
        r = O.Oracle(prob, chain=c).run(7, want_samples=True)
        samples.append(r["samples"][2:])
    x = np.concatenate(samples)
    np.testing.assert_allclose(mean, x.mean(axis=0), rtol=1e-12)
    np.testing.assert_allclose(var, x.var(axis=0), rtol=1e-8, atol=1e-12)
    R = prob.L // 2
    np.testing.assert_array_equal(crop, mean[R:-R, R:-R])


def test_fp32_cumulant_cache_tracks_exact_after_sweeps():
    # the float sweep scores most window pixels from cached photon-posterior
    # cumulants that are tilted after each accepted update, and keeps mu and
    # the patch spectra by float increments; after many sweeps without a
    # refresh its dL and dP are compared with the double kernel's at the same
    # (float) state.  Errors of 1e-3 in a log acceptance ratio move the
    # acceptance probability by 0.1%: far below the Monte Carlo error.
    prob = synth.small_problem(H=30, W=28, L=7, maps=True, seed=41, refresh_every=0)
    s = bdecon.Sampler(prob, precision=bdecon.BDECON_FP32, max_sweeps=64)
    s.sweep(40)
    rho, _ = s.get_state()
    assert s.accept_counts().sum() > 0
    e = bdecon.Sampler(prob, precision=bdecon.BDECON_FP64, max_sweeps=4)
    e.set_state(rho, 0)
    Ho, Wo = prob.object_shape()
    rng = np.random.default_rng(9)
    errs = []
    for m in list(rng.integers(0, Ho * Wo, 24)) + [(Ho // 2) * Wo + Wo // 2]:
        new = float(np.float32(rho.flat[m] * math.exp(rng.normal(0, 0.2))))
        ok, dl, dp = s.delta(int(m), new)
        ok64, dl64, dp64 = e.delta(int(m), new)
        assert ok and ok64
        errs.append((abs(dl - dl64), abs(dp - dp64), abs(dl64), abs(dp64)))
    err = np.array(errs)
    print("max |dL err| %.3g  max |dP err| %.3g" % (err[:, 0].max(), err[:, 1].max()))
    assert (err[:, 0] <= 1e-3 + 1e-5 * err[:, 2]).all()
    assert (err[:, 1] <= 1e-3 + 1e-4 * err[:, 3]).all()
    s.close()
    e.close()


def test_wait_timeout_is_reported_and_context_survives():
    # a block that never publishes its progress (a flag nothing sets): its
    # neighbours' bounded waits run out, the device error flag is raised, every
    # block returns, and the host reads BDECON_ERR_TIMEOUT; no GPU fault
    prob = synth.small_problem(H=20, W=20, L=5, seed=51)
    s = bdecon.Sampler(prob, precision=bdecon.BDECON_FP32, max_sweeps=16)
    s.set_fault(3, 200_000_000)
    s.sweep(2)
    with pytest.raises(bdecon.BdeconError) as ei:
        s.sync()
    assert ei.value.status == 4
    with pytest.raises(bdecon.BdeconError) as ei:
        s.sweep(1)
    assert ei.value.status == 5
    s.close()
    t = bdecon.Sampler(prob, precision=bdecon.BDECON_FP32, max_sweeps=16)
    t.sweep(3)
    t.sync()
    assert np.isfinite(t.trace()).all()
    t.close()


def test_non_finite_expected_image_is_reported():
    # an object that overflows float gives an infinite expected image: the
    # refresh raises the numeric flag, read on the host as BDECON_ERR_NUMERIC
    prob = synth.small_problem(H=12, W=12, L=3, seed=52)
    s = bdecon.Sampler(prob, precision=bdecon.BDECON_FP32, max_sweeps=8)
    rho = np.full(prob.object_shape(), 1e300)
    with pytest.raises(bdecon.BdeconError) as ei:
        s.set_state(rho, 0)
    assert ei.value.status == 6
    s.close()


@pytest.mark.parametrize("team_warps", [1, 3])
def test_fp64_exact_chain_with_explicit_team(team_warps):
    # the team size fixes only the order of the per-update reductions; every
    # team gives the oracle's chain in double precision
    prob = synth.small_problem(H=22, W=21, L=11, sigma=1.6, seed=71, maps=True, refresh_every=4, burn_in=2)
    prob.team_warps = team_warps
    _compare_exact(prob, 8)


@pytest.mark.parametrize("plan", [(3, 3, 2), (2, 4, 2)])
def test_fp64_exact_chain_two_teams_several_rounds(plan):
    # blocks of two one-warp update teams over tiles of several patches: after
    # a class step's first round each team synchronises on its own barrier and
    # the block meets at the step's end; the chain is still the oracle's
    prob = synth.small_problem(H=30, W=27, L=5, seed=13, maps=True, n_chains=2, refresh_every=4, burn_in=2)
    _compare_exact(prob, 10, plan=plan)


def test_fp64_exact_chain_with_airy_psf():
    # the paper's widefield PSF shape (pixel-integrated Airy pattern, NA 1.4,
    # 520 nm, 65 nm pixels) on a 13 x 13 support, sCMOS maps
    prob = synth.small_problem(H=30, W=26, L=13, maps=True, seed=19, refresh_every=6, burn_in=2)
    prob.psf = synth.airy_psf(1.4, 520.0, 65.0, 13)
    _compare_exact(prob, 15)


def test_lowsnr2048_float_first_class_sampled_and_trace():
    # the float form on the 2048x2048 low-SNR frame (L = 31, 4 chains, the
    # streamed multi-round plan): sampled first-class updates match the
    # oracle and every chain's trace is finite
    test_full_frame_first_class_sampled("lowsnr_2048", (0, 3), bdecon.BDECON_FP32)
