"""Batched sampling: many problems of different sizes, PSFs and chain counts
share launches (one cooperative launch per PSF side).  Each problem's chains
must be bit-identical to the same problem run alone -- its arithmetic does
not depend on what else is in the batch -- and, in double precision, equal
to the oracle's chains."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2411_00991_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2411_00991_gb300 import bdecon  # noqa: E402


def _mix():
    return [
        synth.small_problem(H=20, W=24, L=5, seed=61, refresh_every=4, burn_in=2),
        synth.small_problem(H=17, W=13, L=3, maps=True, seed=62, n_chains=2, refresh_every=4, burn_in=2),
        synth.small_problem(H=16, W=19, L=5, stride=7, seed=63, refresh_every=4, burn_in=2),
        synth.small_problem(H=26, W=22, L=11, sigma=1.8, seed=64, refresh_every=4, burn_in=2),
    ]


def _collect(s, p, n_chains):
    out = []
    for c in range(n_chains):
        rho, t = s.get_state(p, c)
        tr = s.trace(p, c)
        # equal traces compare equal even when infinite: check that they are finite
        assert np.isfinite(tr).all() and np.isfinite(rho).all()
        out.append((rho, tr, s.get_mu(p, c), s.accept_counts(p, c)))
    return out, s.posterior_mean(p)


@pytest.mark.parametrize("precision", [bdecon.BDECON_FP64, bdecon.BDECON_FP32])
def test_batch_equals_alone(precision):
    probs = _mix()
    T = 9
    b = bdecon.Sampler(probs, precision=precision, max_sweeps=T + 4)
    b.sweep(T)
    b.sync()
    plans = [b.get_plan(p) for p in range(len(probs))]
    assert len({pl["warps"] for pl in plans}) >= 2        # launch groups with different team sizes
    mixed = [_collect(b, p, pr.n_chains) for p, pr in enumerate(probs)]
    b.close()
    for p, pr in enumerate(probs):
        a = bdecon.Sampler(pr, precision=precision, max_sweeps=T + 4)
        a.sweep(T)
        alone = _collect(a, 0, pr.n_chains)
        a.close()
        for c in range(pr.n_chains):
            for x, y in zip(mixed[p][0][c], alone[0][c]):
                np.testing.assert_array_equal(x, y)
        np.testing.assert_array_equal(mixed[p][1], alone[1])


def test_batch_fp64_matches_oracle():
    probs = _mix()
    T = 7
    b = bdecon.Sampler(probs, precision=bdecon.BDECON_FP64, max_sweeps=T + 4, flags=bdecon.FLAG_ACCEPT_LOG)
    b.sweep(T)
    b.sync()
    for p, pr in enumerate(probs):
        for c in range(pr.n_chains):
            ref = O.Oracle(pr, chain=c).run(T, want_acc_log=True)
            np.testing.assert_array_equal(b.accept_log(p, c), ref["acc_log"])
            rho, _ = b.get_state(p, c)
            np.testing.assert_allclose(rho, ref["rho"], rtol=1e-12)
            np.testing.assert_allclose(b.trace(p, c), ref["trace"], rtol=1e-12)
    b.close()


@pytest.mark.parametrize("precision", [bdecon.BDECON_FP64, bdecon.BDECON_FP32])
def test_one_launch_and_autotuned_plans_are_bit_identical(precision):
    # every problem in one launch (block = the largest team), and the plan the
    # autotuner picks after timing its trials (the trials' sweeps are undone)
    probs = _mix()
    T = 9
    ref = bdecon.Sampler(probs, precision=precision, max_sweeps=T + 8)
    ref.sweep(T)
    want = [_collect(ref, p, pr.n_chains) for p, pr in enumerate(probs)]
    ref.close()

    one = bdecon.Sampler(probs, precision=precision, max_sweeps=T + 8)
    one.set_grouping(True)
    plans = [one.get_plan(p) for p in range(len(probs))]
    assert len({pl["blocks"] for pl in plans}) == 1 and len({pl["warps"] for pl in plans}) == 1
    one.sweep(4)
    one.set_grouping(False)                 # regrouping between sweeps changes nothing either
    one.sweep(T - 4)
    got_one = [_collect(one, p, pr.n_chains) for p, pr in enumerate(probs)]
    one.close()

    tuned = bdecon.Sampler(probs, precision=precision, max_sweeps=T + 8)
    tuned.sweep(2)
    info = tuned.autotune(trial_sweeps=3)
    assert info["ms_per_sweep"] > 0
    rho, t = tuned.get_state(0, 0)
    assert t == 2
    assert tuned.trace(0, 0).size == 2
    tuned.sweep(T - 2)
    got_tuned = [_collect(tuned, p, pr.n_chains) for p, pr in enumerate(probs)]
    tuned.close()

    for got in (got_one, got_tuned):
        for p, pr in enumerate(probs):
            for c in range(pr.n_chains):
                for x, y in zip(got[p][0][c], want[p][0][c]):
                    np.testing.assert_array_equal(x, y)
            np.testing.assert_array_equal(got[p][1], want[p][1])


def test_tuning_cache_reuses_the_tuned_plan_and_changes_no_result():
    # a handle created after an autotune of the same shapes starts with the
    # tuned plan; with the cache off it starts with the automatic one; the
    # chains are the same either way
    probs = _mix()
    T = 6
    bdecon.set_tuning_cache(True)
    auto = bdecon.Sampler(probs, precision=bdecon.BDECON_FP32, max_sweeps=T + 8)
    auto_plans = [auto.get_plan(p) for p in range(len(probs))]
    auto.sweep(T)
    want = [_collect(auto, p, pr.n_chains) for p, pr in enumerate(probs)]
    auto.close()

    tuned = bdecon.Sampler(probs, precision=bdecon.BDECON_FP32, max_sweeps=T + 8)
    tuned.sweep(1)
    tuned.set_grouping(True)                 # a shape the automatic plan never takes,
    tuned.autotune(trial_sweeps=1)           # unless the autotuner keeps it
    tuned_plans = [tuned.get_plan(p) for p in range(len(probs))]
    tuned.close()

    again = bdecon.Sampler(probs, precision=bdecon.BDECON_FP32, max_sweeps=T + 8)
    assert [again.get_plan(p) for p in range(len(probs))] == tuned_plans
    again.sweep(T)
    got = [_collect(again, p, pr.n_chains) for p, pr in enumerate(probs)]
    again.close()
    other = bdecon.Sampler(probs[:3], precision=bdecon.BDECON_FP32, max_sweeps=T + 8)   # another key
    assert [other.get_plan(p) for p in range(3)] == auto_plans[:3]
    other.close()
    bdecon.set_tuning_cache(False)
    off = bdecon.Sampler(probs, precision=bdecon.BDECON_FP32, max_sweeps=T + 8)
    assert [off.get_plan(p) for p in range(len(probs))] == auto_plans
    off.close()
    bdecon.set_tuning_cache(True)
    for p, pr in enumerate(probs):
        for c in range(pr.n_chains):
            for x, y in zip(got[p][0][c], want[p][0][c]):
                np.testing.assert_array_equal(x, y)
        np.testing.assert_array_equal(got[p][1], want[p][1])


def test_lean_form_is_bit_identical():
    # the lean kernel form holds fewer window cells in flight per thread and
    # has a smaller register budget; the cells, their order and the reductions
    # are those of the default form, so chains are bit-identical -- with the
    # form forced on, off, and switched between sweeps, on multi-patch tiles
    # (one- and two-team blocks, several rounds per class step)
    probs = _mix()
    T = 9

    def run(modes):
        s = bdecon.Sampler(probs, precision=bdecon.BDECON_FP32, max_sweeps=T + 4)
        for p in range(len(probs)):
            s.set_plan(2, 3, 2 if p % 2 else 0, p=p)
        done = 0
        for mode, n in modes:
            s.set_lean(mode)
            lean = [s.lean(p) for p in range(len(probs))]
            assert all(lean) if mode == 1 else not any(lean)
            s.sweep(n)
            done += n
        assert done == T
        out = [_collect(s, p, pr.n_chains) for p, pr in enumerate(probs)]
        s.close()
        return out

    want = run([(0, T)])
    for got in (run([(1, T)]), run([(1, 4), (0, T - 4)])):
        for p, pr in enumerate(probs):
            for c in range(pr.n_chains):
                for x, y in zip(got[p][0][c], want[p][0][c]):
                    np.testing.assert_array_equal(x, y)
            np.testing.assert_array_equal(got[p][1], want[p][1])
    d = bdecon.Sampler(probs, precision=bdecon.BDECON_FP64, max_sweeps=4)
    d.set_plan(2, 3, 0, p=0)
    d.set_lean(1)
    assert not any(d.lean(p) for p in range(len(probs)))   # a float form only
    d.close()


def test_warps_only_plan_override():
    probs = _mix()
    s = bdecon.Sampler(probs, precision=bdecon.BDECON_FP32, max_sweeps=8)
    auto = s.get_plan(3)
    s.set_plan(0, 0, 8, p=3)                 # automatic tiles, 8 warps for the L = 11 group
    pl = s.get_plan(3)
    assert pl["warps"] == 8 and auto["warps"] < 8
    with pytest.raises(bdecon.BdeconError):
        s.set_plan(0, 0, 9, p=3)
    assert s.get_plan(3) == pl                # a refused plan keeps the previous one
    s.set_plan(0, 0, 0, p=3)
    assert s.get_plan(3) == auto
    s.close()


@pytest.mark.parametrize("precision", [bdecon.BDECON_FP64, bdecon.BDECON_FP32])
def test_graph_mode_is_bit_identical(precision):
    # sweep calls of 3 and 5 sweeps across refreshes every 4 sweeps: the
    # segment sequences repeat, so later calls replay captured graphs
    probs = _mix()
    calls = [3, 5, 3, 5, 2]
    ref = bdecon.Sampler(probs, precision=precision, max_sweeps=32)
    for n in calls:
        ref.sweep(n)
    want = [_collect(ref, p, pr.n_chains) for p, pr in enumerate(probs)]
    want_launches = ref.launch_count()
    ref.close()
    g = bdecon.Sampler(probs, precision=precision, max_sweeps=32)
    g.set_graph(True)
    for n in calls:
        g.sweep(n)
    got = [_collect(g, p, pr.n_chains) for p, pr in enumerate(probs)]
    assert g.launch_count() == want_launches
    g.close()
    for p, pr in enumerate(probs):
        for c in range(pr.n_chains):
            for x, y in zip(got[p][0][c], want[p][0][c]):
                np.testing.assert_array_equal(x, y)
        np.testing.assert_array_equal(got[p][1], want[p][1])


def test_staged_windows_are_bit_identical():
    # window staging (TMA copies of each update's expected-image and cumulant
    # window, and of a streamed plan's patch spectrum, into shared memory)
    # changes where the sweep reads its data, not what it computes: default,
    # user-tiled and one-launch plans give the unstaged chains bit for bit
    probs = _mix()
    T = 9
    ref = bdecon.Sampler(probs, precision=bdecon.BDECON_FP32, max_sweeps=T + 8)
    ref.sweep(T)
    want = [_collect(ref, p, pr.n_chains) for p, pr in enumerate(probs)]
    ref.close()
    runs = []
    for variant in ("default", "tiles", "one_launch"):
        s = bdecon.Sampler(probs, precision=bdecon.BDECON_FP32, max_sweeps=T + 8)
        s.set_staging(True)
        if variant == "tiles":
            s.set_plan(2, 3, 0, p=3)
        if variant == "one_launch":
            s.set_grouping(True)
        staged = [s.staged(p) for p in range(len(probs))]
        # one-patch one-team plans keep their own kernel form; tiled plans stage
        if variant == "tiles":
            assert staged[3] == 1
        if variant == "one_launch":
            assert all(x == 1 for x in staged)
        s.sweep(4)
        s.set_staging(False)                # switching between sweeps changes nothing either
        assert all(x != 1 for x in (s.staged(p) for p in range(len(probs))))
        s.sweep(2)
        s.set_staging(True)
        s.sweep(T - 6)
        runs.append([_collect(s, p, pr.n_chains) for p, pr in enumerate(probs)])
        s.close()
    for got in runs:
        for p, pr in enumerate(probs):
            for c in range(pr.n_chains):
                for x, y in zip(got[p][0][c], want[p][0][c]):
                    np.testing.assert_array_equal(x, y)
            np.testing.assert_array_equal(got[p][1], want[p][1])


def test_staged_lowsnr_crop_matches_oracle_trace():
    # the low-SNR recipe (L = 31, sCMOS maps, 4 chains) staged: the float trace
    # stays the oracle's Eq. 9 of each chain's state across a refresh
    from oracle import oracle as O
    prob = synth.lowsnr_2048(crop=128)
    prob.refresh_every = 10
    orc = O.Oracle(prob)
    s = bdecon.Sampler(prob, precision=bdecon.BDECON_FP32, max_sweeps=32)
    s.set_staging(True)
    s.set_plan(2, 2, 0)                     # tiles of 2 x 2 patches: a staged multi-round plan
    assert s.staged(0) == 1
    s.sweep(12)
    s.sync()
    for c in range(prob.n_chains):
        rho, t = s.get_state(0, c)
        tr = s.trace(0, c)
        assert t == 12 and np.isfinite(tr).all()
        ref = orc.log_posterior_fft(rho)
        assert abs(tr[-1] - ref) <= 1e-5 * abs(ref), (c, tr[-1], ref)
    s.close()
