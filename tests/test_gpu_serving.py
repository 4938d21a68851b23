"""The serving loop (bdecon_server_*): continuous batching of deconvolution
jobs on the GPU.

Jobs of different frame sizes, PSFs (hence update teams), chain counts,
sweep counts and refresh schedules arrive while others run; the server
admits them as slots and device memory free up and sweeps every running job
in one shared launch per segment.  Each job's chains keep their own sweep
counter and random stream, so its posterior mean must be bit-identical to
the same job run alone through a Sampler handle -- in both precisions --
whatever else shared the launches.
"""
import time

import numpy as np
import pytest

from paper_2411_00991_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2411_00991_gb300 import bdecon  # noqa: E402


def _jobs():
    specs = [  # (H, W, L, chains, sweeps, refresh_every, burn_in)
        (48, 52, 5, 1, 37, 10, 5),
        (33, 40, 11, 2, 21, 0, 0),
        (64, 64, 9, 1, 50, 16, 10),
        (29, 31, 3, 3, 12, 5, 2),
        (40, 72, 15, 1, 30, 7, 3),
        (57, 45, 7, 2, 44, 0, 20),
    ]
    out = []
    for k, (H, W, L, nc, sw, rf, bi) in enumerate(specs):
        p = synth.small_problem(H=H, W=W, L=L, maps=(k % 2 == 0), seed=100 + k)
        p.n_chains, p.refresh_every, p.burn_in = nc, rf, bi
        out.append((p, sw))
    return out


def _alone(prob, sweeps, precision):
    s = bdecon.Sampler(prob, precision=precision, max_sweeps=sweeps)
    s.sweep(sweeps)
    m = s.posterior_mean()
    s.close()
    return m


@pytest.mark.parametrize("precision", [bdecon.BDECON_FP64, bdecon.BDECON_FP32])
def test_each_job_identical_alone_and_in_the_mix(precision):
    jobs = _jobs()
    ref = [_alone(p, sw, precision) for p, sw in jobs]
    srv = bdecon.Server(mem_budget=8 << 30, max_jobs=4, segment_sweeps=8, precision=precision)
    try:
        ids = []
        for k, (p, sw) in enumerate(jobs):
            ids.append(srv.submit(p, sw))
            if k == 1:
                time.sleep(0.05)     # later jobs arrive while the first ones run
        res = [srv.result(i, timeout=300) for i in ids]
        st = srv.stats()
    finally:
        srv.close()
    for k, ((m, t), r) in enumerate(zip(res, ref)):
        assert np.array_equal(m, r), f"job {k}: max diff {np.max(np.abs(m - r))}"
        assert t[0] <= t[1] <= t[2]
    assert st["done"] == len(jobs)
    assert st["mem_used"] == 0
    assert st["segments"] >= 7        # the longest job alone needs 50 / 8 segments


def test_admission_by_device_memory():
    jobs = _jobs()
    need = [bdecon.Sampler.workspace_size(p, precision=bdecon.BDECON_FP32, max_sweeps=sw) for p, sw in jobs]
    budget = max(need) + min(need)      # never more than two of these jobs at once
    srv = bdecon.Server(mem_budget=budget, max_jobs=64, segment_sweeps=4, precision=bdecon.BDECON_FP32)
    try:
        ids = [srv.submit(p, sw) for p, sw in jobs]
        peak_running, peak_mem = 0, 0
        while True:
            st = srv.stats()
            peak_running = max(peak_running, st["running"])
            peak_mem = max(peak_mem, st["mem_used"])
            if st["done"] == len(jobs):
                break
            time.sleep(0.002)
        times = [srv.poll(i)[1] for i in ids]
    finally:
        srv.close()
    assert peak_mem <= budget
    assert 1 <= peak_running <= 2
    # first come, first served: admission order follows submission order
    starts = [t[1] for t in times]
    assert starts == sorted(starts)


def test_oversized_job_fails_and_bad_precision_is_refused():
    p, sw = _jobs()[0]
    srv = bdecon.Server(mem_budget=1 << 16, max_jobs=2, segment_sweeps=4, precision=bdecon.BDECON_FP32)
    try:
        jid = srv.submit(p, sw)
        state, _ = srv.poll(jid)
        assert state == bdecon.JOB_FAILED
        with pytest.raises(bdecon.BdeconError, match="device memory"):
            srv.result(jid, timeout=5)
    finally:
        srv.close()
    srv = bdecon.Server(mem_budget=1 << 30, max_jobs=2, segment_sweeps=4, precision=bdecon.BDECON_FP64)
    try:
        keep = []
        prob = bdecon._problem(p, bdecon.BDECON_FP32, sw, 0, keep)
        jid = bdecon.C.c_int64()
        st = srv.L.bdecon_server_submit(srv.s, bdecon.C.byref(prob), sw, bdecon.C.byref(jid))
        assert st == 1
        assert "precision" in srv.L.bdecon_last_error(None).decode()
    finally:
        srv.close()


def test_stop_with_queued_jobs_frees_everything():
    jobs = _jobs()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    srv = bdecon.Server(mem_budget=8 << 30, max_jobs=1, segment_sweeps=2, precision=bdecon.BDECON_FP32)
    ids = [srv.submit(p, sw) for p, sw in jobs]
    time.sleep(0.02)
    srv.close()                      # returns: the running segment completes, every job ends failed or done
    free1, _ = torch.cuda.mem_get_info()
    assert free1 >= free0 - (64 << 20)


def test_light_job_takes_more_sweeps_per_segment_and_finishes_first():
    # a 320x320 job with 4 chains has more patches than the GPU holds blocks,
    # so its blocks take several patches in turn; a small job in the same
    # launch group takes proportionally more sweeps per segment and is done
    # long before the large one, with a result still identical to running alone
    big = synth.small_problem(H=320, W=320, L=9, seed=201)
    big.n_chains = 4
    small = synth.small_problem(H=24, W=24, L=9, seed=202)
    srv = bdecon.Server(mem_budget=8 << 30, max_jobs=4, segment_sweeps=4, precision=bdecon.BDECON_FP32)
    try:
        ib = srv.submit(big, 30)
        i_s = srv.submit(small, 30)
        ms, ts = srv.result(i_s, timeout=300)
        mb, tb = srv.result(ib, timeout=300)
    finally:
        srv.close()
    assert ts[2] < tb[2]
    np.testing.assert_array_equal(ms, _alone(small, 30, bdecon.BDECON_FP32))
    np.testing.assert_array_equal(mb, _alone(big, 30, bdecon.BDECON_FP32))
