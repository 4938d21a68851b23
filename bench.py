"""Benchmark of the posterior-sampling sweep (pixel-updates/s).

Headline (value): the float form, batched -- 64 frames of uneven sizes
(sides 128..1024, Gaussian PSF sigma 1..4 px on 2 ceil(3 sigma)+1 support,
peak 3..200 photons) x 4 chains each in one handle, launch shapes picked by
the library's autotuner, every sweep call replayed as one CUDA graph.  One
step = 10 sweeps of every chain followed by the double refresh (expected
image, spectra, cumulant cache, log posterior) and the trace: every row of
the hot path (propose, window likelihood change, patch prior change,
accept/write, class schedule, running mean, refresh).  The chains' state
(~5 GB) is far larger than L2, so no flush is needed between steps.

e2e       the same metric through the C ABI from pinned host buffers: create
          (H2D of the 64 frames, set-up, first refresh; the launch plan comes
          from the library's tuning cache, filled by the headline's autotune),
          one step of sweeps, posterior means of every frame (D2H)
roofline  the sweep kernel against the plain-ALU peak (SMs x 128 FP32 lanes x
          2 x max SM clock), with the algorithmic work per update
          L^2 (4 n + 10) + 12 S^2 (n the photon counts carrying >= 2^-26 of a
          pixel's photon posterior); bw_roofline: 68 algorithmic bytes per
          update against the measured HBM copy bandwidth
legs      fp64_plain (the plain double sampler on frames of the same batch),
          widefield_512 (512x512 sCMOS frame, L = 17, 1 chain, float and double),
          widefield_64 (64x64 frame, L = 9, double, 200 sweeps),
          lowsnr_2048 (2048x2048 low-SNR frame, L = 31, 4 chains, float and double),
          serving (Poisson arrivals at 20 jobs/s, float and double arms)
cpu_baseline  the C oracle timed on the host cores on a bounded sample of the
          batch (crops of its frames, one chain per core); the same leg then
          evaluates, with the oracle, the error of each GPU result

--impl reference runs the oracle (the CPU restatement of the method) as the
reference arm on the host cores, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import copy
import json
import math
import multiprocessing as mp
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2411_00991_gb300 import synth  # noqa: E402

METRIC = "pixel-updates/s, FP32 batched vs FP64 plain on one GB300; % of BW roofline"
SWEEPS_PER_STEP = 10
N_IMAGES = 64
CROP = 96
FP64_PEAK_TFLOPS = 1.25     # GB300 nominal FP64 rate (no measured figure on this machine)


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return dict(hbm_gbs=float(d["hbm_gbs"]), sm_max_mhz=float(d.get("sm_max_mhz", 2070.0)),
                    source="measured (MEASURED_PEAKS.json)")
    except Exception:
        return dict(hbm_gbs=6800.0, sm_max_mhz=2070.0, source="fallback")


# ------------------------------------------------------------------ clocks --
class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.rows = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True,
                                     timeout=5).stdout.strip()
                if out:
                    self.rows.append([x.strip() for x in out.split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        self._t.join(timeout=10)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4)
                          if len(r) > 5 + k and r[5 + k].lower().startswith("active")})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(self.rows)}


# ------------------------------------------------------------ workloads --
def batch_problems(rank=0, n_images=N_IMAGES):
    """The batched workload (64 uneven frames x 4 chains); each rank of a
    multi-GPU run takes its own frames (seeds offset by rank)."""
    probs = synth.batch_uneven(n_images, seed0=3000 + 1000 * rank)
    for q in probs:
        q.burn_in = 0                     # every sweep enters the running mean
        q.refresh_every = SWEEPS_PER_STEP
        q.truth = None
    return probs


def obj_updates(probs):
    return sum((q.H + 2 * q.R) * (q.W + 2 * q.R) * q.n_chains for q in probs)


# ------------------------------------------------------------ op counting --
def photon_terms(prob, mu, max_pixels=40000):
    """Mean number of photon counts carrying >= 2^-26 of a camera pixel's
    photon posterior p(phi | w, mu) at the current expected image (a seeded
    sample of at most max_pixels pixels)."""
    from scipy.special import gammaln
    g, o, v = prob.maps()
    c = ((prob.image.astype(np.float64) - o) / g).ravel()
    s2 = (v / g ** 2).ravel()
    mu = np.maximum(np.asarray(mu, dtype=np.float64).ravel(), 1e-12)
    if c.size > max_pixels:
        idx = np.random.default_rng(0).choice(c.size, max_pixels, replace=False)
        c, s2, mu = c[idx], s2[idx], mu[idx]
    phi = np.arange(0, int(max(c.max(), mu.max()) + 60))[:, None]
    lt = -(c[None, :] - phi) ** 2 / (2 * s2[None, :]) + phi * np.log(mu[None, :]) - gammaln(phi + 1)
    lt -= lt.max(axis=0, keepdims=True)
    w = np.exp(lt)
    w /= w.sum(axis=0, keepdims=True)
    return float((w >= 2.0 ** -26).sum(axis=0).mean())


def flops_per_update(L, S, nterms):
    """Algorithmic FP32 operations of one pixel update: L^2 window pixels at
    4 per photon-count term + 10, and 12 per patch spectrum entry (S^2)."""
    return L * L * (4.0 * nterms + 10.0) + 12.0 * S * S


BYTES_PER_UPDATE = 68.0      # rho, mu, cumulant cache r/w; w, o, var; spectrum r/w; double mean r/w


def alu_peak_tflops(dev, sm_mhz):
    import torch
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    return sms * 128 * 2 * sm_mhz * 1e6 / 1e12, sms


def roofline(flops, kernel_ms, launches, updates, dev, peaks, kernel, fp64=False):
    """Roofline of a sweep kernel from its algorithmic work and its measured
    device time (summed over `launches` launches)."""
    sec = kernel_ms / 1e3
    if fp64:
        peak, src = FP64_PEAK_TFLOPS, "GB300 nominal FP64 rate (no measured FP64 figure)"
        sms = None
    else:
        peak, sms = alu_peak_tflops(dev, peaks["sm_max_mhz"])
        src = f"{sms} SMs (device query) x 128 FP32 lanes x 2 x {peaks['sm_max_mhz']:.0f} MHz max SM clock"
    ach = flops / sec / 1e12
    gbs = BYTES_PER_UPDATE * (2 if fp64 else 1) * updates / sec / 1e9
    return ({"bound": "alu", "kernel": kernel, "achieved": ach, "peak": peak, "unit": "TFLOP/s",
             "frac": ach / peak, "traffic": None, "flops_per_launch": flops / max(launches, 1),
             "launch_ms": kernel_ms / max(launches, 1), "launches": launches,
             "flops_formula": "updates x [L^2 (4 n + 10) + 12 S^2]", "peak_source": src},
            {"achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": gbs / peaks["hbm_gbs"],
             "bytes_per_update": BYTES_PER_UPDATE * (2 if fp64 else 1), "peak_source": peaks["source"]})


# ----------------------------------------------------------- CPU baseline --
def crop_problem(prob, side=CROP, y0=None, x0=None):
    """A side x side region of a frame with its maps: a bounded sample of the
    same workload (same PSF, camera model, structure density)."""
    q = copy.copy(prob)
    y0 = (prob.H - side) // 2 if y0 is None else y0
    x0 = (prob.W - side) // 2 if x0 is None else x0
    sl = (slice(y0, y0 + side), slice(x0, x0 + side))
    q.image = np.ascontiguousarray(prob.image[sl])
    for k in ("offset", "var", "gain"):
        v = getattr(prob, k)
        setattr(q, k, v if np.isscalar(v) else np.ascontiguousarray(v[sl]))
    q.truth = None
    q.name = prob.name + f"_crop{side}"
    return q


def _oracle_job(k):
    from oracle import oracle as O
    prob = crop_problem(synth.batch_frame(k % N_IMAGES))
    prob.burn_in, prob.refresh_every = 0, SWEEPS_PER_STEP
    orc = O.Oracle(prob)
    t = time.perf_counter()
    orc.run(1)
    dt = time.perf_counter() - t
    Ho, Wo = prob.object_shape()
    return Ho * Wo, dt


def cpu_baseline(cores=None):
    """The oracle as it stands, one independent chain per host core (spawned
    processes), one sweep of a 96x96 crop of batch frame k on core k, all
    cores at once; returns the updates of all cores over the longest core's
    sweep time."""
    from oracle import oracle as O
    O.build()
    n = cores or min(os.cpu_count() or 1, 16)
    with mp.get_context("spawn").Pool(n) as pool:
        res = pool.map(_oracle_job, range(n))
    upd = sum(r[0] for r in res)
    slowest = max(r[1] for r in res)
    return dict(value=upd / slowest, unit="pixel-updates/s", cores=n, kind="oracle",
                sample=f"one sweep of a {CROP}x{CROP} crop of batch frame k on core k (k < {n}, PSF sides "
                       f"{sorted({synth.batch_frame(k).L for k in range(n)})}), one chain per core, "
                       f"longest core {slowest:.1f} s",
                per_core=float(np.mean([r[0] / r[1] for r in res])))


def _rel(a, b):
    return abs(a - b) / abs(b)


def _eval_job(args):
    prob, rho = args
    from oracle import oracle as O
    return O.Oracle(prob).log_posterior_fft(rho)


def oracle_errors(checks, exact64):
    """Error of the GPU results against the oracle: each trace value (the
    float chains' double running sum) against the oracle's Eq. 9 of the
    chain's own state; the double chain on the 64x64 frame against the
    oracle's chain (accept decisions, object, trace)."""
    from oracle import oracle as O
    out = {}
    with mp.get_context("spawn").Pool(min(len(checks), os.cpu_count() or 4, 16)) as pool:
        refs = pool.map(_eval_job, [(c["prob"], c["rho"]) for c in checks])
    for c, ref in zip(checks, refs):
        out.setdefault(c["leg"], []).append({"what": c["what"], "trace": c["trace"], "oracle": ref,
                                             "rel_err": _rel(c["trace"], ref)})
    if exact64 is not None:
        prob, g = exact64
        ref = O.Oracle(prob).run(g["sweeps"], want_acc_log=True)
        out["widefield_64"] = {"what": f"double chain vs the oracle's chain, {g['sweeps']} sweeps",
                               "accept_mismatches": int((g["acc"] != ref["acc_log"]).sum()),
                               "rho_max_rel_err": float(np.max(np.abs(g["rho"] - ref["rho"]) / ref["rho"])),
                               "trace_max_rel_err": float(np.max(np.abs(g["trace"] - ref["trace"]) /
                                                                 np.abs(ref["trace"])))}
    return out


# -------------------------------------------------------------- helpers --
def _events(torch):
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def timed_sweeps(s, n, stream, torch):
    e0, e1 = _events(torch)
    e0.record(stream)
    s.sweep(n)
    e1.record(stream)
    torch.cuda.synchronize()
    s.sync()
    return e0.elapsed_time(e1)


def kernel_time(s, n):
    """Device time of the sweep-kernel launches of n plain (non-graph) sweeps."""
    s.set_timing(True)
    s.sweep_kernel_time()
    s.sweep(n)
    s.sync()
    ms, launches = s.sweep_kernel_time()
    s.set_timing(False)
    return ms, launches


def _pinned_copy(prob, torch):
    """The problem with its frame and maps in pinned host memory."""
    q = copy.copy(prob)
    for k in ("image", "offset", "var", "gain"):
        v = getattr(prob, k)
        if not np.isscalar(v):
            t = torch.empty(np.asarray(v).shape, dtype=torch.float32, pin_memory=True)
            a = t.numpy()
            a[...] = v
            setattr(q, k, a)
    return q


# ----------------------------------------------------------------- legs --
def leg_fp64_batch(bd, stream, torch, dev, peaks, rank, n_images=8):
    """The plain double sampler on the first n_images frames of the batch,
    against the float form on the same frames (same sweeps)."""
    probs = batch_problems(rank)[:n_images]
    upd = obj_updates(probs)
    out = {"workload": f"frames 0..{n_images - 1} of the batch ({[q.H for q in probs]} px sides, "
                       f"L {[q.L for q in probs]}), 4 chains each, 1 sweep"}
    for name, prec in (("fp64", bd.BDECON_FP64), ("fp32", bd.BDECON_FP32)):
        s = bd.Sampler(probs, precision=prec, max_sweeps=8, stream=stream.cuda_stream)
        s.sweep(1)
        s.sync()
        ms = timed_sweeps(s, 1, stream, torch)
        if name == "fp64":
            kms, nl = kernel_time(s, 1)
            flops = sum((q.H + 2 * q.R) * (q.W + 2 * q.R) * q.n_chains *
                        flops_per_update(q.L, q.S, photon_terms(q, s.get_mu(p, 0))) for p, q in enumerate(probs))
            out["roofline"], out["bw_roofline"] = roofline(flops, kms, nl, upd, dev, peaks, "k_sweep<double>",
                                                           fp64=True)
        s.close()
        out[name] = {"value": upd / (ms / 1e3), "unit": "pixel-updates/s", "ms_per_sweep": ms}
    out["fp32_over_fp64"] = out["fp32"]["value"] / out["fp64"]["value"]
    return out


def leg_widefield512(bd, stream, torch, dev, peaks, flush, checks, steps=3, sweeps=50):
    prob = synth.widefield_512()
    prob.burn_in = 0
    prob.refresh_every = sweeps
    Ho, Wo = prob.object_shape()
    s = bd.Sampler(prob, precision=bd.BDECON_FP32, max_sweeps=(steps + 2) * sweeps + 8, stream=stream.cuda_stream)
    s.sweep(sweeps)
    s.sync()
    ms = 0.0
    for _ in range(steps):
        flush()
        ms += timed_sweeps(s, sweeps, stream, torch)
    kms, nl = kernel_time(s, sweeps)
    nt = photon_terms(prob, s.get_mu())
    upd_launch = Ho * Wo * sweeps
    rf, bw = roofline(flops_per_update(prob.L, prob.S, nt) * upd_launch, kms, nl, upd_launch, dev, peaks,
                      "k_sweep<float> one-team form")
    rho, t = s.get_state()
    checks.append(dict(leg="widefield_512", what=f"float chain, trace after sweep {t}", prob=prob, rho=rho,
                       trace=float(s.trace()[-1])))
    out = {"workload": "512x512 sCMOS frame, PSF sigma 1.2 px on 17x17, 1 chain, refresh every 50, L2 flushed "
                       "between steps", "plan": s.get_plan(),
           "fp32": {"value": Ho * Wo * sweeps * steps / (ms / 1e3), "unit": "pixel-updates/s",
                    "ms_per_sweep": ms / (steps * sweeps)},
           "roofline": rf, "bw_roofline": bw, "mean_photon_terms": nt,
           "acceptance": float(s.accept_counts()[-sweeps:].sum() / (sweeps * Ho * Wo))}
    s.close()
    s64 = bd.Sampler(prob, precision=bd.BDECON_FP64, max_sweeps=32, stream=stream.cuda_stream)
    s64.sweep(2)
    s64.sync()
    flush()
    ms64 = timed_sweeps(s64, 10, stream, torch)
    s64.close()
    out["fp64"] = {"value": Ho * Wo * 10 / (ms64 / 1e3), "unit": "pixel-updates/s", "ms_per_sweep": ms64 / 10}
    out["fp32_over_fp64"] = out["fp32"]["value"] / out["fp64"]["value"]
    return out


def leg_widefield64(bd, stream, torch):
    """The plain double sampler on the 64x64 frame, 200 sweeps (and a 10-sweep
    chain kept for the oracle comparison)."""
    prob = synth.widefield_64()
    Ho, Wo = prob.object_shape()
    out = {"workload": "64x64 frame, 12 blobs + 3 lines, PSF sigma 1.5 px on 9x9, 1 chain, 200 sweeps"}
    for name, prec in (("fp64", bd.BDECON_FP64), ("fp32", bd.BDECON_FP32)):
        s = bd.Sampler(prob, precision=prec, max_sweeps=208, stream=stream.cuda_stream)
        torch.cuda.synchronize()
        ms = timed_sweeps(s, 200, stream, torch)
        s.close()
        out[name] = {"value": Ho * Wo * 200 / (ms / 1e3), "unit": "pixel-updates/s", "ms_per_sweep": ms / 200}
    s = bd.Sampler(prob, precision=bd.BDECON_FP64, max_sweeps=16, flags=bd.FLAG_ACCEPT_LOG,
                   stream=stream.cuda_stream)
    s.sweep(10)
    s.sync()
    exact = dict(sweeps=10, acc=s.accept_log(), rho=s.get_state()[0], trace=s.trace())
    s.close()
    return out, (prob, exact)


def leg_lowsnr2048(bd, stream, torch, dev, peaks, checks):
    prob = synth.lowsnr_2048()
    Ho, Wo = prob.object_shape()
    upd = Ho * Wo * prob.n_chains
    out = {"workload": "2048x2048 low-SNR frame, peak 5 / background 1 photons, PSF sigma 4 px on 31x31, "
                       "sCMOS maps, 4 chains, double refresh every 50 sweeps"}
    s = bd.Sampler(prob, precision=bd.BDECON_FP32, max_sweeps=32, stream=stream.cuda_stream)
    s.sweep(1)
    s.sync()
    ms = timed_sweeps(s, 5, stream, torch)
    kms, nl = kernel_time(s, 2)
    nt = photon_terms(prob, s.get_mu(0, 0))
    out["roofline"], out["bw_roofline"] = roofline(flops_per_update(prob.L, prob.S, nt) * upd * 2, kms, nl,
                                                   upd * 2, dev, peaks, "k_sweep<float>")
    out["plan"] = s.get_plan()
    out["fp32"] = {"value": upd * 5 / (ms / 1e3), "unit": "pixel-updates/s", "ms_per_sweep": ms / 5}
    rho, t = s.get_state(0, 0)
    checks.append(dict(leg="lowsnr_2048", what=f"float chain 0, trace after sweep {t}", prob=prob, rho=rho,
                       trace=float(s.trace(0, 0)[-1])))
    s.close()
    s64 = bd.Sampler(prob, precision=bd.BDECON_FP64, max_sweeps=4, stream=stream.cuda_stream)
    torch.cuda.synchronize()
    ms64 = timed_sweeps(s64, 1, stream, torch)
    s64.close()
    out["fp64"] = {"value": upd / (ms64 / 1e3), "unit": "pixel-updates/s", "ms_per_sweep": ms64}
    out["fp32_over_fp64"] = out["fp32"]["value"] / out["fp64"]["value"]
    return out


def run_serving(bd, precision, n_jobs=8, sweeps=500, rate=20.0, budget_gb=120):
    """The serving form: deconvolution jobs (filament frames, sides
    log-uniform in 128..2048 rounded to 32, PSF sigma U[1, 4] px, sCMOS maps,
    one chain, refresh every 50, burn-in 250) arrive as a Poisson stream of
    the given rate and are submitted to the library's serving loop, which
    admits them under a device-memory budget and sweeps all running jobs in
    shared launches.  The first n_jobs arrivals are served; latency = finish
    - arrival."""
    ta, sides, sig = synth.serving_arrivals(n_jobs, rate=rate, seed=4)
    jobs = [synth.serving_job(int(sides[k]), float(sig[k]), seed=1000 + k) for k in range(n_jobs)]
    for q in jobs:
        q.burn_in = min(q.burn_in, sweeps // 2)
    upd = sum((q.H + 2 * q.R) * (q.W + 2 * q.R) * q.n_chains * sweeps for q in jobs)
    srv = bd.Server(mem_budget=int(budget_gb) << 30, max_jobs=64, segment_sweeps=25, precision=precision)
    t0 = time.perf_counter()
    ids = []
    for k, q in enumerate(jobs):
        while time.perf_counter() - t0 < ta[k] - ta[0]:
            time.sleep(0.0005)
        ids.append(srv.submit(q, sweeps))
    res = [srv.result(i, timeout=1800) for i in ids]
    wall = time.perf_counter() - t0
    stats = srv.stats()
    srv.close()
    lat = np.array([r[1][2] - r[1][0] for r in res])
    for m, _ in res:
        assert np.isfinite(m).all()
    return dict(value=upd / wall, unit="pixel-updates/s", jobs=n_jobs, sweeps_per_job=sweeps,
                arrival_rate_per_s=rate, sides=[int(x) for x in sides], psf_sigma=[round(float(x), 3) for x in sig],
                memory_budget_gb=budget_gb, wall_s=wall, jobs_per_s=n_jobs / wall,
                latency_p50_s=float(np.percentile(lat, 50)), latency_p99_s=float(np.percentile(lat, 99)),
                queue_wait_p50_s=float(np.percentile([r[1][1] - r[1][0] for r in res], 50)),
                segments=stats["segments"])


# ---------------------------------------------------------------- our arm --
def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2411_00991_gb300 import bdecon as bd

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    peaks = _peaks()
    W, K, S = args.warmup, args.steps, SWEEPS_PER_STEP

    # ---- headline: the batched float form
    probs = batch_problems(rank)
    upd_sweep = obj_updates(probs)
    ws_bytes = bd.Sampler.workspace_size(probs, bd.BDECON_FP32, (W + K + 4) * S + 8)
    s = bd.Sampler(probs, precision=bd.BDECON_FP32, max_sweeps=(W + K + 4) * S + 8, stream=stream.cuda_stream)
    s.sweep(1)
    s.sync()
    t = time.perf_counter()
    tune = s.autotune(trial_sweeps=1)
    tune_s = time.perf_counter() - t
    s.set_graph(True)
    s.sweep(S - 1)                      # align the sweep counter with the refresh period
    for _ in range(W):
        s.sweep(S)
    s.sync()
    n0 = s.launch_count()
    evs = [_events(torch) for _ in range(K)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for k in range(K):
            evs[k][0].record(stream)
            s.sweep(S)
            evs[k][1].record(stream)
        torch.cuda.synchronize()
    s.sync()
    ms = sum(a.elapsed_time(b) for a, b in evs)
    launches = s.launch_count() - n0
    if world > 1:
        tt = torch.tensor([ms], dtype=torch.float64, device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ms = float(tt.item())
    value = world * upd_sweep * S * K / (ms / 1e3)
    plans = sorted({json.dumps(s.get_plan(p), sort_keys=True) for p in range(len(probs))})

    if rank != 0:
        s.close()
        if world > 1:
            dist.destroy_process_group()
        return

    # kernel-only time of one step (plain launches, one per launch group and segment)
    s.set_graph(False)
    kms, nl = kernel_time(s, S)
    nts = [photon_terms(q, s.get_mu(p, 0)) for p, q in enumerate(probs)]
    flops = S * sum((q.H + 2 * q.R) * (q.W + 2 * q.R) * q.n_chains * flops_per_update(q.L, q.S, nt)
                    for q, nt in zip(probs, nts))
    rf, bw = roofline(flops, kms, nl, upd_sweep * S, dev, peaks, "k_sweep<float> (batched launch groups)")
    checks = []
    order = np.argsort([q.H for q in probs])
    for p in (int(order[0]), int(order[len(order) // 2]), int(order[-1])):
        rho, t = s.get_state(p, 0)
        checks.append(dict(leg="batched", what=f"frame {p} ({probs[p].H}x{probs[p].W}, L {probs[p].L}) chain 0, "
                                               f"trace after sweep {t}", prob=probs[p], rho=rho,
                           trace=float(s.trace(p, 0)[-1])))
    acc = sum(float(s.accept_counts(p, c)[-S:].sum()) for p, q in enumerate(probs) for c in range(q.n_chains))
    s.close()

    # end to end through the C ABI from pinned host buffers
    e2e = None
    if not args.no_e2e:
        pin = [_pinned_copy(q, torch) for q in probs]
        h2d = sum(np.asarray(getattr(q, k)).nbytes for q in pin for k in ("image", "offset", "var", "psf")
                  if not np.isscalar(getattr(q, k)))
        d2h = sum((q.H + 2 * q.R) * (q.W + 2 * q.R) * 8 for q in pin)
        torch.cuda.synchronize()
        t = time.perf_counter()
        se = bd.Sampler(pin, precision=bd.BDECON_FP32, max_sweeps=S + 4, stream=stream.cuda_stream)
        se.sweep(S)
        means = [se.posterior_mean(p) for p in range(len(pin))]
        se.close()
        dt = time.perf_counter() - t
        assert all(np.isfinite(m).all() for m in means)
        e2e = dict(value=upd_sweep * S / dt, unit="pixel-updates/s", h2d_bytes_per_step=int(h2d),
                   d2h_bytes_per_step=int(d2h), ms_per_step=dt * 1e3,
                   step="create from pinned host buffers (launch plan from the library's tuning cache, "
                        "filled by the autotune above) + 10 sweeps + posterior means of all 64 frames")

    flush_buf = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def flush():
        flush_buf.fill_(1.0)

    legs = {}
    exact64 = None
    if not args.no_legs:
        legs["fp64_plain"] = leg_fp64_batch(bd, stream, torch, dev, peaks, rank)
        legs["widefield_512"] = leg_widefield512(bd, stream, torch, dev, peaks, flush, checks)
        legs["widefield_64"], exact64 = leg_widefield64(bd, stream, torch)
        legs["lowsnr_2048"] = leg_lowsnr2048(bd, stream, torch, dev, peaks, checks)
    if not args.no_serve:
        legs["serving"] = {"fp32": run_serving(bd, bd.BDECON_FP32, n_jobs=args.serve_jobs),
                           "fp64": run_serving(bd, bd.BDECON_FP64, n_jobs=args.serve_jobs, sweeps=5)}
        legs["serving"]["note"] = ("the double arm serves the same arrival stream with 5 sweeps per job "
                                   "(500 would take ~1 h): compare throughput, not latency")

    line = {
        "metric": METRIC,
        "value": value,
        "unit": "pixel-updates/s",
        "n_gpus": world,
        "steps": K,
        "warmup": W,
        "ms_per_step": ms / K,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (seeded filament+blob objects, Poisson photons, Gaussian read noise)",
        "config": {"workload": "batched: 64 frames, sides uniform from {128,256,384,512,768,1024}, Gaussian PSF "
                               "sigma U[1,4] px on 2 ceil(3 sigma)+1, peak log-U[3,200] photons, background 1, "
                               "gain 2.0 / offset 100 / read sd 1.6, 4 chains each; float sweeps, double refresh "
                               "every 10 sweeps; autotuned launch shapes, CUDA graph",
                   "sweeps_per_step": S, "updates_per_sweep": upd_sweep, "images": len(probs),
                   "chains": sum(q.n_chains for q in probs), "workspace_bytes": int(ws_bytes),
                   "l2": "inputs larger than L2 (chain state ~%.1f GB vs 129 MB), no flush" % (ws_bytes / 1e9),
                   "plans": [json.loads(x) for x in plans],
                   "autotune": dict(one_launch=tune["one_launch"], trial_ms_per_sweep=tune["ms_per_sweep"],
                                    seconds=tune_s)},
        "e2e": e2e,
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
        "roofline": rf,
        "bw_roofline": bw,
        "mean_photon_terms": float(np.average(nts, weights=[q.L * q.L for q in probs])),
        "acceptance": acc / (upd_sweep * S),
        "legs": legs,
    }
    if not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline()
        line["oracle_error"] = oracle_errors(checks, exact64)
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    W, K = args.warmup, args.steps
    vals = []
    r = None
    for k in range(W + K):
        r = cpu_baseline()
        if k >= W:
            vals.append(r["value"])
    v = float(np.mean(vals))
    line = {
        "impl": "reference",
        "metric": METRIC,
        "value": v,
        "unit": "pixel-updates/s",
        "n_gpus": world,
        "steps": K,
        "warmup": W,
        "ms_per_step": (CROP + 24) ** 2 * r["cores"] / v * 1e3,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic (seeded filament+blob objects, Poisson photons, Gaussian read noise)",
        "config": {"workload": "batched: 64 uneven frames x 4 chains (as the GPU arm); reference = the C oracle, "
                               f"one sweep of a {CROP}x{CROP} crop of batch frame k per host core k per step"},
        "cpu_baseline": {"value": v, "unit": "pixel-updates/s", "cores": r["cores"], "kind": "oracle",
                         "sample": r["sample"]},
        "e2e": {"value": v, "unit": "pixel-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_profile(args):
    """Small cases for ncu: --profile N runs one launch of N sweeps of the
    512x512 frame after a warm-up launch; --profile-batch L runs two sweeps of
    the batch frames whose PSF side is L (one launch group); --profile-lowsnr
    runs two one-sweep launches of the 2048x2048 low-SNR frame (4 chains)."""
    import torch
    from paper_2411_00991_gb300 import bdecon as bd
    st = torch.cuda.current_stream().cuda_stream
    if args.profile_batch:
        # the batch frames of this PSF side with many updates per class step
        # (chains x patches >= 2048): one launch group
        probs = [q for q in batch_problems() if q.L == args.profile_batch and
                 q.n_chains * math.ceil((q.H + 2 * q.R) / q.S) * math.ceil((q.W + 2 * q.R) / q.S) >= 2048]
        s = bd.Sampler(probs, precision=bd.BDECON_FP32, max_sweeps=16, stream=st)
        s.sweep(1)
        s.sync()
        s.sweep(1)
        s.sync()
        print(json.dumps({"profile_batch_L": args.profile_batch, "images": len(probs), "sides": [q.H for q in probs],
                          "updates_per_sweep": obj_updates(probs), "plan": s.get_plan()}))
        s.close()
        return
    if args.profile_lowsnr:
        prob = synth.lowsnr_2048()
        prob.truth = None
        s = bd.Sampler(prob, precision=bd.BDECON_FP32, max_sweeps=16, stream=st)
        s.sweep(1)
        s.sync()
        s.sweep(1)
        s.sync()
        print(json.dumps({"profile_lowsnr": True, "updates_per_sweep": obj_updates([prob]), "plan": s.get_plan(),
                          "lean": s.lean()}))
        s.close()
        return
    prob = synth.widefield_512()
    prob.burn_in = 0
    prob.refresh_every = 0
    prec = bd.BDECON_FP64 if args.profile_fp64 else bd.BDECON_FP32
    s = bd.Sampler(prob, precision=prec, max_sweeps=args.profile + 8, stream=st)
    s.sweep(2)
    s.sync()
    s.sweep(args.profile)
    s.sync()
    print(json.dumps({"profile_sweeps": args.profile, "plan": s.get_plan(), "trace_last": float(s.trace()[-1])}))
    s.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-legs", action="store_true", help="headline only (no per-config legs)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--serve-jobs", type=int, default=8)
    ap.add_argument("--profile", type=int, default=0, help="ncu mode: one launch of this many sweeps")
    ap.add_argument("--profile-fp64", action="store_true")
    ap.add_argument("--profile-batch", type=int, default=0, help="ncu mode: the batch frames of this PSF side")
    ap.add_argument("--profile-lowsnr", action="store_true", help="ncu mode: the 2048x2048 low-SNR frame")
    args = ap.parse_args()
    if args.profile or args.profile_batch or args.profile_lowsnr:
        run_profile(args)
        return
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
