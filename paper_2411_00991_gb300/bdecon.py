"""ctypes binding of libbdecon (include/bdecon.h): argument marshalling only.

Every step of the sampler runs in the library's CUDA kernels; this module
converts numpy arrays to the C structs, passes the CUDA stream, and turns
status codes into exceptions.  It fails loudly when the library cannot be
loaded: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

from . import build as _build

_lib = None

BDECON_FP64 = 0
BDECON_FP32 = 1
FLAG_ACCEPT_LOG = 1
FLAG_SECOND_MOMENT = 2
FLAG_AUGMENTED = 4

STATUS = {0: "OK", 1: "INVALID", 2: "NOMEM", 3: "CUDA", 4: "TIMEOUT", 5: "STATE", 6: "NUMERIC"}


class BdeconError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"bdecon {STATUS.get(status, status)}: {msg}")
        self.status = status


class _ServerConfig(C.Structure):
    _fields_ = [("mem_budget", C.c_size_t), ("max_jobs", C.c_int32), ("segment_sweeps", C.c_int32),
                ("precision", C.c_int32), ("device", C.c_int32), ("one_launch", C.c_int32)]


class _Problem(C.Structure):
    _fields_ = [("H", C.c_int32), ("W", C.c_int32), ("image", C.c_void_p),
                ("L", C.c_int32), ("psf", C.c_void_p),
                ("gain_map", C.c_void_p), ("gain", C.c_double),
                ("offset_map", C.c_void_p), ("offset", C.c_double),
                ("var_map", C.c_void_p), ("read_var", C.c_double),
                ("stride", C.c_int32), ("n_chains", C.c_int32), ("seed", C.c_uint64),
                ("step", C.c_double), ("burn_in", C.c_int32), ("refresh_every", C.c_int32),
                ("precision", C.c_int32), ("max_sweeps", C.c_int32), ("flags", C.c_int32),
                ("team_warps", C.c_int32), ("sample_every", C.c_int32), ("n_samples", C.c_int32),
                ("adapt_target", C.c_double), ("subpixel", C.c_int32)]


EXPORTS = ["bdecon_workspace_size", "bdecon_create", "bdecon_batch_create", "bdecon_create_in",
           "bdecon_destroy", "bdecon_last_error", "bdecon_sweep", "bdecon_sync",
           "bdecon_posterior_mean", "bdecon_posterior_var", "bdecon_log_posterior_trace",
           "bdecon_accept_counts", "bdecon_accept_log", "bdecon_get_state", "bdecon_set_state",
           "bdecon_get_mu", "bdecon_log_posterior", "bdecon_delta", "bdecon_set_plan",
           "bdecon_get_plan", "bdecon_launch_count", "bdecon_set_timing", "bdecon_sweep_kernel_time",
           "bdecon_log_posterior_static", "bdecon_set_fault", "bdecon_server_start",
           "bdecon_server_submit", "bdecon_server_poll", "bdecon_server_wait", "bdecon_server_stats",
           "bdecon_server_stop", "bdecon_set_grouping", "bdecon_autotune", "bdecon_set_graph",
           "bdecon_posterior_std", "bdecon_posterior_cv", "bdecon_get_samples", "bdecon_posterior_quantiles",
           "bdecon_get_steps", "bdecon_get_phi", "bdecon_set_staging", "bdecon_get_staging",
           "bdecon_set_tuning_cache", "bdecon_set_lean", "bdecon_get_lean"]

JOB_QUEUED, JOB_RUNNING, JOB_DONE, JOB_FAILED = 0, 1, 2, 3


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libbdecon.so (building it in-tree first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError(f"libbdecon.so not found at {_build.LIB}; run __graft_entry__.build()")
    L = C.CDLL(_build.LIB)
    vp, i32, i64, sz, dp = C.c_void_p, C.c_int32, C.c_int64, C.c_size_t, C.POINTER(C.c_double)
    P = C.POINTER(_Problem)
    H = C.c_void_p
    sig = {
        "bdecon_workspace_size": [P, i32, C.POINTER(sz)],
        "bdecon_create": [P, vp, C.POINTER(H)],
        "bdecon_batch_create": [P, i32, vp, C.POINTER(H)],
        "bdecon_create_in": [P, i32, vp, vp, sz, C.POINTER(H)],
        "bdecon_sweep": [H, i32],
        "bdecon_sync": [H],
        "bdecon_posterior_mean": [H, i32, vp, i32],
        "bdecon_posterior_var": [H, i32, vp, i32],
        "bdecon_posterior_std": [H, i32, vp, i32],
        "bdecon_posterior_cv": [H, i32, vp, i32],
        "bdecon_get_samples": [H, i32, i32, vp, sz, C.POINTER(sz)],
        "bdecon_posterior_quantiles": [H, i32, vp, i32, vp, i32],
        "bdecon_log_posterior_trace": [H, i32, i32, vp, sz, C.POINTER(sz)],
        "bdecon_accept_counts": [H, i32, i32, vp, sz, C.POINTER(sz)],
        "bdecon_accept_log": [H, i32, i32, vp, sz, C.POINTER(sz)],
        "bdecon_get_state": [H, i32, i32, vp, C.POINTER(i64)],
        "bdecon_set_state": [H, i32, i32, vp, i64],
        "bdecon_get_mu": [H, i32, i32, vp],
        "bdecon_get_steps": [H, i32, i32, vp],
        "bdecon_get_phi": [H, i32, i32, vp],
        "bdecon_log_posterior": [H, i32, i32, dp],
        "bdecon_delta": [H, i32, i32, i64, C.c_double, dp, dp, C.POINTER(i32)],
        "bdecon_set_plan": [H, i32, i32, i32, i32],
        "bdecon_get_plan": [H, i32, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32), C.POINTER(i32)],
        "bdecon_set_staging": [H, i32],
        "bdecon_get_staging": [H, i32, C.POINTER(i32)],
        "bdecon_set_lean": [H, i32],
        "bdecon_get_lean": [H, i32, C.POINTER(i32)],
        "bdecon_launch_count": [H, C.POINTER(i64)],
        "bdecon_set_timing": [H, i32],
        "bdecon_sweep_kernel_time": [H, dp, C.POINTER(i64)],
        "bdecon_set_fault": [H, i32, i64],
        "bdecon_set_grouping": [H, i32],
        "bdecon_set_graph": [H, i32],
        "bdecon_autotune": [H, i32, C.POINTER(i32), dp],
        "bdecon_set_tuning_cache": [i32],
        "bdecon_server_start": [C.POINTER(_ServerConfig), C.POINTER(vp)],
        "bdecon_server_submit": [vp, P, i32, C.POINTER(i64)],
        "bdecon_server_poll": [vp, i64, C.POINTER(i32), vp, vp, sz],
        "bdecon_server_wait": [vp, i64, C.c_double, C.POINTER(i32)],
        "bdecon_server_stats": [vp, C.POINTER(i64), C.POINTER(i64), C.POINTER(i64), C.POINTER(sz),
                                C.POINTER(i64)],
        "bdecon_server_stop": [vp],
        "bdecon_log_posterior_static": [i32, i32, vp, i32, vp, vp, C.c_double, vp, C.c_double, vp,
                                        C.c_double, i32, vp, vp, vp],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = C.c_int
    L.bdecon_destroy.argtypes = [H]
    L.bdecon_destroy.restype = None
    L.bdecon_last_error.argtypes = [H]
    L.bdecon_last_error.restype = C.c_char_p
    _lib = L
    return L


def _p(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _as_map_or_scalar(v, H, W):
    if np.isscalar(v):
        return None, float(v)
    a = np.ascontiguousarray(np.asarray(v, dtype=np.float32))
    if a.shape != (H, W):
        raise ValueError(f"map shape {a.shape} != {(H, W)}")
    return a, 0.0


def _problem(pr, precision, max_sweeps, flags, keep) -> _Problem:
    """Fill a bdecon_problem from a ``synth.Problem``-like object; the numpy
    arrays it points at are appended to ``keep`` (the caller holds them until
    the library has copied them)."""
    img = np.ascontiguousarray(np.asarray(pr.image, dtype=np.float32))
    psf = np.ascontiguousarray(np.asarray(pr.psf, dtype=np.float64))
    H, W = img.shape
    g, gs = _as_map_or_scalar(pr.gain, H, W)
    o, os_ = _as_map_or_scalar(pr.offset, H, W)
    v, vs = _as_map_or_scalar(pr.var, H, W)
    keep += [img, psf, g, o, v]
    return _Problem(H, W, _p(img), psf.shape[0], _p(psf), _p(g), gs, _p(o), os_, _p(v), vs,
                    int(pr.stride), int(pr.n_chains), int(pr.seed), float(pr.step),
                    int(pr.burn_in), int(pr.refresh_every), int(precision), int(max_sweeps),
                    int(flags) | (FLAG_AUGMENTED if getattr(pr, "augmented", False) else 0),
                    int(getattr(pr, "team_warps", 0)), int(getattr(pr, "sample_every", 0)),
                    int(getattr(pr, "n_samples", 0)), float(getattr(pr, "adapt_target", 0.0)),
                    int(getattr(pr, "subpixel", 1)))


def set_tuning_cache(enable: bool = True) -> None:
    """Clear the process-wide tuning cache and turn it on (default) or off.

    While on, every successful Sampler.autotune stores its launch choices
    keyed by the device, precision and problem shapes, and a Sampler created
    later for the same shapes starts with them (results never depend on the
    plan, only the speed does)."""
    rc = load().bdecon_set_tuning_cache(int(bool(enable)))
    if rc != 0:
        raise RuntimeError("bdecon_set_tuning_cache failed (%d)" % rc)


def log_posterior_static(H, W, image_ptr, L, psf_ptr, gain, offset, var, stride, rho_ptr, out_ptr,
                         stream=None):
    """Allocation-free log posterior (bdecon_log_posterior_static): every
    array argument is a device pointer (int); gain / offset / var are a
    device-pointer int for a map or a float scalar (pass ``("map", ptr)``
    for a map).  Returns nothing: the value is written to out_ptr on the
    stream."""
    L_ = load()

    def split(x):
        if isinstance(x, tuple):
            return C.c_void_p(x[1]), 0.0
        return None, float(x)

    g, gs = split(gain)
    o, os_ = split(offset)
    v, vs = split(var)
    s = L_.bdecon_log_posterior_static(int(H), int(W), C.c_void_p(image_ptr), int(L), C.c_void_p(psf_ptr), g, gs,
                                       o, os_, v, vs, int(stride), C.c_void_p(rho_ptr), C.c_void_p(out_ptr),
                                       C.c_void_p(stream) if stream else None)
    if s != 0:
        raise BdeconError(s, L_.bdecon_last_error(None).decode(errors="replace"))


class Sampler:
    """A libbdecon handle over one or more problems (``synth.Problem``-like
    objects with image, psf, gain, offset, var, stride, n_chains, seed, step,
    burn_in, refresh_every)."""

    def __init__(self, problems, precision: int = BDECON_FP32, max_sweeps: int = 4096,
                 flags: int = 0, stream: Optional[int] = None, workspace=None):
        self.L = load()
        if not isinstance(problems, (list, tuple)):
            problems = [problems]
        self.problems = list(problems)
        self._keep = []
        arr = (_Problem * len(problems))()
        for k, pr in enumerate(problems):
            arr[k] = _problem(pr, precision, max_sweeps, flags, self._keep)
        self._arr = arr
        self.precision = precision
        h = C.c_void_p()
        st = C.c_void_p(stream) if stream else None
        if workspace is not None:
            ptr, nbytes = workspace
            s = self.L.bdecon_create_in(arr, len(problems), st, C.c_void_p(ptr), nbytes, C.byref(h))
        else:
            s = self.L.bdecon_batch_create(arr, len(problems), st, C.byref(h))
        if s != 0:
            raise BdeconError(s, self.L.bdecon_last_error(None).decode(errors="replace"))
        self.h = h
        self._keep = []   # inputs were copied by the library

    @staticmethod
    def workspace_size(problems, precision=BDECON_FP32, max_sweeps=4096, flags=0) -> int:
        L = load()
        if not isinstance(problems, (list, tuple)):
            problems = [problems]
        keep = []
        arr = (_Problem * len(problems))()
        for k, pr in enumerate(problems):
            arr[k] = _problem(pr, precision, max_sweeps, flags, keep)
        n = C.c_size_t()
        s = L.bdecon_workspace_size(arr, len(problems), C.byref(n))
        if s != 0:
            raise BdeconError(s, L.bdecon_last_error(None).decode(errors="replace"))
        return int(n.value)

    # ----------------------------------------------------------- plumbing --
    def _ck(self, s):
        if s != 0:
            raise BdeconError(s, self.L.bdecon_last_error(self.h).decode(errors="replace"))

    def close(self):
        if getattr(self, "h", None):
            self.L.bdecon_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _shape(self, p):
        """(crop rows, crop cols, object rows, object cols) of problem p: the
        crop is the object area under the camera, f H x f W for subpixel f."""
        pr = self.problems[p]
        H, W = np.asarray(pr.image).shape
        R = np.asarray(pr.psf).shape[0] // 2
        f = max(1, int(getattr(pr, "subpixel", 1)))
        return f * H, f * W, f * H + 2 * R, f * W + 2 * R

    # ----------------------------------------------------------- sampling --
    def sweep(self, n: int):
        self._ck(self.L.bdecon_sweep(self.h, int(n)))

    def sync(self):
        self._ck(self.L.bdecon_sync(self.h))

    def posterior_mean(self, p: int = 0, crop: bool = False) -> np.ndarray:
        H, W, Ho, Wo = self._shape(p)
        out = np.empty((H, W) if crop else (Ho, Wo))
        self._ck(self.L.bdecon_posterior_mean(self.h, p, _p(out), int(crop)))
        return out

    def posterior_var(self, p: int = 0, crop: bool = False) -> np.ndarray:
        H, W, Ho, Wo = self._shape(p)
        out = np.empty((H, W) if crop else (Ho, Wo))
        self._ck(self.L.bdecon_posterior_var(self.h, p, _p(out), int(crop)))
        return out

    def posterior_std(self, p: int = 0, crop: bool = False) -> np.ndarray:
        H, W, Ho, Wo = self._shape(p)
        out = np.empty((H, W) if crop else (Ho, Wo))
        self._ck(self.L.bdecon_posterior_std(self.h, p, _p(out), int(crop)))
        return out

    def posterior_cv(self, p: int = 0, crop: bool = False) -> np.ndarray:
        """Coefficient of variation std / mean (relative uncertainty)."""
        H, W, Ho, Wo = self._shape(p)
        out = np.empty((H, W) if crop else (Ho, Wo))
        self._ck(self.L.bdecon_posterior_cv(self.h, p, _p(out), int(crop)))
        return out

    def samples(self, p: int = 0, c: int = 0) -> np.ndarray:
        """Kept objects of chain c, (k, H+2R, W+2R), oldest first."""
        H, W, Ho, Wo = self._shape(p)
        n = C.c_size_t()
        self._ck(self.L.bdecon_get_samples(self.h, p, c, None, 0, C.byref(n)))
        out = np.empty(n.value)
        self._ck(self.L.bdecon_get_samples(self.h, p, c, _p(out), out.size, C.byref(n)))
        return out.reshape(-1, Ho, Wo)

    def posterior_quantiles(self, q, p: int = 0, crop: bool = False) -> np.ndarray:
        """Per-pixel quantiles of the kept objects of all chains, (len(q), ...)."""
        H, W, Ho, Wo = self._shape(p)
        qa = np.ascontiguousarray(np.atleast_1d(np.asarray(q, dtype=np.float64)))
        out = np.empty((qa.size, H, W) if crop else (qa.size, Ho, Wo))
        self._ck(self.L.bdecon_posterior_quantiles(self.h, p, _p(qa), qa.size, _p(out), int(crop)))
        return out

    def trace(self, p: int = 0, c: int = 0) -> np.ndarray:
        n = C.c_size_t()
        self._ck(self.L.bdecon_log_posterior_trace(self.h, p, c, None, 0, C.byref(n)))
        out = np.empty(n.value)
        self._ck(self.L.bdecon_log_posterior_trace(self.h, p, c, _p(out), out.size, C.byref(n)))
        return out

    def accept_counts(self, p: int = 0, c: int = 0) -> np.ndarray:
        n = C.c_size_t()
        self._ck(self.L.bdecon_accept_counts(self.h, p, c, None, 0, C.byref(n)))
        out = np.empty(n.value, dtype=np.int64)
        self._ck(self.L.bdecon_accept_counts(self.h, p, c, _p(out), out.size, C.byref(n)))
        return out

    def accept_log(self, p: int = 0, c: int = 0) -> np.ndarray:
        H, W, Ho, Wo = self._shape(p)
        n = C.c_size_t()
        self._ck(self.L.bdecon_accept_log(self.h, p, c, None, 0, C.byref(n)))
        out = np.empty(n.value, dtype=np.uint8)
        self._ck(self.L.bdecon_accept_log(self.h, p, c, _p(out), out.size, C.byref(n)))
        return out.reshape(-1, Ho, Wo)

    def get_state(self, p: int = 0, c: int = 0):
        H, W, Ho, Wo = self._shape(p)
        rho = np.empty((Ho, Wo))
        t = C.c_int64()
        self._ck(self.L.bdecon_get_state(self.h, p, c, _p(rho), C.byref(t)))
        return rho, int(t.value)

    def set_state(self, rho: np.ndarray, sweeps: int, p: int = 0, c: int = 0):
        rho = np.ascontiguousarray(rho, dtype=np.float64)
        self._ck(self.L.bdecon_set_state(self.h, p, c, _p(rho), int(sweeps)))

    def get_phi(self, p: int = 0, c: int = 0) -> np.ndarray:
        """Photon counts of an augmented chain, (H, W) camera pixels."""
        H, W = np.asarray(self.problems[p].image).shape
        out = np.empty((H, W))
        self._ck(self.L.bdecon_get_phi(self.h, p, c, _p(out)))
        return out

    def get_steps(self, p: int = 0, c: int = 0) -> np.ndarray:
        """Per-pixel proposal scales (adapted during burn-in when adapt_target > 0)."""
        H, W, Ho, Wo = self._shape(p)
        out = np.empty((Ho, Wo))
        self._ck(self.L.bdecon_get_steps(self.h, p, c, _p(out)))
        return out

    def get_mu(self, p: int = 0, c: int = 0) -> np.ndarray:
        """Expected image of chain c, (H, W) camera pixels."""
        H, W = np.asarray(self.problems[p].image).shape
        mu = np.empty((H, W))
        self._ck(self.L.bdecon_get_mu(self.h, p, c, _p(mu)))
        return mu

    def log_posterior(self, p: int = 0, c: int = 0) -> float:
        v = C.c_double()
        self._ck(self.L.bdecon_log_posterior(self.h, p, c, C.byref(v)))
        return v.value

    def delta(self, m: int, rho_new: float, p: int = 0, c: int = 0):
        dl, dp, ok = C.c_double(), C.c_double(), C.c_int32()
        self._ck(self.L.bdecon_delta(self.h, p, c, int(m), float(rho_new), C.byref(dl), C.byref(dp),
                                     C.byref(ok)))
        return bool(ok.value), dl.value, dp.value

    def set_plan(self, tile_i: int, tile_j: int, warps: int, p: int = 0):
        self._ck(self.L.bdecon_set_plan(self.h, p, int(tile_i), int(tile_j), int(warps)))

    def set_graph(self, enable: bool = True):
        """Run each sweep() call as one CUDA-graph launch (captured once per segment sequence)."""
        self._ck(self.L.bdecon_set_graph(self.h, int(bool(enable))))

    def set_grouping(self, one_launch: bool):
        self._ck(self.L.bdecon_set_grouping(self.h, int(bool(one_launch))))

    def autotune(self, trial_sweeps: int = 2):
        """Time the candidate launch shapes, keep the fastest; chains unchanged."""
        one, ms = C.c_int32(), C.c_double()
        self._ck(self.L.bdecon_autotune(self.h, int(trial_sweeps), C.byref(one), C.byref(ms)))
        return dict(one_launch=bool(one.value), ms_per_sweep=ms.value)

    def get_plan(self, p: int = 0):
        b, w, ti, tj = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
        self._ck(self.L.bdecon_get_plan(self.h, p, C.byref(b), C.byref(w), C.byref(ti), C.byref(tj)))
        return dict(blocks=b.value, warps=w.value, tile_i=ti.value, tile_j=tj.value)

    def set_staging(self, enable: bool = True):
        self._ck(self.L.bdecon_set_staging(self.h, int(bool(enable))))

    def set_lean(self, mode: int = -1):
        """Lean kernel form: -1 automatic (default), 0 never, 1 wherever eligible."""
        self._ck(self.L.bdecon_set_lean(self.h, int(mode)))

    def lean(self, p: int = 0) -> int:
        """1 when problem p's launch group runs the lean kernel form, else 0."""
        v = C.c_int32()
        self._ck(self.L.bdecon_get_lean(self.h, p, C.byref(v)))
        return int(v.value)

    def staged(self, p: int = 0) -> int:
        """1 when problem p's launch group runs with window staging, else 0."""
        v = C.c_int32()
        self._ck(self.L.bdecon_get_staging(self.h, p, C.byref(v)))
        return int(v.value)

    def set_fault(self, silent_block: int, wait_ns: int = 4_000_000_000):
        self._ck(self.L.bdecon_set_fault(self.h, int(silent_block), int(wait_ns)))

    def set_timing(self, enable: bool = True):
        self._ck(self.L.bdecon_set_timing(self.h, int(bool(enable))))

    def sweep_kernel_time(self):
        """(summed device ms, launches) of the sweep kernel since the last call."""
        ms, n = C.c_double(), C.c_int64()
        self._ck(self.L.bdecon_sweep_kernel_time(self.h, C.byref(ms), C.byref(n)))
        return ms.value, int(n.value)

    def launch_count(self) -> int:
        n = C.c_int64()
        self._ck(self.L.bdecon_launch_count(self.h, C.byref(n)))
        return int(n.value)


class Server:
    """The library's serving loop (bdecon_server_*): jobs are queued, admitted
    by device memory and run together in shared launches by a library
    thread; ``result`` blocks until a job is done and returns its posterior
    mean with its (submit, start, finish) host times."""

    def __init__(self, mem_budget: int, max_jobs: int = 64, segment_sweeps: int = 16,
                 precision: int = BDECON_FP32, device: int = 0, one_launch: bool = False):
        self.L = load()
        cfg = _ServerConfig(int(mem_budget), int(max_jobs), int(segment_sweeps), int(precision), int(device),
                            int(bool(one_launch)))
        self.precision = precision
        s = C.c_void_p()
        self._ck(self.L.bdecon_server_start(C.byref(cfg), C.byref(s)))
        self.s = s
        self._shape = {}

    def _ck(self, st):
        if st != 0:
            raise BdeconError(st, self.L.bdecon_last_error(None).decode(errors="replace"))

    def submit(self, problem, sweeps: int) -> int:
        keep = []
        p = _problem(problem, self.precision, sweeps, 0, keep)
        jid = C.c_int64()
        self._ck(self.L.bdecon_server_submit(self.s, C.byref(p), int(sweeps), C.byref(jid)))
        H, W = np.asarray(problem.image).shape
        R = np.asarray(problem.psf).shape[0] // 2
        self._shape[jid.value] = (H + 2 * R, W + 2 * R)
        return int(jid.value)

    def poll(self, job: int):
        """(state, (t_submit, t_start, t_done)) of a job."""
        st = C.c_int32()
        t = np.zeros(3)
        r = self.L.bdecon_server_poll(self.s, int(job), C.byref(st), _p(t), None, 0)
        if r != 0 and st.value != JOB_FAILED:
            self._ck(r)
        return int(st.value), tuple(t)

    def result(self, job: int, timeout: float = 600.0):
        """Block until the job ends; (posterior mean, (t_submit, t_start, t_done))."""
        st = C.c_int32()
        self._ck(self.L.bdecon_server_wait(self.s, int(job), float(timeout), C.byref(st)))
        if st.value not in (JOB_DONE, JOB_FAILED):
            raise TimeoutError(f"job {job} not finished after {timeout} s")
        out = np.empty(self._shape[job])
        t = np.zeros(3)
        self._ck(self.L.bdecon_server_poll(self.s, int(job), C.byref(st), _p(t), _p(out), out.size))
        return out, tuple(t)

    def stats(self):
        q, r, d, seg = C.c_int64(), C.c_int64(), C.c_int64(), C.c_int64()
        m = C.c_size_t()
        self._ck(self.L.bdecon_server_stats(self.s, C.byref(q), C.byref(r), C.byref(d), C.byref(m),
                                            C.byref(seg)))
        return dict(queued=q.value, running=r.value, done=d.value, mem_used=m.value, segments=seg.value)

    def close(self):
        if getattr(self, "s", None):
            self.L.bdecon_server_stop(self.s)
            self.s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
