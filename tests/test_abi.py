"""C-ABI checks that need no GPU: the library builds, loads and exports every
function include/bdecon.h declares; argument validation refuses bad
problems with a message and leaves nothing allocated; the workspace size is
computed on the host."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2411_00991_gb300 import bdecon, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "bdecon.h")).read()
    return sorted(set(re.findall(r"\b(bdecon_[a-z0-9_]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    L = bdecon.load()
    names = _declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(bdecon.EXPORTS)


def _problem_struct(prob, **over):
    s = bdecon.Sampler.__new__(bdecon.Sampler)
    img = np.ascontiguousarray(prob.image, dtype=np.float32)
    psf = np.ascontiguousarray(prob.psf, dtype=np.float64)
    keep = [img, psf]
    p = bdecon._Problem(prob.H, prob.W, img.ctypes.data, prob.L, psf.ctypes.data, None, 2.0, None, 100.0,
                        None, 2.56, 0, 1, 0, 0.2, 0, 10, bdecon.BDECON_FP32, 64, 0, 0, 0, 0, 0.0, 0)
    for k, v in over.items():
        setattr(p, k, v)
    return p, keep


@pytest.mark.parametrize("field,value,msg", [
    ("L", 4, "odd"),
    ("L", 65, "odd"),
    ("stride", 3, "stride"),
    ("n_chains", 0, "n_chains"),
    ("precision", 7, "precision"),
    ("gain", -1.0, "gain"),
    ("read_var", 0.0, "read_var"),
    ("H", 0, "frame size"),
    ("step", float("nan"), "step"),
    ("refresh_every", -1, "negative"),
    ("team_warps", 9, "team_warps"),
    ("n_samples", -1, "n_samples"),
    ("adapt_target", 1.0, "adapt_target"),
    ("adapt_target", float("nan"), "adapt_target"),
    ("subpixel", 9, "subpixel"),
])
def test_invalid_problem_refused(field, value, msg):
    L = bdecon.load()
    prob = synth.small_problem(H=8, W=9, L=5)
    p, keep = _problem_struct(prob, **{field: value})
    h = C.c_void_p()
    st = L.bdecon_create(C.byref(p), None, C.byref(h))
    assert st == 1
    assert h.value is None
    assert msg in L.bdecon_last_error(None).decode()
    n = C.c_size_t()
    assert L.bdecon_workspace_size(C.byref(p), 1, C.byref(n)) == 1


def test_bad_psf_and_image_refused():
    L = bdecon.load()
    prob = synth.small_problem(H=8, W=9, L=5)
    prob.psf = -prob.psf
    p, keep = _problem_struct(prob)
    h = C.c_void_p()
    assert L.bdecon_create(C.byref(p), None, C.byref(h)) == 1
    assert "PSF" in L.bdecon_last_error(None).decode()
    prob = synth.small_problem(H=8, W=9, L=5)
    prob.image = prob.image.copy()
    prob.image[3, 4] = np.nan
    p, keep = _problem_struct(prob)
    assert L.bdecon_create(C.byref(p), None, C.byref(h)) == 1
    assert "image" in L.bdecon_last_error(None).decode()


def test_null_handle_calls_are_refused():
    L = bdecon.load()
    assert L.bdecon_sweep(None, 1) == 1
    assert L.bdecon_sync(None) == 1
    n = C.c_int64()
    assert L.bdecon_launch_count(None, C.byref(n)) == 1
    L.bdecon_destroy(None)


def test_workspace_size_grows_with_kept_objects():
    prob = synth.small_problem(H=30, W=31, L=5)
    a = bdecon.Sampler.workspace_size(prob)
    prob.n_samples = 10
    b = bdecon.Sampler.workspace_size(prob)
    assert b - a >= 10 * (30 + 4) * (31 + 4) * 4


def test_workspace_size_grows_with_chains():
    prob = synth.small_problem(H=30, W=31, L=5)
    a = bdecon.Sampler.workspace_size(prob)
    prob.n_chains = 3
    b = bdecon.Sampler.workspace_size(prob)
    assert b > a > 30 * 31 * 4
    assert a % 256 == 0


@pytest.mark.parametrize("field,value", [("max_jobs", 0), ("segment_sweeps", 0), ("segment_sweeps", 65),
                                         ("mem_budget", 0), ("precision", 5)])
def test_bad_server_config_refused(field, value):
    L = bdecon.load()
    cfg = bdecon._ServerConfig(1 << 30, 4, 8, bdecon.BDECON_FP32, 0, 0)
    setattr(cfg, field, value)
    s = C.c_void_p()
    assert L.bdecon_server_start(C.byref(cfg), C.byref(s)) == 1
    assert s.value is None
    assert "server config" in L.bdecon_last_error(None).decode()
