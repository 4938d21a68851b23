"""The allocation-free entry point bdecon_log_posterior_static.

Some callers cannot allocate device memory while they run (all device
memory reserved up front for frame buffers, or a device allocator owned by
another framework).  For them the library evaluates the log posterior of an
object with its scratch in a fixed array inside the library.  These tests
call it through the C ABI with device buffers the test itself allocated and
compare it with the handle-based bdecon_log_posterior and with the CPU
oracle's Eq. 9, at the 1e-12 relative tolerance of the double-precision
parity tests, on consecutive calls (the scratch keeps the previous call's
contents), and check that warm calls leave the device's free memory
unchanged.
"""
import ctypes as C

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


def _handle_value(prob, rho):
    s = bdecon.Sampler(prob, precision=bdecon.BDECON_FP64, max_sweeps=4)
    s.set_state(rho, 0)
    v = s.log_posterior()
    s.close()
    return v


def _dev(x, dtype):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda")


def _static_value(prob, rho, out):
    img = _dev(prob.image, torch.float32)
    psf = _dev(prob.psf, torch.float64)
    r = _dev(rho, torch.float64)
    keep = [img, psf, r]

    def arg(v):
        if np.isscalar(v):
            return float(v)
        t = _dev(v, torch.float32)
        keep.append(t)
        return ("map", t.data_ptr())

    out.fill_(float("nan"))
    bdecon.log_posterior_static(prob.H, prob.W, img.data_ptr(), prob.L, psf.data_ptr(), arg(prob.gain),
                                arg(prob.offset), arg(prob.var), prob.stride, r.data_ptr(), out.data_ptr(),
                                torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return float(out.item())


def test_static_matches_handle_on_consecutive_calls():
    a = synth.small_problem(H=40, W=37, L=7, maps=True, stride=9, seed=31)   # ragged patches, sCMOS maps
    b = synth.small_problem(H=23, W=29, L=5, seed=32)                        # scalar camera, other size
    rho_a = synth.random_state(a, 4)
    rho_b = synth.random_state(b, 5)
    ref_a, ref_b = _handle_value(a, rho_a), _handle_value(b, rho_b)
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    first = _static_value(a, rho_a, out)
    second = _static_value(a, rho_a, out)
    assert first == pytest.approx(ref_a, rel=RTOL)
    assert second == pytest.approx(ref_a, rel=RTOL)
    third = _static_value(b, rho_b, out)          # a smaller problem after a larger one
    assert third == pytest.approx(ref_b, rel=RTOL)
    # the oracle's Eq. 9 of the same objects
    assert first == pytest.approx(O.Oracle(a).log_posterior(rho_a), rel=RTOL)
    assert third == pytest.approx(O.Oracle(b).log_posterior(rho_b), rel=RTOL)


def test_static_warm_calls_leave_free_device_memory_unchanged():
    # every device buffer is made before the measured calls, so only the
    # entry point itself could change the device's free memory
    a = synth.small_problem(H=33, W=30, L=5, maps=True, seed=33)
    rho = synth.random_state(a, 6)
    img, psf, r = _dev(a.image, torch.float32), _dev(a.psf, torch.float64), _dev(rho, torch.float64)
    off, var = _dev(a.offset, torch.float32), _dev(a.var, torch.float32)
    out = torch.empty(4, dtype=torch.float64, device="cuda")
    st = torch.cuda.current_stream().cuda_stream

    def call(k):
        bdecon.log_posterior_static(a.H, a.W, img.data_ptr(), a.L, psf.data_ptr(), float(a.gain),
                                    ("map", off.data_ptr()), ("map", var.data_ptr()), a.stride, r.data_ptr(),
                                    out[k:].data_ptr(), st)

    call(0)                                       # set-up: the scratch address is looked up
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for k in (1, 2, 3):
        call(k)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    v = out.cpu().numpy()
    assert v[0] == pytest.approx(O.Oracle(a).log_posterior(rho), rel=RTOL)
    assert (v[1:] == v[0]).all()


def test_static_refuses_problems_beyond_its_scratch():
    L = bdecon.load()
    dummy = torch.zeros(4, dtype=torch.float64, device="cuda")
    p = C.c_void_p(dummy.data_ptr())
    st = L.bdecon_log_posterior_static(12000, 12000, p, 5, p, None, 2.0, None, 100.0, None, 2.56, 0, p, p, None)
    assert st == 1
    assert "static scratch" in L.bdecon_last_error(None).decode()
