"""ctypes binding of the plain FP64 C oracle (bdecon_oracle.c).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the CPU
baseline leg of the benchmark are the only callers.  The product path (the
CUDA library and its Python binding) never imports this module.

Each function cites the part of the paper it follows (see the C source for
the definitions written out).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import sys
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bdecon_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no FMA contraction, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
               "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


class OrProblem(C.Structure):
    _fields_ = [("H", C.c_int), ("W", C.c_int), ("L", C.c_int), ("S", C.c_int),
                ("w", C.c_void_p), ("gain", C.c_void_p), ("offset", C.c_void_p),
                ("var", C.c_void_p), ("psf", C.c_void_p),
                ("seed", C.c_uint64), ("chain", C.c_int), ("step", C.c_double),
                ("burn_in", C.c_int), ("refresh_every", C.c_int), ("adapt_target", C.c_double),
                ("aug", C.c_int), ("sub", C.c_int)]


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        dp, ip = C.POINTER(C.c_double), C.POINTER(C.c_int)
        L.or_philox4x32_10.argtypes = [C.POINTER(C.c_uint32), C.POINTER(C.c_uint32), C.POINTER(C.c_uint32)]
        L.or_uniform.argtypes = [C.c_uint32]
        L.or_uniform.restype = C.c_double
        L.or_draw.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, dp, dp]
        L.or_loglik.argtypes = [C.c_double] * 5
        L.or_loglik.restype = C.c_double
        L.or_convolve.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_int, C.c_void_p]
        L.or_patch_dft.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p]
        L.or_alpha.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p]
        L.or_log_prior_patch.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]
        L.or_log_prior_patch.restype = C.c_double
        L.or_log_posterior.argtypes = [C.POINTER(OrProblem), C.c_void_p]
        L.or_log_posterior.restype = C.c_double
        L.or_log_likelihood.argtypes = [C.POINTER(OrProblem), C.c_void_p]
        L.or_log_likelihood.restype = C.c_double
        L.or_eff_kernel.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_void_p]
        L.or_eff_kernel.restype = None
        L.or_expected.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_int, C.c_int, C.c_void_p]
        L.or_expected.restype = None
        L.or_log_joint.argtypes = [C.POINTER(OrProblem), C.c_void_p, C.c_void_p]
        L.or_log_joint.restype = C.c_double
        L.or_sample_phi.argtypes = [C.c_double] * 6
        L.or_sample_phi.restype = C.c_long
        L.or_phi_uniform.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32]
        L.or_phi_uniform.restype = C.c_double
        L.or_logjoint_pixel.argtypes = [C.c_double] * 5 + [C.c_long]
        L.or_logjoint_pixel.restype = C.c_double
        L.or_init.argtypes = [C.POINTER(OrProblem), C.c_void_p]
        L.or_delta.argtypes = [C.POINTER(OrProblem), C.c_void_p, C.c_int, C.c_double, dp, dp]
        L.or_delta.restype = C.c_int
        L.or_run.argtypes = [C.POINTER(OrProblem), C.c_int, C.c_int, C.c_int, C.c_void_p,
                             C.c_void_p, C.c_void_p, C.c_void_p, ip, C.c_void_p, C.c_void_p,
                             C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        L.or_run.restype = C.c_int
        L.or_single_update.argtypes = [C.POINTER(OrProblem), C.c_void_p, C.c_int, C.c_int, ip, dp, dp, dp]
        L.or_single_update.restype = C.c_int
        _lib = L
    return _lib


def _p(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


# ------------------------------------------------------------- primitives --

def philox4x32_10(ctr, key):
    """Philox4x32-10 block (Salmon et al., SC'11) -> 4 uint32."""
    c = (C.c_uint32 * 4)(*[int(x) & 0xffffffff for x in ctr])
    k = (C.c_uint32 * 2)(*[int(x) & 0xffffffff for x in key])
    o = (C.c_uint32 * 4)()
    lib().or_philox4x32_10(c, k, o)
    return [int(x) for x in o]


def uniform(x: int) -> float:
    """((x >> 9) + 1/2) / 2^23, exact in float32."""
    return lib().or_uniform(int(x) & 0xffffffff)


def draw(seed: int, m: int, t: int, chain: int):
    """(z, u) of the proposal at pixel m, sweep t, chain."""
    z, u = C.c_double(), C.c_double()
    lib().or_draw(int(seed), int(m), int(t), int(chain), C.byref(z), C.byref(u))
    return z.value, u.value


def expected(rho, H, W, K, f) -> np.ndarray:
    """Eq. 1 on a lattice f times finer than the camera (oracle)."""
    K = np.ascontiguousarray(K, dtype=np.float64)
    L = K.shape[0]
    Le = L + f - 1
    Ke = np.empty((Le, Le))
    lib().or_eff_kernel(_p(K), L, int(f), _p(Ke))
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    mu = np.empty((H, W))
    lib().or_expected(_p(rho), int(H), int(W), _p(Ke), Le, int(f), _p(mu))
    return mu


def sample_phi(w, o, G, var, mu, u) -> int:
    """Photon count drawn from p(phi | w, mu) by inverse CDF at u."""
    return int(lib().or_sample_phi(float(w), float(o), float(G), float(var), float(mu), float(u)))


def phi_uniform(seed, n, t, chain) -> float:
    return lib().or_phi_uniform(int(seed), int(n), int(t), int(chain))


def logjoint_pixel(w, o, G, var, mu, phi) -> float:
    return lib().or_logjoint_pixel(float(w), float(o), float(G), float(var), float(mu), int(phi))


def loglik(w, o, G, var, mu) -> float:
    """Eq. 6 for one pixel (photon count summed out)."""
    return lib().or_loglik(float(w), float(o), float(G), float(var), float(mu))


def convolve(rho: np.ndarray, K: np.ndarray) -> np.ndarray:
    """Eq. 1-2: valid true convolution of the padded object with K."""
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    K = np.ascontiguousarray(K, dtype=np.float64)
    L = K.shape[0]
    H, W = rho.shape[0] - (L - 1), rho.shape[1] - (L - 1)
    mu = np.empty((H, W))
    lib().or_convolve(_p(rho), H, W, _p(K), L, _p(mu))
    return mu


def patch_dft(x: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float64)
    ph, pw = x.shape
    re, im = np.empty((ph, pw)), np.empty((ph, pw))
    lib().or_patch_dft(_p(x), pw, ph, pw, _p(re), _p(im))
    return re + 1j * im


def alpha(K: np.ndarray, ph: int, pw: int) -> np.ndarray:
    """Eq. 8 hyperparameter |OTF| / sum |OTF| on a ph x pw patch."""
    K = np.ascontiguousarray(K, dtype=np.float64)
    a = np.empty((ph, pw))
    lib().or_alpha(_p(K), K.shape[0], ph, pw, _p(a))
    return a


def log_prior_patch(spec: np.ndarray, a: np.ndarray) -> float:
    re = np.ascontiguousarray(spec.real, dtype=np.float64).ravel()
    im = np.ascontiguousarray(spec.imag, dtype=np.float64).ravel()
    a = np.ascontiguousarray(a, dtype=np.float64).ravel()
    return lib().or_log_prior_patch(_p(re), _p(im), _p(a), a.size)


# ----------------------------------------------------------------- problem --

class Oracle:
    """Oracle view of a ``synth.Problem`` (maps expanded to float64)."""

    def __init__(self, prob, chain: int = 0):
        self.prob = prob
        self.w = np.ascontiguousarray(prob.image, dtype=np.float64)
        g, o, v = prob.maps()
        self.g, self.o, self.v = (np.ascontiguousarray(x) for x in (g, o, v))
        self.psf = np.ascontiguousarray(prob.psf, dtype=np.float64)
        self.c = OrProblem(prob.H, prob.W, prob.L, prob.S, _p(self.w), _p(self.g), _p(self.o),
                           _p(self.v), _p(self.psf), int(prob.seed), int(chain), float(prob.step),
                           int(prob.burn_in), int(prob.refresh_every), float(getattr(prob, "adapt_target", 0.0)),
                           int(bool(getattr(prob, "augmented", False))), int(getattr(prob, "subpixel", 1)))
        self.Ho, self.Wo = prob.object_shape()

    def log_joint(self, rho: np.ndarray, phi: np.ndarray) -> float:
        """Log of the augmented joint density p(w, phi, rho) (Eq. 5 with the prior)."""
        rho = np.ascontiguousarray(rho, dtype=np.float64)
        phi = np.ascontiguousarray(phi, dtype=np.float64)
        return lib().or_log_joint(C.byref(self.c), _p(rho), _p(phi))

    def log_posterior(self, rho: np.ndarray) -> float:
        rho = np.ascontiguousarray(rho, dtype=np.float64)
        assert rho.shape == (self.Ho, self.Wo)
        return lib().or_log_posterior(C.byref(self.c), _p(rho))

    def log_likelihood(self, rho: np.ndarray) -> float:
        """Eq. 6 summed over the camera pixels at the expected image of rho."""
        rho = np.ascontiguousarray(rho, dtype=np.float64)
        assert rho.shape == (self.Ho, self.Wo)
        return lib().or_log_likelihood(C.byref(self.c), _p(rho))

    def log_posterior_fft(self, rho: np.ndarray) -> float:
        """Eq. 9 for large frames: the likelihood as in log_posterior, the patch
        spectra of Eq. 8 taken by numpy's FFT (a library routine standing in
        for the definitional DFT, which costs O(P^4) per patch) and passed to
        the same patch log prior.  Equal to log_posterior up to rounding."""
        rho = np.ascontiguousarray(rho, dtype=np.float64)
        S = self.prob.S
        alphas = {}
        lp = 0.0
        for i0 in range(0, self.Ho, S):
            for j0 in range(0, self.Wo, S):
                x = rho[i0:i0 + S, j0:j0 + S]
                sh = x.shape
                if sh not in alphas:
                    alphas[sh] = alpha(self.psf / self.psf.sum(), sh[0], sh[1])
                lp += log_prior_patch(np.fft.fft2(x), alphas[sh])
        return self.log_likelihood(rho) + lp

    def init(self) -> np.ndarray:
        rho = np.empty((self.Ho, self.Wo))
        lib().or_init(C.byref(self.c), _p(rho))
        return rho

    def delta(self, rho: np.ndarray, m: int, rho_new: float):
        rho = np.ascontiguousarray(rho, dtype=np.float64)
        dl, dp = C.c_double(), C.c_double()
        ok = lib().or_delta(C.byref(self.c), _p(rho), int(m), float(rho_new), C.byref(dl), C.byref(dp))
        return bool(ok), dl.value, dp.value

    def single_update(self, rho: np.ndarray, m: int, t: int):
        """(accept, rho_new, dL, dP) of one update from state rho, local quantities only."""
        rho = np.ascontiguousarray(rho, dtype=np.float64)
        acc, rn, dl, dp = C.c_int(), C.c_double(), C.c_double(), C.c_double()
        lib().or_single_update(C.byref(self.c), _p(rho), int(m), int(t), C.byref(acc), C.byref(rn),
                               C.byref(dl), C.byref(dp))
        return bool(acc.value), rn.value, dl.value, dp.value

    def run(self, T: int, t0: int = 0, rho_in: Optional[np.ndarray] = None, order: int = 0,
            want_acc_log: bool = False, want_samples: bool = False):
        """Run sweeps t0+1..t0+T; returns a dict of numpy results."""
        Ho, Wo, H, W = self.Ho, self.Wo, self.prob.H, self.prob.W
        rho_out, mu_out, sum_out = np.empty((Ho, Wo)), np.empty((H, W)), np.empty((Ho, Wo))
        trace = np.empty(T)
        n_acc = np.empty(T, dtype=np.int64)
        acc = np.empty((T, Ho, Wo), dtype=np.uint8) if want_acc_log else None
        smp = np.empty((T, Ho, Wo)) if want_samples else None
        steps = np.empty((Ho, Wo))
        phi = np.empty((H, W))
        ns = C.c_int()
        rin = None if rho_in is None else np.ascontiguousarray(rho_in, dtype=np.float64)
        lib().or_run(C.byref(self.c), int(t0), int(T), int(order), _p(rin), _p(rho_out), _p(mu_out),
                     _p(sum_out), C.byref(ns), _p(trace), _p(acc), _p(smp), _p(n_acc), _p(steps), _p(phi))
        n = ns.value
        return dict(rho=rho_out, mu=mu_out, sum=sum_out, n_sum=n,
                    mean=(sum_out / n if n > 0 else None), trace=trace, acc_log=acc,
                    samples=smp, n_acc=n_acc, steps=steps, phi=phi)


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
