"""Seeded synthetic microscopy inputs for the deconvolution sampler.

This module only *simulates data*: it draws a ground-truth object, a
pixel-integrated Gaussian PSF and a noisy camera frame following the
image-formation model of the paper's Methods (Eq. 1-4: blur, Poisson
photon emission, gain/offset/read noise).  It holds none of the sampler's
arithmetic (no likelihood, prior, proposal or update), so both the CUDA
path and the CPU oracle consume exactly the same arrays from here.

Workload shapes follow the paper's experiments (Results, "Simulated Data"
and "Experimental Data": NA 1.3-1.4 Gaussian/Airy-like PSFs at 65 nm pixels,
sCMOS offset ~100 ADU and gain ~2 ADU/e-, up to ~150 photons per pixel).
The paper's own images (TestImages.jl object, HeLa mitochondria frames) are
not available; these synthetic objects stand in for them.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np


@dataclasses.dataclass
class Problem:
    """One deconvolution problem: a camera frame plus calibration and PSF.

    Arrays are host numpy arrays.  ``gain``/``offset``/``var`` are either
    float scalars or (H, W) float32 maps (the paper allows both, Methods
    after Eq. 4).  ``psf`` is (L, L) float64, L odd, not necessarily
    normalised.  ``truth`` is the (H+2R, W+2R) object used to simulate the
    frame (for sanity checks only; the sampler never sees it).
    """
    image: np.ndarray            # (H, W) float32, ADU
    psf: np.ndarray              # (L, L) float64
    gain: object = 2.0
    offset: object = 100.0
    var: object = 2.56
    stride: int = 0              # 0 -> L
    n_chains: int = 1
    seed: int = 0
    step: float = 0.2
    burn_in: int = 0
    refresh_every: int = 50
    truth: Optional[np.ndarray] = None
    name: str = ""
    team_warps: int = 0          # 0 -> chosen by the library from the problem alone
    sample_every: int = 0        # keep every k-th post-burn-in object (0 -> 1)
    n_samples: int = 0           # kept objects per chain (0 -> none)
    adapt_target: float = 0.0    # > 0: adapt each pixel's proposal scale during burn-in toward this acceptance
    augmented: bool = False      # photon-count augmented sampler (completed likelihood, Eq. 5)
    subpixel: int = 1            # object lattice cells per camera pixel side (psf given on that lattice)

    @property
    def H(self) -> int:
        return int(self.image.shape[0])

    @property
    def W(self) -> int:
        return int(self.image.shape[1])

    @property
    def L(self) -> int:
        return int(self.psf.shape[0])

    @property
    def R(self) -> int:
        return self.L // 2

    @property
    def S(self) -> int:
        # the default stride covers the camera window of one update (L + f - 1)
        return self.stride if self.stride else self.L + max(1, int(self.subpixel)) - 1

    def maps(self):
        """(gain, offset, var) expanded to float64 (H, W) maps."""
        out = []
        for v in (self.gain, self.offset, self.var):
            if np.isscalar(v):
                out.append(np.full((self.H, self.W), float(v), dtype=np.float64))
            else:
                out.append(np.asarray(v, dtype=np.float64))
        return tuple(out)

    def object_shape(self):
        f = max(1, int(self.subpixel))
        return (f * self.H + 2 * self.R, f * self.W + 2 * self.R)


# ---------------------------------------------------------------- PSF ----

def gaussian_psf(sigma: float, L: int) -> np.ndarray:
    """Gaussian PSF integrated over each unit pixel (erf differences), truncated
    to L x L and normalised to sum 1.  Pixel integration of the PSF is the
    A_n integral of Eq. 1."""
    if L % 2 != 1:
        raise ValueError("L must be odd")
    R = L // 2
    x = np.arange(-R, R + 1, dtype=np.float64)
    s = sigma * math.sqrt(2.0)
    erf = np.vectorize(math.erf)
    prof = 0.5 * (erf((x + 0.5) / s) - erf((x - 0.5) / s))
    k = np.outer(prof, prof)
    return k / k.sum()


def airy_psf(na: float, wavelength_nm: float, pixel_nm: float, L: int, sub: int = 16) -> np.ndarray:
    """Airy PSF of a circular pupil, (2 J1(x) / x)^2 with x = 2 pi NA r / lambda
    (r in nm), integrated over each pixel by a sub x sub midpoint rule,
    truncated to L x L and normalised to sum 1 (the pixel integral of Eq. 1)."""
    from scipy.special import j1
    if L % 2 != 1:
        raise ValueError("L must be odd")
    R = L // 2
    off = (np.arange(sub) + 0.5) / sub - 0.5
    coords = (np.arange(-R, R + 1)[:, None] + off[None, :]).ravel() * pixel_nm
    yy, xx = np.meshgrid(coords, coords, indexing="ij")
    x = 2.0 * math.pi * na * np.hypot(yy, xx) / wavelength_nm
    with np.errstate(invalid="ignore", divide="ignore"):
        amp = np.where(x > 1e-12, 2.0 * j1(x) / x, 1.0)
    inten = (amp * amp).reshape(L, sub, L, sub).sum(axis=(1, 3))
    return inten / inten.sum()


def psf_sigma_from_optics(na: float, wavelength_nm: float, pixel_nm: float) -> float:
    """Gaussian approximation of the Airy core, sigma = 0.21 lambda / NA, in pixels."""
    return 0.21 * wavelength_nm / na / pixel_nm


# ------------------------------------------------------------- objects ----

def _blobs(shape, n, sig_lo, sig_hi, amp_lo, amp_hi, rng):
    Hh, Ww = shape
    yy, xx = np.mgrid[0:Hh, 0:Ww].astype(np.float64)
    out = np.zeros(shape)
    for _ in range(n):
        cy, cx = rng.uniform(0, Hh), rng.uniform(0, Ww)
        s = rng.uniform(sig_lo, sig_hi)
        a = rng.uniform(amp_lo, amp_hi)
        r = int(math.ceil(4 * s))
        y0, y1 = max(0, int(cy) - r), min(Hh, int(cy) + r + 1)
        x0, x1 = max(0, int(cx) - r), min(Ww, int(cx) + r + 1)
        out[y0:y1, x0:x1] += a * np.exp(-((yy[y0:y1, x0:x1] - cy) ** 2 +
                                          (xx[y0:y1, x0:x1] - cx) ** 2) / (2 * s * s))
    return out


def _lines(shape, n, rng):
    Hh, Ww = shape
    out = np.zeros(shape)
    for _ in range(n):
        y0, x0, y1, x1 = rng.uniform(0, Hh), rng.uniform(0, Ww), rng.uniform(0, Hh), rng.uniform(0, Ww)
        steps = int(max(abs(y1 - y0), abs(x1 - x0))) + 1
        ys = np.clip(np.rint(np.linspace(y0, y1, steps)).astype(int), 0, Hh - 1)
        xs = np.clip(np.rint(np.linspace(x0, x1, steps)).astype(int), 0, Ww - 1)
        out[ys, xs] = 1.0
    return out


def _filaments(shape, n, len_lo, len_hi, rng):
    """1-pixel-wide smooth random curves (direction random walk)."""
    Hh, Ww = shape
    out = np.zeros(shape)
    for _ in range(n):
        y, x = rng.uniform(0, Hh), rng.uniform(0, Ww)
        th = rng.uniform(0, 2 * math.pi)
        length = int(rng.uniform(len_lo, len_hi))
        dth = rng.normal(0.0, 0.08, size=length)
        for k in range(length):
            iy, ix = int(y), int(x)
            if 0 <= iy < Hh and 0 <= ix < Ww:
                out[iy, ix] = 1.0
            th += dth[k]
            y += math.sin(th)
            x += math.cos(th)
    return out


def _scale(struct, peak, background):
    m = struct.max()
    if m <= 0:
        return np.full(struct.shape, float(background))
    return background + struct * ((peak - background) / m)


# -------------------------------------------------------------- camera ----

def expected_image(truth: np.ndarray, psf: np.ndarray, subpixel: int = 1) -> np.ndarray:
    """Eq. 1 for the generator: valid blur of the padded object on its lattice,
    then the f x f lattice cells of each camera pixel summed (f = subpixel)."""
    from scipy.signal import fftconvolve
    fine = fftconvolve(truth, psf, mode="valid")
    f = max(1, int(subpixel))
    if f == 1:
        return fine
    H, W = fine.shape[0] // f, fine.shape[1] // f
    return fine[:H * f, :W * f].reshape(H, f, W, f).sum(axis=(1, 3))


def simulate_frame(truth: np.ndarray, psf: np.ndarray, gain, offset, var,
                   rng: np.random.Generator, subpixel: int = 1) -> np.ndarray:
    """Camera frame from the object (Eq. 1-4): valid blur of the padded object,
    binned to camera pixels, Poisson photons, gain and offset, Gaussian read
    noise; float32 ADU, not rounded."""
    mu = expected_image(truth, psf, subpixel)
    mu = np.maximum(mu, 0.0)
    phot = rng.poisson(mu).astype(np.float64)
    g = np.asarray(gain, dtype=np.float64)
    o = np.asarray(offset, dtype=np.float64)
    v = np.asarray(var, dtype=np.float64)
    w = g * phot + o + rng.normal(0.0, 1.0, size=mu.shape) * np.sqrt(v)
    return w.astype(np.float32)


def scmos_maps(H, W, rng, offset_mean=100.0, offset_sd=2.0, var_shape=2.0, var_scale=1.0):
    """Per-pixel sCMOS offset map ~ N(100, 2) ADU and variance map ~ Gamma(2, 1) ADU^2."""
    off = rng.normal(offset_mean, offset_sd, size=(H, W)).astype(np.float32)
    var = rng.gamma(var_shape, var_scale, size=(H, W)).astype(np.float32)
    var = np.maximum(var, np.float32(1e-3))
    return off, var


# ------------------------------------------------------------- workloads ----

def small_problem(H=20, W=24, L=5, sigma=1.0, peak=20.0, background=2.0,
                  seed=7, maps=False, stride=0, n_chains=1, refresh_every=7,
                  burn_in=0, step=0.2, subpixel=1) -> Problem:
    """A few-tile problem for parity tests (ragged patch tail when the padded
    size is not a multiple of the stride).  With subpixel = f the object lives
    on a lattice f times finer than the camera (PSF side L and sigma in
    lattice units), the photon levels per camera pixel unchanged."""
    rng = np.random.default_rng(seed)
    R = L // 2
    f = max(1, int(subpixel))
    shape = (f * H + 2 * R, f * W + 2 * R)
    struct = _blobs(shape, max(2, H * W // 120), 1.0 * f, 2.5 * f, 0.3, 1.0, rng) + _lines(shape, 2, rng)
    truth = _scale(struct, peak, background) / (f * f)
    psf = gaussian_psf(sigma, L)
    if maps:
        off, var = scmos_maps(H, W, rng)
        gain = 2.1
    else:
        off, var, gain = 100.0, 2.56, 2.0
    img = simulate_frame(truth, psf, gain, off, var, rng, subpixel=f)
    return Problem(image=img, psf=psf, gain=gain, offset=off, var=var, stride=stride,
                   n_chains=n_chains, seed=seed, step=step, burn_in=burn_in,
                   refresh_every=refresh_every, truth=truth, name=f"small{H}x{W}L{L}f{f}",
                   subpixel=f)


def widefield_64(seed=0) -> Problem:
    """64x64 frame, 12 Gaussian blobs (sigma 1-3 px) + 3 one-pixel lines, peak 20,
    background 2 photons/px; Gaussian PSF sigma 1.5 px on 9x9; gain 2.0,
    offset 100 ADU, read-noise sd 1.6 ADU; 1 chain."""
    rng = np.random.default_rng(seed)
    L, sigma = 9, 1.5
    R = L // 2
    shape = (64 + 2 * R, 64 + 2 * R)
    struct = _blobs(shape, 12, 1.0, 3.0, 0.3, 1.0, rng) + _lines(shape, 3, rng)
    truth = _scale(struct, 20.0, 2.0)
    psf = gaussian_psf(sigma, L)
    img = simulate_frame(truth, psf, 2.0, 100.0, 1.6 ** 2, rng)
    return Problem(image=img, psf=psf, gain=2.0, offset=100.0, var=1.6 ** 2,
                   n_chains=1, seed=seed, refresh_every=50, burn_in=100,
                   truth=truth, name="widefield64_L9")


def _filament_frame(side, n_fil, n_blob, peak, background, sigma, L, seed, gain=2.1):
    rng = np.random.default_rng(seed)
    R = L // 2
    shape = (side + 2 * R, side + 2 * R)
    struct = _filaments(shape, n_fil, 20, 200, rng) + _blobs(shape, n_blob, 1.0, 3.0, 0.3, 1.0, rng)
    truth = _scale(struct, peak, background)
    psf = gaussian_psf(sigma, L)
    off, var = scmos_maps(side, side, rng)
    img = simulate_frame(truth, psf, gain, off, var, rng)
    return img, psf, gain, off, var, truth


def widefield_512(seed=1) -> Problem:
    """512x512 sCMOS frame: 200 filaments + 50 blobs, peak 50, background 1
    photons/px; Gaussian approximation of the NA 1.4 / 520 nm / 65 nm Airy core
    (sigma ~1.2 px) on 17x17; offset map N(100, 2) ADU, variance map
    Gamma(2, 1) ADU^2, gain 2.1."""
    sigma = psf_sigma_from_optics(1.4, 520.0, 65.0)
    img, psf, gain, off, var, truth = _filament_frame(512, 200, 50, 50.0, 1.0, sigma, 17, seed)
    return Problem(image=img, psf=psf, gain=gain, offset=off, var=var, n_chains=1,
                   seed=seed, refresh_every=50, burn_in=1000, truth=truth,
                   name="widefield512_L17")


def lowsnr_2048(seed=2, crop: Optional[int] = None) -> Problem:
    """2048x2048 low-SNR frame: 3200 filaments + 800 blobs, peak 5, background 1
    photons/px; Gaussian PSF sigma 4 px on 31x31; sCMOS maps as the 512 frame;
    4 chains, refresh every 50 sweeps.  ``crop`` generates the same recipe at
    crop x crop (filament/blob counts scaled by area) as its own problem."""
    side = 2048 if crop is None else int(crop)
    frac = (side / 2048.0) ** 2
    img, psf, gain, off, var, truth = _filament_frame(
        side, max(1, int(round(3200 * frac))), max(1, int(round(800 * frac))),
        5.0, 1.0, 4.0, 31, seed)
    return Problem(image=img, psf=psf, gain=gain, offset=off, var=var, n_chains=4,
                   seed=seed, refresh_every=50, burn_in=500, truth=truth,
                   name=f"lowsnr{side}_L31")


def batch_uneven(n_images=64, seed0=3000, sides=(128, 256, 384, 512, 768, 1024),
                 n_chains=4) -> List[Problem]:
    """Batch of uneven frames: side uniform from ``sides``, PSF sigma U[1, 4] px
    with support 2*ceil(3 sigma)+1, peak log-U[3, 200], background 1, camera
    scalars gain 2.0 / offset 100 / read sd 1.6; 4 chains each."""
    return [batch_frame(i, seed0, sides, n_chains) for i in range(n_images)]


def batch_frame(i, seed0=3000, sides=(128, 256, 384, 512, 768, 1024), n_chains=4) -> Problem:
    """Frame i of ``batch_uneven`` alone (each frame depends only on seed0 + i)."""
    rng = np.random.default_rng(seed0 + i)
    side = int(rng.choice(sides))
    sigma = float(rng.uniform(1.0, 4.0))
    L = 2 * int(math.ceil(3 * sigma)) + 1
    peak = float(math.exp(rng.uniform(math.log(3.0), math.log(200.0))))
    R = L // 2
    shape = (side + 2 * R, side + 2 * R)
    frac = (side / 512.0) ** 2
    struct = _filaments(shape, max(1, int(200 * frac)), 20, 200, rng) + \
        _blobs(shape, max(1, int(50 * frac)), 1.0, 3.0, 0.3, 1.0, rng)
    truth = _scale(struct, peak, 1.0)
    psf = gaussian_psf(sigma, L)
    img = simulate_frame(truth, psf, 2.0, 100.0, 1.6 ** 2, rng)
    return Problem(image=img, psf=psf, gain=2.0, offset=100.0, var=1.6 ** 2,
                   n_chains=n_chains, seed=seed0 + i, refresh_every=50,
                   burn_in=250, truth=truth, name=f"batch{i}_{side}_L{L}")


def serving_arrivals(n_jobs=300, rate=20.0, seed=4, lo=128, hi=2048):
    """Poisson arrival times (s) and job sides (log-uniform in [lo, hi], rounded
    to multiples of 32) with PSF sigma U[1, 4]."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=n_jobs))
    sides = np.exp(rng.uniform(math.log(lo), math.log(hi), size=n_jobs))
    sides = np.maximum(32, (np.rint(sides / 32.0) * 32).astype(int))
    sig = rng.uniform(1.0, 4.0, size=n_jobs)
    return t, sides, sig


def serving_job(side: int, sigma: float, seed: int, n_chains: int = 1) -> Problem:
    """One serving job: filament frame of the given side with sCMOS maps."""
    L = 2 * int(math.ceil(3 * sigma)) + 1
    frac = (side / 512.0) ** 2
    img, psf, gain, off, var, truth = _filament_frame(
        side, max(1, int(200 * frac)), max(1, int(50 * frac)), 50.0, 1.0, sigma, L, seed)
    return Problem(image=img, psf=psf, gain=gain, offset=off, var=var, n_chains=n_chains,
                   seed=seed, refresh_every=50, burn_in=250, truth=truth,
                   name=f"job{seed}_{side}_L{L}")


def random_state(prob: Problem, seed: int, lo=0.2, hi=30.0) -> np.ndarray:
    """A seeded positive object (H+2R, W+2R) float64 for evaluation tests."""
    rng = np.random.default_rng(seed)
    return np.exp(rng.uniform(math.log(lo), math.log(hi), size=prob.object_shape()))
