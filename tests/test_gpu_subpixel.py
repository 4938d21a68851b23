"""Object lattice finer than the camera (subpixel f > 1) on the GPU.

Each camera pixel sums the f x f lattice cells of its area (Eq. 1), so an
update's window is the camera pixels its effective kernel (PSF (x) box_f)
reaches at the pixel's sub-cell phase.  Double precision: the GPU chain is
the oracle's chain (identical accept decisions; object, expected image and
trace within 1e-12) for f = 2 and 3, sCMOS maps, two chains, the augmented
sampler; batches mixing f = 1 and f = 2 and another launch plan give
bit-identical chains in both precisions; the cropped maps are f H x f W.
"""
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


@pytest.mark.parametrize("kw", [
    dict(H=12, W=14, L=3, seed=131, subpixel=2, refresh_every=4),
    dict(H=10, W=9, L=5, seed=132, subpixel=2, maps=True, n_chains=2, burn_in=2),
    dict(H=8, W=9, L=3, seed=133, subpixel=3, maps=True),
    dict(H=9, W=11, L=3, seed=134, subpixel=2, stride=6),
])
@pytest.mark.parametrize("augmented", [False, True])
def test_fp64_fine_lattice_chain_matches_oracle(kw, augmented):
    p = synth.small_problem(**kw)
    p.augmented = augmented
    T = 10
    s = bdecon.Sampler(p, precision=bdecon.BDECON_FP64, max_sweeps=T + 4, flags=bdecon.FLAG_ACCEPT_LOG)
    s.sweep(T)
    for c in range(p.n_chains):
        ref = O.Oracle(p, chain=c).run(T, want_acc_log=True)
        mism = np.argwhere(s.accept_log(0, c) != ref["acc_log"])
        assert mism.size == 0, f"{len(mism)} accept decisions differ, first {mism[:3]}"
        np.testing.assert_allclose(s.get_state(0, c)[0], ref["rho"], rtol=RTOL)
        np.testing.assert_allclose(s.get_mu(0, c), ref["mu"], rtol=RTOL)
        np.testing.assert_allclose(s.trace(0, c), ref["trace"], rtol=RTOL)
    f = p.subpixel
    assert s.posterior_mean(crop=True).shape == (f * p.H, f * p.W) if T > p.burn_in else True
    s.close()


@pytest.mark.parametrize("precision", [bdecon.BDECON_FP64, bdecon.BDECON_FP32])
def test_fine_lattice_in_batches_and_plans_is_bit_identical(precision):
    probs = [synth.small_problem(H=12, W=14, L=3, seed=135, subpixel=2, refresh_every=4, burn_in=2),
             synth.small_problem(H=17, W=13, L=3, seed=136, refresh_every=4, burn_in=2),
             synth.small_problem(H=10, W=9, L=5, seed=137, subpixel=2, maps=True, refresh_every=4, burn_in=2)]
    T = 8
    ref = []
    for pr in probs:
        a = bdecon.Sampler(pr, precision=precision, max_sweeps=T)
        a.sweep(T)
        ref.append((a.get_state()[0], a.trace(), a.posterior_mean()))
        a.close()
    for mode in ("batch", "plan"):
        b = bdecon.Sampler(probs, precision=precision, max_sweeps=T)
        if mode == "plan":
            b.set_plan(2, 2, 4, p=2)
        b.sweep(T)
        for k in range(len(probs)):
            got = (b.get_state(k)[0], b.trace(k), b.posterior_mean(k))
            for x, y in zip(got, ref[k]):
                np.testing.assert_array_equal(x, y, err_msg=f"{mode} problem {k}")
        b.close()
