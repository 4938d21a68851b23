"""Uncertainty maps: the paper's candidate images (kept posterior samples),
their per-pixel quantiles, and the standard deviation and coefficient of
variation of the posterior (Results, "Uncertainty"; Fig. 4).

In double precision the GPU chain is the oracle's chain, so the kept objects
equal the oracle's objects after the same sweeps, and the quantiles equal
numpy's linear-interpolation quantiles of those objects (a library routine
applied to the oracle's output).  In single precision the device sort is
checked against numpy on the chain's own kept objects, with enough values
per pixel to exercise every stage of the sorting network.
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
Q = [0.0, 0.025, 0.25, 0.5, 0.75, 0.975, 1.0]


def _problem():
    p = synth.small_problem(H=20, W=24, L=5, maps=True, seed=71, n_chains=2, burn_in=3, refresh_every=5)
    p.sample_every, p.n_samples = 2, 5
    return p


def test_fp64_kept_objects_quantiles_std_cv_match_oracle():
    p = _problem()
    T = 16
    s = bdecon.Sampler(p, precision=bdecon.BDECON_FP64, max_sweeps=T + 4, flags=bdecon.FLAG_SECOND_MOMENT)
    s.sweep(T)
    kept = [s.samples(0, c) for c in range(p.n_chains)]
    qs = s.posterior_quantiles(Q)
    qs_crop = s.posterior_quantiles(Q, crop=True)
    std, cv, mean = s.posterior_std(), s.posterior_cv(), s.posterior_mean()
    s.close()
    # sweeps t = 5, 7, 9, 11, 13 are kept (every 2nd past burn-in 3; 5 slots)
    t_kept = [5, 7, 9, 11, 13]
    ref_kept, ref_all = [], []
    for c in range(p.n_chains):
        r = O.Oracle(p, chain=c).run(T, want_samples=True)
        assert kept[c].shape == (len(t_kept),) + p.object_shape()
        ref = r["samples"][[t - 1 for t in t_kept]]
        np.testing.assert_allclose(kept[c], ref, rtol=RTOL)
        ref_kept.append(ref)
        ref_all.append(r["samples"][p.burn_in:])
    pooled = np.concatenate(ref_kept)
    want = np.quantile(pooled, Q, axis=0)
    np.testing.assert_allclose(qs, want, rtol=RTOL)
    R = p.L // 2
    np.testing.assert_allclose(qs_crop, want[:, R:-R, R:-R], rtol=RTOL)
    x = np.concatenate(ref_all)
    np.testing.assert_allclose(mean, x.mean(axis=0), rtol=RTOL)
    np.testing.assert_allclose(std, x.std(axis=0), rtol=1e-7, atol=1e-10)
    np.testing.assert_allclose(cv, x.std(axis=0) / x.mean(axis=0), rtol=1e-7, atol=1e-10)


def test_fp32_device_quantiles_match_numpy_on_many_values():
    # 3 chains x 110 kept objects = 330 values per pixel (padded to 512, two
    # elements per thread in every stage of the network)
    p = synth.small_problem(H=14, W=15, L=3, seed=72, n_chains=3, burn_in=10, refresh_every=25)
    p.sample_every, p.n_samples = 1, 110
    s = bdecon.Sampler(p, precision=bdecon.BDECON_FP32, max_sweeps=130)
    s.sweep(125)                         # 115 past burn-in, 110 slots: the last 5 are not kept
    kept = np.concatenate([s.samples(0, c) for c in range(3)])
    assert kept.shape[0] == 330
    qs = s.posterior_quantiles(Q + [0.333, 0.9])
    s.close()
    np.testing.assert_allclose(qs, np.quantile(kept, Q + [0.333, 0.9], axis=0), rtol=RTOL)


def test_resume_drops_objects_kept_before_the_resume_point():
    p = _problem()
    s = bdecon.Sampler(p, precision=bdecon.BDECON_FP64, max_sweeps=40)
    s.sweep(9)                           # kept: t = 5, 7, 9
    assert s.samples(0, 0).shape[0] == 3
    rho, t = s.get_state(0, 0)
    s.set_state(rho, t, 0, 0)
    assert s.samples(0, 0).shape[0] == 0
    with pytest.raises(bdecon.BdeconError, match="no object kept"):
        s.posterior_quantiles([0.5])
    s.sweep(4)                           # t = 11, 13
    assert s.samples(0, 0).shape[0] == 2
    s.close()


def test_quantile_arguments_are_checked():
    p = _problem()
    s = bdecon.Sampler(p, precision=bdecon.BDECON_FP32, max_sweeps=12)
    s.sweep(6)
    for bad in ([1.5], [-0.1], [float("nan")], [0.5] * 65):
        with pytest.raises(bdecon.BdeconError):
            s.posterior_quantiles(bad)
    s.close()
    q = synth.small_problem(H=10, W=10, L=3, seed=73)
    s = bdecon.Sampler(q, precision=bdecon.BDECON_FP32, max_sweeps=8)
    s.sweep(3)
    with pytest.raises(bdecon.BdeconError, match="n_samples"):
        s.posterior_quantiles([0.5])
    with pytest.raises(bdecon.BdeconError, match="SECOND_MOMENT"):
        s.posterior_cv()
    s.close()
