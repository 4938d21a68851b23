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
        out.append((rho, s.trace(p, c), s.get_mu(p, c), s.accept_counts(p, c)))
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
