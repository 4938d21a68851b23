"""Pins of the oracle's counter-based random numbers (no GPU).

Philox4x32-10 is checked against the published known-answer vectors; the
23-bit uniform mapping against its closed form; Box-Muller normals and the
uniforms against their distributions.
"""
import math
import os

import numpy as np
import pytest
from scipy import stats

from oracle import oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat():
    rows = []
    for line in open(GOLD):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        v = [int(x, 16) for x in line.split()]
        rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,out", _kat())
def test_philox_known_answers(ctr, key, out):
    assert O.philox4x32_10(ctr, key) == out


def test_uniform_closed_form():
    assert O.uniform(0) == 0.5 / 2 ** 23
    assert O.uniform(0xFFFFFFFF) == 1.0 - 0.5 / 2 ** 23
    assert O.uniform(0x80000000) == (2 ** 22 + 0.5) / 2 ** 23
    rng = np.random.default_rng(1)
    for x in rng.integers(0, 2 ** 32, size=400, dtype=np.uint64):
        x = int(x)
        # the low 9 bits are dropped; u(x) + u(~x) == 1 (symmetry)
        assert O.uniform(x) == O.uniform(x & 0xFFFFFE00)
        assert O.uniform(x) + O.uniform(x ^ 0xFFFFFFFF) == 1.0
        # exact in float32
        assert float(np.float32(O.uniform(x))) == O.uniform(x)


def test_draws_distribution():
    n = 40000
    zs = np.empty(n)
    us = np.empty(n)
    for m in range(n):
        zs[m], us[m] = O.draw(12345, m, 3, 1)
    assert abs(zs.mean()) < 4.0 / math.sqrt(n)
    assert abs(zs.var() - 1.0) < 5.0 * math.sqrt(2.0 / n)
    assert stats.kstest(zs, "norm").pvalue > 1e-3
    assert stats.kstest(us, "uniform").pvalue > 1e-3
    hist, _ = np.histogram(us, bins=64, range=(0, 1))
    assert stats.chisquare(hist).pvalue > 1e-3
    # different counters decorrelate (sweep and chain are part of the key space)
    z2 = np.array([O.draw(12345, m, 4, 1)[0] for m in range(2000)])
    z3 = np.array([O.draw(12345, m, 3, 2)[0] for m in range(2000)])
    assert abs(np.corrcoef(zs[:2000], z2)[0, 1]) < 0.1
    assert abs(np.corrcoef(zs[:2000], z3)[0, 1]) < 0.1


def test_draw_counter_layout():
    # (pixel, sweep, chain, 0) with the 64-bit seed split into (lo, hi) key words
    seed = (7 << 32) | 99
    x = O.philox4x32_10([5, 6, 2, 0], [99, 7])
    z, u = O.draw(seed, 5, 6, 2)
    u0, u1 = O.uniform(x[0]), O.uniform(x[1])
    assert u == O.uniform(x[2])
    assert z == pytest.approx(math.sqrt(-2 * math.log(u0)) * math.cos(2 * math.pi * u1), rel=1e-15)
