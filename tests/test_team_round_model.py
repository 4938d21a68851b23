"""Executable model of an update team's rounds in the lean sweep-kernel form
(no GPU).

After a class step's first round, a team of warps runs each round with one
barrier: every warp reads the round's proposal from a ring of 32 slots,
writes its partial sums, meets the others at the barrier, and reads every
warp's partial sums to take the decision; the drawing warp then draws
proposals ahead.  There is no second barrier before the next round, which
is safe when (a) the partial sums alternate between two sets by round
parity and (b) proposals are drawn two rounds ahead (16 at a time, every
16th round, when a sweep has more than 32 rounds), so that a draw is
published by the barrier of the round before its own and a slot is only
overwritten after its last reader.

The model interleaves the warps at random, one action at a time, with a
real barrier, and checks every read.  Drawing one round ahead, or a single
set of partial sums, must fail for some interleaving: the check has power.
"""
import random

import pytest

RING = 32


def run(seed, n_warps=2, rounds=70, wide=True, dist=2, double=True):
    rng = random.Random(seed)
    pwarp = n_warps - 1
    ring = [None] * RING
    bufs = [[None] * n_warps for _ in range(2 if double else 1)]

    def draw(e):
        ring[e % RING] = e

    if wide:
        for e in range(18 if dist == 2 else RING):
            draw(e)
    else:
        for e in range(dist):
            draw(e)
    # per warp: (round, phase); phases: 0 read proposal, 1 write partials,
    # 2 barrier arrival, 3 read partials, 4 draw (drawing warp), then next round
    state = [[0, 0] for _ in range(n_warps)]
    arrived = {}

    def after_draws(e):
        if wide:
            if dist == 2:
                if e % 16 == 0 and e > 0:
                    for k in range(2, 18):
                        draw(e + k)
            elif e % RING == RING - 1:
                for k in range(1, RING + 1):
                    draw(e + k)
        else:
            draw(e + dist)

    while any(st[0] < rounds for st in state):
        runnable = []
        for w, (e, ph) in enumerate(state):
            if e >= rounds:
                continue
            if ph == 3 and arrived.get(e, 0) < n_warps:
                continue          # waiting at the barrier
            runnable.append(w)
        w = rng.choice(runnable)
        e, ph = state[w]
        b = bufs[e % 2 if double else 0]
        if ph == 0:
            if ring[e % RING] != e:
                return f"warp {w} read slot {e % RING} holding {ring[e % RING]} in round {e}"
        elif ph == 1:
            b[w] = e
        elif ph == 2:
            arrived[e] = arrived.get(e, 0) + 1
        elif ph == 3:
            if any(x != e for x in b):
                return f"warp {w} read partial sums {b} in round {e}"
        elif ph == 4:
            if w == pwarp:
                after_draws(e)
        if ph == 4:
            state[w] = [e + 1, 0]
        else:
            state[w][1] = ph + 1
    return None


@pytest.mark.parametrize("wide", [True, False])
@pytest.mark.parametrize("n_warps", [2, 4])
def test_one_barrier_rounds_are_safe(wide, n_warps):
    for seed in range(300):
        err = run(seed, n_warps=n_warps, wide=wide)
        assert err is None, f"seed {seed}: {err}"


@pytest.mark.parametrize("wide", [True, False])
def test_drawing_one_round_ahead_fails_without_the_second_barrier(wide):
    errs = [run(seed, wide=wide, dist=1) for seed in range(300)]
    assert any(e is not None and "slot" in e for e in errs)


def test_a_single_set_of_partial_sums_fails_without_the_second_barrier():
    errs = [run(seed, double=False) for seed in range(300)]
    assert any(e is not None and "partial" in e for e in errs)
