"""Executable model of the sweep kernel's neighbour protocol (no GPU).

The sweep kernel updates one pixel per tile and class step.  Pixels of one
class are conditionally independent (their windows are disjoint), so every
tile may score its step-k update while its neighbours still run step k-1,
and it re-scores only if a neighbour changed data in its window meanwhile.
Each tile publishes a progress word: the number of steps it has published
and two change marks (it changed data its neighbours read at its last and at
its previous published step).  A tile at step k waits until every neighbour
has published k steps; a neighbour can then show k or k+1 published steps,
and the step is stale if the marks of steps k-1 or k are set.

This model runs tiles on a line with random interleavings of those actions
and checks every tile-step against the sequential schedule (all updates of
class step k after all of step k-1).  Weakened staleness rules must fail,
so the check has power against a wrong rule.
"""
import random

import pytest

S, R = 4, 1          # pixels per tile (classes per sweep) and window radius: 2R < S


def window(t, k, n_cells):
    """Cells read by tile t's update at class step k: the window of its pixel."""
    pos = t * S + (k % S)
    return [c for c in range(pos - R, pos + R + 1) if 0 <= c < n_cells]


def decide(vals, t, k):
    """A deterministic accept decision that depends on every value read."""
    h = hash((tuple(vals), t, k)) & 0xFFFF
    return h % 3 == 0


def sequential(n_tiles, steps):
    """Reference: class step by class step, tiles in any order."""
    n_cells = n_tiles * S
    data = [0] * n_cells
    seen = {}
    for k in range(steps):
        reads = {t: [data[c] for c in window(t, k, n_cells)] for t in range(n_tiles)}
        for t in range(n_tiles):
            seen[(t, k)] = reads[t]
            if decide(reads[t], t, k):
                for c in window(t, k, n_cells):
                    data[c] = data[c] * 31 + 7 * t + k + 1
    return data, seen


def stale_rule(rule, word, k):
    steps, c0, c1 = word
    if rule == "both":        # the kernel's rule: marks of steps k-1 and k
        return (c0 or c1) if steps > k else c0
    if rule == "last":        # weakened: only the last published step's mark
        return c0
    if rule == "none":
        return False
    raise ValueError(rule)


def concurrent(n_tiles, steps, rng, rule):
    """Random interleaving of the tiles' actions under the protocol."""
    n_cells = n_tiles * S
    data = [0] * n_cells
    words = [(0, False, False)] * n_tiles        # (steps published, changed last, changed before)
    seen = {}
    # per tile: step, phase, speculative values
    st = [dict(k=0, phase="score", vals=None) for _ in range(n_tiles)]
    nbrs = [[u for u in (t - 1, t + 1) if 0 <= u < n_tiles] for t in range(n_tiles)]
    active = set(range(n_tiles))
    while active:
        t = rng.choice(sorted(active))
        p = st[t]
        k = p["k"]
        if p["phase"] == "score":                 # speculative read, before the wait
            p["vals"] = [data[c] for c in window(t, k, n_cells)]
            p["phase"] = "wait"
        elif p["phase"] == "wait":
            if any(words[u][0] < k for u in nbrs[t]):
                continue                          # a neighbour has not published step k-1
            stale = any(stale_rule(rule, words[u], k) for u in nbrs[t]) if k > 0 else False
            if stale:                             # re-score on the current data
                p["vals"] = [data[c] for c in window(t, k, n_cells)]
            seen[(t, k)] = p["vals"]
            acc = decide(p["vals"], t, k)
            if acc:
                for c in window(t, k, n_cells):
                    data[c] = data[c] * 31 + 7 * t + k + 1
            words[t] = (k + 1, acc, words[t][1])  # publish with the change marks
            p["k"] = k + 1
            p["phase"] = "score"
            if p["k"] == steps:
                active.discard(t)
    return data, seen


@pytest.mark.parametrize("seed", range(40))
def test_protocol_matches_sequential_schedule(seed):
    rng = random.Random(seed)
    n_tiles, steps = rng.choice([3, 5, 8]), rng.choice([9, 17, 33])
    ref_data, ref_seen = sequential(n_tiles, steps)
    data, seen = concurrent(n_tiles, steps, rng, "both")
    assert seen == ref_seen
    assert data == ref_data


@pytest.mark.parametrize("rule", ["last", "none"])
def test_weakened_staleness_rules_fail(rule):
    failures = 0
    for seed in range(60):
        rng = random.Random(1000 + seed)
        ref_data, ref_seen = sequential(6, 25)
        data, seen = concurrent(6, 25, rng, rule)
        failures += seen != ref_seen
    assert failures > 0, f"rule {rule!r} never disagreed with the sequential schedule"


def test_window_geometry_of_the_model():
    # same-class windows of neighbouring tiles are disjoint, adjacent classes overlap
    n_cells = 4 * S
    for k in range(S):
        assert not set(window(0, k, n_cells)) & set(window(1, k, n_cells))
    assert set(window(0, S - 1, n_cells)) & set(window(1, S, n_cells))
