"""The prune kernel's greedy scan (a7) against Algorithm 1's loop, on the CPU.

Candidates are numbered in processing order (by rank), so the next argmin of
the live set is its lowest set bit. Row p of the domination mask holds the
later candidates p removes at the target's alpha. Algorithm 1 keeps the lowest
live candidate, clears its row from the live set, and stops after R kept.

For rows of at most 64 candidates the kernel takes two steps per round. It
reads the masks of the two lowest live candidates together, keeps the first,
and keeps the second only if the first left it live, because the second is
then the next argmin. This file restates both loops and checks them equal on
random masks of every density, on R from 1 to past m, and on the degenerate
rows (none live, everything dominated, nothing dominated).
"""
import numpy as np
import pytest


def _low(x: int) -> int:
    return (x & -x).bit_length() - 1


def algorithm1(masks, live: int, R: int):
    kept = []
    while live and len(kept) < R:
        p = _low(live)
        kept.append(p)
        live &= ~(masks[p] | (1 << p))
    return kept


def two_step(masks, live: int, R: int):
    kept = []
    while len(kept) < R and live:
        p1 = _low(live)
        rest = live & (live - 1)
        p2 = _low(rest) if rest else p1
        m1, m2 = masks[p1], masks[p2]
        kept.append(p1)
        live = rest & ~m1
        if len(kept) < R and (live >> p2) & 1:
            kept.append(p2)
            live &= ~(m2 | (1 << p2))
    return kept


def _masks(rng, m: int, density: float):
    """Row p dominates later candidates c > p with probability `density`."""
    out = []
    for p in range(64):
        bits = 0
        if p < m:
            for c in range(p + 1, m):
                if rng.random() < density:
                    bits |= 1 << c
        out.append(bits)
    return out


@pytest.mark.parametrize("density", [0.0, 0.02, 0.1, 0.3, 0.6, 1.0])
def test_two_step_scan_is_algorithm_1(density):
    rng = np.random.default_rng(int(density * 1000) + 7)
    for trial in range(300):
        m = int(rng.integers(0, 65))
        masks = _masks(rng, m, density)
        live = (1 << m) - 1
        for R in (1, 2, 3, 5, 17, 32, 48, 64, 100):
            assert two_step(masks, live, R) == algorithm1(masks, live, R), (density, trial, m, R)


def test_degenerate_rows():
    none = [0] * 64
    full = [((1 << 64) - 1) & ~((1 << (p + 1)) - 1) for p in range(64)]  # p removes every later one
    assert two_step(none, 0, 64) == [] == algorithm1(none, 0, 64)
    assert two_step(none, (1 << 64) - 1, 64) == list(range(64))
    assert two_step(full, (1 << 64) - 1, 64) == [0] == algorithm1(full, (1 << 64) - 1, 64)
    assert two_step(none, (1 << 64) - 1, 5) == [0, 1, 2, 3, 4]
