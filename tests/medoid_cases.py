"""Float datasets whose start vertex turns on the last bit of the mean.

The start vertex (§4.1) is the point nearest to the mean vector, with the
mean's sums taken in index order in binary64 and ties going to the smaller id.
In :func:`tie_case` one column decides:
- rows 0 and 1 hold two adjacent float32 values a < b;
- the rows after them hold values down to 2^-60 in size, so the running sum
  rounds many times;
- the last rows steer the running sum, by exact additions, to n * mid + k ulp,
  where mid = (a + b) / 2 is exact in binary64.

With n a power of two the mean is mid + k ulp(mid) exactly. Every other column
is constant, so it adds nothing to any distance. Rows 0 and 1 are then the two
points nearest to the mean:
- k < 0 gives row 0;
- k = 0 is a tie, and the smaller id, row 0, wins;
- k > 0 gives row 1.

A mean one unit in the last place off, in either direction, changes the
answer of one of k = 0 and k = 1.
"""
from fractions import Fraction

import numpy as np


def sequential_sum(values) -> float:
    """Index-order binary64 sum (Python floats are binary64)."""
    s = 0.0
    for x in np.asarray(values, dtype=np.float64).tolist():
        s += x
    return s


def tie_case(col: int, k: int, d: int = 96, p: int = 14, seed: int = 0):
    """(X, expected start vertex) for the construction in the module docstring."""
    n = 1 << p
    rng = np.random.default_rng(seed * 1000 + col * 10 + (k + 1))
    a = np.float32(0.0390625 + float(rng.random()) * 1e-3)
    b = np.nextafter(a, np.float32(1.0))
    mid = (float(a) + float(b)) / 2.0
    assert Fraction(mid) == (Fraction(float(a)) + Fraction(float(b))) / 2
    target = n * mid + k * float(np.spacing(n * mid))

    m = n - 8  # rows 0 .. m-1: a, b and the drivers; then the steering rows; then zeros
    v = np.empty(m, dtype=np.float32)
    v[0], v[1] = a, b
    rest = m - 2
    near = (mid * (1.0 + (rng.random(rest) - 0.5) * 0.5)).astype(np.float32)
    small = ((rng.random(rest) - 0.3) * 2.0 ** -rng.integers(20, 61, rest)).astype(np.float32)
    v[2:] = np.where(rng.random(rest) < 0.9, near, small)
    s = sequential_sum(v)
    assert Fraction(s) != sum(Fraction(float(x)) for x in v), "the drivers must make the sum round"

    steer = []
    while s != target:
        f = np.float32(target - s)
        t = s + float(f)
        assert Fraction(t) == Fraction(s) + Fraction(float(f)), "steering additions must be exact"
        steer.append(f)
        s = t
        assert len(steer) <= 4
    column = np.zeros(n, dtype=np.float32)
    column[:m] = v
    column[m:m + len(steer)] = steer
    assert sequential_sum(column) == target

    X = np.empty((n, d), dtype=np.float32)
    X[:] = (np.arange(d, dtype=np.float32) * np.float32(0.125))[None, :]
    X[:, col] = column
    return X, (1 if k > 0 else 0)
