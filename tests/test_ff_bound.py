"""The float-float squared distance of the search's middle ordering tier
(`ff_d2` in csrc/search.cu), emulated step for step in IEEE single precision,
against exact rational arithmetic: its error must stay within the bound the
kernel uses, (3d + 13) 2^-48 d2 + (4d + 4) 2^-149, on rows of ordinary,
concentrated, wide-exponent, equal and subnormal values.  The GPU parity tests
check the kernel itself against the oracle; this pins the bound."""
from fractions import Fraction

import numpy as np
import pytest

f32 = np.float32


def _round32(v: Fraction) -> np.float32:
    """v rounded to the nearest float32, ties to even."""
    r = f32(float(v))
    best, key = None, None
    for z in (r, np.nextafter(r, f32(np.inf)), np.nextafter(r, f32(-np.inf))):
        k = (abs(Fraction(float(z)) - v), int(np.array(z, np.float32).view(np.uint32)) & 1)
        if key is None or k < key:
            best, key = z, k
    return f32(best)


def _fma(a, b, c):
    return _round32(Fraction(float(a)) * Fraction(float(b)) + Fraction(float(c)))


def _ff_step(x, y, sh, sl):
    th = f32(x - y)  # two-sum of x and -y
    bv = f32(th - x)
    tl = f32(f32(x - f32(th - bv)) + f32(f32(f32(0) - y) - bv))
    ph = f32(th * th)
    pl = _fma(th, th, -ph)
    xt = _fma(f32(2) * th, tl, pl)
    s1 = f32(sh + ph)  # two-sum of sh and ph
    b1 = f32(s1 - sh)
    e = f32(f32(sh - f32(s1 - b1)) + f32(ph - b1))
    l1 = f32(sl + f32(e + xt))
    sh = f32(s1 + l1)  # renormalise
    sl = f32(l1 - f32(sh - s1))
    return sh, sl


def _check(a, b):
    d = a.shape[0]
    sh, sl = f32(0), f32(0)
    with np.errstate(over="ignore", under="ignore"):
        for x, y in zip(a, b):
            sh, sl = _ff_step(x, y, sh, sl)
    ff = Fraction(float(np.float64(sh) + np.float64(sl)))
    exact = sum((Fraction(float(x)) - Fraction(float(y))) ** 2 for x, y in zip(a, b))
    bound = Fraction((3 * d + 13), 2 ** 48) * exact + Fraction(4 * d + 4, 2 ** 149)
    assert abs(ff - exact) <= bound, (float(abs(ff - exact)), float(bound))


@pytest.mark.parametrize("seed", range(4))
def test_concentrated_rows(seed):
    rng = np.random.default_rng(seed)
    a = np.abs(rng.normal(size=960))
    a = (a / np.linalg.norm(a)).astype(np.float32)
    b = (a + rng.normal(size=960) * 10.0 ** -rng.uniform(2, 6)).astype(np.float32)
    _check(a, b)


@pytest.mark.parametrize("seed", range(3))
def test_wide_exponent_rows(seed):
    rng = np.random.default_rng(100 + seed)
    a = (rng.normal(size=256) * np.exp(rng.uniform(-30, 30, 256))).astype(np.float32)
    b = (rng.normal(size=256) * np.exp(rng.uniform(-30, 30, 256))).astype(np.float32)
    _check(a, b)


def test_equal_subnormal_and_long_rows():
    rng = np.random.default_rng(7)
    a = rng.normal(size=96).astype(np.float32)
    _check(a, a.copy())  # d2 = 0 exactly
    tiny = (rng.integers(1, 50, 64) * 2.0 ** -149).astype(np.float32)  # subnormal differences
    _check(tiny, np.zeros(64, np.float32))
    _check(tiny, (tiny * 2).astype(np.float32))
    a = rng.normal(size=4096).astype(np.float32)
    _check(a, (a + rng.normal(size=4096) * 1e-3).astype(np.float32))
