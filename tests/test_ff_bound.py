"""The error bounds of the float ordering tiers, pinned by emulating the
kernels' arithmetic step for step in IEEE single precision (fused
multiply-adds rounded once) against exact rational arithmetic, on rows of
ordinary, concentrated, wide-exponent, equal and subnormal values:

* the float-float squared distance of the search's middle tier (`ff_d2` in
  csrc/search.cu): (3d + 13) 2^-48 d2 + (4d + 4) 2^-149;
* the single-precision distance summed per 32-dimension slice, the first tier
  of the prune, the search and the exact kNN: (min(d, 32) + ceil(d / 32) + 8)
  2^-24 d2 + 4 (d + 1) 2^-149;
* the float prune's split-f16 Gram: eps_ip |u||v| + 2^-36 sqrt(d) (|u| + |v|) /
  scale, summed in one of the tensor core's possible orders;
* and, for the uint8 prune, that the sign of a rounded difference of two
  integers below 2^24 in magnitude is exactly their order.

The GPU parity tests check the kernels themselves against the oracle; these
check that the bounds the kernels decide with hold for their arithmetic."""
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


# ---- the single-precision tier: d2 summed per 32-dimension slice, each
# difference rounded and its square added by a fused multiply-add, the slice
# sums then added in order; its bound (slice_rel_bound, abs_bound in
# csrc/common.cuh) is (min(d, 32) + ceil(d / 32) + 8) 2^-24 d2 + (d + 1) 2^-149 4.

def _sliced_d2(a, b, interleaved=False):
    # interleaved: the prune kernel's pivot keys, where each slice keeps two
    # running sums (dimensions 8c .. 8c+3 and 8c+4 .. 8c+7 of each group of
    # eight) added together at the slice's end
    acc = f32(0)
    with np.errstate(over="ignore", under="ignore"):
        for c0 in range(0, a.shape[0], 32):
            part = [f32(0), f32(0)]
            for i, (x, y) in enumerate(zip(a[c0:c0 + 32], b[c0:c0 + 32])):
                t = f32(x - y)
                j = ((i // 4) & 1) if interleaved else 0
                part[j] = _fma(t, t, part[j])
            acc = f32(acc + f32(part[0] + part[1]))
    return acc


def _check_sliced(a, b):
    for interleaved in (False, True):
        _check_sliced_order(a, b, interleaved)


def _check_sliced_order(a, b, interleaved):
    d = a.shape[0]
    got = Fraction(float(_sliced_d2(a, b, interleaved)))
    exact = sum((Fraction(float(x)) - Fraction(float(y))) ** 2 for x, y in zip(a, b))
    rel = Fraction(min(d, 32) + (d + 31) // 32 + 8, 2 ** 24)
    bound = rel * exact + Fraction(4 * (d + 1), 2 ** 149)
    assert abs(got - exact) <= bound, (float(abs(got - exact)), float(bound))


@pytest.mark.parametrize("d,seed", [(24, 0), (96, 1), (128, 2), (960, 3), (1000, 4)])
def test_single_precision_slice_bound(d, seed):
    rng = np.random.default_rng(200 + seed)
    a = np.abs(rng.normal(size=d)).astype(np.float32)
    _check_sliced(a, (a + rng.normal(size=d) * 1e-2).astype(np.float32))
    w = (rng.normal(size=d) * np.exp(rng.uniform(-20, 20, d))).astype(np.float32)
    _check_sliced(w, (rng.normal(size=d) * np.exp(rng.uniform(-20, 20, d))).astype(np.float32))
    _check_sliced((rng.integers(1, 9, d) * 2.0 ** -149).astype(np.float32), np.zeros(d, np.float32))


# ---- the float prune's Gram tier: rows scaled by a power of two into [-1, 1],
# split into f16 hi and lo (hi = f16(x), lo = f16(2^11 (x - hi))), the two
# accumulators hi hi^T and hi lo^T + lo hi^T summed in f32, combined as
# fma(D2, 2^-11, D1).  Bound (csrc/prune.cu): |G~ - G| <= eps_ip |u||v| +
# 2^-36 sqrt(d) (|u| + |v|) / scale, eps_ip = 4 2^-22 + 2^-23 + d 2^-22.  The
# emulation sums in k order, one of the orders the tensor core may take; the
# bound's factor-4 accumulation allowance is what covers the others.

def _split(x):
    hi = x.astype(np.float16)
    lo = ((x - hi.astype(np.float32)) * f32(2048)).astype(np.float16)  # exact difference and scaling
    return hi.astype(np.float32), lo.astype(np.float32)


def _gram_tier(u, v, scale):
    hu, lu = _split((u * scale).astype(np.float32))
    hv, lv = _split((v * scale).astype(np.float32))
    d1 = f32(0)
    d2 = f32(0)
    for k in range(u.shape[0]):  # f16 x f16 products are exact in f32
        d1 = f32(d1 + f32(hu[k] * hv[k]))
        d2 = f32(d2 + f32(hu[k] * lv[k]))
        d2 = f32(d2 + f32(lu[k] * hv[k]))
    return Fraction(float(_fma(d2, f32(2.0 ** -11), d1))) / Fraction(float(scale)) ** 2


@pytest.mark.parametrize("d,seed", [(32, 0), (96, 1), (960, 2)])
def test_split_f16_gram_bound(d, seed):
    rng = np.random.default_rng(300 + seed)
    for trial in range(3):
        u = rng.normal(size=d).astype(np.float32)
        v = (u + rng.normal(size=d) * 0.3).astype(np.float32)
        if trial == 1:  # components spread over many binades: low halves go subnormal in f16
            u = (u * np.exp(rng.uniform(-12, 0, d))).astype(np.float32)
            v = (v * np.exp(rng.uniform(-12, 0, d))).astype(np.float32)
        mx = float(max(np.abs(u).max(), np.abs(v).max()))
        scale = f32(2.0 ** -np.frexp(mx)[1])  # a power of two bringing max |x| to at most 1
        got = _gram_tier(u, v, scale)
        exact = sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(u, v))
        nu = float(np.sqrt(np.sum(u.astype(np.float64) ** 2)))
        nv = float(np.sqrt(np.sum(v.astype(np.float64) ** 2)))
        eps_ip = 4 * 2.0 ** -22 + 2.0 ** -23 + d * 2.0 ** -22
        bound = eps_ip * nu * nv + 2.0 ** -36 * np.sqrt(d) * (nu + nv) / float(scale)
        assert abs(float(got - exact)) <= bound, (float(got - exact), bound)


# ---- the uint8 prune's mask bits: x = 2 G - |t|^2 and q are integers of
# magnitude below 2^24 held exactly in single precision; the sign bit of the
# rounded x - q is exactly "x < q" (+0 at equality, and rounding never crosses
# zero), which the kernel funnel-shifts into a "not removed" word.

def test_sign_of_rounded_integer_difference():
    rng = np.random.default_rng(9)
    lim = 2 ** 24 - 1
    x = rng.integers(-lim, lim + 1, 200000)
    q = rng.integers(-lim, lim + 1, 200000)
    edge = np.array([0, 1, -1, lim, -lim, lim - 1, 2 ** 23, -(2 ** 23)])
    x = np.concatenate([x, np.repeat(edge, edge.size), edge, edge])
    q = np.concatenate([q, np.tile(edge, edge.size), edge, edge + 1])
    diff = x.astype(np.float32) - q.astype(np.float32)  # one rounding
    sign = np.signbit(diff)
    assert np.array_equal(sign, x < q)
