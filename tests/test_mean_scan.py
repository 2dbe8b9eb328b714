"""The float mean kernel's step, emulated on the CPU against the index-order
binary64 sum it must reproduce bit for bit (the start vertex of §4.1).

The kernel adds up to 64 rows per warp step. While the running sum s stays in
one binade with grid u, every addition rounds to that grid. So it converts each
value to integer units q = rne(x / u), prefix-sums them onto s's significand,
and keeps the leading elements whose running significand T stays in
[2^52 + 1, 2^53] (no tie). The first element outside is added in binary64.
s = +0 skips zeros and takes the first nonzero value. Rows come in blocks of
1024, and steps stop at a block's end. This file restates that arithmetic in
numpy (the kernel's element order; lanes are pairs of consecutive elements) and
checks it on the data that exercise each branch: rounding in every step,
binade changes both ways, exact ties, cancellation to zero, subnormal values
and sums, and huge dynamic range.
"""
import struct

import numpy as np
import pytest

import datagen
import medoid_cases

LO, HI = (1 << 52) + 1, 1 << 53


def _bits(s: float) -> int:
    return struct.unpack("<Q", struct.pack("<d", s))[0]


def _double(b: int) -> float:
    return struct.unpack("<d", struct.pack("<Q", b))[0]


def _units(xb: np.ndarray, e52: int, neg: int):
    """q = rne(x / 2^e52) in the sign frame of s, and whether it may be kept."""
    xb = xb.astype(np.int64)
    ex = (xb >> 23) & 0xFF
    m = (xb & 0x7FFFFF) | np.where(ex != 0, 0x800000, 0)
    k = np.where(ex != 0, ex, 1) - 150 - e52
    up = (k >= 0) & (k <= 30)
    v = np.where(up, m << np.clip(k, 0, 30), 0)
    ok = ~((k > 30) & (m != 0))
    sh = np.clip(-k, 1, 25)
    down = (k < 0) & (-k < 26)
    rem = m & ((1 << sh) - 1)
    half = 1 << (sh - 1)
    v = np.where(down, (m >> sh) + (rem > half), v)
    ok &= ~(down & (rem == half) & (m != 0))
    v = np.where(((xb >> 31) & 1) != neg, -v, v)
    return v, ok


def warp_step_sum(x: np.ndarray, block: int = 1024) -> float:
    x = np.ascontiguousarray(x, dtype=np.float32)
    xb = x.view(np.uint32)
    n = x.size
    s, i = 0.0, 0
    while i < n:
        bend = min(n, (i // block + 1) * block)
        avail = min(64, bend - i)
        sb = _bits(s)
        eb = (sb >> 52) & 0x7FF
        if sb == 0:
            nz = np.nonzero(xb[i:i + avail] & 0x7FFFFFFF)[0]
            if nz.size == 0:
                i += avail
                continue
            s = float(x[i + nz[0]])
            i += int(nz[0]) + 1
            continue
        if eb in (0, 0x7FF):
            s = s + float(x[i])
            i += 1
            continue
        neg = sb >> 63
        S = (sb & ((1 << 52) - 1)) | (1 << 52)
        q, ok = _units(xb[i:i + avail], eb - 1075, neg)
        T = S + np.cumsum(q)
        valid = ok & (T >= LO) & (T <= HI)
        bad = np.nonzero(~valid)[0]
        fi = int(bad[0]) if bad.size else avail
        top = np.nonzero(valid & (T == HI))[0]
        fe = int(top[0]) if top.size else 64
        c = min(fi, fe + 1)
        if c > 0:
            t = int(T[c - 1])
            sign = neg << 63
            s = _double(sign | ((eb + 1) << 52) if t == HI else sign | (eb << 52) | (t - (1 << 52)))
        used = c
        if c < avail and c == fi:
            s = s + float(x[i + c])
            used = c + 1
        i += used
    return s


def _columns():
    rng = np.random.default_rng(20260214)
    n = 20000
    cases = {
        "normal": rng.standard_normal(n),
        "biased": rng.standard_normal(n) * 0.1 + 0.01,
        "uniform negative": -rng.random(n) * 3,
        "2^-60 .. 2^60": np.where(rng.random(n) < 0.5, -1, 1) * 2.0 ** rng.uniform(-60, 60, n),
        "2^-125 .. 2^125": np.where(rng.random(n) < 0.5, -1, 1) * 2.0 ** rng.uniform(-125, 125, n),
        "subnormal values": (rng.integers(0, 1 << 23, n).astype(np.uint32)
                             | (rng.integers(0, 2, n).astype(np.uint32) << 31)).view(np.float32),
        "subnormals and normals": np.where(np.arange(n) % 7 == 0, rng.standard_normal(n),
                                           rng.standard_normal(n) * 1e-40),
        "ties: 2^30 and 2^-24": np.where(np.arange(n) % 3 == 0, 2.0 ** 30, 2.0 ** -24),
        "grid values": np.ldexp(rng.integers(0, 4096, n).astype(np.float64), rng.integers(-12, 28, n)),
        "powers of two +-": np.where(rng.random(n) < 0.5, -1, 1) * np.ldexp(1.0, rng.integers(-20, 40, n)),
        "cancel to zero": np.where(np.arange(n) < n // 2, 1e30, -1e30),
        "cancel then small": np.concatenate([[1e30, -1e30], rng.standard_normal(n - 2) * 1e-3]),
        "2^24 + small ints": 2.0 ** 24 + rng.integers(0, 3, n),
        "1 and 1 + ulp": 1.0 + np.ldexp(rng.integers(0, 2, n).astype(np.float64), -23),
        "zeros and signed zeros": np.where(np.arange(n) % 5 == 0, -0.0, 0.0),
        "alternating +-1": np.where(np.arange(3000) % 2 == 0, 1.0, -1.0),
        # the sum hovers at 1.0 in steps of about an ulp, so it crosses the binade
        # boundary both ways with fractions of the grid below and above it
        "hovering at a power of two": np.concatenate(
            [[1.0], np.where(rng.random(n) < 0.5, -1, 1) * rng.uniform(0.25, 2.0, n) * 2.0 ** -52]),
        "ragged: 1": rng.standard_normal(1),
        "ragged: 1025": rng.standard_normal(1025),
    }
    for name, v in cases.items():
        yield name, np.asarray(v).astype(np.float32)
    for col in (0, 40):
        for k in (-1, 0, 1):
            yield f"last-bit case col {col} k {k}", medoid_cases.tie_case(col, k)[0][:, col]
    deep = datagen.dataset("deep", 20000)
    for j in (0, 17, 95):
        yield f"deep column {j}", deep[:, j]
    gist = datagen.dataset("gist", 5000)
    for j in (0, 480, 959):
        yield f"gist column {j}", gist[:, j]


@pytest.mark.parametrize("name,x", list(_columns()), ids=[c[0] for c in _columns()])
def test_warp_step_sum_is_the_sequential_sum(name, x):
    want = medoid_cases.sequential_sum(x)
    got = warp_step_sum(x)
    assert _bits(got) == _bits(want), (name, got, want)
