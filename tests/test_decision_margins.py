"""The prune kernel's single-precision domination tests, emulated on the CPU,
never contradict the canonical binary64 decision of Algorithm 1.

Canonical (reading of Algorithm 1's test alpha D(p*, v) <= D(p, v) on squared
distances, alpha = A / 1000): v is removed iff fl(A^2 d2a) <= fl(1e6 d2b) in
binary64, with d2a = D(p*, v)^2 and d2b = D(p, v)^2 the canonical distances.

The kernel knows d2b only as a single-precision key kacc with
|kacc - d2b| <= E_rel d2b + E_abs, and d2a as dv with |dv - d2a| <= err, where
err includes the floor d 2^-125. Per column and alpha it forms
qlo = (kacc (1 - E_rel) - E_abs) kappa 0.999998 and
qhi = (kacc (1 + E_rel) + E_abs) kappa 1.000002, with kappa = fl32(1e6 / A^2).
"Surely removed" is hi < qlo and "surely kept" is lo > qhi, where
lo, hi = fl32(dv -+ err). The recheck tier's sure_dominates compares
A^2 (d2a (1 -+ E) -+ Eabs) with 1e6 (d2b (1 -+ E) -+ Eabs) the same way. Its
E and Eabs hold slack over the distances' own error: 6 ulps relative, and
four times the underflow allowance. That slack is what keeps the test sure
only when it is right where the products round in the subnormal range.

Each case puts d2a within 2e-6 or 1e-5 of the boundary (and some far from
it), with keys from 2^-140 (where the thresholds are subnormal) to 2^100. It takes the worst
admissible kacc, dv and err, and evaluates the formulas in float32 both with
and without the multiply-add fused. A sure answer must then equal the
canonical one.
"""
import numpy as np
import pytest

F = np.float32


def _bounds(d: int):
    e_rel = F((min(d, 32) + (d + 31) // 32 + 8) * 5.9604645e-08)
    e_abs = F(F(d + 1) * F(1.4012985e-45) * F(4.0))
    return e_rel, e_abs


def _fma32(a, b, c):
    """fl32(a * b + c) with one rounding (a, b float32: the product is exact in binary64)."""
    return F(float(a) * float(b) + float(c))


def _thresholds(kacc, e_rel, e_abs, kappa, fused):
    one_m, one_p = F(F(1) - e_rel), F(F(1) + e_rel)
    if fused:
        lo_key = _fma32(kacc, one_m, -e_abs)
        hi_key = _fma32(kacc, one_p, e_abs)
    else:
        lo_key = F(F(kacc * one_m) - e_abs)
        hi_key = F(F(kacc * one_p) + e_abs)
    qlo = F(F(lo_key * kappa) * F(0.999998))
    qhi = F(F(hi_key * kappa) * F(1.000002))
    return qlo, qhi


def _sure_dominates(A2, d2a, d2b, E, Eabs):
    one_p, one_m = F(F(1) + E), F(F(1) - E)
    lhs_hi = F(A2 * F(F(d2a * one_p) + Eabs))
    lhs_lo = F(A2 * F(F(d2a * one_m) - Eabs))
    rhs_hi = F(F(1.0e6) * F(F(d2b * one_p) + Eabs))
    rhs_lo = F(F(1.0e6) * F(F(d2b * one_m) - Eabs))
    if not (np.isfinite(lhs_hi) and np.isfinite(rhs_hi)):
        return -1
    if lhs_hi < rhs_lo:
        return 1
    if lhs_lo > rhs_hi:
        return 0
    return -1


def _inward(lo: float, hi: float):
    """The float32 values nearest the ends of [lo, hi] that lie inside it."""
    a, b = F(lo), F(hi)
    if float(a) < lo:
        a = np.nextafter(a, F(np.inf))
    if float(b) > hi:
        b = np.nextafter(b, F(-np.inf))
    return a, b


def _cases(rng, count):
    for _ in range(count):
        A = int(rng.choice([1000, 1001, 1010, 1050, 1100, 1150, 1200, 1500, 2000, 4000]))
        d = int(rng.choice([8, 32, 96, 128, 960]))
        # a third of the keys where float32 is subnormal or nearly so
        d2b = float(2.0 ** (rng.uniform(-140, -118) if rng.random() < 0.3 else rng.uniform(-118, 100)))
        r = rng.random()
        delta = rng.uniform(-2e-6, 2e-6) if r < 0.4 else rng.uniform(-1e-5, 1e-5) if r < 0.8 else \
            rng.uniform(-0.5, 0.5)
        d2a = d2b * 1e6 / (A * A) * (1.0 + delta)
        yield A, d, d2a, d2b


@pytest.mark.parametrize("seed", range(4))
def test_gram_tier_thresholds_never_contradict_the_canonical_test(seed):
    rng = np.random.default_rng(seed)
    n_sure = 0
    for A, d, d2a, d2b in _cases(rng, 3000):
        canonical_remove = float(A * A) * d2a <= 1e6 * d2b
        e_rel, e_abs = _bounds(d)
        kappa = F(1.0e6 / (A * A))
        k_lo, k_hi = _inward(d2b - float(e_rel) * d2b - float(e_abs), d2b + float(e_rel) * d2b + float(e_abs))
        floor = float(d) * 2.0 ** -125
        for kacc in (k_lo, k_hi, F(d2b)):
            if not np.isfinite(kacc):
                continue
            for rel in (1e-7, 1e-5, 1e-3):
                err = F(max(floor, d2a * rel) * 1.0001)
                dv_lo, dv_hi = _inward(d2a - float(err), d2a + float(err))
                for dv in (dv_lo, dv_hi, F(d2a)):
                    lo, hi = F(dv - err), F(dv + err)
                    for fused in (False, True):
                        qlo, qhi = _thresholds(kacc, e_rel, e_abs, kappa, fused)
                        if hi < qlo:
                            assert canonical_remove, (A, d, d2a, d2b, kacc, dv, err, fused)
                            n_sure += 1
                        if lo > qhi:
                            assert not canonical_remove, (A, d, d2a, d2b, kacc, dv, err, fused)
                            n_sure += 1
    assert n_sure > 1000  # the far cases are decided


@pytest.mark.parametrize("seed", range(4))
def test_recheck_tier_never_contradicts_the_canonical_test(seed):
    rng = np.random.default_rng(100 + seed)
    decided = 0
    for A, d, d2a, d2b in _cases(rng, 4000):
        canonical_remove = float(A * A) * d2a <= 1e6 * d2b
        E, Eabs = _bounds(d)  # what the kernel passes to sure_dominates
        # The distances' own error: E less its 6 ulps of slack, relative, plus (d + 1) 2^-149
        # for terms that underflow (Eabs is four times that). The slack is what absorbs the
        # roundings of sure_dominates' own products, which are absolute in the subnormal range.
        rel = float(E) - 6 * 2.0 ** -24
        ab = (d + 1) * 2.0 ** -149
        a_lo, a_hi = _inward(d2a - rel * d2a - ab, d2a + rel * d2a + ab)
        b_lo, b_hi = _inward(d2b - rel * d2b - ab, d2b + rel * d2b + ab)
        for fa in (a_lo, a_hi, F(d2a)):
            for fb in (b_lo, b_hi, F(d2b)):
                if not (np.isfinite(fa) and np.isfinite(fb)):
                    continue
                r = _sure_dominates(F(A * A), fa, fb, E, Eabs)
                if r == 1:
                    assert canonical_remove, (A, d, d2a, d2b, fa, fb)
                elif r == 0:
                    assert not canonical_remove, (A, d, d2a, d2b, fa, fb)
                decided += r >= 0
    assert decided > 1000


def _sure_less(a, b, E, Eabs):
    return F(F(a * F(F(1) + E)) + Eabs) < F(F(b * F(F(1) - E)) - Eabs)


@pytest.mark.parametrize("seed", range(4))
def test_sure_less_never_misorders_keys(seed):
    """sure_less(a, b) orders two pivot keys in single precision only when their
    binary64 values are strictly ordered the same way; equal values (which the
    id orders) are never claimed. Keys carry the distances' own error, as above."""
    rng = np.random.default_rng(300 + seed)
    claimed = 0
    for _ in range(6000):
        d = int(rng.choice([8, 32, 96, 128, 960]))
        E, Eabs = _bounds(d)
        rel = float(E) - 6 * 2.0 ** -24
        ab = (d + 1) * 2.0 ** -149
        tb = float(2.0 ** (rng.uniform(-149, -118) if rng.random() < 0.3 else rng.uniform(-118, 100)))
        r = rng.random()
        ta = tb if r < 0.2 else tb * (1.0 + (rng.uniform(-1e-5, 1e-5) if r < 0.8 else rng.uniform(-0.5, 0.5)))
        a_lo, a_hi = _inward(ta - rel * ta - ab, ta + rel * ta + ab)
        b_lo, b_hi = _inward(tb - rel * tb - ab, tb + rel * tb + ab)
        for fa in (a_lo, a_hi, F(ta)):
            for fb in (b_lo, b_hi, F(tb)):
                if _sure_less(fa, fb, E, Eabs):
                    assert ta < tb, (d, ta, tb, fa, fb)
                    claimed += 1
    assert claimed > 1000
