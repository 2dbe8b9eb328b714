"""Pins for the CPU oracle: what the paper and plain mathematics fix, independent
of the oracle's own code.

* Lemma 3.5 (collinear construction, unsorted) and the sorted counterpart,
* Lemma 3.7 (general-metric distance matrix, sorted),
* Appendix A (Euclidean construction of Lemma 3.8) and the worked numbers
  printed after Table 1 (tests/golden/worked_example_alpha3_alpha2.json),
* Lemma 2.2 (slow preprocessing gives an alpha-reachable graph),
* Theorems 3.1 / 3.2 (reachability after RP-Tuning is at least the worst case),
* Algorithm 1 invariants (characterisation of the kept set, subgraph,
  idempotence, R-prefix, duplicate handling),
* Algorithm 2 traced by hand (tests/golden/greedy_search_line.json) and its
  reduction to exact kNN on a complete graph,
* exact kNN against scipy's brute-force distances.
"""
import json
import math
import os

import numpy as np
import pytest

import datagen
import oracle
import medoid_cases
from closed_forms import (appendix_a_points, beta_euc, sorted_euclid_bound,
                          sorted_general_bound, unsorted_bound,
                          unsorted_bound_as_printed)

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _gold(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def _csr(rows):
    row_ptr = np.zeros(len(rows) + 1, dtype=np.int64)
    np.cumsum([len(r) for r in rows], out=row_ptr[1:])
    col = np.concatenate([np.asarray(r, dtype=np.int32) for r in rows]) if rows else np.zeros(0, np.int32)
    return row_ptr, col.astype(np.int32)


def _canon_d2_matrix(X):
    """Exact squared distances: int64 for uint8; for float32 the binary64 sum
    in index order, which is the canonical reading of the Euclidean distance."""
    if X.dtype == np.uint8:
        Y = X.astype(np.int64)
        return ((Y[:, None, :] - Y[None, :, :]) ** 2).sum(-1)
    Y = X.astype(np.float64)
    s = np.zeros((X.shape[0], X.shape[0]))
    for i in range(X.shape[1]):
        t = Y[:, None, i] - Y[None, :, i]
        s = s + t * t
    return s


def _dominated(D2, A, u, v, p):
    if D2.dtype == np.int64:
        return A * A * int(D2[u, v]) <= 1_000_000 * int(D2[p, v])
    return float(A * A) * D2[u, v] <= 1e6 * D2[p, v]


# ---------------------------------------------------------------- Lemma 3.5

@pytest.mark.parametrize("dtype", [np.uint8, np.float32])
def test_lemma_3_5_collinear_unsorted_is_tight(dtype):
    # alpha1 = alpha2 = 2: p=0, z=1*4, y=z+z/alpha1=6, x=y+y/alpha2=9 on a line.
    a1 = a2 = 2.0
    X = np.array([[0], [4], [6], [9]], dtype=dtype)  # ids: p=0, z=1, y=2, x=3
    p, z, y, x = 0, 1, 2, 3
    # N_out(p) = {x, y} with x stored first; every other node links to all others.
    assert oracle.robust_prune(X, p, [x, y], a2, variant="unsorted").tolist() == [x]
    assert oracle.robust_prune(X, p, [x, y], a2, variant="sorted").tolist() == [y]
    base = [[x, y], [0, 2, 3], [0, 1, 3], [0, 1, 2]]
    rp, col = _csr(base)
    # G is alpha1-reachable: z is reached from p through y with equality.
    assert oracle.reachability(X, rp, col) == pytest.approx(a1, rel=1e-12)
    after = [oracle.robust_prune(X, p, [x, y], a2, variant="unsorted").tolist()] + base[1:]
    rp2, col2 = _csr(after)
    # Theorem 3.1 is attained: alpha* = alpha1 alpha2 / (alpha1 + alpha2 + 1) = 0.8.
    assert oracle.reachability(X, rp2, col2) == pytest.approx(unsorted_bound(a1, a2), rel=1e-12)
    assert unsorted_bound(a1, a2) == pytest.approx(0.8)
    assert unsorted_bound_as_printed(a1, a2) <= unsorted_bound(a1, a2)
    after_s = [oracle.robust_prune(X, p, [x, y], a2, variant="sorted").tolist()] + base[1:]
    rp3, col3 = _csr(after_s)
    # Sorted processing keeps y, the witness for z: the pattern is ruled out (§3.2).
    assert oracle.reachability(X, rp3, col3) >= a2 - 1e-12


# ---------------------------------------------------------------- Lemma 3.7

def _lemma37_matrix(a1, a2):
    # ids: p=0, x=1, y=2, z=3; D(p,.)=1, D(y,z)=1/a1, D(x,y)=1/a2,
    # D(x,z)=(a1+a2)/(a1 a2).  (The printed matrix swaps the labels x and z;
    # this labelling is the one that satisfies the constraints of Lemma 3.6.)
    D = np.zeros((4, 4))
    D[0, 1:] = D[1:, 0] = 1.0
    D[2, 3] = D[3, 2] = 1.0 / a1
    D[1, 2] = D[2, 1] = 1.0 / a2
    D[1, 3] = D[3, 1] = (a1 + a2) / (a1 * a2)
    return D


@pytest.mark.parametrize("a1,a2", [(4.0, 2.0), (2.0, 2.0)])
def test_lemma_3_7_general_metric_sorted_is_tight(a1, a2):
    D = _lemma37_matrix(a1, a2)
    p, x, y, z = 0, 1, 2, 3
    # Equal distances from p: the tie goes to the smaller id, so x is taken first
    # and prunes y (alpha2 * D(x, y) = 1 <= D(p, y) = 1).
    assert oracle.robust_prune_dmat(D, p, [y, x], a2, variant="sorted").tolist() == [x]
    base = [[x, y], [0, 2, 3], [0, 1, 3], [0, 1, 2]]
    rp, col = _csr(base)
    assert oracle.reachability_dmat(D, rp, col) == pytest.approx(a1, rel=1e-12)
    after = [oracle.robust_prune_dmat(D, p, [y, x], a2).tolist()] + base[1:]
    rp2, col2 = _csr(after)
    assert oracle.reachability_dmat(D, rp2, col2) == pytest.approx(sorted_general_bound(a1, a2), rel=1e-12)


def test_worked_example_general_metric_value():
    g = _gold("worked_example_alpha3_alpha2.json")
    a1, a2 = g["alpha1"], g["alpha2"]
    D = _lemma37_matrix(a1, a2)
    kept = oracle.robust_prune_dmat(D, 0, [2, 1], a2)
    assert kept.tolist() == [1]
    ratio = D[0, 3] / D[kept[0], 3]
    assert round(ratio, g["printed_digits"]) == g["general_sorted"]


# ---------------------------------------------------------------- Appendix A

@pytest.mark.parametrize("a1,a2", [(3.0, 2.0), (1.5, 1.2), (1.5, 1.1), (2.0, 1.5)])
def test_appendix_a_euclidean_construction(a1, a2):
    pts = appendix_a_points(a1, a2)  # p, x, y, z
    P = np.array(pts, dtype=np.float64)
    D = np.sqrt(((P[:, None, :] - P[None, :, :]) ** 2).sum(-1))
    D[0, 1:] = D[1:, 0] = 1.0  # x, y, z lie on the unit circle around p
    # The constraints of Lemma 3.8 hold with equality in the reals ...
    assert D[2, 3] == pytest.approx(1.0 / a1, rel=1e-12)
    assert D[1, 2] == pytest.approx(1.0 / a2, rel=1e-12)
    # ... so prune with alpha2 a hair below its value to stay on the pruning side.
    kept = oracle.robust_prune_dmat(D, 0, [2, 1], a2 * (1 - 1e-9))
    assert kept.tolist() == [1]
    ratio = D[0, 3] / D[1, 3]
    assert ratio == pytest.approx(1.0 / beta_euc(a1, a2), rel=1e-12)
    assert ratio >= sorted_general_bound(a1, a2)  # the Euclidean case is better (Table 1)


def test_worked_example_euclidean_value():
    g = _gold("worked_example_alpha3_alpha2.json")
    a1, a2 = g["alpha1"], g["alpha2"]
    P = np.array(appendix_a_points(a1, a2))
    D = np.sqrt(((P[:, None, :] - P[None, :, :]) ** 2).sum(-1))
    D[0, 1:] = D[1:, 0] = 1.0
    kept = oracle.robust_prune_dmat(D, 0, [2, 1], a2 * (1 - 1e-9))
    ratio = D[0, 3] / D[kept[0], 3]
    assert round(ratio, g["printed_digits"]) == g["euclidean_sorted_approx"]
    assert round(sorted_euclid_bound(a1, a2), 3) == g["euclidean_sorted_approx"]


def test_appendix_a_vector_form_float32():
    # The same construction as float32 vectors, nudged off the equality
    # boundaries (x moved towards y and inwards) so the decisions are strict.
    a1, a2 = 3.0, 2.0
    t1 = math.asin(1 / (2 * a1))
    t2 = math.asin(1 / (2 * a2)) * (1 - 1e-3)
    y = (math.cos(2 * t1), math.sin(2 * t1))
    x = tuple((1 - 1e-3) * c for c in (math.cos(2 * (t1 + t2)), math.sin(2 * (t1 + t2))))
    X = np.array([(0, 0), x, y, (1, 0)], dtype=np.float32)
    assert oracle.robust_prune(X, 0, [2, 1], a2).tolist() == [1]
    d = lambda a, b: math.dist(X[a].astype(float), X[b].astype(float))
    assert d(0, 3) / d(1, 3) == pytest.approx(1 / beta_euc(a1, a2), rel=5e-3)


# ---------------------------------------------------------------- Algorithm 1 invariants

def _check_prune_invariants(X, D2, p, cand, A, R, variant, kept):
    V = []
    for v in cand:
        if v != p and v not in V:
            V.append(int(v))
    kept = [int(v) for v in kept]
    assert set(kept) <= set(V), "output must be a subset of the candidates"
    assert len(set(kept)) == len(kept)
    assert len(kept) <= R
    if variant == "sorted":
        order = sorted(V, key=lambda v: (D2[p, v], v))
    else:
        order = V
    pos = {v: i for i, v in enumerate(order)}
    assert [pos[v] for v in kept] == sorted(pos[v] for v in kept), "kept in processing order"
    # every kept point is not dominated by an earlier kept point
    for i, v in enumerate(kept):
        for u in kept[:i]:
            assert not _dominated(D2, A, u, v, p)
    # every dropped point is dominated by a kept point processed before it,
    # unless the degree bound was reached before it came up
    last = pos[kept[-1]] if kept else -1
    for v in V:
        if v in kept:
            continue
        dom = any(_dominated(D2, A, u, v, p) for u in kept if pos[u] < pos[v])
        assert dom or (len(kept) == R and pos[v] > last)
    # the set is uniquely determined by those two facts: rebuild it greedily
    K = []
    for v in order:
        if len(K) == R:
            break
        if not any(_dominated(D2, A, u, v, p) for u in K):
            K.append(v)
    assert K == kept


@pytest.mark.parametrize("dtype", [np.uint8, np.float32])
@pytest.mark.parametrize("variant", ["sorted", "unsorted"])
def test_robust_prune_characterisation(dtype, variant):
    rng = np.random.default_rng(7)
    for trial in range(40):
        n = int(rng.integers(5, 40))
        d = int(rng.choice([1, 2, 3, 8, 17]))
        if dtype == np.uint8:
            X = rng.integers(0, 6 if trial % 3 == 0 else 256, size=(n, d)).astype(np.uint8)
        else:
            X = rng.normal(size=(n, d)).astype(np.float32)
            if trial % 4 == 0:
                X[1] = X[2]  # identical vectors: distance 0
        D2 = _canon_d2_matrix(X)
        p = int(rng.integers(0, n))
        cand = rng.integers(0, n, size=int(rng.integers(0, 2 * n))).tolist() + [p]
        rng.shuffle(cand)
        for alpha in (1.0, 1.05, 1.2, 1.5, 2.0):
            A = int(round(alpha * 1000))
            for R in (1, 3, oracle.R_INF):
                kept = oracle.robust_prune(X, p, cand, alpha, R, variant)
                _check_prune_invariants(X, D2, p, cand, A, R, variant, kept)


def test_duplicates_and_self_loops_are_ignored():
    X = datagen.dataset("tiny", 50)
    cand = [3, 7, 3, 0, 12, 7, 0, 40, 12]
    ref = oracle.robust_prune(X, 0, [3, 7, 12, 40], 1.1)
    assert oracle.robust_prune(X, 0, cand, 1.1).tolist() == ref.tolist()
    # unsorted: first occurrences keep their positions
    assert oracle.robust_prune(X, 0, cand, 1.1, variant="unsorted").tolist() == \
        oracle.robust_prune(X, 0, [3, 7, 12, 40], 1.1, variant="unsorted").tolist()


@pytest.fixture(scope="module")
def tiny_base():
    X = datagen.dataset("tiny")
    rp, col = oracle.slow_base(X, 1.5)
    return X, rp, col


def test_lemma_2_2_slow_preprocessing_is_alpha_reachable(tiny_base):
    X, rp, col = tiny_base
    assert oracle.reachability(X, rp, col) >= 1.5
    # and on integer data
    U = datagen.dataset("sift", 300)
    rpu, colu = oracle.slow_base(U, 1.2)
    assert oracle.reachability(U, rpu, colu) >= 1.2


@pytest.mark.parametrize("a2", [1.2, 1.1])
def test_theorems_3_1_3_2_reachability_after_tuning(tiny_base, a2):
    X, rp, col = tiny_base
    a1 = 1.5
    rps, cols = oracle.rp_tune(X, rp, col, a2, oracle.R_INF, "sorted")
    assert oracle.reachability(X, rps, cols) >= sorted_euclid_bound(a1, a2)
    rpu, colu = oracle.rp_tune(X, rp, col, a2, oracle.R_INF, "unsorted")
    assert oracle.reachability(X, rpu, colu) >= unsorted_bound(a1, a2)


def _rows(rp, col):
    return [col[rp[i]:rp[i + 1]].tolist() for i in range(rp.shape[0] - 1)]


def test_subgraph_idempotence_and_r_prefix(tiny_base):
    X, rp, col = tiny_base
    base_rows = _rows(rp, col)
    # identity: re-pruning the base at its own alpha with no bound changes nothing
    rpi, coli = oracle.rp_tune(X, rp, col, 1.5, oracle.R_INF)
    assert _rows(rpi, coli) == base_rows
    for a in (1.2, 1.0):
        rpa, cola = oracle.rp_tune(X, rp, col, a, 32)
        rows = _rows(rpa, cola)
        assert all(set(r) <= set(b) for r, b in zip(rows, base_rows))
        rpb, colb = oracle.rp_tune(X, rpa, cola, a, 32)
        assert _rows(rpb, colb) == rows
        rpc, colc = oracle.rp_tune(X, rp, col, a, 8)
        assert _rows(rpc, colc) == [r[:8] for r in rows]


# ---------------------------------------------------------------- Algorithm 2

def test_greedy_search_hand_trace():
    g = _gold("greedy_search_line.json")
    X = np.array(g["points_1d_u8"], dtype=np.uint8)[:, None]
    n = X.shape[0]
    rows = [[v for v in (i - 1, i + 1) if 0 <= v < n] for i in range(n)]
    rp, col = _csr(rows)
    Q = np.array([[g["query_1d_u8"]]], dtype=np.uint8)
    ids, d2, exp = oracle.greedy_search(X, rp, col, g["start"], Q, g["L"], g["k"])
    assert ids[0].tolist() == g["expected_ids"]
    assert d2[0].tolist() == g["expected_d2"]
    assert int(exp[0]) == g["expected_expansions"]


@pytest.mark.parametrize("dtype", [np.uint8, np.float32])
def test_greedy_search_complete_graph_is_exact(dtype):
    scipy_dist = pytest.importorskip("scipy.spatial.distance")
    rng = np.random.default_rng(3)
    n, d = 120, 6
    X = (rng.integers(0, 4, size=(n, d)) if dtype == np.uint8 else rng.normal(size=(n, d))).astype(dtype)
    Q = (rng.integers(0, 4, size=(9, d)) if dtype == np.uint8 else rng.normal(size=(9, d))).astype(dtype)
    rows = [[v for v in range(n) if v != i] for i in range(n)]
    rp, col = _csr(rows)
    for L, k in ((10, 10), (40, 7)):
        ids, _, _ = oracle.greedy_search(X, rp, col, 5, Q, L, k)
        D = scipy_dist.cdist(Q.astype(np.float64), X.astype(np.float64), "sqeuclidean")
        for i in range(Q.shape[0]):
            ref = np.lexsort((np.arange(n), D[i]))[:k]
            assert ids[i].tolist() == ref.tolist()


def test_greedy_search_pads_unreachable():
    X = np.arange(6, dtype=np.uint8)[:, None]
    rows = [[1], [0], [3], [2], [5], [4]]  # three components
    rp, col = _csr(rows)
    ids, d2, _ = oracle.greedy_search(X, rp, col, 0, np.array([[5]], np.uint8), 4, 4)
    assert ids[0].tolist() == [1, 0, -1, -1]
    assert np.isinf(d2[0, 2:]).all()


# ---------------------------------------------------------------- kNN and medoid

@pytest.mark.parametrize("dtype", [np.uint8, np.float32])
def test_knn_matches_library_brute_force(dtype):
    scipy_dist = pytest.importorskip("scipy.spatial.distance")
    rng = np.random.default_rng(11)
    n, d, k = 500, 12, 25
    X = (rng.integers(0, 3, size=(n, d)) if dtype == np.uint8 else rng.normal(size=(n, d))).astype(dtype)
    Q = X[:30] if dtype == np.uint8 else rng.normal(size=(30, d)).astype(dtype)
    ids, d2 = oracle.knn(X, k, Q=Q)
    D = scipy_dist.cdist(Q.astype(np.float64), X.astype(np.float64), "sqeuclidean")
    for i in range(Q.shape[0]):
        ref = np.lexsort((np.arange(n), D[i]))[:k]  # many exact ties for uint8
        assert ids[i].tolist() == ref.tolist()
        np.testing.assert_allclose(d2[i], D[i, ref], rtol=1e-12)
    # base points as queries exclude themselves
    ids2, _ = oracle.knn(X, k, qid=np.arange(10))
    for i in range(10):
        Di = scipy_dist.cdist(X[i:i + 1].astype(np.float64), X.astype(np.float64), "sqeuclidean")[0]
        order = [v for v in np.lexsort((np.arange(n), Di)) if v != i][:k]
        assert ids2[i].tolist() == order


def test_medoid_is_nearest_to_mean():
    X = datagen.dataset("tiny")
    m = X.astype(np.float64).mean(0)
    d = ((X.astype(np.float64) - m) ** 2).sum(1)
    assert oracle.medoid(X) == int(np.argmin(d))
    U = datagen.dataset("sift", 3000)
    mu = U.astype(np.float64).mean(0)
    du = ((U.astype(np.float64) - mu) ** 2).sum(1)
    assert oracle.medoid(U) == int(np.argmin(du))


@pytest.mark.parametrize("col", [0, 40, 95])
@pytest.mark.parametrize("k", [-1, 0, 1])
def test_medoid_follows_the_index_order_mean_to_the_last_bit(col, k):
    """§4.1's start vertex under the binary64 index-order reading of the mean:
    the constructed mean sits on, or one ulp either side of, the midpoint of
    rows 0 and 1, so only the exact sequential rounding gives the answer."""
    X, expect = medoid_cases.tie_case(col, k)
    assert oracle.medoid(X) == expect


def test_medoid_tie_cases_see_one_ulp():
    """The construction is sensitive: a mean one ulp up breaks the k = 0 tie
    towards row 1, and one ulp down turns the k = 1 case to row 0; the exactly
    rounded sum (another reading of the mean) changes some answer too."""
    def nearest(X, mean):
        return int(np.argmin(((X.astype(np.float64) - mean) ** 2).sum(1)))

    n_changed = 0
    for col in (0, 40, 95):
        for k, nudge, flipped in ((0, +1, 1), (1, -1, 0)):
            X, _ = medoid_cases.tie_case(col, k)
            m = np.array([medoid_cases.sequential_sum(X[:, j]) for j in range(X.shape[1])]) / X.shape[0]
            m[col] = np.nextafter(m[col], nudge * np.inf)
            assert nearest(X, m) == flipped
        for k in (-1, 0, 1):
            X, expect = medoid_cases.tie_case(col, k)
            exact = np.array([math.fsum(X[:, j].astype(np.float64).tolist()) for j in range(X.shape[1])]) / X.shape[0]
            n_changed += nearest(X, exact) != expect
    assert n_changed > 0


def test_canonical_distances_are_exact_or_within_the_sum_bound():
    """d2_pairs / d2_query: uint8 distances are exact integers; float32 ones are
    index-order binary64 sums of exactly formed squares' roundings, within
    (d + 1) 2^-53 of the exact rational value; id -1 gives +inf."""
    from fractions import Fraction
    rng = np.random.default_rng(31)
    n, d = 60, 37
    a = rng.integers(0, n, 150)
    b = rng.integers(0, n, 150)
    U = rng.integers(0, 256, (n, d), dtype=np.uint8)
    want = ((U[a].astype(np.int64) - U[b].astype(np.int64)) ** 2).sum(1)
    assert np.array_equal(oracle.d2_pairs(U, a, b), want.astype(np.float64))
    F = rng.standard_normal((n, d)).astype(np.float32)

    def exact(x, y):
        return sum((Fraction(float(u)) - Fraction(float(v))) ** 2 for u, v in zip(x, y))

    got = oracle.d2_pairs(F, a, b)
    for i in range(a.size):
        e = exact(F[a[i]], F[b[i]])
        assert abs(Fraction(got[i]) - e) <= Fraction(d + 1, 2 ** 53) * e
    assert (oracle.d2_pairs(F, a, a) == 0).all()
    Q = rng.standard_normal((5, d)).astype(np.float32)
    ids = rng.integers(-1, n, (5, 7)).astype(np.int32)
    ids[0, 0] = -1
    dq = oracle.d2_query(F, Q, ids)
    for i in range(5):
        for j in range(7):
            if ids[i, j] < 0:
                assert dq[i, j] == np.inf
            else:
                e = exact(Q[i], F[ids[i, j]])
                assert abs(Fraction(dq[i, j]) - e) <= Fraction(d + 1, 2 ** 53) * e
    dqu = oracle.d2_query(U, U[:3], np.array([[0, 1], [2, -1], [5, 2]], np.int32))
    assert dqu[0, 0] == 0 and dqu[1, 1] == np.inf
    assert dqu[2, 0] == float(((U[2].astype(np.int64) - U[5].astype(np.int64)) ** 2).sum())


def test_knn_base_reduces_to_the_knn_lists():
    """The kNN-candidate base, RobustPrune(p, kNN_k(p), alpha, R):
    - alpha so large that no candidate dominates another keeps every list whole
      and in distance order, i.e. exactly the kNN lists;
    - R = 1 keeps each point's nearest neighbour (Algorithm 1 keeps the argmin
      first), i.e. the 1-NN graph;
    - any alpha gives lists that start with the nearest neighbour and hold
      only kNN candidates."""
    rng = np.random.default_rng(32)
    n, k = 300, 12
    X = rng.standard_normal((n, 8)).astype(np.float32)
    ids, _ = oracle.knn(X, k, qid=np.arange(n))
    rp_, col = oracle.knn_base(X, k, 1000.0, k)
    assert np.array_equal(np.diff(rp_), np.full(n, k))
    assert np.array_equal(col.reshape(n, k), ids)
    rp1, col1 = oracle.knn_base(X, k, 1.2, 1)
    assert np.array_equal(np.diff(rp1), np.ones(n, np.int64)) and np.array_equal(col1, ids[:, 0])
    rpa, cola = oracle.knn_base(X, k, 1.2, k)
    for p in range(n):
        row = cola[rpa[p]:rpa[p + 1]]
        assert row[0] == ids[p, 0] and set(row.tolist()) <= set(ids[p].tolist())
    assert np.diff(rpa).mean() < k  # alpha = 1.2 does prune
    rows = oracle.knn_base(X, k, 1.2, k, nodes=np.array([7, 3]))
    assert [r.tolist() for r in rows] == [cola[rpa[7]:rpa[8]].tolist(), cola[rpa[3]:rpa[4]].tolist()]


def test_reachability_small_line():
    # points 0, 1, 3 on a line; edges 0->1, 1->2, 2->1
    X = np.array([[0], [1], [3]], dtype=np.uint8)
    rp, col = _csr([[1], [2], [1]])
    # non-edges: (0,2): D(0,2)/D(1,2) = 3/2; (1,0): D(1,0)/D(2,0) = 1/3; (2,0): D(2,0)/D(1,0) = 3
    assert oracle.reachability(X, rp, col) == pytest.approx(1 / 3, rel=1e-12)


def test_reachability_per_node_terms():
    """Definition 2.1 per node, distances pair by pair: the line worked by hand
    above, the closed forms (a node with no out-neighbour gives 0, a node
    adjacent to every other point gives +inf), Lemma 2.2 on the slow
    preprocessing base, and the minimum over nodes against the all-pairs
    routine on several graphs."""
    X = np.array([[0], [1], [3]], dtype=np.uint8)
    rp, col = _csr([[1], [2], [1]])
    # node 0: q=2 via p'=1: 3/2; node 1: q=0 via p'=2: 1/3; node 2: q=0 via p'=1: 3/1
    np.testing.assert_array_equal(oracle.reachability_nodes(X, rp, col), [1.5, 1 / 3, 3.0])
    np.testing.assert_array_equal(oracle.reachability_nodes(X, rp, col, nodes=[2, 0]), [3.0, 1.5])
    rp, col = _csr([[], [0, 2], [1]])  # node 0 has no out-neighbour; node 1 reaches everything
    np.testing.assert_array_equal(oracle.reachability_nodes(X, rp, col), [0.0, np.inf, 3.0])
    T = datagen.dataset("tiny", 400)
    rpb, colb = oracle.slow_base(T, 1.5)
    assert oracle.reachability_nodes(T, rpb, colb).min() >= 1.5  # Lemma 2.2
    for R in (8, 32):
        rpt, colt = oracle.rp_tune(T, rpb, colb, 1.1, R)
        assert oracle.reachability_nodes(T, rpt, colt).min() == oracle.reachability(T, rpt, colt)
    U = datagen.dataset("sift", 300)
    rpu, colu = oracle.slow_base(U, 1.2)
    per = oracle.reachability_nodes(U, rpu, colu)
    assert per.min() == oracle.reachability(U, rpu, colu) and per.min() >= 1.2


# ---- k-recall@k (§4): |returned ∩ true top-k| / k, averaged over the queries.
# Each case is worked by hand; a plausible slip (counting the -1 padding of
# Algorithm 2's short answers, counting a repeated id twice, or reading past k
# in either list) changes at least one of the expected values.
@pytest.mark.parametrize("found,truth,k,expected", [
    # padding: two real ids, both true; the two -1 entries must not match each other
    ([[1, 2, -1, -1]], [[1, 2, 3, 4]], 4, 2 / 4),
    ([[1, 2, -1, -1]], [[1, 2, -1, -1]], 4, 2 / 4),
    # a repeated id in the returned list counts once
    ([[5, 5, 6, 7]], [[5, 6, 8, 9]], 4, 2 / 4),
    # only the first k entries of each list count: 9 and 8 are past k in `found`,
    # 7 and 6 past k in `truth`
    ([[1, 2, 3, 9, 8]], [[9, 8, 7, 6, 5]], 3, 0 / 3),
    ([[9, 1, 2, 8]], [[9, 3, 4, 8]], 3, 1 / 3),
    # order inside the first k does not matter
    ([[3, 2, 1]], [[1, 2, 3]], 3, 3 / 3),
    # the mean over queries, not over returned ids
    ([[1, 2], [7, -1]], [[1, 2], [8, 9]], 2, (2 + 0) / (2 * 2)),
    ([[0, 1, 2, 3], [4, 5, 6, 7], [8, 9, 10, 11]], [[0, 1, 2, 3], [4, 5, 0, 1], [1, 2, 3, 4]], 4,
     (4 + 2 + 0) / 12),
])
def test_recall_at_k_hand_worked(found, truth, k, expected):
    assert oracle.recall_at_k(np.array(found), np.array(truth), k) == pytest.approx(expected, abs=0)


def test_recall_at_k_of_exact_search_is_one():
    """GreedySearch on a complete graph with L >= k is exact kNN (Alg. 2), so its
    recall against the exact kNN is 1; a list shifted by one place loses the
    k-th true neighbour and gains the (k+1)-th, which is not in the truth."""
    X = datagen.dataset("tiny", 300)
    Q = datagen.queries("tiny", 20)
    n = X.shape[0]
    row_ptr = np.arange(0, n * (n - 1) + 1, n - 1, dtype=np.int64)
    col = np.array([j for i in range(n) for j in range(n) if j != i], dtype=np.int32)
    ids, _, _ = oracle.greedy_search(X, row_ptr, col, 0, Q, 40, 10)
    truth, _ = oracle.knn(X, 11, Q=Q)
    assert oracle.recall_at_k(ids, truth[:, :10], 10) == 1.0
    assert oracle.recall_at_k(truth[:, 1:11], truth[:, :10], 10) == pytest.approx(9 / 10, abs=1e-15)


# ---- Vamana (§2.1 "fast preprocessing"; §4.1 builds its bases with it), the
# batched reading the oracle states.
def test_vamana_hand_trace_on_a_line():
    g = _gold("vamana_line.json")
    X = np.asarray(g["x"], dtype=np.float32)[:, None]
    rp_, col, over = oracle.vamana(X, g["perm"], g["alphas"], g["R"], g["L"], g["vcap"], g["max_batch"],
                                   g["start"])
    rows = [col[rp_[p]:rp_[p + 1]].tolist() for p in range(X.shape[0])]
    assert rows == g["rows"]
    assert over == 0


@pytest.mark.parametrize("dtype", ["u8", "f32"])
def test_vamana_graph_is_valid_and_navigable(dtype):
    """Every list holds at most R distinct points other than its owner, the
    last pass's RobustPrune makes every list obey Algorithm 1's degree bound,
    and the graph does what the construction is for: GreedySearch from the
    start finds most true nearest neighbours (recall@10 at L = 64)."""
    if dtype == "u8":
        X = datagen.dataset("sift", 1500)[:, :32]
        X = np.ascontiguousarray(X)
        Q = np.ascontiguousarray(datagen.queries("sift", 100)[:, :32])
    else:
        X = datagen.dataset("tiny", 1500)
        Q = datagen.queries("tiny", 100)
    n = X.shape[0]
    perm = np.random.default_rng(9).permutation(n).astype(np.int32)
    s = oracle.medoid(X)
    R = 24
    rp_, col, over = oracle.vamana(X, perm, [1.0, 1.2], R, 40, 160, 64, s)
    deg = np.diff(rp_)
    assert deg.max() <= R and deg.min() >= 1
    for p in range(n):
        row = col[rp_[p]:rp_[p + 1]]
        assert p not in row and len(set(row.tolist())) == row.shape[0]
    ids, _, _ = oracle.greedy_search(X, rp_, col, s, Q, 64, 10)
    truth, _ = oracle.knn(X, 10, Q=Q)
    assert oracle.recall_at_k(ids, truth, 10) >= 0.9
