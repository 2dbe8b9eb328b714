"""GPU parity: the CUDA path through the C ABI against the CPU oracle, element by
element on the same seeded inputs.  Edge lists must be identical, order
included (Algorithm 1 output order = the order points were kept); search
results must be identical (Algorithm 2, ties by id)."""
import numpy as np
import pytest

import datagen
import medoid_cases
import oracle

rp = pytest.importorskip("paper_2602_08097_gb300")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_08097_gb300 import build as b
    b.build()
    c = rp.rp_create(0)
    yield c
    rp.rp_destroy(c)


@pytest.fixture(scope="module")
def tiny():
    X = datagen.dataset("tiny")
    row_ptr, col = oracle.slow_base(X, 1.5)
    return X, row_ptr, col


def _same_csr(got, ref, what=""):
    grp, gcol = got
    rrp, rcol = ref
    assert grp.shape == rrp.shape, what
    if not np.array_equal(grp, rrp):
        bad = int(np.nonzero(grp != rrp)[0][0])
        raise AssertionError(f"{what}: row_ptr differs first at {bad}: {grp[bad]} vs {rrp[bad]}")
    if not np.array_equal(gcol, rcol):
        bad = int(np.nonzero(gcol != rcol)[0][0])
        node = int(np.searchsorted(rrp, bad, side="right") - 1)
        raise AssertionError(f"{what}: col differs first at edge {bad} (node {node}): "
                             f"{gcol[rrp[node]:rrp[node + 1]].tolist()} vs {rcol[rrp[node]:rrp[node + 1]].tolist()}")


# ------------------------------------------------------------------ tuning

@pytest.mark.parametrize("variant", ["sorted", "unsorted"])
def test_tiny_tune_matches_oracle(ctx, tiny, variant):
    X, row_ptr, col = tiny
    v = rp.RP_SORTED if variant == "sorted" else rp.RP_UNSORTED
    g = rp.rp_load_graph(ctx, X, row_ptr, col)
    for alpha, R in ((1.2, 32), (1.1, 32), (1.0, 32), (1.2, rp.RP_R_INF), (1.1, rp.RP_R_INF), (1.5, rp.RP_R_INF)):
        t = rp.rp_tune(ctx, g, alpha, R, v)
        _same_csr(rp.rp_graph_export(ctx, t), oracle.rp_tune(X, row_ptr, col, alpha, R, variant),
                  f"tiny {variant} alpha={alpha} R={R}")
        rp.rp_graph_free(ctx, t)
    rp.rp_graph_free(ctx, g)


def test_batch_equals_plain_and_replays(ctx, tiny):
    X, row_ptr, col = tiny
    g = rp.rp_load_graph(ctx, X, row_ptr, col)
    alphas = [1.2, 1.15, 1.1, 1.05, 1.0, 1.0]
    Rs = [32, 32, 64, 16, 32, 1]
    for rep in range(3):  # the second and third calls replay the captured graph
        outs = rp.rp_tune_batch(ctx, g, alphas, Rs)
        for t, a, r in zip(outs, alphas, Rs):
            _same_csr(rp.rp_graph_export(ctx, t), oracle.rp_tune(X, row_ptr, col, a, r), f"batch a={a} R={r}")
            rp.rp_graph_free(ctx, t)
    assert rp.rp_stats(ctx)["graph_replays"] >= 2
    rp.rp_graph_free(ctx, g)


@pytest.mark.parametrize("dtype", ["u8", "f32"])
@pytest.mark.parametrize("deg_hi", [5, 64, 128, 300])
def test_random_graphs_all_paths(ctx, dtype, deg_hi):
    # uneven degrees that exercise the 64-, 128- and large-degree kernels,
    # with duplicate entries and self loops in the input
    n = 3000
    if dtype == "u8":
        X = datagen.dataset("sift", n)
    else:
        X = datagen.dataset("deep", n)
    row_ptr, col = datagen.random_graph(n, 0, deg_hi, seed=deg_hi, dup_frac=0.05, self_frac=0.02)
    g = rp.rp_load_graph(ctx, X, row_ptr, col)
    for variant in ("sorted", "unsorted"):
        v = rp.RP_SORTED if variant == "sorted" else rp.RP_UNSORTED
        for alpha, R in ((1.0, 8), (1.2, 64), (1.05, rp.RP_R_INF)):
            t = rp.rp_tune(ctx, g, alpha, R, v)
            _same_csr(rp.rp_graph_export(ctx, t), oracle.rp_tune(X, row_ptr, col, alpha, R, variant),
                      f"{dtype} deg<={deg_hi} {variant} a={alpha} R={R}")
            rp.rp_graph_free(ctx, t)
    st = rp.rp_stats(ctx)
    assert st["self_loops_dropped"] > 0 and st["duplicates_dropped"] > 0
    rp.rp_graph_free(ctx, g)



@pytest.mark.parametrize("dtype", ["u8", "f32"])
@pytest.mark.parametrize("variant", ["sorted", "unsorted"])
def test_lists_in_and_out_of_algorithm_order(ctx, dtype, variant):
    """A list that RobustPrune wrote is already in Algorithm 1's processing
    order, and the kernel then takes each rank from the stored position; a
    reordered list takes the counted ranks.  Both kinds share launches and
    slots here (every third list reversed, one in seven rotated by one)."""
    X = datagen.dataset("sift" if dtype == "u8" else "deep", 3000)
    row_ptr, col = oracle.knn_base(X, 64, 1.2, 64)
    col = col.copy()
    for v in range(len(row_ptr) - 1):
        a, b = row_ptr[v], row_ptr[v + 1]
        if v % 3 == 0:
            col[a:b] = col[a:b][::-1]
        elif v % 7 == 0 and b - a > 1:
            col[a:b] = np.roll(col[a:b], 1)
    vt = rp.RP_SORTED if variant == "sorted" else rp.RP_UNSORTED
    g = rp.rp_load_graph(ctx, X, row_ptr, col)
    targets = [(1.15, 64), (1.05, 40), (1.0, 16)]
    outs = rp.rp_tune_batch(ctx, g, [t[0] for t in targets], [t[1] for t in targets], vt)
    for t, o in zip(targets, outs):
        _same_csr(rp.rp_graph_export(ctx, o), oracle.rp_tune(X, row_ptr, col, *t, variant), f"{dtype} {variant} {t}")
        rp.rp_graph_free(ctx, o)
    rp.rp_graph_free(ctx, g)


@pytest.mark.parametrize("name,n,alpha,variant", [("tiny", 2000, 1.5, "sorted"), ("tiny", 2000, 1.2, "unsorted"),
                                                  ("sift", 1200, 1.2, "sorted")])
def test_slow_preprocessing_base_on_the_gpu(ctx, name, n, alpha, variant):
    """§2.1's slow preprocessing, RobustPrune of every point over all the
    others, through the library: the complete graph (lists in id order),
    tuned at (alpha, unbounded R) on the wide-degree path."""
    X = datagen.dataset(name, n)
    ids = np.arange(n, dtype=np.int32)
    col = np.concatenate([np.delete(ids, p) for p in range(n)])
    row_ptr = np.arange(n + 1, dtype=np.int64) * (n - 1)
    g = rp.rp_load_graph(ctx, X, row_ptr, col)
    vt = rp.RP_SORTED if variant == "sorted" else rp.RP_UNSORTED
    t = rp.rp_tune(ctx, g, alpha, rp.RP_R_INF, vt)
    _same_csr(rp.rp_graph_export(ctx, t), oracle.slow_base(X, alpha, variant=variant),
              f"slow base {name} alpha={alpha} {variant}")
    rp.rp_graph_free(ctx, t)
    rp.rp_graph_free(ctx, g)

def test_ties_and_duplicate_vectors(ctx):
    # many identical vectors and exact distance ties (uint8 values in {0, 1})
    rng = np.random.default_rng(5)
    for dtype in (np.uint8, np.float32):
        X = rng.integers(0, 2, size=(400, 8)).astype(dtype)
        row_ptr, col = datagen.random_graph(400, 10, 120, seed=9)
        g = rp.rp_load_graph(ctx, X, row_ptr, col)
        for alpha, R in ((1.0, 20), (1.5, rp.RP_R_INF), (2.0, 3)):
            for variant, v in (("sorted", rp.RP_SORTED), ("unsorted", rp.RP_UNSORTED)):
                t = rp.rp_tune(ctx, g, alpha, R, v)
                _same_csr(rp.rp_graph_export(ctx, t), oracle.rp_tune(X, row_ptr, col, alpha, R, variant),
                          f"ties {dtype.__name__} {variant} a={alpha} R={R}")
                rp.rp_graph_free(ctx, t)
        rp.rp_graph_free(ctx, g)


def test_near_ties_in_float_keys(ctx):
    # points on a sphere around each node make many pivot keys agree to
    # within single precision, exercising the binary64 recheck
    rng = np.random.default_rng(8)
    n, d = 600, 24
    base = rng.normal(size=(n, d))
    X = np.empty((n, d), np.float32)
    X[0] = 0
    X[1:] = (base[1:] / np.linalg.norm(base[1:], axis=1, keepdims=True) * (1 + 1e-7 * rng.random((n - 1, 1))))
    rows = [list(range(1, 200))] + [list(rng.integers(0, n, 40)) for _ in range(n - 1)]
    row_ptr = np.zeros(n + 1, np.int64)
    np.cumsum([len(r) for r in rows], out=row_ptr[1:])
    col = np.concatenate([np.asarray(r, np.int32) for r in rows])
    rp.rp_stats(ctx, reset=True)
    g = rp.rp_load_graph(ctx, X, row_ptr, col)
    for alpha in (1.0, 1.3):
        t = rp.rp_tune(ctx, g, alpha, rp.RP_R_INF)
        _same_csr(rp.rp_graph_export(ctx, t), oracle.rp_tune(X, row_ptr, col, alpha), f"near-ties a={alpha}")
        rp.rp_graph_free(ctx, t)
    assert rp.rp_stats(ctx)["fp64_sort_keys"] > 0
    rp.rp_graph_free(ctx, g)


def test_near_and_exact_ties_on_the_tensor_core_path(ctx):
    """Rows of at most 64 candidates (the tensor-core kernel): keys that agree
    to single precision are ordered by float-float distances, and exact ties
    (copies of one point under different ids) fall through to binary64 and
    then to the smaller id, as Algorithm 1's argmin with ties by id reads."""
    rng = np.random.default_rng(21)
    n, d = 400, 24
    base = rng.normal(size=(n, d))
    X = (base / np.linalg.norm(base, axis=1, keepdims=True) * (1 + 1e-7 * rng.random((n, 1)))).astype(np.float32)
    X[0] = 0
    X[10:20] = X[5]  # ten copies of point 5: equal keys for every node
    rows = [list(range(1, 60))] + [list(rng.choice(np.arange(1, n), 48, replace=False)) for _ in range(n - 1)]
    row_ptr = np.zeros(n + 1, np.int64)
    np.cumsum([len(r) for r in rows], out=row_ptr[1:])
    col = np.concatenate([np.asarray(r, np.int32) for r in rows])
    rp.rp_stats(ctx, reset=True)
    g = rp.rp_load_graph(ctx, X, row_ptr, col)
    for alpha in (1.0, 1.3):
        for variant in (rp.RP_SORTED, rp.RP_UNSORTED):
            t = rp.rp_tune(ctx, g, alpha, rp.RP_R_INF, variant)
            ref = oracle.rp_tune(X, row_ptr, col, alpha, variant="sorted" if variant == rp.RP_SORTED else "unsorted")
            _same_csr(rp.rp_graph_export(ctx, t), ref, f"ties a={alpha} v={variant}")
            rp.rp_graph_free(ctx, t)
    st = rp.rp_stats(ctx)
    assert st["generic_nodes"] == 0
    assert st["fp64_sort_keys"] > 0  # the exact ties
    rp.rp_graph_free(ctx, g)


def test_degenerate_graphs(ctx):
    X = datagen.dataset("sift", 50)
    # no edges at all
    g = rp.rp_load_graph(ctx, X)
    t = rp.rp_tune(ctx, g, 1.0, 1)
    r, c = rp.rp_graph_export(ctx, t)
    assert r.tolist() == [0] * 51 and c.shape[0] == 0
    # a single point
    g1 = rp.rp_load_graph(ctx, X[:1], np.array([0, 1], np.int64), np.array([0], np.int32))
    r1, c1 = rp.rp_graph_export(ctx, rp.rp_tune(ctx, g1, 1.2, 5))
    assert r1.tolist() == [0, 0]
    # R = 1 keeps exactly the nearest candidate
    row_ptr, col = datagen.random_graph(50, 1, 49, seed=1)
    g2 = rp.rp_load_graph(ctx, X, row_ptr, col)
    _same_csr(rp.rp_graph_export(ctx, rp.rp_tune(ctx, g2, 1.0, 1)), oracle.rp_tune(X, row_ptr, col, 1.0, 1), "R=1")


def test_max_degree(ctx):
    n = 8300
    X = datagen.dataset("sift", n)
    rows = [np.arange(1, 8193)] + [np.array([0, (i * 7) % n], np.int64) for i in range(1, n)]
    row_ptr = np.zeros(n + 1, np.int64)
    np.cumsum([len(r) for r in rows], out=row_ptr[1:])
    col = np.concatenate(rows).astype(np.int32)
    g = rp.rp_load_graph(ctx, X, row_ptr, col)
    t = rp.rp_tune(ctx, g, 1.1, rp.RP_R_INF)
    _same_csr(rp.rp_graph_export(ctx, t), oracle.rp_tune(X, row_ptr, col, 1.1), "degree 8192")
    bad = np.concatenate([[0], np.full(1, 8193)]).astype(np.int64)
    with pytest.raises(rp.RPError):
        rp.rp_load_graph(ctx, X[:8194], np.concatenate([[0, 8193], np.full(8193, 8193)]).astype(np.int64),
                         np.arange(1, 8194).astype(np.int32))
    del bad


def test_invalid_inputs_are_rejected(ctx):
    X = datagen.dataset("tiny", 20)
    row_ptr, col = datagen.random_graph(20, 1, 5, seed=2)
    g = rp.rp_load_graph(ctx, X, row_ptr, col)
    for alpha in (0.999, 1.0005, float("nan"), 1e9):
        with pytest.raises(rp.RPError) as e:
            rp.rp_tune(ctx, g, alpha, 4)
        assert e.value.code == rp.RP_EINVAL
    with pytest.raises(rp.RPError):
        rp.rp_tune(ctx, g, 1.1, 0)
    with pytest.raises(rp.RPError) as e:
        rp.rp_tune(ctx, 987654, 1.1, 4)
    assert e.value.code == rp.RP_ENOTFOUND
    bad_col = col.copy()
    bad_col[3] = 20  # out of range
    with pytest.raises(rp.RPError) as e:
        rp.rp_load_graph(ctx, X, row_ptr, bad_col)
    assert e.value.code == rp.RP_EINVAL
    Xn = X.copy()
    Xn[4, 2] = np.nan
    with pytest.raises(rp.RPError):
        rp.rp_load_graph(ctx, Xn, row_ptr, col)
    Xb = X.copy()
    Xb[7, 0] = 2.0 ** 51  # finite, but its squared distances could leave single precision
    with pytest.raises(rp.RPError) as e:
        rp.rp_load_graph(ctx, Xb, row_ptr, col)
    assert e.value.code == rp.RP_EINVAL
    Xb[7, 0] = 2.0 ** 50  # the largest magnitude accepted
    rp.rp_graph_free(ctx, rp.rp_load_graph(ctx, Xb, row_ptr, col))
    with pytest.raises(rp.RPError):
        rp.rp_search(ctx, g, X[:2], 5, 10)  # L < k
    # the context still works after the errors
    t = rp.rp_tune(ctx, g, 1.1, 4)
    _same_csr(rp.rp_graph_export(ctx, t), oracle.rp_tune(X, row_ptr, col, 1.1, 4), "after errors")


def test_budget_is_enforced(ctx):
    small = rp.rp_create(0, hbm_budget_bytes=64 << 10)
    try:
        with pytest.raises(rp.RPError) as e:
            rp.rp_load_graph(small, datagen.dataset("sift", 2000))
        assert e.value.code == rp.RP_ENOMEM
    finally:
        rp.rp_destroy(small)


# ------------------------------------------------------------------ kNN and base graphs

@pytest.mark.parametrize("name", ["sift", "deep", "tiny"])
def test_knn_matches_oracle(ctx, name):
    X = datagen.dataset(name, 5000 if name != "tiny" else None)
    Q = datagen.queries(name, 100)
    g = rp.rp_load_graph(ctx, X)
    ids, dist = rp.rp_knn(ctx, g, Q, 100)
    ref, refd = oracle.knn(X, 100, Q=Q)
    assert np.array_equal(ids, ref)
    np.testing.assert_allclose(dist, refd, rtol=1e-5)
    # base points as queries, each excluded from its own list
    ids2, _ = rp.rp_knn(ctx, g, None, 64, nq=300)
    ref2, _ = oracle.knn(X, 64, qid=np.arange(300))
    assert np.array_equal(ids2, ref2)


def test_knn_candidate_base_matches_oracle(ctx):
    X = datagen.dataset("sift", 6000)
    g = rp.rp_load_graph(ctx, X)
    b = rp.rp_build_knn_base(ctx, g, 128, 1.2, 64)
    got = rp.rp_graph_export(ctx, b)
    ref = oracle.knn_base(X, 128, 1.2, 64)
    _same_csr(got, ref, "kNN-128 base at (1.2, 64)")
    for alpha, R in ((1.1, 64), (1.05, 48), (1.0, 32)):
        t = rp.rp_tune(ctx, b, alpha, R)
        _same_csr(rp.rp_graph_export(ctx, t), oracle.rp_tune(X, ref[0], ref[1], alpha, R), f"sift tune {alpha},{R}")


def test_float_knn_candidate_base_matches_oracle(ctx):
    X = datagen.dataset("deep", 4000)
    g = rp.rp_load_graph(ctx, X)
    b = rp.rp_build_knn_base(ctx, g, 128, 1.2, 64)
    _same_csr(rp.rp_graph_export(ctx, b), oracle.knn_base(X, 128, 1.2, 64), "deep kNN-128 base")


# ------------------------------------------------------------------ start vertex

@pytest.mark.parametrize("n", [1, 2, 63, 64, 65, 129, 1151, 4097])
def test_float_medoid_of_a_ramp(ctx, n):
    """The float mean adds rows in index order, 64 rows a group plus a ragged tail.
    Rows on a ramp (x = i in three columns, one of them in each 32-column group)
    put the mean at (n-1)/2, so the medoid (§4.1, ties to the smaller id) is row
    (n-1)//2; a skipped or repeated group moves it."""
    X = np.zeros((n, 96), dtype=np.float32)
    for c in (0, 40, 95):
        X[:, c] = np.arange(n, dtype=np.float32)
    g = rp.rp_load_graph(ctx, X)
    assert rp.rp_graph_info(ctx, g)["start"] == (n - 1) // 2
    rp.rp_graph_free(ctx, g)


@pytest.mark.parametrize("col", [0, 40, 95])
@pytest.mark.parametrize("k", [-1, 0, 1])
def test_float_medoid_to_the_last_bit(ctx, col, k):
    """The mean is on, or one ulp either side of, the midpoint of rows 0 and 1
    (the sum rounds thousands of times on the way): a mean one ulp off in
    either direction changes one of these answers."""
    X, expect = medoid_cases.tie_case(col, k)
    g = rp.rp_load_graph(ctx, X)
    assert rp.rp_graph_info(ctx, g)["start"] == expect
    rp.rp_graph_free(ctx, g)


def _medoid_data(kind, n, d, rng):
    X = rng.standard_normal((n, d)).astype(np.float32)
    if kind == "far rows":
        X[rng.integers(0, n, 8)] *= 40.0  # pull the mean off the origin
    elif kind == "wide range":
        X *= (2.0 ** rng.integers(-100, 44, (n, d))).astype(np.float32)  # loads take |x| <= 2^50
    elif kind == "zero and subnormal columns":
        X[:, ::3] = 0.0
        X[:, 1::3] *= np.float32(1e-40)  # subnormal float32 values
    elif kind == "alternating":
        X[:, 0] = np.where(np.arange(n) % 2 == 0, 1.0, -1.0)
    return X


@pytest.mark.parametrize("kind,n,d", [("far rows", 4097, 96), ("far rows", 20011, 100), ("far rows", 3001, 17),
                                      ("wide range", 5000, 96), ("zero and subnormal columns", 3003, 40),
                                      ("alternating", 2500, 8)])
def test_float_medoid_matches_oracle(ctx, kind, n, d):
    X = _medoid_data(kind, n, d, np.random.default_rng(n + d))
    g = rp.rp_load_graph(ctx, X)
    assert rp.rp_graph_info(ctx, g)["start"] == oracle.medoid(X)
    rp.rp_graph_free(ctx, g)


# ------------------------------------------------------------------ search

@pytest.mark.parametrize("L,k", [(64, 10), (32, 32), (100, 7)])
def test_tiny_search_matches_oracle(ctx, tiny, L, k):
    X, row_ptr, col = tiny
    Q = datagen.queries("tiny")
    g = rp.rp_load_graph(ctx, X, row_ptr, col)
    t = rp.rp_tune(ctx, g, 1.1, 32)
    trp, tcol = rp.rp_graph_export(ctx, t)
    start = rp.rp_graph_info(ctx, t)["start"]
    assert start == oracle.medoid(X)
    ids, dists = rp.rp_search(ctx, t, Q, L, k)
    ref, refd, _ = oracle.greedy_search(X, trp, tcol, start, Q, L, k)
    assert np.array_equal(ids, ref)
    np.testing.assert_allclose(dists, refd, rtol=1e-5)


def test_u8_search_and_recall_match_oracle(ctx):
    X = datagen.dataset("sift", 6000)
    Q = datagen.queries("sift", 200)
    g = rp.rp_load_graph(ctx, X)
    b = rp.rp_build_knn_base(ctx, g, 64, 1.2, 32)
    brp, bcol = rp.rp_graph_export(ctx, b)
    start = rp.rp_graph_info(ctx, b)["start"]
    assert start == oracle.medoid(X)
    ids, dists = rp.rp_search(ctx, b, Q, 128, 100)
    ref, refd, _ = oracle.greedy_search(X, brp, bcol, start, Q, 128, 100)
    assert np.array_equal(ids, ref)
    assert np.array_equal(dists.astype(np.float64), refd)  # exact integers
    gt, _ = rp.rp_knn(ctx, g, Q, 100)
    hits = rp.rp_recall(ctx, ids, gt, 100)
    assert hits / (100 * Q.shape[0]) == pytest.approx(oracle.recall_at_k(ref, gt, 100), abs=0)



@pytest.mark.parametrize("name", ["sift", "deep"])
def test_every_search_plan_gives_the_oracle_lists(ctx, name):
    """rp_set_search_config only moves work between CTAs and the id cache:
    every plan must return Algorithm 2's lists (a cache miss costs a distance,
    never a result)."""
    X = datagen.dataset(name, 3000)
    Q = datagen.queries(name, 150)
    brp, bcol = oracle.knn_base(X, 48, 1.2, 32)
    g = rp.rp_load_graph(ctx, X, brp, bcol)
    start = rp.rp_graph_info(ctx, g)["start"]
    ref, _, _ = oracle.greedy_search(X, brp, bcol, start, Q, 96, 50)
    try:
        for bits, ctas in [(0, 0), (8, 0), (9, 0), (12, 0), (8, 1), (10, 3), (11, 16), (0, 2)]:
            rp.rp_set_search_config(ctx, bits, ctas)
            ids, _ = rp.rp_search(ctx, g, Q, 96, 50)
            assert np.array_equal(ids, ref), (bits, ctas)
        for bits, ctas in [(7, 0), (13, 0), (-1, 0), (0, -1), (0, 17)]:
            with pytest.raises(rp.RPError):
                rp.rp_set_search_config(ctx, bits, ctas)
    finally:
        rp.rp_set_search_config(ctx, 0, 0)
    rp.rp_graph_free(ctx, g)

def test_search_unreachable_pads(ctx):
    X = np.arange(6, dtype=np.uint8)[:, None]
    row_ptr = np.array([0, 1, 2, 3, 4, 5, 6], np.int64)
    col = np.array([1, 0, 3, 2, 5, 4], np.int32)
    g = rp.rp_load_graph(ctx, X, row_ptr, col, start=0)
    ids, d = rp.rp_search(ctx, g, np.array([[5]], np.uint8), 4, 4)
    assert ids[0].tolist() == [1, 0, -1, -1]
    assert np.isinf(d[0, 2:]).all()


def test_device_buffers(ctx, tiny):
    torch = pytest.importorskip("torch")
    X, row_ptr, col = tiny
    dev = torch.device("cuda:0")
    Xt = torch.from_numpy(X).to(dev)
    g = rp.rp_load_graph(ctx, Xt, torch.from_numpy(row_ptr).to(dev), torch.from_numpy(col).to(dev))
    t = rp.rp_tune(ctx, g, 1.05, 16)
    r, c = rp.rp_graph_export(ctx, t, device=dev)
    _same_csr((r.cpu().numpy(), c.cpu().numpy()), oracle.rp_tune(X, row_ptr, col, 1.05, 16), "device buffers")
    Q = torch.from_numpy(datagen.queries("tiny", 50)).to(dev)
    ids, _ = rp.rp_search(ctx, t, Q, 40, 10)
    rp.rp_sync(ctx)
    ref, _, _ = oracle.greedy_search(X, r.cpu().numpy(), c.cpu().numpy(), rp.rp_graph_info(ctx, t)["start"],
                                     Q.cpu().numpy(), 40, 10)
    assert np.array_equal(ids.cpu().numpy(), ref)


def test_uint8_wide_rows_take_the_exact_path(ctx):
    # d = 384: bf16 partial sums could pass 2^24, so these rows must be pruned
    # on the exact integer path
    rng = np.random.default_rng(21)
    X = rng.integers(0, 256, size=(700, 384)).astype(np.uint8)
    row_ptr, col = datagen.random_graph(700, 10, 100, seed=4)
    g = rp.rp_load_graph(ctx, X, row_ptr, col)
    for alpha, R in ((1.0, 16), (1.2, rp.RP_R_INF)):
        t = rp.rp_tune(ctx, g, alpha, R)
        _same_csr(rp.rp_graph_export(ctx, t), oracle.rp_tune(X, row_ptr, col, alpha, R), f"u8 d=384 a={alpha}")
        rp.rp_graph_free(ctx, t)


@pytest.mark.parametrize("dtype", ["u8", "f32"])
def test_sixteen_targets_in_one_launch(ctx, dtype):
    n = 3000
    X = datagen.dataset("sift" if dtype == "u8" else "deep", n)
    row_ptr, col = datagen.random_graph(n, 0, 128, seed=16)
    g = rp.rp_load_graph(ctx, X, row_ptr, col)
    alphas = [1.0 + 0.013 * i for i in range(16)]
    Rs = [8 + 4 * i for i in range(16)]
    for variant in (rp.RP_SORTED, rp.RP_UNSORTED):
        outs = rp.rp_tune_batch(ctx, g, alphas, Rs, variant)
        for t, a, r in zip(outs, alphas, Rs):
            _same_csr(rp.rp_graph_export(ctx, t),
                      oracle.rp_tune(X, row_ptr, col, a, r, "sorted" if variant == rp.RP_SORTED else "unsorted"),
                      f"{dtype} 16 targets a={a} R={r}")
            rp.rp_graph_free(ctx, t)


@pytest.mark.parametrize("variant", ["sorted", "unsorted"])
def test_gist_shaped_wide_float_rows(ctx, variant):
    # d = 960: eight 128-dim slices per row on the tensor-core path, degrees
    # across all three buckets
    n = 2000
    X = datagen.dataset("gist", n)
    row_ptr, col = datagen.random_graph(n, 0, 150, seed=960, dup_frac=0.02, self_frac=0.01)
    g = rp.rp_load_graph(ctx, X, row_ptr, col)
    clean = rp.rp_graph_export(ctx, g)
    v = rp.RP_SORTED if variant == "sorted" else rp.RP_UNSORTED
    targets = [(1.175, 64), (1.1, 64), (1.025, 64), (1.0, 32)]
    outs = rp.rp_tune_batch(ctx, g, [a for a, _ in targets], [r for _, r in targets], v)
    for (a, r), o in zip(targets, outs):
        _same_csr(rp.rp_graph_export(ctx, o), oracle.rp_tune(X, clean[0], clean[1], a, r, variant),
                  f"gist {variant} a={a} R={r}")
        rp.rp_graph_free(ctx, o)
    rp.rp_graph_free(ctx, g)


def test_gist_shaped_knn_base_and_search(ctx):
    n = 3000
    X = datagen.dataset("gist", n)
    Q = datagen.queries("gist", 50)
    data = rp.rp_load_graph(ctx, X)
    base = rp.rp_build_knn_base(ctx, data, 64, 1.2, 48)
    got = rp.rp_graph_export(ctx, base)
    ref = oracle.knn_base(X, 64, 1.2, 48)
    _same_csr(got, ref, "gist kNN-64 base")
    start = rp.rp_graph_info(ctx, base)["start"]
    ids, dists = rp.rp_search(ctx, base, Q, 200, 100)
    ref_i, ref_d, _ = oracle.greedy_search(X, ref[0], ref[1], start, Q, 200, 100)
    assert np.array_equal(ids, ref_i)
    # float distances feeding recall: error against the binary64 reading
    rel = np.abs(dists.astype(np.float64) - ref_d) / np.maximum(ref_d, 1e-30)
    print(f"gist search distances: max relative error vs binary64 {rel.max():.3e}")
    assert rel.max() <= (960 + 8) * 2.0**-24
    rp.rp_graph_free(ctx, base)
    rp.rp_graph_free(ctx, data)
