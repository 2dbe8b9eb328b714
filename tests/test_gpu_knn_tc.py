"""Exact kNN on the tensor cores (rp_set_knn_method RP_KNN_TENSOR): the f16
Gram only filters candidates, so the lists must equal the CUDA-core scan's
and the oracle's exactly, distances included, for uint8 and float rows."""
import numpy as np
import pytest

import datagen
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
    rp.rp_set_knn_method(c, rp.RP_KNN_AUTO)
    rp.rp_destroy(c)


def _both(ctx, g, Q, k, nq=None):
    out = {}
    for m in (rp.RP_KNN_TENSOR, rp.RP_KNN_CUDA_CORE):
        rp.rp_set_knn_method(ctx, m)
        out[m] = rp.rp_knn(ctx, g, Q, k, nq=nq)
        assert rp.rp_stats(ctx)["knn_method"] == m
    rp.rp_set_knn_method(ctx, rp.RP_KNN_AUTO)
    return out[rp.RP_KNN_TENSOR], out[rp.RP_KNN_CUDA_CORE]


@pytest.mark.parametrize("name,n,k", [("sift", 5000, 100), ("sift", 1000, 128), ("deep", 4000, 100),
                                      ("tiny", 2000, 10), ("deep", 300, 128)])
def test_queries_match_the_cuda_core_scan_and_the_oracle(ctx, name, n, k):
    X = datagen.dataset(name, n)
    Q = datagen.queries(name, 300)
    g = rp.rp_load_graph(ctx, X)
    (ti, td), (ci, cd) = _both(ctx, g, Q, k)
    assert np.array_equal(ti, ci) and np.array_equal(td, cd)
    ref_i, ref_d = oracle.knn(X, k, Q=Q)
    assert np.array_equal(ti, ref_i)
    rp.rp_graph_free(ctx, g)


@pytest.mark.parametrize("name,n", [("sift", 4000), ("deep", 3000)])
def test_base_points_exclude_themselves(ctx, name, n):
    X = datagen.dataset(name, n)
    g = rp.rp_load_graph(ctx, X)
    (ti, td), (ci, cd) = _both(ctx, g, None, 64, nq=n)
    assert np.array_equal(ti, ci) and np.array_equal(td, cd)
    assert not np.any(ti == np.arange(n)[:, None])
    sel = np.arange(0, n, 97)
    ref_i, _ = oracle.knn(X, 64, qid=sel)
    assert np.array_equal(ti[sel], ref_i)
    rp.rp_graph_free(ctx, g)


def test_duplicates_and_exact_ties(ctx):
    # many repeated rows: equal distances are ordered by id
    rng = np.random.default_rng(4)
    base = rng.integers(0, 6, size=(40, 128), dtype=np.uint8)
    X = np.ascontiguousarray(base[rng.integers(0, 40, 3000)])
    Q = np.ascontiguousarray(base[:50])
    g = rp.rp_load_graph(ctx, X)
    (ti, td), (ci, cd) = _both(ctx, g, Q, 20)
    assert np.array_equal(ti, ci) and np.array_equal(td, cd)
    ref_i, _ = oracle.knn(X, 20, Q=Q)
    assert np.array_equal(ti, ref_i)
    rp.rp_graph_free(ctx, g)


def test_base_built_on_either_path_is_the_same(ctx):
    X = datagen.dataset("deep", 6000)
    g = rp.rp_load_graph(ctx, X)
    graphs = []
    for m in (rp.RP_KNN_TENSOR, rp.RP_KNN_CUDA_CORE):
        rp.rp_set_knn_method(ctx, m)
        b = rp.rp_build_knn_base(ctx, g, 64, 1.2, 48)
        graphs.append(rp.rp_graph_export(ctx, b))
        rp.rp_graph_free(ctx, b)
    rp.rp_set_knn_method(ctx, rp.RP_KNN_AUTO)
    assert np.array_equal(graphs[0][0], graphs[1][0]) and np.array_equal(graphs[0][1], graphs[1][1])
    rp.rp_graph_free(ctx, g)


def test_method_limits(ctx):
    X = datagen.dataset("sift", 500)
    g = rp.rp_load_graph(ctx, X)
    Q = datagen.queries("sift", 5)
    rp.rp_set_knn_method(ctx, rp.RP_KNN_TENSOR)
    with pytest.raises(rp.RPError):
        rp.rp_knn(ctx, g, Q, 200)  # k above 128
    rp.rp_set_knn_method(ctx, rp.RP_KNN_AUTO)
    ids, _ = rp.rp_knn(ctx, g, Q, 200)  # falls back to the CUDA-core scan
    assert rp.rp_stats(ctx)["knn_method"] == rp.RP_KNN_CUDA_CORE
    assert np.array_equal(ids, oracle.knn(X, 200, Q=Q)[0])
    with pytest.raises(rp.RPError):
        rp.rp_set_knn_method(ctx, 9)
    rp.rp_graph_free(ctx, g)
    G = datagen.dataset("gist", 300)  # d = 960: beyond the tensor-core path
    gg = rp.rp_load_graph(ctx, G)
    rp.rp_set_knn_method(ctx, rp.RP_KNN_TENSOR)
    with pytest.raises(rp.RPError):
        rp.rp_knn(ctx, gg, G[:3].copy(), 10)
    rp.rp_set_knn_method(ctx, rp.RP_KNN_AUTO)
    rp.rp_graph_free(ctx, gg)


def _splitmix64(x):
    # splitmix64 (Steele, Lea and Flood; Vigna's reference form), on uint64 arrays
    x = (x + np.uint64(0x9E3779B97F4A7C15)).astype(np.uint64)
    x = ((x ^ (x >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)).astype(np.uint64)
    x = ((x ^ (x >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)).astype(np.uint64)
    return x ^ (x >> np.uint64(31))


@pytest.mark.parametrize("name", ["deep", "sift"])
def test_random_candidate_base_matches_the_oracle(ctx, name):
    n, kk, nr, seed = 3000, 32, 16, 77
    X = datagen.dataset(name, n)
    g = rp.rp_load_graph(ctx, X)
    b = rp.rp_build_knn_random_base(ctx, g, kk, nr, seed, 1.2, 40)
    got = rp.rp_graph_export(ctx, b)
    # the candidate rows: exact kNN, then nr draws over the other points
    knn_ids, _ = oracle.knn(X, kk, qid=np.arange(n))
    with np.errstate(over="ignore"):
        p = np.repeat(np.arange(n, dtype=np.uint64), nr)
        j = np.tile(np.arange(nr, dtype=np.uint64), n)
        h = _splitmix64(np.uint64(seed) ^ _splitmix64(p * np.uint64(131) + j))
    v = (h % np.uint64(n - 1)).astype(np.int64).reshape(n, nr)
    v += v >= np.arange(n)[:, None]
    cand = np.concatenate([knn_ids.astype(np.int64), v], axis=1).astype(np.int32)
    row_ptr = np.arange(n + 1, dtype=np.int64) * (kk + nr)
    ref = oracle.rp_tune(X, row_ptr, cand.ravel(), 1.2, 40)
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])
    # the base now links far points: some kept edge is not among the kNN candidates
    assert any(set(got[1][got[0][q]:got[0][q + 1]]) - set(knn_ids[q]) for q in range(0, n, 10))
    with pytest.raises(rp.RPError):
        rp.rp_build_knn_random_base(ctx, g, kk, 200, seed, 1.2, 40)
    rp.rp_graph_free(ctx, b)
    rp.rp_graph_free(ctx, g)
