"""Vamana construction on the GPU (§2.1 "fast preprocessing"; §4.1 builds the
paper's base indices with it) against the oracle's batched reading: the same
insertion order and batch schedule must give the same graph, every list
element by element, order included.  Covers the hand-traced line, float and
uint8 rows, one and two passes, batches small enough that many back-edge
lists overflow R and are pruned again, and searches whose visited sets are
cut to vcap."""
import json
import os

import numpy as np
import pytest

import datagen
import oracle

rp = pytest.importorskip("paper_2602_08097_gb300")
pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden")


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


def test_hand_traced_line(ctx):
    with open(os.path.join(GOLD, "vamana_line.json")) as f:
        g = json.load(f)
    X = np.asarray(g["x"], dtype=np.float32)[:, None]
    data = rp.rp_load_graph(ctx, X, start=g["start"])
    v, cut = rp.rp_build_vamana(ctx, data, g["alphas"], g["R"], g["L"], g["vcap"], g["max_batch"], g["perm"])
    rp_, col = rp.rp_graph_export(ctx, v)
    assert [col[rp_[p]:rp_[p + 1]].tolist() for p in range(X.shape[0])] == g["rows"]
    assert cut == 0


def _rows(name, n, dims=None):
    X = datagen.dataset(name, n)
    if dims is not None:
        X = np.ascontiguousarray(X[:, :dims])
    return X


# (workload, n, dims, alphas, R, L, vcap, max_batch)
CASES = [
    ("tiny", 2000, None, [1.0, 1.2], 24, 40, 160, 64),
    ("deep", 3000, None, [1.0, 1.2], 32, 50, 200, 128),
    ("sift", 3000, None, [1.2], 32, 50, 200, 256),
    ("sift", 2500, 48, [1.0, 1.1], 16, 32, 24, 100),   # vcap below the expansions: cut visited sets
    ("gist", 1500, None, [1.2], 40, 60, 240, 32),
]


@pytest.mark.parametrize("name,n,dims,alphas,R,L,vcap,max_batch", CASES)
def test_matches_oracle(ctx, name, n, dims, alphas, R, L, vcap, max_batch):
    X = _rows(name, n, dims)
    perm = np.random.default_rng(n + R).permutation(n).astype(np.int32)
    data = rp.rp_load_graph(ctx, X)
    start = rp.rp_graph_info(ctx, data)["start"]
    assert start == oracle.medoid(X)
    v, cut = rp.rp_build_vamana(ctx, data, alphas, R, L, vcap, max_batch, perm)
    got_rp, got_col = rp.rp_graph_export(ctx, v)
    ref_rp, ref_col, ref_cut = oracle.vamana(X, perm, alphas, R, L, vcap, max_batch, start)
    assert cut == ref_cut
    assert np.array_equal(got_rp, ref_rp)
    assert np.array_equal(got_col, ref_col)
    assert np.diff(got_rp).max() <= R
    rp.rp_graph_free(ctx, v)
    rp.rp_graph_free(ctx, data)


def test_identity_order_and_defaults(ctx):
    """perm = NULL inserts 0 .. n-1; the default batch cap is n // 50 and vcap 4 L."""
    X = datagen.dataset("tiny", 1200)
    data = rp.rp_load_graph(ctx, X)
    start = rp.rp_graph_info(ctx, data)["start"]
    v, cut = rp.rp_build_vamana(ctx, data, [1.2], 20, 30)
    ref_rp, ref_col, ref_cut = oracle.vamana(X, np.arange(1200), [1.2], 20, 30, 120, 24, start)
    got_rp, got_col = rp.rp_graph_export(ctx, v)
    assert np.array_equal(got_rp, ref_rp) and np.array_equal(got_col, ref_col) and cut == ref_cut


def test_rejects_bad_arguments(ctx):
    X = datagen.dataset("tiny", 100)
    data = rp.rp_load_graph(ctx, X)
    for kw in (dict(alphas=[0.9]), dict(alphas=[1.0001]), dict(R=0), dict(L=0), dict(perm=np.zeros(100, np.int32))):
        args = dict(alphas=[1.2], R=8, L=16, vcap=0, max_batch=0, perm=None)
        args.update(kw)
        with pytest.raises(rp.RPError):
            rp.rp_build_vamana(ctx, data, args["alphas"], args["R"], args["L"], args["vcap"], args["max_batch"],
                               args["perm"])


def test_hub_takes_at_most_512_back_edges_a_batch(ctx):
    # Point 0 sits at the centre of a thin shell of 2,999 points in 64 dimensions,
    # nearer to each of them than any other point, so every point keeps it (first
    # in its processing order), and the batches of 1,024 and 953 points name it
    # that many times: its senders are cut to the 512 smallest ids (found by the
    # bisection on the id value) before the merge and the prune.
    rng = np.random.default_rng(11)
    n = 3000
    U = rng.normal(size=(n, 64))
    U /= np.linalg.norm(U, axis=1, keepdims=True)
    X = (U * (1.0 + 0.05 * rng.random((n, 1)))).astype(np.float32)
    X[0] = 0.0
    perm = rng.permutation(n).astype(np.int32)
    data = rp.rp_load_graph(ctx, X)
    start = rp.rp_graph_info(ctx, data)["start"]
    assert start == oracle.medoid(X) == 0
    for alphas in ([1.2], [1.0, 1.2]):
        v, cut = rp.rp_build_vamana(ctx, data, alphas, 16, 32, 128, 2048, perm)
        got_rp, got_col = rp.rp_graph_export(ctx, v)
        ref_rp, ref_col, ref_cut = oracle.vamana(X, perm, alphas, 16, 32, 128, 2048, start)
        assert all(0 in ref_col[ref_rp[p]:ref_rp[p + 1]] for p in range(1, n))
        assert cut == ref_cut
        assert np.array_equal(got_rp, ref_rp) and np.array_equal(got_col, ref_col)
        rp.rp_graph_free(ctx, v)
    rp.rp_graph_free(ctx, data)
