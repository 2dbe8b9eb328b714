"""alpha-reachability (Definition 2.1) through the C ABI (rp_reachability)
against the oracle's per-node terms, exactly: both sides take D = sqrt of the
exact (uint8) or canonical binary64 (float) squared distance and divide in
binary64.  Also Lemma 2.2 on the slow preprocessing base, the closed forms and
the edge cases."""
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
    rp.rp_destroy(c)


def test_slow_base_and_its_tunings(ctx):
    X = datagen.dataset("tiny", 600)
    rpb, colb = oracle.slow_base(X, 1.5)
    g = rp.rp_load_graph(ctx, X, rpb, colb)
    a, per = rp.rp_reachability(ctx, g)
    ref = oracle.reachability_nodes(X, rpb, colb)
    assert np.array_equal(per, ref) and a == ref.min()
    assert a >= 1.5  # Lemma 2.2
    for alpha, R, variant in [(1.1, 16, rp.RP_SORTED), (1.2, rp.RP_R_INF, rp.RP_UNSORTED), (1.0, 8, rp.RP_SORTED)]:
        t = rp.rp_tune(ctx, g, alpha, R, variant)
        trp, tcol = rp.rp_graph_export(ctx, t)
        a, per = rp.rp_reachability(ctx, t)
        ref = oracle.reachability_nodes(X, trp, tcol)
        assert np.array_equal(per, ref), (alpha, R, variant)
        assert a == ref.min()
        rp.rp_graph_free(ctx, t)
    rp.rp_graph_free(ctx, g)


@pytest.mark.parametrize("name,n", [("sift", 1500), ("deep", 1200)])
def test_knn_bases(ctx, name, n):
    X = datagen.dataset(name, n)
    brp, bcol = oracle.knn_base(X, 32, 1.2, 24)
    g = rp.rp_load_graph(ctx, X, brp, bcol)
    a, per = rp.rp_reachability(ctx, g)
    assert np.array_equal(per, oracle.reachability_nodes(X, brp, bcol))
    nodes = np.array([n - 1, 0, 17, 17, n // 2], dtype=np.int64)
    a2, per2 = rp.rp_reachability(ctx, g, nodes)
    assert np.array_equal(per2, per[nodes]) and a2 == per[nodes].min()
    rp.rp_graph_free(ctx, g)


def test_sampled_nodes_of_a_larger_graph(ctx):
    X = datagen.dataset("sift", 20000)
    data = rp.rp_load_graph(ctx, X)
    base = rp.rp_build_knn_base(ctx, data, 64, 1.2, 48)
    t = rp.rp_tune(ctx, base, 1.05, 32)
    nodes = np.random.default_rng(5).choice(20000, 24, replace=False).astype(np.int64)
    for g in (base, t):
        g_rp, g_col = rp.rp_graph_export(ctx, g)
        a, per = rp.rp_reachability(ctx, g, nodes)
        ref = oracle.reachability_nodes(X, g_rp, g_col, nodes)
        assert np.array_equal(per, ref) and a == ref.min()
    for g in (t, base, data):
        rp.rp_graph_free(ctx, g)


def test_closed_forms_and_edge_cases(ctx):
    # points 0, 1, 3 on a line
    X = np.array([[0], [1], [3]], dtype=np.uint8)
    g = rp.rp_load_graph(ctx, X, np.array([0, 1, 2, 3], np.int64), np.array([1, 2, 1], np.int32), start=0)
    a, per = rp.rp_reachability(ctx, g)
    assert per.tolist() == [1.5, 1 / 3, 3.0] and a == 1 / 3  # worked by hand
    h = rp.rp_load_graph(ctx, X, np.array([0, 0, 2, 3], np.int64), np.array([0, 2, 1], np.int32), start=1)
    _, per = rp.rp_reachability(ctx, h)
    assert per.tolist() == [0.0, np.inf, 3.0]  # no out-neighbour; adjacent to all; 3 / 1
    a, per = rp.rp_reachability(ctx, g, np.zeros(0, np.int64))
    assert a == np.inf and per.size == 0
    for bad in ([3], [-1]):
        with pytest.raises(rp.RPError):
            rp.rp_reachability(ctx, g, np.array(bad, np.int64))
    # a duplicate of q among p's out-neighbours reaches q at every alpha
    Y = np.array([[0, 0], [5, 0], [5, 0], [9, 9]], dtype=np.float32)
    k = rp.rp_load_graph(ctx, Y, np.array([0, 1, 2, 2, 3], np.int64), np.array([1, 0, 1], np.int32), start=0)
    k_rp, k_col = rp.rp_graph_export(ctx, k)
    _, per = rp.rp_reachability(ctx, k)
    assert np.array_equal(per, oracle.reachability_nodes(Y, k_rp, k_col))
    for x in (g, h, k):
        rp.rp_graph_free(ctx, x)
