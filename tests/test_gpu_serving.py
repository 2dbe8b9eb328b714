"""GPU parity of the serving path: the mixed search launch (rp_search_multi)
and the scheduler over a context (rp_server_create).  A query's result must
not depend on the batch it was served in: every mixed result is compared
element by element with the oracle's answer for that query alone, and with
rp_search on the same graph."""
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


@pytest.fixture(scope="module", params=["sift", "tiny"])
def world(request, ctx):
    name = request.param
    n = 6000 if name == "sift" else 2000
    X = datagen.dataset(name, n)
    base_rp, base_col = oracle.knn_base(X, 64, 1.2, 40)
    base = rp.rp_load_graph(ctx, X, base_rp, base_col)
    Q = datagen.queries(name, 256)
    start = rp.rp_graph_info(ctx, base)["start"]
    yield name, X, (base_rp, base_col), base, Q, start
    rp.rp_graph_free(ctx, base)


TARGETS = [(1.15, 40), (1.1, 32), (1.05, 24), (1.0, 16)]


def test_mixed_launch_matches_each_query_alone(ctx, world):
    name, X, (brp, bcol), base, Q, start = world
    tuned = rp.rp_tune_batch(ctx, base, [a for a, _ in TARGETS], [r for _, r in TARGETS])
    graphs = [base] + tuned
    rng = np.random.default_rng(5)
    nq, k = Q.shape[0], 20
    q_graph = rng.integers(0, len(graphs), nq).astype(np.int32)
    q_L = rng.choice([20, 33, 64, 100, 257], nq).astype(np.int32)
    ids, dists = rp.rp_search_multi(ctx, graphs, q_graph, q_L, Q, k)
    csr = [(brp, bcol)] + [oracle.rp_tune(X, brp, bcol, a, r) for a, r in TARGETS]
    for gi in range(len(graphs)):
        for L in np.unique(q_L):
            sel = np.nonzero((q_graph == gi) & (q_L == L))[0]
            if sel.size == 0:
                continue
            ref_i, ref_d, _ = oracle.greedy_search(X, csr[gi][0], csr[gi][1], start, Q[sel], int(L), k)
            assert np.array_equal(ids[sel], ref_i), f"graph {gi} L={L}"
            if name == "sift":
                assert np.array_equal(dists[sel].astype(np.float64), ref_d)
            alone_i, alone_d = rp.rp_search(ctx, graphs[gi], Q[sel], int(L), k)
            assert np.array_equal(alone_i, ids[sel]) and np.array_equal(alone_d, dists[sel])
    for t in tuned:
        rp.rp_graph_free(ctx, t)


def test_mixed_launch_rejects_bad_tables(ctx, world):
    name, X, _, base, Q, start = world
    with pytest.raises(rp.RPError):
        rp.rp_search_multi(ctx, [base], np.array([0, 1], np.int32), np.array([10, 10], np.int32), Q[:2], 10)
    with pytest.raises(rp.RPError):
        rp.rp_search_multi(ctx, [base], np.array([0, 0], np.int32), np.array([10, 5], np.int32), Q[:2], 10)
    with pytest.raises(rp.RPError):
        rp.rp_search_multi(ctx, [base], np.array([0, 0], np.int32), np.array([10, 2000], np.int32), Q[:2], 10)
    other = rp.rp_load_graph(ctx, X[:100].copy(), np.zeros(101, np.int64), np.zeros(0, np.int32))
    with pytest.raises(rp.RPError):  # graphs over different vectors
        rp.rp_search_multi(ctx, [base, other], np.array([0, 1], np.int32), np.array([10, 10], np.int32), Q[:2], 10)
    rp.rp_graph_free(ctx, other)


@pytest.mark.parametrize("serial", [False, True])
def test_server_stream_matches_each_request_alone(ctx, world, serial):
    from paper_2602_08097_gb300.serving import make_requests, replay
    name, X, (brp, bcol), base, Q, start = world
    stream = datagen.poisson_stream(60, 2000.0, seed=17, prune_frac=0.15)
    for e in stream:
        if e["kind"] == "search":
            e["nq"] = min(e["nq"], 64)
    reqs = make_requests(stream, Q, seed=17)
    gb = rp.rp_graph_shape(ctx, base)["adj_bytes"]
    srv = rp.rp_server_create(ctx, base, graph_budget_bytes=3 * gb, serial=serial)
    try:
        rep = replay(srv, reqs, time_scale=0.0)
    finally:
        rp.rp_server_destroy(srv)
    st = rep["stats"]
    assert st["requests_done"] == len(reqs) and st["peak_resident_graphs"] <= 3
    if serial:
        assert st["rounds"] == len(reqs)
    cache = {}
    for r in reqs:
        if r.kind != "search":
            continue
        key = (r.alpha, r.R)
        if key not in cache:
            cache[key] = oracle.rp_tune(X, brp, bcol, r.alpha, r.R)
        g_rp, g_col = cache[key]
        ref_i, ref_d, _ = oracle.greedy_search(X, g_rp, g_col, start, r.queries, max(r.L, r.k), r.k)
        assert np.array_equal(r.ids, ref_i), f"request alpha={r.alpha} R={r.R} L={r.L}"


def test_server_searches_the_base(ctx, world):
    name, X, (brp, bcol), base, Q, start = world
    srv = rp.rp_server_create(ctx, base)
    try:
        rid, ids, _ = rp.rp_submit_search(srv, 0.0, 0, Q[:16], 64, 10)
        info = rp.rp_poll(srv, rid, 60000)
    finally:
        rp.rp_server_destroy(srv)
    assert info["status"] == rp.RP_OK and info["graph"] == base
    ref_i, _, _ = oracle.greedy_search(X, brp, bcol, start, Q[:16], 64, 10)
    assert np.array_equal(ids, ref_i)


@pytest.mark.parametrize("chunks", [1, 3, 17])
def test_async_tuning_equals_batched_tuning(ctx, world, chunks):
    """rp_tune_batch_async (lowest-priority stream, the prune cut into node-range
    chunks) gives rp_tune_batch's graphs edge for edge; searches launched on
    the context's stream while it runs return the oracle's lists."""
    name, X, (brp, bcol), base, Q, start = world
    al, Rs = [a for a, _ in TARGETS], [r for _, r in TARGETS]
    ref = rp.rp_tune_batch(ctx, base, al, Rs)
    outs, ticket = rp.rp_tune_batch_async(ctx, base, al, Rs, chunks=chunks)
    ids, _ = rp.rp_search(ctx, base, Q[:32], 40, 10)  # on the ctx stream, meanwhile
    assert rp.rp_tune_wait(ctx, ticket, 60000)
    ref_i, _, _ = oracle.greedy_search(X, brp, bcol, start, Q[:32], 40, 10)
    assert np.array_equal(ids, ref_i)
    for g, r in zip(outs, ref):
        a_rp, a_col = rp.rp_graph_export(ctx, g)
        r_rp, r_col = rp.rp_graph_export(ctx, r)
        assert np.array_equal(a_rp, r_rp) and np.array_equal(a_col, r_col)
        rp.rp_graph_free(ctx, g)
        rp.rp_graph_free(ctx, r)
    with pytest.raises(rp.RPError):
        rp.rp_tune_wait(ctx, ticket + 5)
