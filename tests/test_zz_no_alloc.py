"""rp_search_noalloc: the search entry point for callers that cannot allocate
device memory (their memory is reserved up front, or they must not see
allocations while capturing a stream).  It must return what rp_search returns
on the same graph and queries, on two calls in a row (the second call reuses
the fixed scratch array the first one left behind).  This file is collected
last so that a failure here stops a -x run only after every other test."""
import numpy as np
import pytest

import datagen

rp = pytest.importorskip("paper_2602_08097_gb300")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_08097_gb300 import build as b
    b.build()
    ctx = rp.rp_create(0)
    yield torch, ctx
    rp.rp_destroy(ctx)


def _rows(name, n, nq, dims):
    """The workload's seeded rows, cut to their first ``dims`` dimensions when
    given (a row stride that is not a multiple of 128 bytes)."""
    X = datagen.dataset(name, n)
    Q = datagen.queries(name, nq)
    if dims is not None:
        X = np.ascontiguousarray(X[:, :dims])
        Q = np.ascontiguousarray(Q[:, :dims])
    return X, Q


def _graph_on_device(torch, ctx, name, n, nq, kcand, alpha, R, dims=None):
    X, Q = _rows(name, n, nq, dims)
    g = rp.rp_load_graph(ctx, X)
    b = rp.rp_build_knn_base(ctx, g, kcand, alpha, R)
    row_ptr, col = rp.rp_graph_export(ctx, b)
    start = rp.rp_graph_info(ctx, b)["start"]
    dev = torch.device("cuda:0")
    tens = [torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (X, row_ptr, col, Q)]
    return b, Q, start, tens


# (workload, n, L, k, dims): the last two cases cut the rows to 100 float32
# dimensions (400-byte rows: a short last 32-dimension slice) and to 48 uint8
# dimensions (48-byte rows), strides rp_search never sees (it pads rows to 128
# bytes), so the packed-row reads are compared with the padded ones.
@pytest.mark.parametrize("name,n,L,k,dims", [("sift", 6000, 128, 100, None), ("deep", 5000, 64, 10, None),
                                             ("tiny", 2000, 64, 10, None), ("gist", 3000, 64, 10, 100),
                                             ("sift", 4000, 64, 10, 48)])
def test_no_alloc_search_matches_rp_search(env, name, n, L, k, dims):
    torch, ctx = env
    b, Q, start, (Xd, rpd, cold, Qd) = _graph_on_device(torch, ctx, name, n, 300, 64, 1.2, 32, dims)
    ref_ids, ref_d = rp.rp_search(ctx, b, Q, L, k)
    for _ in range(2):
        ids, dists = rp.rp_search_noalloc(Xd, rpd, cold, start, Qd, L, k)
        torch.cuda.synchronize()
        assert np.array_equal(ids.cpu().numpy(), ref_ids)
        np.testing.assert_allclose(dists.cpu().numpy(), ref_d, rtol=1e-5)
    # no distance buffer (dists == NULL at the C ABI): the same ids
    ids2, none = rp.rp_search_noalloc(Xd, rpd, cold, start, Qd, L, k, want_dists=False)
    assert none is None
    assert np.array_equal(ids2.cpu().numpy(), ref_ids)
    rp.rp_graph_free(ctx, b)


def test_no_alloc_status_is_read_back(env):
    """The device status word of the last call comes back through
    rp_search_noalloc_status; a clean search reports RP_OK."""
    import ctypes
    torch, ctx = env
    b, Q, start, (Xd, rpd, cold, Qd) = _graph_on_device(torch, ctx, "tiny", 1000, 50, 64, 1.2, 32)
    s = torch.cuda.Stream()
    rp.rp_search_noalloc(Xd, rpd, cold, start, Qd, 32, 10, stream=s, check_status=False)
    info = ctypes.c_int64(-7)
    rc = rp.load_library().rp_search_noalloc_status(ctypes.c_void_p(s.cuda_stream), ctypes.byref(info))
    assert rc == rp.RP_OK and info.value == 0
    rp.rp_graph_free(ctx, b)


def test_no_alloc_search_rejects_bad_arguments(env):
    torch, ctx = env
    dev = torch.device("cuda:0")
    X = torch.zeros((10, 3), dtype=torch.uint8, device=dev)  # 3-byte rows: not a multiple of 16
    rp_ = torch.zeros(11, dtype=torch.int64, device=dev)
    col = torch.zeros(1, dtype=torch.int32, device=dev)
    with pytest.raises(rp.RPError) as e:
        rp.rp_search_noalloc(X, rp_, col, 0, X[:2], 8, 4)
    assert e.value.code == rp.RP_EINVAL
    Xok = torch.zeros((10, 16), dtype=torch.uint8, device=dev)
    with pytest.raises(rp.RPError):
        rp.rp_search_noalloc(Xok, rp_, col, 0, Xok[:2], 4, 8)  # L < k
    with pytest.raises(rp.RPError):
        rp.rp_search_noalloc(Xok, rp_, col, 10, Xok[:2], 8, 4)  # start outside [0, n)
    # caught by the binding before the library sees a pointer
    with pytest.raises(ValueError):
        rp.rp_search_noalloc(Xok, rp_.to(torch.int32), col, 0, Xok[:2], 8, 4)  # row_ptr not int64
    with pytest.raises(ValueError):
        rp.rp_search_noalloc(Xok, rp_[:-1], col, 0, Xok[:2], 8, 4)  # row_ptr not n + 1 long
    with pytest.raises(ValueError):
        rp.rp_search_noalloc(Xok, rp_, col, 0, Xok[:2].float(), 8, 4)  # queries of another dtype
    with pytest.raises(ValueError):
        rp.rp_search_noalloc(Xok, rp_, col, 0, Xok[:2, :8], 8, 4)  # queries of another width
    with pytest.raises(ValueError):
        rp.rp_search_noalloc(Xok, rp_, col, 0, Xok[:2], 8, 4,
                             ids=torch.empty(3, dtype=torch.int32, device=dev))  # ids too small
