"""Python binding of librp.so (the C ABI in include/rp.h), argument marshalling only.

Every function here has the name of the C entry point it calls and does no
computation of its own: numpy arrays are passed as host memory
(RP_MEM_HOST), CUDA torch tensors as device memory (RP_MEM_DEVICE), and all
work runs in the library's kernels.  There is no fallback: if librp.so is
missing or cannot be loaded, :func:`load_library` raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "librp.so")

RP_OK, RP_EINVAL, RP_ENOMEM, RP_ECUDA, RP_ETIMEOUT, RP_ENOTFOUND, RP_EDEVICE = 0, -1, -2, -3, -4, -5, -6
RP_U8, RP_F32 = 1, 2
RP_SORTED, RP_UNSORTED = 0, 1
RP_MEM_HOST, RP_MEM_DEVICE = 0, 1
RP_R_INF = 2**31 - 1
RP_MAX_DEGREE = 8192
RP_MAX_L = 1024
RP_TUNING_AUTO, RP_TUNING_FIXED = 0, 1
RP_KNN_AUTO, RP_KNN_CUDA_CORE, RP_KNN_TENSOR = 0, 1, 2

_NAMES = {RP_EINVAL: "RP_EINVAL", RP_ENOMEM: "RP_ENOMEM", RP_ECUDA: "RP_ECUDA", RP_ETIMEOUT: "RP_ETIMEOUT",
          RP_ENOTFOUND: "RP_ENOTFOUND", RP_EDEVICE: "RP_EDEVICE"}


class RPError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


class rp_stats_t(ctypes.Structure):
    _fields_ = [("nodes_pruned", ctypes.c_int64), ("fp64_decisions", ctypes.c_int64),
                ("fp64_sort_keys", ctypes.c_int64), ("fp64_search_dists", ctypes.c_int64),
                ("self_loops_dropped", ctypes.c_int64), ("duplicates_dropped", ctypes.c_int64),
                ("generic_nodes", ctypes.c_int64), ("graph_replays", ctypes.c_int64),
                ("bytes_in_use", ctypes.c_uint64), ("bytes_peak", ctypes.c_uint64),
                ("kernel_launches", ctypes.c_int64), ("last_prune_ms", ctypes.c_float),
                ("last_emit_ms", ctypes.c_float), ("last_search_ms", ctypes.c_float),
                ("tile0", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("knn_method", ctypes.c_int32), ("pad_", ctypes.c_int32),
                ("f32_rechecks", ctypes.c_int64)]


class rp_request_info(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int32), ("status", ctypes.c_int32), ("graph", ctypes.c_int64),
                ("L_eff", ctypes.c_int32), ("round", ctypes.c_int32), ("submit_ns", ctypes.c_int64),
                ("start_ns", ctypes.c_int64), ("done_ns", ctypes.c_int64)]


class rp_server_stats_t(ctypes.Structure):
    _fields_ = [(name, ctypes.c_int64) for name in (
        "requests_done", "requests_failed", "queries_done", "rounds", "tune_launches", "targets_tuned",
        "search_launches", "evictions", "l_clamps", "resident_graphs", "peak_resident_graphs", "busy_ns")]


TUNE_FN = ctypes.CFUNCTYPE(ctypes.c_int32, ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_double),
                           ctypes.POINTER(ctypes.c_int32), ctypes.c_int32, ctypes.POINTER(ctypes.c_int64))
SEARCH_FN = ctypes.CFUNCTYPE(ctypes.c_int32, ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64), ctypes.c_int32,
                             ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32), ctypes.c_void_p,
                             ctypes.c_int64, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                             ctypes.POINTER(ctypes.c_float))
FREE_FN = ctypes.CFUNCTYPE(ctypes.c_int32, ctypes.c_void_p, ctypes.c_int64)
TUNE_START_FN = ctypes.CFUNCTYPE(ctypes.c_int32, ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_double),
                                 ctypes.POINTER(ctypes.c_int32), ctypes.c_int32, ctypes.POINTER(ctypes.c_int64),
                                 ctypes.POINTER(ctypes.c_int64))
TUNE_READY_FN = ctypes.CFUNCTYPE(ctypes.c_int32, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32)


class rp_executor(ctypes.Structure):
    _fields_ = [("user", ctypes.c_void_p), ("tune_batch", TUNE_FN), ("search_multi", SEARCH_FN),
                ("graph_free", FREE_FN), ("tune_start", TUNE_START_FN), ("tune_ready", TUNE_READY_FN)]


class rp_server_config(ctypes.Structure):
    _fields_ = [("base", ctypes.c_int64), ("d", ctypes.c_int32), ("dtype", ctypes.c_int32),
                ("graph_bytes", ctypes.c_uint64), ("graph_budget_bytes", ctypes.c_uint64),
                ("max_batch_queries", ctypes.c_int64), ("serial", ctypes.c_int32)]


_lib = None


def load_library(path: str = LIB_PATH):
    """Load librp.so (built by ``paper_2602_08097_gb300.build.build()``); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"librp.so not found at {path}: build it with __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    P, i32, i64, u64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
    sig = {
        "rp_create": [ctypes.POINTER(P), i32, u64, P],
        "rp_destroy": [P],
        "rp_sync": [P],
        "rp_load_graph": [P, P, i32, i64, i32, P, P, i32, i32, ctypes.POINTER(i64)],
        "rp_tune": [P, i64, dbl, i32, i32, ctypes.POINTER(i64)],
        "rp_tune_batch": [P, i64, P, P, i32, i32, P],
        "rp_tune_batch_async": [P, i64, P, P, i32, i32, i32, P, ctypes.POINTER(i64)],
        "rp_graph_attach": [P, i64, P, P, i32, ctypes.POINTER(i64)],
        "rp_debug_gram": [P, i64, P, P, i64, P],
        "rp_tune_wait": [P, i64, i32],
        "rp_graph_info": [P, i64, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i32), ctypes.POINTER(i64)],
        "rp_graph_export": [P, i64, P, P, i64, i32],
        "rp_search": [P, i64, P, i64, i32, i32, P, P, i32],
        "rp_knn": [P, i64, P, i64, i32, P, P, i32],
        "rp_recall": [P, P, i32, P, i32, i64, i32, ctypes.POINTER(i64), i32],
        "rp_reachability": [P, i64, P, i64, P, ctypes.POINTER(ctypes.c_double)],
        "rp_build_knn_base": [P, i64, i32, dbl, i32, ctypes.POINTER(i64)],
        "rp_build_knn_random_base": [P, i64, i32, i32, u64, dbl, i32, ctypes.POINTER(i64)],
        "rp_build_vamana": [P, i64, P, i32, P, i32, i32, i32, i64, ctypes.POINTER(i64), ctypes.POINTER(i64)],
        "rp_graph_free": [P, i64],
        "rp_stats": [P, ctypes.POINTER(rp_stats_t), i32],
        "rp_search_noalloc": [P, i32, i64, i32, P, P, i64, P, i64, i32, i32, P, P, P],
        "rp_search_noalloc_status": [P, ctypes.POINTER(i64)],
        "rp_search_multi": [P, P, i32, P, P, P, i64, i32, P, P, i32],
        "rp_graph_shape": [P, i64, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(u64)],
        "rp_graph_slice": [P, i64, i64, i64, ctypes.POINTER(i64)],
        "rp_set_tuning": [P, i32, i32, i32],
        "rp_set_knn_method": [P, i32],
        "rp_set_search_config": [P, i32, i32],
        "rp_server_create": [P, i64, u64, i64, i32, ctypes.POINTER(P)],
        "rp_server_create_ex": [ctypes.POINTER(rp_executor), ctypes.POINTER(rp_server_config), ctypes.POINTER(P)],
        "rp_server_destroy": [P],
        "rp_submit_tune": [P, dbl, i32, ctypes.POINTER(i64)],
        "rp_submit_search": [P, dbl, i32, P, i64, i32, i32, P, P, ctypes.POINTER(i64)],
        "rp_poll": [P, i64, i32, ctypes.POINTER(rp_request_info)],
        "rp_server_stats": [P, ctypes.POINTER(rp_server_stats_t)],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = i32
    lib.rp_last_error.argtypes = [P]
    lib.rp_last_error.restype = ctypes.c_char_p
    lib.rp_server_last_error.argtypes = [P]
    lib.rp_server_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _check(ctx, rc):
    if rc != RP_OK:
        msg = load_library().rp_last_error(ctx).decode(errors="replace") if ctx else ""
        raise RPError(rc, msg)


def _is_torch(x):
    return type(x).__module__.split(".")[0] == "torch"


def _mem(*arrays):
    kinds = {("dev" if (_is_torch(a) and a.is_cuda) else "host") for a in arrays if a is not None}
    if len(kinds) > 1:
        raise TypeError("mix of host and device buffers in one call")
    return RP_MEM_DEVICE if kinds == {"dev"} else RP_MEM_HOST


def _ptr(a):
    if a is None:
        return None
    if _is_torch(a):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(a.data_ptr())
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous")
    return ctypes.c_void_p(a.ctypes.data)


def _dtype_code(x):
    name = str(x.dtype).split(".")[-1]
    if name == "uint8":
        return RP_U8
    if name == "float32":
        return RP_F32
    raise TypeError(f"vectors must be uint8 or float32, got {x.dtype}")


def _empty_like_mem(mem, shape, np_dtype, device=None):
    if mem == RP_MEM_HOST:
        return np.empty(shape, dtype=np_dtype)
    import torch
    tdt = {np.int32: torch.int32, np.float32: torch.float32, np.int64: torch.int64}[np_dtype]
    return torch.empty(shape, dtype=tdt, device=device)


def rp_create(device: int = 0, hbm_budget_bytes: int = 0, stream=None):
    """Returns an opaque context handle.  ``stream``: a torch.cuda.Stream, a raw handle or None."""
    lib = load_library()
    h = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
    out = ctypes.c_void_p()
    rc = lib.rp_create(ctypes.byref(out), int(device), int(hbm_budget_bytes), ctypes.c_void_p(h) if h else None)
    _check(None, rc)
    return out


def rp_destroy(ctx):
    _check(None, load_library().rp_destroy(ctx))


def rp_last_error(ctx) -> str:
    return load_library().rp_last_error(ctx).decode(errors="replace")


def rp_sync(ctx):
    _check(ctx, load_library().rp_sync(ctx))


def rp_load_graph(ctx, vectors, row_ptr=None, col=None, start: int = -1) -> int:
    mem = _mem(vectors, row_ptr, col)
    n, d = int(vectors.shape[0]), int(vectors.shape[1])
    out = ctypes.c_int64()
    _check(ctx, load_library().rp_load_graph(ctx, _ptr(vectors), _dtype_code(vectors), n, d, _ptr(row_ptr),
                                             _ptr(col), int(start), mem, ctypes.byref(out)))
    return out.value


def rp_tune(ctx, src: int, alpha: float, R: int = RP_R_INF, variant: int = RP_SORTED) -> int:
    out = ctypes.c_int64()
    _check(ctx, load_library().rp_tune(ctx, int(src), float(alpha), int(R), int(variant), ctypes.byref(out)))
    return out.value


def rp_tune_batch(ctx, src: int, alphas, Rs, variant: int = RP_SORTED):
    T = len(alphas)
    a = (ctypes.c_double * T)(*[float(x) for x in alphas])
    r = (ctypes.c_int32 * T)(*[int(x) for x in Rs])
    outs = (ctypes.c_int64 * T)()
    _check(ctx, load_library().rp_tune_batch(ctx, int(src), a, r, T, int(variant), outs))
    return list(outs)


def rp_debug_gram(ctx, g: int, rows, centres=None) -> np.ndarray:
    """Test support: the prune kernel's split-f16 Gram of float rows, 128 at a time,
    each 64-row half centred on its row of ``centres`` (one per half) if given;
    returns float32[len(rows) // 128, 128, 128]."""
    rows = np.ascontiguousarray(rows, dtype=np.int32)
    if centres is not None:
        centres = np.ascontiguousarray(centres, dtype=np.int32)
        if centres.shape != (rows.shape[0] // 64,):
            raise ValueError("centres needs one row id per 64 rows")
    out = np.empty((rows.shape[0] // 128, 128, 128), dtype=np.float32)
    _check(ctx, load_library().rp_debug_gram(ctx, int(g), _ptr(rows), _ptr(centres), rows.shape[0], _ptr(out)))
    return out


def rp_graph_attach(ctx, data: int, row_ptr, col) -> int:
    """A graph over the vectors of ``data`` from a CSR (numpy arrays or CUDA tensors)."""
    mem = _mem(row_ptr, col)
    out = ctypes.c_int64()
    _check(ctx, load_library().rp_graph_attach(ctx, int(data), _ptr(row_ptr), _ptr(col), mem, ctypes.byref(out)))
    return out.value


def rp_tune_batch_async(ctx, src: int, alphas, Rs, chunks: int = 16, variant: int = RP_SORTED):
    """rp_tune_batch on the low-priority stream in `chunks` launches; returns (graphs, ticket).
    The graphs may be used once rp_tune_wait(ctx, ticket) returns True."""
    T = len(alphas)
    a = (ctypes.c_double * T)(*[float(x) for x in alphas])
    r = (ctypes.c_int32 * T)(*[int(x) for x in Rs])
    outs = (ctypes.c_int64 * T)()
    ticket = ctypes.c_int64()
    _check(ctx, load_library().rp_tune_batch_async(ctx, int(src), a, r, T, int(variant), int(chunks), outs,
                                                   ctypes.byref(ticket)))
    return list(outs), ticket.value


def rp_tune_wait(ctx, ticket: int, timeout_ms: int = 0) -> bool:
    """True once tuning job `ticket` is finished, False if still running after timeout_ms."""
    rc = load_library().rp_tune_wait(ctx, int(ticket), int(timeout_ms))
    if rc == RP_ETIMEOUT:
        return False
    _check(ctx, rc)
    return True


def rp_graph_info(ctx, g: int):
    n, nnz, start = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    md = ctypes.c_int32()
    _check(ctx, load_library().rp_graph_info(ctx, int(g), ctypes.byref(n), ctypes.byref(nnz), ctypes.byref(md),
                                             ctypes.byref(start)))
    return dict(n=n.value, nnz=nnz.value, max_degree=md.value, start=start.value)


def rp_graph_export(ctx, g: int, device=None):
    """Returns (row_ptr int64[n+1], col int32[nnz]) as numpy arrays, or torch tensors on ``device``."""
    info = rp_graph_info(ctx, g)
    mem = RP_MEM_DEVICE if device is not None else RP_MEM_HOST
    rp = _empty_like_mem(mem, (info["n"] + 1,), np.int64, device)
    col = _empty_like_mem(mem, (max(info["nnz"], 1),), np.int32, device)
    _check(ctx, load_library().rp_graph_export(ctx, int(g), _ptr(rp), _ptr(col), int(col.shape[0]), mem))
    if mem == RP_MEM_DEVICE:
        rp_sync(ctx)
    return rp, col[:info["nnz"]]


def rp_search(ctx, g: int, queries, L: int, k: int, ids=None, dists=None):
    """GreedySearch for every row of ``queries``; returns (ids[nq,k], dists[nq,k])."""
    mem = _mem(queries, ids, dists)
    nq = int(queries.shape[0])
    dev = queries.device if mem == RP_MEM_DEVICE else None
    if ids is None:
        ids = _empty_like_mem(mem, (nq, k), np.int32, dev)
    if dists is None:
        dists = _empty_like_mem(mem, (nq, k), np.float32, dev)
    _check(ctx, load_library().rp_search(ctx, int(g), _ptr(queries), nq, int(L), int(k), _ptr(ids), _ptr(dists), mem))
    return ids, dists


def rp_search_multi(ctx, graphs, q_graph, q_L, queries, k: int, ids=None, dists=None):
    """One search launch where query i runs on graphs[q_graph[i]] with list size q_L[i]."""
    mem = _mem(queries, ids, dists)
    nq = int(queries.shape[0])
    dev = queries.device if mem == RP_MEM_DEVICE else None
    if ids is None:
        ids = _empty_like_mem(mem, (nq, k), np.int32, dev)
    if dists is None:
        dists = _empty_like_mem(mem, (nq, k), np.float32, dev)
    g = np.ascontiguousarray(graphs, dtype=np.int64)
    qg = np.ascontiguousarray(q_graph, dtype=np.int32)
    qL = np.ascontiguousarray(q_L, dtype=np.int32)
    if qg.shape != (nq,) or qL.shape != (nq,):
        raise ValueError("q_graph and q_L need one entry per query")
    _check(ctx, load_library().rp_search_multi(ctx, _ptr(g), int(g.shape[0]), _ptr(qg), _ptr(qL), _ptr(queries), nq,
                                               int(k), _ptr(ids), _ptr(dists), mem))
    return ids, dists


def rp_graph_shape(ctx, g: int) -> dict:
    d, dt, b = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_uint64()
    _check(ctx, load_library().rp_graph_shape(ctx, int(g), ctypes.byref(d), ctypes.byref(dt), ctypes.byref(b)))
    return dict(d=d.value, dtype=dt.value, adj_bytes=b.value)


def rp_graph_slice(ctx, g: int, lo: int, hi: int) -> int:
    """The rows of nodes lo .. hi-1 of graph g (other rows empty), sharing g's vectors."""
    out = ctypes.c_int64()
    _check(ctx, load_library().rp_graph_slice(ctx, int(g), int(lo), int(hi), ctypes.byref(out)))
    return out.value


def rp_knn(ctx, g: int, queries, k: int, nq: int | None = None, ids=None, dists=None):
    """Exact kNN of ``queries`` (or of base points 0..nq-1 when queries is None)."""
    mem = _mem(queries, ids, dists) if queries is not None else (_mem(ids) if ids is not None else RP_MEM_HOST)
    nq = int(queries.shape[0]) if queries is not None else int(nq)
    dev = (queries.device if queries is not None else ids.device) if mem == RP_MEM_DEVICE else None
    if ids is None:
        ids = _empty_like_mem(mem, (nq, k), np.int32, dev)
    if dists is None:
        dists = _empty_like_mem(mem, (nq, k), np.float32, dev)
    _check(ctx, load_library().rp_knn(ctx, int(g), _ptr(queries), nq, int(k), _ptr(ids), _ptr(dists), mem))
    return ids, dists


def rp_recall(ctx, found, truth, k: int) -> int:
    """Total matches between the first k ids of each row of found and truth."""
    mem = _mem(found, truth)
    hits = ctypes.c_int64()
    _check(ctx, load_library().rp_recall(ctx, _ptr(found), int(found.shape[1]), _ptr(truth), int(truth.shape[1]),
                                         int(found.shape[0]), int(k), ctypes.byref(hits), mem))
    return hits.value


def rp_reachability(ctx, g: int, nodes=None):
    """alpha-reachability (Definition 2.1): returns (alpha_star, per-node terms)
    at ``nodes`` (default: every node; at scale pass a sample)."""
    if nodes is None:
        n = rp_graph_info(ctx, g)["n"]
        arr, m = None, n
    else:
        arr = np.ascontiguousarray(nodes, dtype=np.int64)
        m = arr.shape[0]
    per = np.zeros(m, dtype=np.float64)
    a = ctypes.c_double()
    _check(ctx, load_library().rp_reachability(ctx, int(g), None if arr is None else arr.ctypes.data, int(m),
                                               per.ctypes.data, ctypes.byref(a)))
    return a.value, per


def rp_build_knn_base(ctx, data: int, kcand: int, alpha: float, R: int) -> int:
    out = ctypes.c_int64()
    _check(ctx, load_library().rp_build_knn_base(ctx, int(data), int(kcand), float(alpha), int(R), ctypes.byref(out)))
    return out.value


def rp_build_knn_random_base(ctx, data: int, kcand: int, nrand: int, seed: int, alpha: float, R: int) -> int:
    out = ctypes.c_int64()
    _check(ctx, load_library().rp_build_knn_random_base(ctx, int(data), int(kcand), int(nrand), int(seed),
                                                        float(alpha), int(R), ctypes.byref(out)))
    return out.value


def rp_build_vamana(ctx, data: int, alphas, R: int, L: int, vcap: int = 0, max_batch: int = 0, perm=None):
    """Vamana graph (§2.1 fast preprocessing, §4.1 base indices) over the vectors of ``data``:
    one insertion pass per entry of ``alphas``, batches of 1, 2, 4, ... points up to
    ``max_batch`` (default n // 50), visited sets cut to ``vcap`` (default 4 L), insertion
    order ``perm`` (default 0 .. n-1).  Returns (graph, searches whose visited set was cut)."""
    n = rp_graph_info(ctx, data)["n"]
    vcap = int(vcap) if vcap else 4 * int(L)
    max_batch = int(max_batch) if max_batch else max(1, n // 50)
    a = (ctypes.c_double * len(alphas))(*[float(x) for x in alphas])
    pa = None
    if perm is not None:
        pa = np.ascontiguousarray(perm, dtype=np.int32)
        if pa.shape != (n,):
            raise ValueError("perm must hold n entries")
    cut = ctypes.c_int64()
    out = ctypes.c_int64()
    _check(ctx, load_library().rp_build_vamana(ctx, int(data), _ptr(pa), len(alphas), a, int(R), int(L), vcap,
                                               max_batch, ctypes.byref(cut), ctypes.byref(out)))
    return out.value, cut.value


def rp_graph_free(ctx, g: int):
    _check(ctx, load_library().rp_graph_free(ctx, int(g)))


def rp_set_tuning(ctx, mode: int, tile0: int = 0, ctas_per_sm: int = 0):
    _check(ctx, load_library().rp_set_tuning(ctx, int(mode), int(tile0), int(ctas_per_sm)))


def rp_set_search_config(ctx, cache_bits: int = 0, ctas_per_sm: int = 0):
    _check(ctx, load_library().rp_set_search_config(ctx, int(cache_bits), int(ctas_per_sm)))


def rp_set_knn_method(ctx, method: int):
    _check(ctx, load_library().rp_set_knn_method(ctx, int(method)))


def rp_stats(ctx, reset: bool = False) -> dict:
    s = rp_stats_t()
    _check(ctx, load_library().rp_stats(ctx, ctypes.byref(s), int(bool(reset))))
    return {name: getattr(s, name) for name, _ in rp_stats_t._fields_ if name != "pad_"}


def rp_search_noalloc(vectors, row_ptr, col, start: int, queries, L: int, k: int, ids=None, dists=None,
                      stream=None, want_dists: bool = True, check_status: bool = True):
    """GreedySearch with caller-owned CUDA tensors and no device allocation by the library.

    ``vectors``/``queries`` are CUDA tensors of uint8 or float32 rows (same dtype and width);
    ``row_ptr`` (int64, n+1) and ``col`` (int32) the graph, all on one device.  Runs on
    ``stream`` (a torch.cuda.Stream or raw handle; default: the current torch stream of that
    device).  ``want_dists=False`` passes no distance buffer.  With ``check_status`` the call
    waits for the stream and raises RPError(RP_EDEVICE) if the kernel reported a problem.
    Returns (ids, dists) tensors (dists None when not wanted).
    """
    import torch
    tens = {"vectors": vectors, "row_ptr": row_ptr, "col": col, "queries": queries}
    for name, t in tens.items():
        if not (_is_torch(t) and t.is_cuda):
            raise TypeError(f"{name} must be a CUDA tensor")
    dev = queries.device
    if any(t.device != dev for t in tens.values()):
        raise ValueError("vectors, row_ptr, col and queries must be on one device")
    if vectors.dim() != 2 or queries.dim() != 2:
        raise ValueError("vectors and queries must be 2-D (rows x dims)")
    if queries.dtype != vectors.dtype or queries.shape[1] != vectors.shape[1]:
        raise ValueError("queries must have the vectors' dtype and width")
    n = int(vectors.shape[0])
    if row_ptr.dtype != torch.int64 or row_ptr.dim() != 1 or int(row_ptr.numel()) != n + 1:
        raise ValueError("row_ptr must be int64 with n + 1 entries")
    if col.dtype != torch.int32 or col.dim() != 1:
        raise ValueError("col must be 1-D int32")
    nq = int(queries.shape[0])
    if ids is None:
        ids = torch.empty((nq, k), dtype=torch.int32, device=dev)
    if dists is None and want_dists:
        dists = torch.empty((nq, k), dtype=torch.float32, device=dev)
    for name, t, dt in (("ids", ids, torch.int32), ("dists", dists, torch.float32)):
        if t is None:
            continue
        if not (_is_torch(t) and t.is_cuda and t.device == dev and t.dtype == dt):
            raise ValueError(f"{name} must be a {dt} CUDA tensor on the queries' device")
        if int(t.numel()) < nq * k:
            raise ValueError(f"{name} must hold at least nq * k entries")
    with torch.cuda.device(dev):
        if stream is None:
            stream = torch.cuda.current_stream(dev)
        h = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
        hs = ctypes.c_void_p(h) if h else None
        rc = load_library().rp_search_noalloc(_ptr(vectors), _dtype_code(vectors), n, int(vectors.shape[1]),
                                              _ptr(row_ptr), _ptr(col), int(start), _ptr(queries), nq, int(L),
                                              int(k), _ptr(ids), _ptr(dists), hs)
        if rc != RP_OK:
            raise RPError(rc, "rp_search_noalloc rejected its arguments or failed to launch")
        if check_status:
            info = ctypes.c_int64(0)
            rc = load_library().rp_search_noalloc_status(hs, ctypes.byref(info))
            if rc != RP_OK:
                raise RPError(rc, f"rp_search_noalloc: the kernel reported a problem (query {info.value})")
    return ids, dists


def rp_search_noalloc_status(stream=None) -> None:
    """Device status of the last rp_search_noalloc call on the current device: waits for
    ``stream`` (default: the current torch stream) and raises RPError(RP_EDEVICE), naming
    the offending query, if the kernel reported a problem."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    h = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
    info = ctypes.c_int64(0)
    rc = load_library().rp_search_noalloc_status(ctypes.c_void_p(h) if h else None, ctypes.byref(info))
    if rc != RP_OK:
        raise RPError(rc, f"rp_search_noalloc: the kernel reported a problem (query {info.value})")


# ---- serving (rp_server_*): the binding keeps the buffers and callbacks the
# library holds pointers to alive until the request is reaped / the server is
# destroyed.
RP_REQ_QUEUED, RP_REQ_RUNNING, RP_REQ_DONE = 0, 1, 2
_held = {}  # server handle -> {"exec": callbacks, request id -> (ids, dists)}


def _scheck(srv, rc, what):
    if rc != RP_OK:
        msg = load_library().rp_server_last_error(srv).decode(errors="replace") if srv else ""
        raise RPError(rc, f"{what}: {msg}")


def rp_server_create(ctx, base: int, graph_budget_bytes: int = 0, max_batch_queries: int = 0,
                     serial: bool = False):
    out = ctypes.c_void_p()
    _check(ctx, load_library().rp_server_create(ctx, int(base), int(graph_budget_bytes), int(max_batch_queries),
                                                int(bool(serial)), ctypes.byref(out)))
    _held[out.value] = {}
    return out.value


def rp_server_create_ex(tune_batch, search_multi, graph_free, base: int, d: int, dtype: int, graph_bytes: int,
                        graph_budget_bytes: int = 0, max_batch_queries: int = 0, serial: bool = False,
                        tune_start=None, tune_ready=None):
    """A server over Python callables with the rp_executor signatures (raw ctypes arguments);
    tune_start/tune_ready are the optional asynchronous tuning pair."""
    ex = rp_executor(None, TUNE_FN(tune_batch), SEARCH_FN(search_multi), FREE_FN(graph_free),
                     TUNE_START_FN(tune_start) if tune_start else TUNE_START_FN(),
                     TUNE_READY_FN(tune_ready) if tune_ready else TUNE_READY_FN())
    cfg = rp_server_config(int(base), int(d), int(dtype), int(graph_bytes), int(graph_budget_bytes),
                           int(max_batch_queries), int(bool(serial)))
    out = ctypes.c_void_p()
    rc = load_library().rp_server_create_ex(ctypes.byref(ex), ctypes.byref(cfg), ctypes.byref(out))
    if rc != RP_OK:
        raise RPError(rc, "rp_server_create_ex rejected its arguments")
    _held[out.value] = {"exec": ex}
    return out.value


def rp_server_destroy(srv):
    rc = load_library().rp_server_destroy(srv)
    _held.pop(srv, None)
    if rc != RP_OK:
        raise RPError(rc, "rp_server_destroy: freeing a tuned graph failed")


def rp_submit_tune(srv, alpha: float, R: int) -> int:
    rid = ctypes.c_int64()
    _scheck(srv, load_library().rp_submit_tune(srv, float(alpha), int(R), ctypes.byref(rid)), "rp_submit_tune")
    return rid.value


def rp_submit_search(srv, alpha: float, R: int, queries: np.ndarray, L: int, k: int, ids=None, dists=None):
    """Queue a search of host rows ``queries``; returns (request id, ids, dists), the
    arrays being filled by the time rp_poll reports the request finished."""
    queries = np.ascontiguousarray(queries)
    nq = int(queries.shape[0])
    if ids is None:
        ids = np.empty((nq, k), dtype=np.int32)
    if dists is None:
        dists = np.empty((nq, k), dtype=np.float32)
    rid = ctypes.c_int64()
    _scheck(srv, load_library().rp_submit_search(srv, float(alpha), int(R), _ptr(queries), nq, int(L), int(k),
                                                 _ptr(ids), _ptr(dists), ctypes.byref(rid)), "rp_submit_search")
    _held[srv][rid.value] = (ids, dists)
    return rid.value, ids, dists


def rp_poll(srv, request_id: int, timeout_ms: int = 0):
    """None while the request runs; its rp_request_info as a dict once finished."""
    info = rp_request_info()
    rc = load_library().rp_poll(srv, int(request_id), int(timeout_ms), ctypes.byref(info))
    if rc == RP_ETIMEOUT:
        return None
    _scheck(srv, rc, "rp_poll")
    _held.get(srv, {}).pop(int(request_id), None)
    return {name: getattr(info, name) for name, _ in rp_request_info._fields_}


def rp_server_stats(srv) -> dict:
    s = rp_server_stats_t()
    _scheck(srv, load_library().rp_server_stats(srv, ctypes.byref(s)), "rp_server_stats")
    return {name: getattr(s, name) for name, _ in rp_server_stats_t._fields_}


def rp_server_last_error(srv) -> str:
    return load_library().rp_server_last_error(srv).decode(errors="replace")
