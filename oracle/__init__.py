"""CPU oracle for RP-Tuning and GreedySearch -- TEST INFRASTRUCTURE ONLY.

Thin ctypes wrapper around ``oracle.c`` (plain C, fp64 / exact int64).  Only the
test-suite, ``__graft_entry__.smoke()`` and the benchmark's ``cpu_baseline`` /
``--impl reference`` legs may import this module.  It shares no code with the
CUDA library and never calls it.

Every function cites the passage of the paper it follows:

* :func:`robust_prune` -- Algorithm 1 (RobustPrune); ``variant="unsorted"`` is
  UnsortedRobustPrune from §3 (p* is an arbitrary remaining out-neighbour; read
  here as the first one left in stored order).
* :func:`rp_tune` -- §3, "RP-Tuning": RobustPrune(p, N_out(p), alpha2, R) for
  every p, each reading only the input graph.
* :func:`slow_base` -- §2.1 slow preprocessing, RobustPrune(p, P minus p,
  alpha, R) for every p (Lemma 2.2).
* :func:`greedy_search` -- Algorithm 2, from the start vertex of §4.1.
* :func:`knn` -- exact k nearest neighbours, the recall ground truth (§4).
* :func:`reachability` -- alpha* of Definition 2.1 (:func:`reachability_nodes`: its per-node terms).
* :func:`recall_at_k` -- k-recall@k as defined at the start of §4.
* :func:`vamana` -- the Vamana ("fast preprocessing") construction of §2.1 with
  which §4.1 builds its base indices, in a fixed batch schedule.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
R_INF = 2**31 - 1
U8, F32 = 1, 2
SORTED, UNSORTED = 0, 1

_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, -ffp-contract=off)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread",
                               "-ffp-contract=off", "-fno-fast-math", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i64, i32, dbl = ctypes.c_int64, ctypes.c_int32, ctypes.c_double
        ci = ctypes.c_int
        _lib.orc_robust_prune.restype = i64
        _lib.orc_robust_prune.argtypes = [P, ci, i64, ci, i64, P, i64, i32, i32, ci, P]
        _lib.orc_robust_prune_dmat.restype = i64
        _lib.orc_robust_prune_dmat.argtypes = [P, i64, i64, P, i64, dbl, i32, ci, P]
        _lib.orc_rp_tune.restype = ci
        _lib.orc_rp_tune.argtypes = [P, ci, i64, ci, P, P, i32, i32, ci, P, i64, ci, P, P, i64]
        _lib.orc_slow_base.restype = ci
        _lib.orc_slow_base.argtypes = [P, ci, i64, ci, i32, i32, ci, P, i64, ci, P, P, i64]
        _lib.orc_knn.restype = ci
        _lib.orc_knn.argtypes = [P, ci, i64, ci, P, P, i64, ci, ci, P, P]
        _lib.orc_medoid.restype = i64
        _lib.orc_medoid.argtypes = [P, ci, i64, ci]
        _lib.orc_greedy_search.restype = ci
        _lib.orc_greedy_search.argtypes = [P, ci, i64, ci, P, P, i64, P, i64, ci, ci, ci, P, P, P]
        _lib.orc_reachability.restype = dbl
        _lib.orc_reachability.argtypes = [P, ci, i64, ci, P, P, ci]
        _lib.orc_reachability_dmat.restype = dbl
        _lib.orc_reachability_dmat.argtypes = [P, i64, P, P]
        _lib.orc_reachability_nodes.restype = ci
        _lib.orc_reachability_nodes.argtypes = [P, ci, i64, ci, P, P, P, i64, ci, P]
        _lib.orc_d2_pairs.restype = ci
        _lib.orc_d2_pairs.argtypes = [P, ci, ci, P, P, i64, P]
        _lib.orc_d2_query.restype = ci
        _lib.orc_d2_query.argtypes = [P, ci, ci, P, i64, P, ci, P]
        _lib.orc_vamana.restype = ci
        _lib.orc_vamana.argtypes = [P, ci, i64, ci, P, ci, P, i32, i32, i32, i64, i64, ci, P, P, P]
        _lib.orc_num_threads.restype = ci
        _lib.orc_num_threads.argtypes = [ci]
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


def _vecs(X):
    X = np.ascontiguousarray(X)
    if X.dtype == np.uint8:
        return X, U8
    if X.dtype == np.float32:
        return X, F32
    raise TypeError(f"vectors must be uint8 or float32, got {X.dtype}")


def milli(alpha: float) -> int:
    """alpha -> A = round(1000 alpha); alpha must lie on the 0.001 grid and be >= 1."""
    A = int(round(alpha * 1000.0))
    if abs(alpha * 1000.0 - A) > 1e-6 or A < 1000:
        raise ValueError(f"alpha={alpha!r} must be >= 1 and a multiple of 0.001")
    return A


def _variant(v) -> int:
    return {"sorted": SORTED, "unsorted": UNSORTED, SORTED: SORTED, UNSORTED: UNSORTED}[v]


def num_threads(n: int = 0) -> int:
    return int(_load().orc_num_threads(int(n)))


def robust_prune(X, p: int, cand, alpha: float, R: int = R_INF, variant="sorted") -> np.ndarray:
    """Algorithm 1 for one point p; returns the new N_out(p) in the order points were added."""
    X, dt = _vecs(X)
    cand = np.ascontiguousarray(cand, dtype=np.int32)
    out = np.empty(max(1, cand.shape[0]), dtype=np.int32)
    k = _load().orc_robust_prune(_ptr(X), dt, X.shape[0], X.shape[1], int(p), _ptr(cand),
                                 cand.shape[0], milli(alpha), int(R), _variant(variant), _ptr(out))
    return out[:k].copy()


def robust_prune_dmat(D, p: int, cand, alpha: float, R: int = R_INF, variant="sorted") -> np.ndarray:
    """Algorithm 1 over an explicit (general-metric) distance matrix D, real alpha, unsquared."""
    D = np.ascontiguousarray(D, dtype=np.float64)
    cand = np.ascontiguousarray(cand, dtype=np.int32)
    out = np.empty(max(1, cand.shape[0]), dtype=np.int32)
    k = _load().orc_robust_prune_dmat(_ptr(D), D.shape[0], int(p), _ptr(cand), cand.shape[0],
                                      float(alpha), int(R), _variant(variant), _ptr(out))
    return out[:k].copy()


def _to_csr(cnt, padded):
    n = cnt.shape[0]
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(cnt, out=row_ptr[1:])
    cap = padded.shape[1] if padded.ndim == 2 else 0
    mask = np.arange(cap)[None, :] < cnt[:, None]
    return row_ptr, np.ascontiguousarray(padded[mask], dtype=np.int32)


def rp_tune(X, row_ptr, col, alpha: float, R: int = R_INF, variant="sorted", nodes=None,
            nthreads: int = 0):
    """§3 RP-Tuning.  Whole graph -> (row_ptr, col) of G'; with ``nodes`` -> list of rows."""
    X, dt = _vecs(X)
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    n = X.shape[0]
    maxdeg = int(np.max(np.diff(row_ptr))) if n > 0 else 0
    cap = max(1, min(maxdeg, int(R)))
    nodes_arr = None if nodes is None else np.ascontiguousarray(nodes, dtype=np.int64)
    cnt_n = n if nodes_arr is None else nodes_arr.shape[0]
    cnt = np.zeros(cnt_n, dtype=np.int32)
    padded = np.zeros((cnt_n, cap), dtype=np.int32)
    _load().orc_rp_tune(_ptr(X), dt, n, X.shape[1], _ptr(row_ptr), _ptr(col), milli(alpha),
                        int(R), _variant(variant), _ptr(nodes_arr),
                        0 if nodes_arr is None else nodes_arr.shape[0], int(nthreads),
                        _ptr(cnt), _ptr(padded), cap)
    if nodes_arr is not None:
        return [padded[i, :cnt[i]].copy() for i in range(cnt_n)]
    return _to_csr(cnt, padded)


def slow_base(X, alpha: float, R: int = R_INF, variant="sorted", nodes=None, nthreads: int = 0):
    """§2.1 slow preprocessing: RobustPrune(p, P minus p, alpha, R) for every p (Lemma 2.2)."""
    X, dt = _vecs(X)
    n = X.shape[0]
    cap = max(1, min(n - 1, int(R)))
    nodes_arr = None if nodes is None else np.ascontiguousarray(nodes, dtype=np.int64)
    cnt_n = n if nodes_arr is None else nodes_arr.shape[0]
    cnt = np.zeros(cnt_n, dtype=np.int32)
    padded = np.zeros((cnt_n, cap), dtype=np.int32)
    _load().orc_slow_base(_ptr(X), dt, n, X.shape[1], milli(alpha), int(R), _variant(variant),
                          _ptr(nodes_arr), 0 if nodes_arr is None else nodes_arr.shape[0],
                          int(nthreads), _ptr(cnt), _ptr(padded), cap)
    if nodes_arr is not None:
        return [padded[i, :cnt[i]].copy() for i in range(cnt_n)]
    return _to_csr(cnt, padded)


def knn(X, k: int, Q=None, qid=None, nthreads: int = 0):
    """Exact k nearest neighbours ordered by (d2, id).  Queries are the rows of Q, or
    the base points ``qid`` (each excluded from its own list).  Returns (ids, d2)."""
    X, dt = _vecs(X)
    if Q is not None:
        Q = np.ascontiguousarray(Q, dtype=X.dtype)
        nq = Q.shape[0]
        qa = None
    else:
        qa = np.ascontiguousarray(qid, dtype=np.int64)
        nq = qa.shape[0]
    ids = np.empty((nq, k), dtype=np.int32)
    d2 = np.empty((nq, k), dtype=np.float64)
    _load().orc_knn(_ptr(X), dt, X.shape[0], X.shape[1], _ptr(Q), _ptr(qa), nq, int(k),
                    int(nthreads), _ptr(ids), _ptr(d2))
    return ids, d2


def knn_base(X, k: int, alpha: float, R: int, nodes=None, nthreads: int = 0):
    """The kNN-candidate base graph: RobustPrune(p, top-k exact kNN of p, alpha, R).

    Returns the CSR graph over all points, or the list of rows for ``nodes``.
    """
    X, _ = _vecs(X)
    n = X.shape[0]
    sel = np.arange(n, dtype=np.int64) if nodes is None else np.ascontiguousarray(nodes, np.int64)
    ids, _ = knn(X, k, qid=sel, nthreads=nthreads)
    cnt = np.full(sel.shape[0], k, dtype=np.int64)
    cand_ptr = np.zeros(sel.shape[0] + 1, dtype=np.int64)
    np.cumsum(cnt, out=cand_ptr[1:])
    # Prune every selected node against its own candidate list: build a graph
    # whose row i (i-th selected node) is its candidate list, addressed through
    # a full-size row_ptr so that the oracle sees point ids unchanged.
    full_ptr = np.zeros(n + 1, dtype=np.int64)
    deg = np.zeros(n, dtype=np.int64)
    deg[sel] = k
    np.cumsum(deg, out=full_ptr[1:])
    col = np.empty(int(full_ptr[-1]), dtype=np.int32)
    for i, p in enumerate(sel):
        col[full_ptr[p]:full_ptr[p] + k] = ids[i]
    rows = rp_tune(X, full_ptr, col, alpha, R, "sorted", nodes=sel, nthreads=nthreads)
    if nodes is not None:
        return rows
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum([r.shape[0] for r in rows], out=row_ptr[1:])
    return row_ptr, np.concatenate(rows).astype(np.int32) if rows else np.zeros(0, np.int32)


def medoid(X) -> int:
    """Start vertex (§4.1): the point nearest to the fp64 mean vector; ties to the smaller id."""
    X, dt = _vecs(X)
    return int(_load().orc_medoid(_ptr(X), dt, X.shape[0], X.shape[1]))


def greedy_search(X, row_ptr, col, start: int, Q, L: int, k: int, nthreads: int = 0):
    """Algorithm 2 for every row of Q.  Returns (ids[nq,k], d2[nq,k], expansions[nq])."""
    X, dt = _vecs(X)
    Q = np.ascontiguousarray(Q, dtype=X.dtype)
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    nq = Q.shape[0]
    ids = np.empty((nq, k), dtype=np.int32)
    d2 = np.empty((nq, k), dtype=np.float64)
    exp = np.empty(nq, dtype=np.int64)
    rc = _load().orc_greedy_search(_ptr(X), dt, X.shape[0], X.shape[1], _ptr(row_ptr), _ptr(col),
                                   int(start), _ptr(Q), nq, int(L), int(k), int(nthreads),
                                   _ptr(ids), _ptr(d2), _ptr(exp))
    if rc != 0:
        raise ValueError("greedy_search: need L >= k > 0 and a valid start vertex")
    return ids, d2, exp


def reachability(X, row_ptr, col, nthreads: int = 0) -> float:
    """alpha*(G) of Definition 2.1 (brute force over all ordered pairs; small n only)."""
    X, dt = _vecs(X)
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    return float(_load().orc_reachability(_ptr(X), dt, X.shape[0], X.shape[1], _ptr(row_ptr),
                                          _ptr(col), int(nthreads)))


def reachability_nodes(X, row_ptr, col, nodes=None, nthreads: int = 0) -> np.ndarray:
    """Per-node terms of alpha*(G) (Definition 2.1) at ``nodes`` (default: all):
    min over non-neighbours q of max over out-neighbours p' of D(p, q) / D(p', q).
    Distances pair by pair, so any n; alpha*(G) is the minimum over all nodes."""
    X, dt = _vecs(X)
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    nodes_arr = None if nodes is None else np.ascontiguousarray(nodes, dtype=np.int64)
    m = X.shape[0] if nodes_arr is None else nodes_arr.shape[0]
    out = np.zeros(m, dtype=np.float64)
    _load().orc_reachability_nodes(_ptr(X), dt, X.shape[0], X.shape[1], _ptr(row_ptr), _ptr(col),
                                   _ptr(nodes_arr), m, int(nthreads), _ptr(out))
    return out


def reachability_dmat(D, row_ptr, col) -> float:
    """alpha*(G) of Definition 2.1 for an explicit distance matrix (general metric)."""
    D = np.ascontiguousarray(D, dtype=np.float64)
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    return float(_load().orc_reachability_dmat(_ptr(D), D.shape[0], _ptr(row_ptr), _ptr(col)))


def d2_pairs(X, a, b) -> np.ndarray:
    """Canonical squared distances between base points a[i] and b[i]."""
    X, dt = _vecs(X)
    a = np.ascontiguousarray(a, dtype=np.int64)
    b = np.ascontiguousarray(b, dtype=np.int64)
    out = np.empty(a.shape[0], dtype=np.float64)
    _load().orc_d2_pairs(_ptr(X), dt, X.shape[1], _ptr(a), _ptr(b), a.shape[0], _ptr(out))
    return out


def d2_query(X, Q, ids) -> np.ndarray:
    """Canonical squared distances from Q[i] to base points ids[i, j] (+inf for id < 0)."""
    X, dt = _vecs(X)
    Q = np.ascontiguousarray(Q, dtype=X.dtype)
    ids = np.ascontiguousarray(ids, dtype=np.int32)
    out = np.empty(ids.shape, dtype=np.float64)
    _load().orc_d2_query(_ptr(X), dt, X.shape[1], _ptr(Q), Q.shape[0], _ptr(ids), ids.shape[1],
                         _ptr(out))
    return out


def recall_at_k(found, truth, k: int) -> float:
    """k-recall@k (§4): mean over queries of |found[:k] intersect truth[:k]| / k."""
    found = np.asarray(found)
    truth = np.asarray(truth)
    tot = 0
    for f, t in zip(found, truth):
        tot += len(set(int(x) for x in f[:k] if x >= 0) & set(int(x) for x in t[:k] if x >= 0))
    return tot / (k * max(1, found.shape[0]))


def vamana(X, perm, alphas, R: int, L: int, vcap: int, max_batch: int, start: int, nthreads: int = 0):
    """Vamana (§2.1 "fast preprocessing"; §4.1 builds its base indices this way), run in
    batches: the graph starts empty and the points of ``perm`` are inserted in batches of
    1, 2, 4, ... points (at most ``max_batch``), one pass per entry of ``alphas``.  Each
    point of a batch searches the graph as it stood at the batch's start (Algorithm 2,
    list size L, its first ``vcap`` visited points), is pruned over them (Algorithm 1,
    sorted, degree bound R), then every point it kept gets it as a back edge, a list
    growing past R being pruned again (Algorithm 1).  Returns (row_ptr, col, overflows),
    overflows counting searches whose visited set was cut to ``vcap``."""
    X, dt = _vecs(X)
    n = X.shape[0]
    perm = np.ascontiguousarray(perm, dtype=np.int32)
    if perm.shape != (n,) or not np.array_equal(np.sort(perm), np.arange(n, dtype=np.int32)):
        raise ValueError("perm must be a permutation of 0 .. n-1")
    A = np.ascontiguousarray([milli(a) for a in alphas], dtype=np.int32)
    nbr = np.zeros((n, R), dtype=np.int32)
    deg = np.zeros(n, dtype=np.int32)
    over = np.zeros(1, dtype=np.int64)
    rc = _load().orc_vamana(_ptr(X), dt, n, X.shape[1], _ptr(perm), A.shape[0], _ptr(A), int(R), int(L),
                            int(vcap), int(max_batch), int(start), int(nthreads), _ptr(nbr), _ptr(deg), _ptr(over))
    if rc != 0:
        raise ValueError("vamana: bad arguments")
    row_ptr, col = _to_csr(deg, nbr)
    return row_ptr, col, int(over[0])
