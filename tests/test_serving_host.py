"""The serving scheduler of librp.so (rp_server_*), run on the host: its
executor is backed by the oracle through ctypes callbacks, so admission,
batching, eviction, result routing and failure handling are tested without a
GPU.  Every request's result must equal the oracle's answer for that request
alone, whatever the mix it was served in."""
import ctypes
import threading

import numpy as np
import pytest

import datagen
import oracle

rp = pytest.importorskip("paper_2602_08097_gb300")

N, D = 400, 32


@pytest.fixture(scope="module")
def world():
    from paper_2602_08097_gb300 import build as b
    b.build()
    X = datagen.dataset("tiny", N)
    base = oracle.knn_base(X, 32, 1.2, 24)
    start = oracle.medoid(X)
    Q = datagen.queries("tiny", 64)
    return X, base, start, Q


class OracleExec:
    """rp_executor over the oracle; graph handles are small integers."""

    BASE = 7

    def __init__(self, X, base, start, fail_alpha_milli=None, gate=None):
        self.X, self.start = X, start
        self.graphs = {self.BASE: base}
        self.next = 100
        self.fail = fail_alpha_milli
        self.gate = gate
        self.entered = threading.Event()  # set once the scheduler is inside a tuning call
        self.live_peak = 0
        self.tune_calls = []
        self.search_calls = []

    def tune(self, user, src, alphas, Rs, T, outs):
        try:
            self.entered.set()
            if self.gate is not None:
                self.gate.wait(10)
            assert src == self.BASE
            targets = [(alphas[t], Rs[t]) for t in range(T)]
            self.tune_calls.append(targets)
            if self.fail is not None and any(round(a * 1000) == self.fail for a, _ in targets):
                return rp.RP_ENOMEM
            row_ptr, col = self.graphs[self.BASE]
            for t, (a, R) in enumerate(targets):
                h = self.next
                self.next += 1
                self.graphs[h] = oracle.rp_tune(self.X, row_ptr, col, a, R)
                outs[t] = h
            self.live_peak = max(self.live_peak, len(self.graphs) - 1)
            return rp.RP_OK
        except Exception:  # never let an exception cross the C boundary
            return rp.RP_EINVAL

    def search(self, user, graphs, ngraphs, q_graph, q_L, queries, nq, k, ids, dists):
        try:
            qg = np.ctypeslib.as_array(q_graph, shape=(nq,)).copy()
            qL = np.ctypeslib.as_array(q_L, shape=(nq,)).copy()
            Q = np.ctypeslib.as_array(ctypes.cast(queries, ctypes.POINTER(ctypes.c_float)), shape=(nq, D))
            out_i = np.ctypeslib.as_array(ids, shape=(nq, k))
            out_d = np.ctypeslib.as_array(dists, shape=(nq, k))
            hs = [graphs[j] for j in range(ngraphs)]
            self.search_calls.append((tuple(hs), int(nq)))
            for i in range(nq):
                row_ptr, col = self.graphs[hs[qg[i]]]
                gi, gd, _ = oracle.greedy_search(self.X, row_ptr, col, self.start, Q[i:i + 1], int(qL[i]), k)
                out_i[i] = gi[0]
                out_d[i] = gd[0].astype(np.float32)
            return rp.RP_OK
        except Exception:
            return rp.RP_EINVAL

    def free(self, user, g):
        if g not in self.graphs or g == self.BASE:
            return rp.RP_ENOTFOUND
        del self.graphs[g]
        return rp.RP_OK

    def server(self, budget_graphs=0, serial=False, max_batch=0):
        gb = 1000
        return rp.rp_server_create_ex(self.tune, self.search, self.free, self.BASE, D, rp.RP_F32, gb,
                                      budget_graphs * gb, max_batch, serial)


def _expected(X, base, start, r):
    row_ptr, col = base if r.alpha == 0 else oracle.rp_tune(X, base[0], base[1], r.alpha, r.R)
    ids, d2, _ = oracle.greedy_search(X, row_ptr, col, start, r.queries, max(r.L, r.k), r.k)
    return ids, d2.astype(np.float32)


def _stream(Q, n=40, seed=11):
    from paper_2602_08097_gb300.serving import make_requests
    s = datagen.poisson_stream(n, 1000.0, seed=seed, prune_frac=0.25)
    for e in s:  # keep the host-side oracle quick
        if e["kind"] == "search":
            e["nq"] = min(e["nq"], 4)
            e["k"] = 10
            e["L"] = int(e["L"]) // 8
    reqs = make_requests(s, Q, seed=seed)
    reqs[0].alpha, reqs[0].R = 0, 0  # one search on the base itself
    if reqs[0].kind == "tune":
        reqs[0].kind, reqs[0].queries, reqs[0].L, reqs[0].k = "search", Q[:2], 16, 10
    return reqs


@pytest.mark.parametrize("serial", [False, True])
def test_mixed_stream_matches_each_request_alone(world, serial):
    from paper_2602_08097_gb300.serving import replay
    X, base, start, Q = world
    ex = OracleExec(X, base, start)
    srv = ex.server(serial=serial)
    reqs = _stream(Q)
    try:
        rep = replay(srv, reqs, time_scale=0.0)
    finally:
        rp.rp_server_destroy(srv)
    for r in reqs:
        if r.kind == "search":
            ids, d2 = _expected(X, base, start, r)
            assert np.array_equal(r.ids, ids) and np.array_equal(r.dists, d2)
            assert r.info["L_eff"] == max(r.L, r.k)
    st = rep["stats"]
    assert st["requests_done"] == len(reqs) and st["requests_failed"] == 0
    assert st["l_clamps"] == sum(1 for r in reqs if r.kind == "search" and r.L < r.k)
    ntargets = len({(round(r.alpha * 1000), r.R) for r in reqs if r.alpha != 0})
    assert st["targets_tuned"] == ntargets  # unlimited budget: each target tuned once
    if serial:
        assert st["rounds"] == len(reqs)
        assert all(len(c) == 1 for c in ex.tune_calls)
        assert st["search_launches"] == sum(1 for r in reqs if r.kind == "search")
    assert not ex.graphs.keys() - {OracleExec.BASE}  # destroy freed every tuned graph


def test_rounds_batch_what_arrived(world):
    """Requests that arrive while a round runs share the next round's launches."""
    X, base, start, Q = world
    gate = threading.Event()
    ex = OracleExec(X, base, start, gate=gate)
    srv = ex.server()
    try:
        first = rp.rp_submit_tune(srv, 1.15, 24)  # holds the scheduler in its tuning call
        assert ex.entered.wait(10)
        assert rp.rp_poll(srv, first, 50) is None  # still running: the bounded wait runs out
        later = []
        for j, (a, R) in enumerate([(1.1, 24), (1.05, 16), (1.1, 24), (1.0, 16)]):
            later.append(rp.rp_submit_search(srv, a, R, Q[j:j + 3], 12, 10))
        later.append((rp.rp_submit_tune(srv, 1.03, 20), None, None))
        gate.set()
        infos = [rp.rp_poll(srv, rid, 20000) for rid, _, _ in later]
        assert rp.rp_poll(srv, first, 20000)["round"] == 1
        assert {i["round"] for i in infos} == {2}
        st = rp.rp_server_stats(srv)
        assert st["rounds"] == 2 and st["tune_launches"] == 2 and st["search_launches"] == 1
        assert [len(c) for c in ex.tune_calls] == [1, 4]  # (1.1,24) (1.05,16) (1.0,16) (1.03,20)
        assert ex.search_calls[-1][1] == 12
        for (rid, ids, dists), (j, (a, R)) in zip(later[:4], enumerate([(1.1, 24), (1.05, 16), (1.1, 24), (1.0, 16)])):
            rp_, col = oracle.rp_tune(X, base[0], base[1], a, R)
            ref, d2, _ = oracle.greedy_search(X, rp_, col, start, Q[j:j + 3], 12, 10)
            assert np.array_equal(ids, ref)
        with pytest.raises(rp.RPError):
            rp.rp_poll(srv, first)  # already reaped
    finally:
        gate.set()
        rp.rp_server_destroy(srv)



class GatedExec(OracleExec):
    """Tuning call i waits on gates[i] (at most 10 s)."""

    def __init__(self, X, base, start, gates):
        super().__init__(X, base, start)
        self.gates = list(gates)
        self.calls = 0

    def tune(self, user, src, alphas, Rs, T, outs):
        i = self.calls
        self.calls += 1
        self.entered.set()  # the scheduler is inside a tuning call
        if i < len(self.gates):
            self.gates[i].wait(10)
        return super().tune(user, src, alphas, Rs, T, outs)


def test_resident_requests_do_not_wait_for_the_rounds_tuning(world):
    """In a round that tunes, the searches on graphs already resident (and on
    the base) complete before its tuning call returns; the rest after it."""
    X, base, start, Q = world
    g1, g2 = threading.Event(), threading.Event()
    ex = GatedExec(X, base, start, [g1, g2])
    srv = ex.server()
    try:
        first = rp.rp_submit_tune(srv, 1.15, 24)  # round 1: held in its tuning call by g1
        assert ex.entered.wait(10)  # round 1 has started: what follows waits for round 2
        early = [rp.rp_submit_search(srv, 1.15, 24, Q[0:3], 12, 10), rp.rp_submit_search(srv, 0.0, 0, Q[3:5], 12, 10)]
        late = [(rp.rp_submit_tune(srv, 1.1, 24), None, None), rp.rp_submit_search(srv, 1.1, 24, Q[5:8], 12, 10)]
        g1.set()
        assert rp.rp_poll(srv, first, 20000)["round"] == 1
        for rid, _, _ in early:  # round 2's tuning call is still held by g2
            info = rp.rp_poll(srv, rid, 5000)
            assert info is not None and info["round"] == 2 and info["status"] == rp.RP_OK
        assert rp.rp_poll(srv, late[0][0], 50) is None and rp.rp_poll(srv, late[1][0], 50) is None
        g2.set()
        for rid, _, _ in late:
            info = rp.rp_poll(srv, rid, 20000)
            assert info is not None and info["round"] == 2 and info["status"] == rp.RP_OK
        st = rp.rp_server_stats(srv)
        assert st["rounds"] == 2 and st["tune_launches"] == 2 and st["search_launches"] == 2
        for (rid, ids, _), (a, R, rows) in zip(early + late[1:], [(1.15, 24, slice(0, 3)), (0, 0, slice(3, 5)),
                                                                 (1.1, 24, slice(5, 8))]):
            g = base if a == 0 else oracle.rp_tune(X, base[0], base[1], a, R)
            ref, _, _ = oracle.greedy_search(X, g[0], g[1], start, Q[rows], 12, 10)
            assert np.array_equal(ids, ref)
    finally:
        g1.set()
        g2.set()
        rp.rp_server_destroy(srv)

def test_budget_evicts_least_recently_used(world):
    from paper_2602_08097_gb300.serving import Request, replay
    X, base, start, Q = world
    ex = OracleExec(X, base, start)
    srv = ex.server(budget_graphs=2)
    targets = [(1.15, 24), (1.1, 24), (1.15, 24), (1.05, 16), (1.1, 24), (1.0, 16), (1.15, 24)]
    reqs = [Request("search", a, R, 0.0, queries=Q[i:i + 2], L=10, k=10) for i, (a, R) in enumerate(targets)]
    try:
        # one request per round so that the LRU order is the submission order
        for r in reqs:
            replay(srv, [r], time_scale=0.0)
        st = rp.rp_server_stats(srv)
    finally:
        rp.rp_server_destroy(srv)
    assert ex.live_peak <= 2 and st["peak_resident_graphs"] == 2
    # LRU with 2 slots: 1.15 1.1 | 1.15 hit | 1.05 evicts 1.1 | 1.1 evicts 1.15 | 1.0 evicts 1.05 | 1.15 evicts 1.1
    assert st["targets_tuned"] == 6 and st["evictions"] == 4
    for r in reqs:
        ids, d2 = _expected(X, base, start, r)
        assert np.array_equal(r.ids, ids)


def test_admission_respects_the_budget(world):
    """A round admits requests only while their distinct targets fit."""
    X, base, start, Q = world
    gate = threading.Event()
    ex = OracleExec(X, base, start, gate=gate)
    srv = ex.server(budget_graphs=2)
    try:
        hold = rp.rp_submit_tune(srv, 1.2, 24)
        assert ex.entered.wait(10)
        subs = [rp.rp_submit_search(srv, a, 24, Q[i:i + 1], 10, 10) for i, a in enumerate([1.1, 1.05, 1.1, 1.0])]
        gate.set()
        infos = [rp.rp_poll(srv, rid, 20000) for rid, _, _ in subs]
        rp.rp_poll(srv, hold, 20000)
    finally:
        gate.set()
        rp.rp_server_destroy(srv)
    # round 2 takes 1.1 and 1.05 (and the second 1.1); 1.0 would be a third target
    assert [i["round"] for i in infos] == [2, 2, 2, 3]
    assert ex.live_peak <= 2


def test_failures_reach_only_their_requests(world):
    X, base, start, Q = world
    gate = threading.Event()
    ex = OracleExec(X, base, start, fail_alpha_milli=1050, gate=gate)
    srv = ex.server(serial=True)
    try:
        hold = rp.rp_submit_tune(srv, 1.2, 24)
        assert ex.entered.wait(10)
        ok = rp.rp_submit_search(srv, 1.1, 24, Q[:2], 10, 10)
        bad = rp.rp_submit_search(srv, 1.05, 24, Q[:2], 10, 10)
        bad_t = rp.rp_submit_tune(srv, 1.05, 16)
        gate.set()
        assert rp.rp_poll(srv, hold, 20000)["status"] == rp.RP_OK
        assert rp.rp_poll(srv, ok[0], 20000)["status"] == rp.RP_OK
        i_bad = rp.rp_poll(srv, bad[0], 20000)
        assert i_bad["status"] == rp.RP_ENOMEM and i_bad["graph"] == 0
        assert rp.rp_poll(srv, bad_t, 20000)["status"] == rp.RP_ENOMEM
        st = rp.rp_server_stats(srv)
        assert st["requests_failed"] == 2 and st["requests_done"] == 2
        assert "status -2" in rp.rp_server_last_error(srv)
    finally:
        gate.set()
        rp.rp_server_destroy(srv)


def test_invalid_submissions_are_refused(world):
    X, base, start, Q = world
    ex = OracleExec(X, base, start)
    srv = ex.server()
    try:
        for a, R in [(0.9, 24), (1.0005, 24), (101.0, 24), (1.1, 0)]:
            with pytest.raises(rp.RPError) as e:
                rp.rp_submit_tune(srv, a, R)
            assert e.value.code == rp.RP_EINVAL
        with pytest.raises(rp.RPError):
            rp.rp_submit_tune(srv, 0.0, 24)  # the base is not a tuning target
        for kw in [dict(L=10, k=0), dict(L=2000, k=10), dict(L=10, k=1025)]:
            with pytest.raises(rp.RPError):
                rp.rp_submit_search(srv, 1.1, 24, Q[:1], **kw)
        with pytest.raises(rp.RPError):
            rp.rp_submit_search(srv, 1.1, 24, Q[:0], 10, 10)
        with pytest.raises(rp.RPError):
            rp.rp_poll(srv, 12345)
        assert rp.rp_server_stats(srv)["rounds"] == 0
    finally:
        rp.rp_server_destroy(srv)


def test_mixed_round_evicts_only_what_it_does_not_use(world):
    """Budget of 2 tuned graphs, A and B resident: a round that searches A
    (resident, served first) and C (new) evicts B, never A, and a later search
    on A needs no tuning."""
    from paper_2602_08097_gb300.serving import Request, replay
    X, base, start, Q = world
    ex = OracleExec(X, base, start)
    srv = ex.server(budget_graphs=2)
    A, B, C = (1.15, 24), (1.1, 24), (1.05, 16)
    try:
        replay(srv, [Request("tune", *A, 0.0), Request("tune", *B, 0.0)], time_scale=0.0)
        mixed = [Request("search", *A, 0.0, queries=Q[0:3], L=12, k=10),
                 Request("search", *C, 0.0, queries=Q[3:6], L=12, k=10)]
        replay(srv, mixed, time_scale=0.0)
        st = rp.rp_server_stats(srv)
        assert st["evictions"] == 1 and st["targets_tuned"] == 3
        again = [Request("search", *A, 0.0, queries=Q[6:8], L=12, k=10)]
        replay(srv, again, time_scale=0.0)
        st = rp.rp_server_stats(srv)
        assert st["targets_tuned"] == 3 and st["evictions"] == 1  # A stayed resident
        assert ex.live_peak <= 2
        for r in mixed + again:
            ids, d2 = _expected(X, base, start, r)
            assert np.array_equal(r.ids, ids) and np.array_equal(r.dists, d2)
    finally:
        rp.rp_server_destroy(srv)


class AsyncExec(OracleExec):
    """rp_executor with the asynchronous tuning pair: tune_start computes at once
    but a job counts as finished only after its gate is set, so the test holds
    a job "on the device" while the scheduler goes on."""

    def __init__(self, X, base, start, gates=(), fail_alpha_milli=None):
        super().__init__(X, base, start, fail_alpha_milli=fail_alpha_milli)
        self.gates = list(gates)
        self.jobs = {}  # ticket -> (gate index, status)
        self.started = threading.Event()

    def tune_start(self, user, src, alphas, Rs, T, outs, ticket):
        try:
            st = self.tune(user, src, alphas, Rs, T, outs)
            t = len(self.jobs) + 1
            self.jobs[t] = (t - 1, st)
            ticket[0] = t
            self.started.set()
            return rp.RP_OK if st == rp.RP_OK else st
        except Exception:
            return rp.RP_EINVAL

    def tune_ready(self, user, ticket, timeout_ms):
        gi, st = self.jobs[ticket]
        if gi < len(self.gates) and not self.gates[gi].is_set():
            return rp.RP_ETIMEOUT
        return st

    def server(self, budget_graphs=0, serial=False, max_batch=0):
        gb = 1000
        return rp.rp_server_create_ex(self.tune, self.search, self.free, self.BASE, D, rp.RP_F32, gb,
                                      budget_graphs * gb, max_batch, serial, self.tune_start, self.tune_ready)


def test_async_searches_run_while_a_tuning_job_runs(world):
    """With an asynchronous executor a round does not wait for its tuning job:
    a search on a resident graph that arrives while a job runs completes
    before the job does; the requests on the graph being tuned complete after."""
    X, base, start, Q = world
    g1, g2 = threading.Event(), threading.Event()
    ex = AsyncExec(X, base, start, gates=[g1, g2])
    srv = ex.server()
    try:
        g1.set()  # the first job (1.15, 24) finishes at once
        a = rp.rp_submit_search(srv, 1.15, 24, Q[0:3], 12, 10)
        assert rp.rp_poll(srv, a[0], 20000)["status"] == rp.RP_OK
        held = rp.rp_submit_search(srv, 1.1, 24, Q[3:6], 12, 10)  # job 2, held by g2
        for _ in range(200):
            if len(ex.jobs) >= 2:
                break
            threading.Event().wait(0.01)
        assert len(ex.jobs) == 2
        quick = [rp.rp_submit_search(srv, 1.15, 24, Q[6:8], 12, 10), rp.rp_submit_search(srv, 0.0, 0, Q[8:9], 12, 10)]
        for rid, _, _ in quick:  # served while job 2 is still "running"
            info = rp.rp_poll(srv, rid, 5000)
            assert info is not None and info["status"] == rp.RP_OK
        assert rp.rp_poll(srv, held[0], 50) is None
        g2.set()
        assert rp.rp_poll(srv, held[0], 20000)["status"] == rp.RP_OK
        for (rid, ids, _), (al, R, rows) in zip([a, held] + quick, [(1.15, 24, slice(0, 3)), (1.1, 24, slice(3, 6)),
                                                                  (1.15, 24, slice(6, 8)), (0, 0, slice(8, 9))]):
            g = base if al == 0 else oracle.rp_tune(X, base[0], base[1], al, R)
            ref, _, _ = oracle.greedy_search(X, g[0], g[1], start, Q[rows], 12, 10)
            assert np.array_equal(ids, ref)
        st = rp.rp_server_stats(srv)
        assert st["tune_launches"] == 2 and st["targets_tuned"] == 2
    finally:
        g1.set()
        g2.set()
        rp.rp_server_destroy(srv)


def test_async_mixed_stream_and_failures(world):
    """The asynchronous path serves a mixed stream with every result equal to
    the request's answer alone; a failing job fails only its own requests."""
    from paper_2602_08097_gb300.serving import replay
    X, base, start, Q = world
    ex = AsyncExec(X, base, start)
    srv = ex.server()
    reqs = _stream(Q, n=30, seed=5)
    try:
        rep = replay(srv, reqs, time_scale=0.0)
    finally:
        rp.rp_server_destroy(srv)
    for r in reqs:
        if r.kind == "search":
            ids, d2 = _expected(X, base, start, r)
            assert np.array_equal(r.ids, ids) and np.array_equal(r.dists, d2)
    assert rep["stats"]["requests_done"] == len(reqs) and rep["stats"]["requests_failed"] == 0
    assert not ex.graphs.keys() - {OracleExec.BASE}
    ex2 = AsyncExec(X, base, start, fail_alpha_milli=1050)
    srv = ex2.server()
    try:
        ok = rp.rp_submit_search(srv, 1.1, 24, Q[:2], 10, 10)
        assert rp.rp_poll(srv, ok[0], 20000)["status"] == rp.RP_OK
        bad = rp.rp_submit_search(srv, 1.05, 24, Q[:2], 10, 10)
        assert rp.rp_poll(srv, bad[0], 20000)["status"] == rp.RP_ENOMEM
    finally:
        rp.rp_server_destroy(srv)


def test_async_respects_the_budget(world):
    """The asynchronous path never holds more tuned graphs than the budget,
    however many distinct targets are parked at once."""
    from paper_2602_08097_gb300.serving import Request, replay
    X, base, start, Q = world
    ex = AsyncExec(X, base, start)
    srv = ex.server(budget_graphs=2)
    targets = [(1.15, 24), (1.1, 24), (1.05, 16), (1.0, 16), (1.12, 20), (1.15, 24)]
    reqs = [Request("search", a, R, 0.0, queries=Q[i:i + 2], L=10, k=10) for i, (a, R) in enumerate(targets)]
    try:
        replay(srv, reqs, time_scale=0.0)
        st = rp.rp_server_stats(srv)
    finally:
        rp.rp_server_destroy(srv)
    assert st["peak_resident_graphs"] <= 2 and ex.live_peak <= 2
    for r in reqs:
        ids, d2 = _expected(X, base, start, r)
        assert np.array_equal(r.ids, ids)
