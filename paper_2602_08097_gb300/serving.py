"""Serving workload driver over the library's scheduler (rp_server_* in
include/rp.h): turns an arrival stream into prune-to-(alpha, R) jobs and
query batches, submits each at its arrival time and reports latency
percentiles and throughput.

All scheduling (admission, batching, eviction) and all device work happen
inside librp.so; this module only submits, polls and summarises.  Latency is
taken from the library's own timestamps (submission to completion).
"""
from __future__ import annotations

import time
from dataclasses import dataclass

import numpy as np

from . import rp_poll, rp_server_stats, rp_submit_search, rp_submit_tune


@dataclass
class Request:
    kind: str                       # "tune" or "search"
    alpha: float                    # 0 addresses the base graph (search only)
    R: int
    arrival: float                  # seconds from the start of the stream
    queries: np.ndarray | None = None
    rows: np.ndarray | None = None  # which rows of the query set the batch holds
    L: int = 0
    k: int = 0
    rid: int = -1                   # library request id once submitted
    ids: np.ndarray | None = None
    dists: np.ndarray | None = None
    info: dict | None = None        # rp_request_info once finished


def make_requests(stream: list, queries: np.ndarray, seed: int = 0, first_target=(1.1, 64)) -> list:
    """Requests from datagen.poisson_stream: a query batch takes ``nq`` distinct
    rows of ``queries`` (seeded) and addresses one of the targets tuned so far,
    chosen by the stream's uniform draw (``first_target`` before any)."""
    rng = np.random.default_rng(seed)
    reqs, targets = [], [tuple(first_target)]
    for s in stream:
        if s["kind"] == "tune":
            targets.append((s["alpha"], s["R"]))
            reqs.append(Request("tune", s["alpha"], s["R"], s["t"]))
        else:
            a, R = targets[min(int(s["slot_u"] * len(targets)), len(targets) - 1)]
            nq = min(s["nq"], queries.shape[0])
            rows = rng.choice(queries.shape[0], size=nq, replace=False)
            reqs.append(Request("search", a, R, s["t"], queries=np.ascontiguousarray(queries[rows]), rows=rows,
                                L=s["L"], k=s["k"]))
    return reqs


def replay(srv, requests: list, time_scale: float = 1.0, poll_ms: int = 1000, max_wait_s: float = 600.0) -> dict:
    """Submit ``requests`` at arrival * time_scale seconds, wait for all of them,
    and return a summary (latency percentiles in ms, queries per second, the
    server's counters).  A request that failed raises."""
    reqs = sorted(requests, key=lambda r: r.arrival)
    t0 = time.perf_counter()
    for r in reqs:
        wait = r.arrival * time_scale - (time.perf_counter() - t0)
        if wait > 0:
            time.sleep(wait)
        if r.kind == "tune":
            r.rid = rp_submit_tune(srv, r.alpha, r.R)
        else:
            r.rid, r.ids, r.dists = rp_submit_search(srv, r.alpha, r.R, r.queries, r.L, r.k)
    deadline = time.perf_counter() + max_wait_s
    for r in reqs:
        while r.info is None:
            r.info = rp_poll(srv, r.rid, poll_ms)
            if r.info is None and time.perf_counter() > deadline:
                raise TimeoutError(f"request {r.rid} unfinished after {max_wait_s} s")
        if r.info["status"] != 0:
            raise RuntimeError(f"request {r.rid} ({r.kind} alpha={r.alpha} R={r.R}) failed: {r.info['status']}")
    wall = time.perf_counter() - t0
    lat = np.array([(r.info["done_ns"] - r.info["submit_ns"]) / 1e6 for r in reqs])
    slat = np.array([(r.info["done_ns"] - r.info["submit_ns"]) / 1e6 for r in reqs if r.kind == "search"])
    nq = sum(r.queries.shape[0] for r in reqs if r.kind == "search")
    first = min(r.info["submit_ns"] for r in reqs)
    last = max(r.info["done_ns"] for r in reqs)

    def pct(v, q):
        return float(np.percentile(v, q)) if len(v) else None
    return {"requests": len(reqs), "queries": int(nq), "p50_ms": pct(lat, 50), "p99_ms": pct(lat, 99),
            "search_p50_ms": pct(slat, 50), "search_p99_ms": pct(slat, 99),
            "qps": nq / ((last - first) / 1e9) if last > first else None, "wall_s": wall,
            "stats": rp_server_stats(srv)}
