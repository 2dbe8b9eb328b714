#!/usr/bin/env python
"""Benchmark of the RP-Tuning hot path on one GB300 (per rank under torchrun).

Default workload (deep-shaped float, the largest single-GPU configuration):
n = 10,000,000 points, d = 96, float32 unit rows from a 256-centre Gaussian
mixture; base graph = Vamana (§2.1, §4.1: two insertion passes at alpha 1.0
and 1.2, R = 64, L_build = 75), built once by the library on the GPU (not
timed); eight targets (alpha, R) in {1.15, 1.1, 1.05, 1.0} x {64, 48} in one
batched, graph-captured launch; 10,000 queries, L = 100, k = 100.

One timed step = the whole hot path over that input: RP-Tuning of every node
for every target in one batched launch (gather, keys, Gram, sort, domination
bits, scans, CSR emit), GreedySearch of the queries on each tuned graph and
recall@100 of each against the exact kNN ground truth.  `value` = nodes x
targets / second over the timed steps (inputs resident in HBM, L2 flushed
before every step).  `e2e` repeats the step through the C ABI with host
buffers: vectors, base CSR and queries copied in, tuned graphs and search
results copied out, every step.

`--workload sift` runs the integer configuration (1,000,000 x 128 uint8,
rint(min(255, Gamma(0.6, 40))); base RobustPrune(1.2, 64) over each point's
exact 128 nearest neighbours; targets (1.1, 64), (1.05, 48), (1.0, 32);
10,000 queries, L = 128).  `--workload gist` runs the batched high-d float sweep
(1,000,000 x 960 float32 rows, |N(0,1)| * 0.05 then L2-normalised; base over
exact kNN-128; nine targets: alpha 1.175 down to 1.0 at R = 64 plus (1.0, 32),
in one launch; 1,000 queries, L = 200).

`serving` (outside the timed step): a Poisson stream of prune-to-(alpha, R)
jobs and query batches through the library's scheduler (rp_server_*), the
continuous-batching scheduler against the plain serial path, at offered loads
relative to the serial path's capacity; p50/p99 latency, QPS and recall@100.
It runs over the sift base (8 GB of tuned graphs, so the stream evicts) and
over the deep base (120 GB).

Outside the timed step every workload also sweeps L over 100..256 on the base
and on each tuned graph (`recall_qps_frontier`: QPS and recall@100 per L),
measures alpha-reachability (Definition 2.1) at seeded nodes of the base and
of every target tuned with the sorted and the unsorted variant
(`reachability_sample`: min and median of the per-node terms; 64 nodes on the
integer workload, where distances are exact integers, and none on the float
ones, whose binary64 distances over every point take minutes per node on this
part), times the Vamana build against the tuning (`rebuild_vs_tune`: the
analogue of Table 2), and checks that re-pruning a tuned graph at its own
(alpha, R) returns it edge for edge (`idempotence_check`).

`--impl reference` times the CPU oracle (the reference arm of this build) on
a bounded sample of the same workload and prints the same JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import datagen  # noqa: E402

METRIC = "RP-Tuning nodes/s per α (batched vs plain, same GPU); query p50/p99 at recall@100"
UNIT = "nodes/s per alpha"
BASE_ALPHA, BASE_R, KCAND = 1.2, 64, 128
K_SEARCH = 100
# graph budget of the serving leg: 8 GB keeps ~30 sift-sized tuned graphs (the
# stream evicts); the deep stream runs under 120 GB of tuned graphs
SERVE_BUDGET_GB = {"sift": 8, "deep": 120}
SERVE_LOADS = (0.5, 0.8, 1.0, 2.0, 4.0)  # offered load / capacity of the serial path
FRONTIER_L = (100, 128, 160, 200, 256)   # list sizes of the recall-QPS frontier (k = 100)
REACH_SAMPLE = {"sift": 64, "gist": 0, "deep": 0}  # nodes whose alpha-reachability terms are measured
VAMANA = dict(alphas=(1.0, 1.2), L=75)    # §4.1's base construction (alpha1 = 1.2, L_build = 75), R = BASE_R

# The paper-shaped workloads (synthetic; recipes in datagen).  deep is the
# default bench line (the largest single-GPU configuration); sift the integer
# one; gist the batched high-d float sweep (9 targets: alpha 1.175 down to 1.0
# in steps of 0.025 at R=64, plus (1.0, 32)).
WORKLOADS = {
    "sift": dict(dtype="u8", n=1_000_000, d=128, nq=10_000, L=128,
                 targets=[(1.1, 64), (1.05, 48), (1.0, 32)]),
    "gist": dict(dtype="f32", n=1_000_000, d=960, nq=1_000, L=200,
                 targets=[(round(1.175 - 0.025 * i, 3), 64) for i in range(8)] + [(1.0, 32)]),
    "deep": dict(dtype="f32", n=10_000_000, d=96, nq=10_000, L=100,
                 targets=[(a, r) for a in (1.15, 1.1, 1.05, 1.0) for r in (64, 48)],
                 base="vamana"),
}
TARGETS = WORKLOADS["sift"]["targets"]
L_SEARCH = WORKLOADS["sift"]["L"]


def workload_name(n, nq, name="sift"):
    w = WORKLOADS[name]
    shape = {"sift": "sift-shaped uint8", "gist": "gist-shaped float32", "deep": "deep-shaped float32"}[name]
    tl = ",".join(f"({a:g},{r})" for a, r in w["targets"])
    if w.get("base") == "vamana":
        base = (f"base Vamana(alpha {VAMANA['alphas'][0]:g} then {VAMANA['alphas'][1]:g}, R={BASE_R}, "
                f"L_build={VAMANA['L']})")
    else:
        base = "base RobustPrune(1.2,64) over exact kNN-128"
    return f"{shape} n={n:,} d={w['d']}; {base}; tune {tl}; {nq:,} queries L={w['L']} k=100"


def build_base(rp, ctx, data, name):
    """The workload's base graph, built by the library on the GPU (the benchmark's
    untimed fixture; the full-size parity tests build the same one)."""
    W = WORKLOADS[name]
    if W.get("base") == "vamana":  # the points are drawn independently: index order is a random order
        g, _ = rp.rp_build_vamana(ctx, data, VAMANA["alphas"], BASE_R, VAMANA["L"])
        return g
    return rp.rp_build_knn_base(ctx, data, KCAND, BASE_ALPHA, BASE_R)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- reference arm / CPU baseline

def oracle_sample(n_sample, name="sift"):
    """The oracle's own base over the generator's first n points of the workload (no GPU input),
    built the way the workload builds its base."""
    import oracle
    X = datagen.dataset(name, n_sample)
    t0 = time.perf_counter()
    if WORKLOADS[name].get("base") == "vamana":
        base_rp, base_col, _ = oracle.vamana(X, np.arange(n_sample, dtype=np.int32), VAMANA["alphas"], BASE_R,
                                             VAMANA["L"], 4 * VAMANA["L"], max(1, n_sample // 50), oracle.medoid(X))
    else:
        base_rp, base_col = oracle.knn_base(X, KCAND, BASE_ALPHA, BASE_R)
    return X, base_rp, base_col, time.perf_counter() - t0


def time_oracle_tune(X, base_rp, base_col, targets=None):
    import oracle
    t0 = time.perf_counter()
    for a, r in (targets or TARGETS):
        oracle.rp_tune(X, base_rp, base_col, a, r)
    return time.perf_counter() - t0


def cpu_baseline(n_sample=20000, name="sift"):
    import oracle
    w = WORKLOADS[name]
    X, brp, bcol, build_s = oracle_sample(n_sample, name)
    secs, reps = 0.0, 0
    while secs < 10.0 or reps < 1:  # about ten seconds of CPU work
        secs += time_oracle_tune(X, brp, bcol, w["targets"])
        reps += 1
    Q = datagen.queries(name, 200)
    start = oracle.medoid(X)
    t0 = time.perf_counter()
    oracle.greedy_search(X, brp, bcol, start, Q, w["L"], K_SEARCH)
    qs = time.perf_counter() - t0
    T = len(w["targets"])
    return {"value": reps * n_sample * T / secs, "unit": UNIT, "cores": oracle.num_threads(0),
            "kind": "oracle",
            "sample": (f"oracle RP-Tuning of all {n_sample:,} nodes of the generator's first {n_sample:,} points "
                       f"of the workload (its own base, built as the workload's), {T} targets, repeated {reps}x "
                       f"({secs:.1f} s); GreedySearch of 200 queries {200 / qs:.1f} QPS"),
            "search_qps": 200 / qs}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    n_sample = args.ref_sample
    w = WORKLOADS[args.workload]
    X, brp, bcol, _ = oracle_sample(n_sample, args.workload)
    for _ in range(args.warmup):
        time_oracle_tune(X, brp, bcol, w["targets"])
    times = [time_oracle_tune(X, brp, bcol, w["targets"]) for _ in range(args.steps)]
    tot = sum(times)
    value = n_sample * len(w["targets"]) * args.steps / tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": w["dtype"],
            "data": "synthetic", "config": {"workload": workload_name(args.n, args.nq, args.workload),
                                            "reference_sample_nodes": n_sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(0), "kind": "oracle",
                             "sample": (f"RP-Tuning of the generator's first {n_sample:,} points (its own base), "
                                        f"{len(w['targets'])} targets per step")},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- our arm

def run_ours(args):
    import torch
    import paper_2602_08097_gb300 as rp
    from paper_2602_08097_gb300 import build as b

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    b.build()
    W = WORKLOADS[args.workload]
    TARGETS_W = W["targets"]
    L_W = W["L"]
    n, nq, k = args.n, args.nq, K_SEARCH
    X = datagen.dataset(args.workload, n)
    Q = datagen.queries(args.workload, nq)
    row_bytes = X.shape[1] * X.itemsize
    stream = torch.cuda.Stream(device=dev)
    ctx = rp.rp_create(local, stream=stream)
    alphas = [a for a, _ in TARGETS_W]
    Rs = [r for _, r in TARGETS_W]
    T = len(TARGETS_W)

    # ---- fixture (not timed): vectors, base graph, ground truth
    t0 = time.perf_counter()
    data = rp.rp_load_graph(ctx, X)
    torch.cuda.synchronize(dev)
    tb0 = time.perf_counter()
    base = build_base(rp, ctx, data, args.workload)
    torch.cuda.synchronize(dev)
    base_build_s = time.perf_counter() - tb0
    base_rp, base_col = rp.rp_graph_export(ctx, base)
    gt, _ = rp.rp_knn(ctx, data, Q, k)
    fixture_s = time.perf_counter() - t0
    deg = np.diff(base_rp)
    Qd = torch.from_numpy(Q).to(dev)
    gtd = torch.from_numpy(gt).to(dev)
    ids_d = [torch.empty((nq, k), dtype=torch.int32, device=dev) for _ in range(T)]
    dist_d = [torch.empty((nq, k), dtype=torch.float32, device=dev) for _ in range(T)]
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)

    stats_acc = {"prune_ms": [], "emit_ms": [], "search_ms": []}

    # Several GPUs: the nodes split into contiguous id ranges (RP-Tuning treats
    # every node on its own, §3).  Each rank tunes its range, the ranks'
    # slices are all-gathered as device tensors (row lengths and column ids)
    # and registered over the resident vectors, and each rank searches its
    # share of the queries on the assembled graphs.
    split = None
    if ws > 1:
        from paper_2602_08097_gb300 import shard
        lo, hi = shard.node_range(rank, ws, n)
        split = dict(part=rp.rp_graph_slice(ctx, base, lo, hi), lo=lo, hi=hi,
                     q=slice(nq * rank // ws, nq * (rank + 1) // ws))

    def tune_step():
        if split is None:
            return rp.rp_tune_batch(ctx, base, alphas, Rs)
        from paper_2602_08097_gb300 import shard
        outs = []
        for g in rp.rp_tune_batch(ctx, split["part"], alphas, Rs):
            row_ptr, col = rp.rp_graph_export(ctx, g, device=dev)
            rp.rp_graph_free(ctx, g)
            counts = torch.diff(row_ptr[split["lo"]:split["hi"] + 1])
            full_rp, full_col = shard.allgather_csr(counts, col, n)
            outs.append(rp.rp_graph_attach(ctx, base, full_rp, full_col))
        return outs

    def step(record):
        outs = tune_step()
        if record:
            st = rp.rp_stats(ctx)
            stats_acc["prune_ms"].append(st["last_prune_ms"])
            stats_acc["emit_ms"].append(st["last_emit_ms"])
        sms = 0.0
        qs = split["q"] if split else slice(0, nq)
        for i, g in enumerate(outs):
            rp.rp_search(ctx, g, Qd[qs], L_W, k, ids=ids_d[i][qs], dists=dist_d[i][qs])
            if record:
                sms += rp.rp_stats(ctx)["last_search_ms"]
        if record:
            stats_acc["search_ms"].append(sms)
        hits = [rp.rp_recall(ctx, ids_d[i][qs], gtd[qs], k) for i in range(T)]
        return outs, hits

    def free(outs):
        for g in outs:
            rp.rp_graph_free(ctx, g)

    nnz = None
    for _ in range(args.warmup):
        outs, hits = step(False)
        if nnz is None:
            nnz = [rp.rp_graph_info(ctx, g)["nnz"] for g in outs]
        free(outs)
    torch.cuda.synchronize(dev)
    if ws > 1:
        torch.distributed.barrier()
    l0 = rp.rp_stats(ctx)["kernel_launches"]
    times = []
    recalls = None
    with ClockSampler(local) as clocks:
        for _ in range(args.steps):
            with torch.cuda.stream(stream):
                flush.zero_()  # evict L2 (129 MB) before every timed step
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            torch.cuda.nvtx.range_push("bench_step")  # lets a profiler select the timed steps' launches
            outs, hits = step(False)
            torch.cuda.nvtx.range_pop()
            e1.record(stream)
            stream.synchronize()
            times.append(e0.elapsed_time(e1))
            nq_local = (nq * (rank + 1) // ws - nq * rank // ws) if split else nq
            recalls = [h / (nq_local * k) for h in hits]
            if nnz is None:
                nnz = [rp.rp_graph_info(ctx, g)["nnz"] for g in outs]
            free(outs)
    launches = rp.rp_stats(ctx)["kernel_launches"] - l0
    torch.cuda.synchronize(dev)
    tot_ms = sum(times)
    if ws > 1:
        t = torch.tensor([tot_ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        torch.distributed.barrier()
        tot_ms = float(t.item())
    # one graph tuned by all ranks together (split), each rank's share of the queries
    value = n * T * args.steps / (tot_ms / 1000.0)

    # ---- per-kernel timing pass (same step, phase events read between calls)
    for _ in range(max(2, args.steps)):
        with torch.cuda.stream(stream):
            flush.zero_()
        outs, _ = step(True)
        free(outs)
    tuned_cfg = rp.rp_stats(ctx)  # the autotuner's pick for this source and target count
    st_tiers = rp.rp_stats(ctx, reset=True)  # decision tiers over the whole run so far
    tiers = {"f32_rechecks_per_node_target": st_tiers["f32_rechecks"] / max(st_tiers["nodes_pruned"], 1),
             "fp64_decisions_per_node_target": st_tiers["fp64_decisions"] / max(st_tiers["nodes_pruned"], 1),
             "fp64_sort_keys": st_tiers["fp64_sort_keys"], "fp64_search_dists": st_tiers["fp64_search_dists"]}
    prune_ms = statistics.mean(stats_acc["prune_ms"])
    if not prune_ms > 0:
        raise RuntimeError(f"prune kernel time not measured: {stats_acc}")
    emit_ms = statistics.mean(stats_acc["emit_ms"])
    search_ms = statistics.mean(stats_acc["search_ms"])
    deg_r = deg[split["lo"]:split["hi"]] if split else deg  # the nodes this rank's prune launch covers
    alg_bytes = float(((deg_r + 1) * row_bytes + 4 * deg_r + 8).sum() + 4 * sum(nnz) * len(deg_r) / n)
    hbm_peak, peak_kind = load_peaks()
    achieved = alg_bytes / (prune_ms / 1000.0) / 1e9
    traffic = None  # DRAM bytes per launch from the committed ncu summary, if it is of this kernel source
    prof = os.path.join(ROOT, "profiles", f"prune_tc_{W['dtype']}_{args.workload}_full.md")
    if os.path.exists(prof) and n == W["n"]:
        fields = {}
        with open(prof) as f:
            for ln in f:
                if ":" in ln and not ln.startswith(("#", "-", " ", "|")):
                    k_, v_ = ln.split(":", 1)
                    fields[k_.strip()] = v_.strip()
        if fields.get("kernel_source_hash") == kernel_hash():
            traffic = float(fields["traffic_bytes_per_launch"])

    # ---- plain vs batched tuning alone
    def time_tune(batched, reps):
        ts = []
        for r in range(reps + 2):
            with torch.cuda.stream(stream):
                flush.zero_()
            a0 = torch.cuda.Event(enable_timing=True)
            a1 = torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            if batched:
                outs = rp.rp_tune_batch(ctx, base, alphas, Rs)
            else:
                outs = [rp.rp_tune(ctx, base, a, R) for a, R in TARGETS_W]
            a1.record(stream)
            stream.synchronize()
            if r >= 2:
                ts.append(a0.elapsed_time(a1))
            free(outs)
        return statistics.median(ts)

    tb = time_tune(True, args.steps) if not args.quick else float("nan")
    tp = time_tune(False, args.steps) if not args.quick else float("nan")

    # ---- single-query latency (batch size 1), on the (1.05, 48) graph
    outs = rp.rp_tune_batch(ctx, base, alphas, Rs)
    g1 = outs[1]
    lat = []
    q1 = [Qd[i:i + 1] for i in range(min(300 if not args.quick else 22, nq))]
    i1 = torch.empty((1, k), dtype=torch.int32, device=dev)
    d1 = torch.empty((1, k), dtype=torch.float32, device=dev)
    for i, q in enumerate(q1):
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        rp.rp_search(ctx, g1, q, L_W, k, ids=i1, dists=d1)
        a1.record(stream)
        stream.synchronize()
        if i >= 20:
            lat.append(a0.elapsed_time(a1))
    free(outs)
    lat.sort()
    p50 = lat[len(lat) // 2]
    p99 = lat[min(len(lat) - 1, int(0.99 * len(lat)))]

    # ---- recall-QPS frontier over L (outside the timed step): the base and each
    # tuned graph, every query batch at once
    frontier = None
    if not args.quick:
        outs = rp.rp_tune_batch(ctx, base, alphas, Rs)
        ide = torch.empty((nq, k), dtype=torch.int32, device=dev)
        frontier = {}
        for gname, g in [("base", base)] + [(f"{a},{r}", o) for (a, r), o in zip(TARGETS_W, outs)]:
            pts = []
            for Lx in FRONTIER_L:
                rp.rp_search(ctx, g, Qd, Lx, k, ids=ide)
                ms = rp.rp_stats(ctx)["last_search_ms"]
                pts.append({"L": Lx, "qps": nq / (ms / 1000.0),
                            "recall_at_100": rp.rp_recall(ctx, ide, gtd, k) / (nq * k)})
            frontier[gname] = pts
        free(outs)

    # ---- alpha-reachability (Definition 2.1) at a seeded sample of nodes: the base
    # and every target tuned with each of Algorithm 1's variants, the comparison
    # Theorems 3.1-3.2 are about; outside the timed step.  The base's lists come
    # out of RobustPrune already in its processing order, where the unsorted
    # variant would coincide with the sorted one, so the unsorted variant runs on
    # the same lists reversed (farthest first: an arbitrary order, as it allows).
    reach = None
    if not args.quick and REACH_SAMPLE[args.workload] > 0:
        sample = np.sort(np.random.default_rng(5005).choice(n, min(n, REACH_SAMPLE[args.workload]), replace=False))
        reach = {"nodes": int(sample.size), "unsorted_order": "each base list reversed", "graphs": {}}
        r0 = time.perf_counter()
        a_b, per_b = rp.rp_reachability(ctx, base, sample)
        reach["graphs"]["base"] = {"min": a_b, "median": float(np.median(per_b))}
        rev_col = base_col[np.repeat(base_rp[:-1] + base_rp[1:] - 1, deg) - np.arange(base_col.shape[0])]
        rev = rp.rp_load_graph(ctx, X, base_rp, rev_col)
        del rev_col
        for vname, vcode, src in (("sorted", rp.RP_SORTED, base), ("unsorted", rp.RP_UNSORTED, rev)):
            outs = rp.rp_tune_batch(ctx, src, alphas, Rs, vcode)
            for (a, r), g in zip(TARGETS_W, outs):
                a_t, per_t = rp.rp_reachability(ctx, g, sample)
                reach["graphs"][f"{a},{r} {vname}"] = {"min": a_t, "median": float(np.median(per_t))}
            free(outs)
        rp.rp_graph_free(ctx, rev)
        reach["seconds"] = time.perf_counter() - r0

    # ---- idempotence at full size: a tuned graph is RobustPrune output, so
    # re-pruning it at its own (alpha, R) must return it edge for edge, order
    # included (checked on the first target)
    a0, r0 = TARGETS_W[0]
    once = rp.rp_tune(ctx, base, a0, r0)
    twice = rp.rp_tune(ctx, once, a0, r0)
    g_rp, g_col = rp.rp_graph_export(ctx, once)
    b_rp, b_col = rp.rp_graph_export(ctx, twice)
    idempotent = bool(np.array_equal(g_rp, b_rp) and np.array_equal(g_col, b_col))
    rp.rp_graph_free(ctx, twice)
    rp.rp_graph_free(ctx, once)
    del g_rp, g_col, b_rp, b_col

    # ---- rebuild vs tune (the analogue of Table 2): a Vamana graph built at the
    # middle target's alpha against RP-Tuning of the base to it, both on this GPU
    rebuild = None
    if not args.quick and W.get("base") == "vamana":
        am, rm = TARGETS_W[len(TARGETS_W) // 2]
        torch.cuda.synchronize(dev)
        r0_ = time.perf_counter()
        g_re, _ = rp.rp_build_vamana(ctx, data, (VAMANA["alphas"][0], am), rm, VAMANA["L"])
        torch.cuda.synchronize(dev)
        t_rebuild = time.perf_counter() - r0_
        rp.rp_graph_free(ctx, g_re)
        t0_ = time.perf_counter()
        g_tu = rp.rp_tune(ctx, base, am, rm)
        torch.cuda.synchronize(dev)
        t_tune = time.perf_counter() - t0_
        rp.rp_graph_free(ctx, g_tu)
        rebuild = {"alpha": am, "R": rm, "rebuild_s": t_rebuild, "tune_s": t_tune, "speedup": t_rebuild / t_tune,
                   "note": "Vamana rebuild (alpha 1.0 then alpha) vs RP-Tuning of the base, one GPU"}

    # ---- end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e and not args.quick:
        Xh = torch.from_numpy(X).pin_memory()
        rph = torch.from_numpy(base_rp).pin_memory()
        colh = torch.from_numpy(base_col).pin_memory()
        Qh = torch.from_numpy(Q).pin_memory()
        gth = torch.from_numpy(gt).pin_memory()
        idh = [torch.empty((nq, k), dtype=torch.int32).pin_memory() for _ in range(T)]
        dh = [torch.empty((nq, k), dtype=torch.float32).pin_memory() for _ in range(T)]
        out_rp = [torch.empty(n + 1, dtype=torch.int64).pin_memory() for _ in range(T)]
        out_col = [torch.empty(base_col.shape[0], dtype=torch.int32).pin_memory() for _ in range(T)]
        lib = rp.load_library()
        import ctypes
        # a stored index is its vectors, its adjacency and its start vertex
        base_start = rp.rp_graph_info(ctx, base)["start"]

        def e2e_step():
            g = rp.rp_load_graph(ctx, Xh, rph, colh, start=base_start)
            outs = rp.rp_tune_batch(ctx, g, alphas, Rs)
            h2d = X.nbytes + base_rp.nbytes + base_col.nbytes
            d2h = 0
            hits = []
            for i, t in enumerate(outs):
                rp.rp_search(ctx, t, Qh, L_W, k, ids=idh[i], dists=dh[i])
                h2d += Q.nbytes
                d2h += idh[i].numel() * 4 + dh[i].numel() * 4
                hits.append(rp.rp_recall(ctx, idh[i], gth, k))
                h2d += idh[i].numel() * 4 + gth.numel() * 4
                rc = lib.rp_graph_export(ctx, int(t), ctypes.c_void_p(out_rp[i].data_ptr()),
                                         ctypes.c_void_p(out_col[i].data_ptr()), int(out_col[i].numel()),
                                         rp.RP_MEM_HOST)
                if rc != 0:
                    raise rp.RPError(rc, rp.rp_last_error(ctx))
                d2h += (n + 1) * 8 + nnz[i] * 4
            for t in outs:
                rp.rp_graph_free(ctx, t)
            rp.rp_graph_free(ctx, g)
            return h2d, d2h

        for _ in range(1):
            e2e_step()
        torch.cuda.synchronize(dev)
        et = []
        for _ in range(max(2, min(args.steps, 5))):
            t1 = time.perf_counter()
            h2d, d2h = e2e_step()
            torch.cuda.synchronize(dev)
            et.append(time.perf_counter() - t1)
        e2e_s = statistics.mean(et)
        e2e = {"value": n * T / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "ms_per_step": 1000 * e2e_s,
               "step": "load the stored index (vectors, CSR, start vertex) from pinned host memory, tune, "
                       "search with host queries and results, recall, export every tuned graph to host memory"}

    serving = None
    if not args.quick and not args.no_serve and args.workload in SERVE_BUDGET_GB:
        serving = serve_bench(rp, ctx, base, Q, gt, args)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline and not args.quick:
        cpu = cpu_baseline(args.cpu_sample, args.workload)

    rp.rp_destroy(ctx)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": W["dtype"], "data": "synthetic",
            "config": {"workload": workload_name(n, nq, args.workload), "n": n, "d": W["d"], "targets": TARGETS_W,
                       "queries": nq, "L": L_W, "k": k, "l2": "flushed (512 MB write) before every timed step",
                       "parallelism": f"node ranges x{ws} (all-gather of tuned slices)" if ws > 1 else "1 GPU"},
            "roofline": {"bound": "hbm", "kernel": f"prune_tc_kernel<{W['dtype']}, 64, {kernel_tb(W['dtype'], TARGETS_W)}> "
                                                   "(tcgen05 Gram)",
                         "achieved": achieved,
                         "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak, "traffic": traffic,
                         "peak_kind": peak_kind, "algorithmic_bytes_per_launch": alg_bytes,
                         "launch_ms": prune_ms},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": int(launches),
            "clocks": clocks.summary(),
            "tune_batched_nodes_per_s_per_alpha": n * T / (tb / 1000.0),
            "tune_plain_nodes_per_s_per_alpha": n * T / (tp / 1000.0),
            "batched_over_plain": tp / tb,
            "phase_ms": {"prune": prune_ms, "emit": emit_ms, f"search_{T}x": search_ms},
            "decision_tiers": tiers,
            "prune_config": {"tile0": tuned_cfg["tile0"], "ctas_per_sm": tuned_cfg["ctas_per_sm"],
                             "chosen_by": "autotuner (rp_set_tuning RP_TUNING_AUTO)"},
            "search_qps": T * nq / (search_ms / 1000.0),
            "query_latency_ms_bs1": {"p50": p50, "p99": p99},
            "recall_at_100": dict(zip([f"{a},{r}" for a, r in TARGETS_W], recalls)),
            "avg_degree": {"base": float(deg.mean()), **{f"{a},{r}": nz / n for (a, r), nz in zip(TARGETS_W, nnz)}},
            "fixture_s": fixture_s,
            "recall_qps_frontier": frontier,
            "reachability_sample": reach,
            "idempotence_check": {"alpha": a0, "R": r0, "retune_equals_tuned": idempotent},
            "rebuild_vs_tune": rebuild,
            "base_build_s": base_build_s,
            "serving": serving,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def serve_bench(rp, ctx, base, Q, gt, args):
    """Poisson stream of prune jobs (10%) and query batches (1..1024 queries, L in
    64..256 raised to k=100) through the library's scheduler, continuous vs the
    plain serial path, at offered loads relative to the serial path's capacity.
    Latency is submission to completion, from the scheduler's own clock."""
    from paper_2602_08097_gb300.serving import make_requests, replay
    stream = datagen.poisson_stream(args.serve_requests, 1.0, seed=3001, prune_frac=0.10)
    budget_gb = SERVE_BUDGET_GB[args.workload]
    budget = budget_gb << 30

    def run(serial, time_scale):
        reqs = make_requests(stream, Q, seed=3001)
        srv = rp.rp_server_create(ctx, base, graph_budget_bytes=budget, serial=serial)
        try:
            rep = replay(srv, reqs, time_scale=time_scale)
        finally:
            rp.rp_server_destroy(srv)
        found = np.concatenate([r.ids for r in reqs if r.kind == "search"])
        truth = np.ascontiguousarray(np.concatenate([gt[r.rows] for r in reqs if r.kind == "search"]))
        rep["recall_at_100"] = rp.rp_recall(ctx, found, truth, K_SEARCH) / found.size
        rep.pop("wall_s", None)
        return rep

    # capacity of the serial path: everything submitted at once
    sat = run(True, 0.0)
    span_s = stream[-1]["t"]
    cap_rps = sat["requests"] / (sat["stats"]["busy_ns"] / 1e9)
    out = {"requests": args.serve_requests, "graph_budget_gb": budget_gb,
           "serial_capacity_req_per_s": cap_rps, "loads": {}}
    for load in SERVE_LOADS:
        rate = load * cap_rps
        ts = 1.0 / rate  # stream generated at 1 request/s
        entry = {"offered_req_per_s": rate}
        for name, serial in (("serial", True), ("continuous", False)):
            if serial and load > 1.0:
                continue  # the serial queue grows without bound past its capacity
            r = run(serial, ts)
            entry[name] = {k: r[k] for k in ("p50_ms", "p99_ms", "search_p50_ms", "search_p99_ms", "qps",
                                             "recall_at_100")}
            entry[name].update({k: r["stats"][k] for k in ("rounds", "tune_launches", "targets_tuned",
                                                            "search_launches", "evictions", "l_clamps")})
        out["loads"][f"{load:g}x"] = entry
    out["stream_span_s_at_1x"] = span_s / cap_rps
    return out


def kernel_tb(dtype, targets):
    """The prune kernel's TB for a sweep: the power of two at or above the number of
    targets (uint8) or of distinct alphas (float), at most 16."""
    k = len({a for a, _ in targets}) if dtype == "f32" else len(targets)
    tb = 1
    while tb < k:
        tb *= 2
    return min(tb, 16)


def kernel_hash():
    import hashlib
    h = hashlib.sha256()
    for f in ("prune.cu", "common.cuh", "tc.cuh"):
        with open(os.path.join(ROOT, "paper_2602_08097_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="deep")
    ap.add_argument("--n", type=int, default=None)
    ap.add_argument("--nq", type=int, default=None)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=400)
    ap.add_argument("--cpu-sample", type=int, default=20000)
    ap.add_argument("--ref-sample", type=int, default=20000)
    ap.add_argument("--quick", action="store_true",
                    help="timed steps and the per-kernel pass only (for profiler runs)")
    args = ap.parse_args()
    if args.n is None:
        args.n = WORKLOADS[args.workload]["n"]
    if args.nq is None:
        args.nq = WORKLOADS[args.workload]["nq"]
    if args.warmup < 3 and args.impl == "ours":
        print("note: timing rules ask for >= 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
