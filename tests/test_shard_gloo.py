"""Multi-GPU split of RP-Tuning by node ranges (paper_2602_08097_gb300.shard),
run as two gloo ranks on the CPU.  Each rank tunes its own node range (the
oracle stands in for the GPU, which these processes do not have), the
slices are all-gathered and assembled, and the result must equal the
unsharded tuning bit for bit, order included.  Also: the ranges tile 0..n,
and assembly rejects slices that do not."""
import os
import socket

import numpy as np
import pytest

import datagen
import oracle

shard = pytest.importorskip("paper_2602_08097_gb300.shard")

TARGETS = [(1.1, 32), (1.05, 24), (1.0, 16)]
N = 600


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem():
    X = datagen.dataset("tiny", N)
    base_rp, base_col = oracle.knn_base(X, 32, 1.2, 32)
    return X, base_rp, base_col


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        X, base_rp, base_col = _problem()
        lo, hi = shard.node_range(rank, world, N)
        mine = []
        for a, R in TARGETS:
            # the oracle tunes this rank's rows (on a GPU: rp_graph_slice + rp_tune_batch)
            rows = oracle.rp_tune(X, base_rp, base_col, a, R, nodes=np.arange(lo, hi))
            rp_ = np.zeros(hi - lo + 1, dtype=np.int64)
            np.cumsum([len(r) for r in rows], out=rp_[1:])
            col = np.concatenate(rows).astype(np.int32) if rows else np.zeros(0, np.int32)
            mine.append(shard.Slice(lo, hi, rp_, col))
        graphs = shard.gather_slices(mine, N)
        for t, (row_ptr, col) in enumerate(graphs):
            np.save(os.path.join(out_dir, f"r{rank}_t{t}_rp.npy"), row_ptr)
            np.save(os.path.join(out_dir, f"r{rank}_t{t}_col.npy"), col)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_match_the_unsharded_tuning(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    port = _free_port()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, str(tmp_path))) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0, "a rank failed"
    X, base_rp, base_col = _problem()
    for t, (a, R) in enumerate(TARGETS):
        ref_rp, ref_col = oracle.rp_tune(X, base_rp, base_col, a, R)
        for r in range(2):
            got_rp = np.load(tmp_path / f"r{r}_t{t}_rp.npy")
            got_col = np.load(tmp_path / f"r{r}_t{t}_col.npy")
            assert np.array_equal(got_rp, ref_rp) and np.array_equal(got_col, ref_col), f"rank {r} target {t}"


@pytest.mark.parametrize("n,world", [(0, 1), (1, 3), (10, 3), (1000, 7), (5, 8)])
def test_ranges_tile_the_nodes(n, world):
    ranges = [shard.node_range(r, world, n) for r in range(world)]
    assert ranges[0][0] == 0 and ranges[-1][1] == n
    for (a, b), (c, d) in zip(ranges, ranges[1:]):
        assert b == c and a <= b
    sizes = [b - a for a, b in ranges]
    assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard.node_range(world, world, n)


def test_assemble_round_trip_and_rejects_gaps():
    rng = np.random.default_rng(0)
    n = 50
    deg = rng.integers(0, 6, n)
    row_ptr = np.zeros(n + 1, np.int64)
    np.cumsum(deg, out=row_ptr[1:])
    col = rng.integers(0, n, int(row_ptr[-1])).astype(np.int32)
    parts = [shard.slice_of(row_ptr, col, *shard.node_range(r, 4, n)) for r in range(4)]
    got_rp, got_col = shard.assemble(parts[::-1], n)
    assert np.array_equal(got_rp, row_ptr) and np.array_equal(got_col, col)
    with pytest.raises(ValueError):
        shard.assemble(parts[:2] + parts[3:], n)  # a gap
    with pytest.raises(ValueError):
        shard.assemble(parts[:3], n)  # short of n
