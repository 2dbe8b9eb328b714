"""RP-Tuning split by node ranges on the GPU: every rank's slice
(rp_graph_slice -> rp_tune_batch), assembled in range order, must equal the
unsharded tuning bit for bit.  Ranks run one after another on the one GPU
(they never wait on each other: the split has no exchange step)."""
import numpy as np
import pytest

import datagen
import oracle

rp = pytest.importorskip("paper_2602_08097_gb300")
pytestmark = pytest.mark.gpu

TARGETS = [(1.1, 48), (1.05, 32), (1.0, 16)]


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


@pytest.mark.parametrize("name,n,world", [("sift", 6000, 3), ("tiny", 2000, 2), ("deep", 3001, 4)])
def test_slices_assemble_to_the_unsharded_tuning(ctx, name, n, world):
    from paper_2602_08097_gb300 import shard
    X = datagen.dataset(name, n)
    base_rp, base_col = oracle.knn_base(X, 64, 1.2, 48)
    base = rp.rp_load_graph(ctx, X, base_rp, base_col)
    alphas, Rs = [a for a, _ in TARGETS], [r for _, r in TARGETS]
    whole = [rp.rp_graph_export(ctx, g) for g in rp.rp_tune_batch(ctx, base, alphas, Rs)]
    per_rank = [shard.tune_slices(ctx, base, alphas, Rs, r, world) for r in range(world)]
    for t in range(len(TARGETS)):
        got_rp, got_col = shard.assemble([per_rank[r][t] for r in range(world)], n)
        assert np.array_equal(got_rp, whole[t][0]) and np.array_equal(got_col, whole[t][1]), f"target {t}"
        ref_rp, ref_col = oracle.rp_tune(X, base_rp, base_col, *TARGETS[t])
        assert np.array_equal(got_rp, ref_rp) and np.array_equal(got_col, ref_col)
    rp.rp_graph_free(ctx, base)


def test_slice_bounds(ctx):
    X = datagen.dataset("tiny", 300)
    base_rp, base_col = oracle.knn_base(X, 16, 1.2, 16)
    base = rp.rp_load_graph(ctx, X, base_rp, base_col)
    empty = rp.rp_graph_slice(ctx, base, 120, 120)
    assert rp.rp_graph_info(ctx, empty)["nnz"] == 0
    full = rp.rp_graph_slice(ctx, base, 0, 300)
    f_rp, f_col = rp.rp_graph_export(ctx, full)
    assert np.array_equal(f_rp, base_rp) and np.array_equal(f_col, base_col)
    part = rp.rp_graph_slice(ctx, base, 10, 20)
    p_rp, p_col = rp.rp_graph_export(ctx, part)
    assert np.all(np.diff(p_rp)[:10] == 0) and np.all(np.diff(p_rp)[20:] == 0)
    assert np.array_equal(p_col, base_col[base_rp[10]:base_rp[20]])
    for lo, hi in [(-1, 5), (5, 4), (0, 301)]:
        with pytest.raises(rp.RPError):
            rp.rp_graph_slice(ctx, base, lo, hi)
    for g in (empty, full, part, base):
        rp.rp_graph_free(ctx, g)


def test_device_assembly_and_attach(ctx):
    """The multi-GPU step's assembly on the device: each rank's slice as device
    tensors (row lengths of its range, its column ids), concatenated in range
    order with a prefix sum (shard.allgather_csr's arithmetic), registered over
    the resident vectors with rp_graph_attach; the attached graph equals the
    unsharded tuning and its searches return the oracle's lists."""
    import torch
    from paper_2602_08097_gb300 import shard
    X = datagen.dataset("deep", 3000)
    Q = datagen.queries("deep", 40)
    base_rp, base_col = oracle.knn_base(X, 64, 1.2, 48)
    base = rp.rp_load_graph(ctx, X, base_rp, base_col)
    start = rp.rp_graph_info(ctx, base)["start"]
    dev = torch.device("cuda", 0)
    world, n = 3, X.shape[0]
    a, R = TARGETS[1]
    parts = []
    for r in range(world):
        lo, hi = shard.node_range(r, world, n)
        part = rp.rp_graph_slice(ctx, base, lo, hi)
        (g,) = rp.rp_tune_batch(ctx, part, [a], [R])
        rp_d, col_d = rp.rp_graph_export(ctx, g, device=dev)
        parts.append((torch.diff(rp_d[lo:hi + 1]), col_d.clone()))
        rp.rp_graph_free(ctx, g)
        rp.rp_graph_free(ctx, part)
    lengths = torch.cat([c for c, _ in parts])
    row_ptr = torch.zeros(n + 1, dtype=torch.int64, device=dev)
    torch.cumsum(lengths, 0, out=row_ptr[1:])
    col = torch.cat([c for _, c in parts])
    g = rp.rp_graph_attach(ctx, base, row_ptr, col)
    got_rp, got_col = rp.rp_graph_export(ctx, g)
    ref_rp, ref_col = oracle.rp_tune(X, base_rp, base_col, a, R)
    assert np.array_equal(got_rp, ref_rp) and np.array_equal(got_col, ref_col)
    assert rp.rp_graph_info(ctx, g)["start"] == start
    ids, _ = rp.rp_search(ctx, g, Q, 40, 10)
    ref_ids, _, _ = oracle.greedy_search(X, ref_rp, ref_col, start, Q, 40, 10)
    assert np.array_equal(ids, ref_ids)
    bad = col.clone()
    bad[0] = n  # an id out of range is refused
    with pytest.raises(rp.RPError):
        rp.rp_graph_attach(ctx, base, row_ptr, bad)
    rp.rp_graph_free(ctx, g)
    rp.rp_graph_free(ctx, base)
