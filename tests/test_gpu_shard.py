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
