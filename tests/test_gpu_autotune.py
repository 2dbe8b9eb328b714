"""Prune kernel configurations (rp_set_tuning): every fixed (tile, CTAs per SM)
must give the oracle's edge lists, and the autotuner's pick on a source large
enough to trigger it must give the same graphs as the default configuration."""
import numpy as np
import pytest

import datagen
import oracle

rp = pytest.importorskip("paper_2602_08097_gb300")
pytestmark = pytest.mark.gpu

CONFIGS = [(0, 0), (1, 0), (0, 2), (1, 3), (0, 3), (1, 2)]


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_08097_gb300 import build as b
    b.build()
    c = rp.rp_create(0)
    yield c
    rp.rp_set_tuning(c, rp.RP_TUNING_AUTO)
    rp.rp_destroy(c)


@pytest.mark.parametrize("dtype", ["u8", "f32"])
def test_every_fixed_configuration_matches_the_oracle(ctx, dtype):
    n = 2500
    X = datagen.dataset("sift" if dtype == "u8" else "deep", n)
    row_ptr, col = datagen.random_graph(n, 0, 160, seed=11, dup_frac=0.02, self_frac=0.01)
    g = rp.rp_load_graph(ctx, X, row_ptr, col)
    clean_rp, clean_col = rp.rp_graph_export(ctx, g)
    targets = [(1.15, 64), (1.05, 24), (1.0, rp.RP_R_INF)]
    refs = {t: oracle.rp_tune(X, clean_rp, clean_col, *t) for t in targets}
    try:
        for tile0, ctas in CONFIGS:
            rp.rp_set_tuning(ctx, rp.RP_TUNING_FIXED, tile0, ctas)
            outs = rp.rp_tune_batch(ctx, g, [a for a, _ in targets], [r for _, r in targets])
            st = rp.rp_stats(ctx)
            assert (st["tile0"], st["ctas_per_sm"]) == (tile0, ctas)
            for t, o in zip(targets, outs):
                got = rp.rp_graph_export(ctx, o)
                assert np.array_equal(got[0], refs[t][0]) and np.array_equal(got[1], refs[t][1]), (dtype, tile0, ctas, t)
                rp.rp_graph_free(ctx, o)
    finally:
        rp.rp_set_tuning(ctx, rp.RP_TUNING_AUTO)
    rp.rp_graph_free(ctx, g)


def test_autotuned_configuration_gives_the_default_graphs(ctx):
    n = 80_000  # more than the 65,536 degree <= 64 nodes that trigger trials
    X = datagen.dataset("sift", n)
    data = rp.rp_load_graph(ctx, X)
    base = rp.rp_build_knn_base(ctx, data, 64, 1.2, 48)
    alphas, Rs = [1.1, 1.0], [48, 24]
    rp.rp_set_tuning(ctx, rp.RP_TUNING_FIXED, 0, 0)
    ref = [rp.rp_graph_export(ctx, g) for g in rp.rp_tune_batch(ctx, base, alphas, Rs)]
    rp.rp_set_tuning(ctx, rp.RP_TUNING_AUTO)
    for rep in range(2):  # the second call reuses the choice (and replays the captured launch)
        outs = rp.rp_tune_batch(ctx, base, alphas, Rs)
        st = rp.rp_stats(ctx)
        assert (st["tile0"], st["ctas_per_sm"]) in CONFIGS
        for o, r in zip(outs, ref):
            got = rp.rp_graph_export(ctx, o)
            assert np.array_equal(got[0], r[0]) and np.array_equal(got[1], r[1])
            rp.rp_graph_free(ctx, o)
    # a sampled node against the oracle, from the vectors alone
    node = np.array([12345], dtype=np.int64)
    base_row = oracle.knn_base(X, 64, 1.2, 48, nodes=node)[0]
    b_rp, b_col = rp.rp_graph_export(ctx, base)
    assert b_col[b_rp[12345]:b_rp[12346]].tolist() == base_row.tolist()
    with pytest.raises(rp.RPError):
        rp.rp_set_tuning(ctx, rp.RP_TUNING_FIXED, 2, 0)
    with pytest.raises(rp.RPError):
        rp.rp_set_tuning(ctx, 7, 0, 0)
    rp.rp_graph_free(ctx, base)
    rp.rp_graph_free(ctx, data)
