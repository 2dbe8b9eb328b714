"""The error bound of the float Gram tier, measured on the tensor cores.

The prune kernel forms every float Gram entry from the candidate rows centred
on the node's pivot, y = x - p (an f32 subtraction per value), scaled by a
power of two and split into f16 hi and lo (y' = scale y = hi + 2^-11 lo), as
hi hi^T + 2^-11 (hi lo^T + lo hi^T) accumulated in f32 by tcgen05 MMAs, and
trusts
    |G~ - <y_u, y_v>| <= eps_ip |y_u| |y_v| + 2^-36 sqrt(d) (|y_u| + |y_v|) / scale,
    eps_ip = 5 2^-22 + 2^-23 + d 2^-22,
where the d 2^-22 term is four times the f32 accumulation bound for one
summation order: an allowance for whatever order the tensor core sums in,
and one 2^-22 covers the subtractions.  tests/test_ff_bound.py checks the
bound against an emulation of one order; this test reads the entries the
kernel's own operand stores, MMA sequence and combination produce
(rp_debug_gram) for more than a million pairs of deep-shaped (d = 96) and
gist-shaped (d = 960) rows, raw and centred on pivots (each 64-row half on its
own pivot, the rows drawn near it as a node's candidates are), and holds each
against the exact inner product of the f64 differences."""
import math

import numpy as np
import pytest

import datagen

rp = pytest.importorskip("paper_2602_08097_gb300")
pytestmark = pytest.mark.gpu


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


def _near_rows(X, centres, rng):
    # 64 rows per pivot drawn among its 256 nearest points, as a node's candidates are
    out = []
    for c in centres:
        d2 = np.einsum("ij,ij->i", X - X[c], X - X[c])
        near = np.argpartition(d2, 257)[:257]
        near = near[near != c][:256]
        out.append(rng.choice(near, 64, replace=False))
    return np.concatenate(out).astype(np.int32)


@pytest.mark.parametrize("centred", [False, True])
@pytest.mark.parametrize("name,n,nrows", [("deep", 200_000, 8064), ("gist", 20_000, 8064), ("tiny", 2000, 1920)])
def test_split_gram_within_its_bound(ctx, name, n, nrows, centred):
    X = datagen.dataset(name, n)
    g = rp.rp_load_graph(ctx, X)
    rng = np.random.default_rng(nrows)
    centres = None
    if centred:
        centres = rng.choice(n, nrows // 64, replace=False).astype(np.int32)
        rows = _near_rows(X, centres, rng)
    else:
        rows = rng.choice(n, nrows, replace=False).astype(np.int32)
    got = rp.rp_debug_gram(ctx, g, rows, centres).astype(np.float64)
    rp.rp_graph_free(ctx, g)
    d = X.shape[1]
    mx = float(np.max(np.abs(X)))
    e = math.frexp(mx)[1]  # mx < 2^e: the library's power-of-two scale is 2^-e
    scale = math.ldexp(1.0, -e) * (0.5 if centred else 1.0)  # centred rows: half of it
    eps_ip = 5 * 2.0**-22 + 2.0**-23 + d * 2.0**-22
    worst = 0.0
    pairs = 0
    for gi in range(nrows // 128):
        R = X[rows[gi * 128:(gi + 1) * 128]].astype(np.float64)
        if centred:
            R[:64] -= X[centres[2 * gi]]
            R[64:] -= X[centres[2 * gi + 1]]
        exact = R @ R.T  # float64 products of float32 values: error far below the bound
        nrm = np.sqrt(np.einsum("ij,ij->i", R, R))
        bound = eps_ip * np.outer(nrm, nrm) + 2.0**-36 * math.sqrt(d) * (nrm[:, None] + nrm[None, :]) / scale
        bound += 1e-12 * np.outer(nrm, nrm)  # the float64 reference's own rounding
        err = np.abs(got[gi] - exact)
        assert np.all(err <= bound), f"{name}: group {gi}, worst {float(np.max(err / bound)):.3f} of the bound"
        worst = max(worst, float(np.max(err / bound)))
        pairs += 128 * 128
    assert pairs >= (1_000_000 if name != "tiny" else 200_000)
    print(f"{name}{' centred' if centred else ''}: {pairs} pairs, largest error {worst:.4f} of the bound")
