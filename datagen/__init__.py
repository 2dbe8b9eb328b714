"""Seeded synthetic inputs shaped like the paper's workloads (§4.1 Setup).

The paper evaluates on SIFT-1M, GIST-1M, Deep-1M and MSSPACEV-1M (§4.1,
"Datasets").  None of those files exist here, so every workload is drawn from a
seeded ``numpy.random.Generator(PCG64(seed))`` with the same shape, element
type and a value distribution of the same kind:

=====  ==========================================================  =========
name   recipe                                                       seeds
=====  ==========================================================  =========
tiny   n=2,000, d=32, f32; 16 centres ~ N(0, 4 I), x = c_z + N(0,I)  1000/2000
sift   n=1,000,000, d=128, u8 = rint(min(255, Gamma(0.6, 40)))       1001/2001
gist   n=1,000,000, d=960, f32 = |N(0,1)| * 0.05, rows L2-normalised 1002/2002
deep   n=10,000,000, d=96, f32; 256 centres ~ N(0, I), component     1003/2003
       covariance diag(s_i^2) with s_i = 1.5 i^-0.75 (i = 1 .. 96),
       rows unit-normalised in f64 then cast to f32
=====  ==========================================================  =========

Deep's 96 values are PCA outputs of network embeddings: their variance falls
off with the component index and the local intrinsic dimension is far below
96.  The deep mixture's components have that shape (a maximum-likelihood
estimate of the intrinsic dimension from 20 nearest neighbours is about 15);
an isotropic component of the same dimension (about 38 by that estimate)
would make every graph index far harder to search than the data it stands
for.

Rows are drawn in fixed chunks of ``CHUNK`` rows so that a prefix of ``n`` rows
is the same whatever total is asked for; a smaller ``n`` therefore gives the
first ``n`` points of the full-size set.  Queries come from a second generator
(seed 2000 + config index) and reuse the base set's mixture centres.

This module holds none of the pruning or search arithmetic: it only draws
numbers and assembles arrays.  Both the CUDA path (through its tests and the
benchmark) and the CPU oracle consume what it returns.
"""
from __future__ import annotations

import numpy as np

CHUNK = 65536

# Config index -> (dtype, d, n_full, n_queries)
CONFIGS = {
    "tiny": dict(index=0, dtype="f32", d=32, n=2000, nq=200),
    "sift": dict(index=1, dtype="u8", d=128, n=1_000_000, nq=10_000),
    "gist": dict(index=2, dtype="f32", d=960, n=1_000_000, nq=1_000),
    "deep": dict(index=3, dtype="f32", d=96, n=10_000_000, nq=10_000),
}

# deep: per-dimension standard deviation of a mixture component, 1.5 i^-0.75
DEEP_SPREAD = 1.5 * np.arange(1, 97, dtype=np.float64) ** -0.75


def _gen(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _unit_rows_f32(x64: np.ndarray) -> np.ndarray:
    nrm = np.sqrt(np.einsum("ij,ij->i", x64, x64))
    nrm[nrm == 0.0] = 1.0
    return (x64 / nrm[:, None]).astype(np.float32)


def _tiny_centres(rng: np.random.Generator) -> np.ndarray:
    return rng.normal(0.0, 2.0, size=(16, 32))


def _deep_centres(rng: np.random.Generator, d: int) -> np.ndarray:
    return rng.normal(0.0, 1.0, size=(256, d))


def _rows(name: str, n: int, rng: np.random.Generator, centres) -> np.ndarray:
    cfg = CONFIGS[name]
    d = cfg["d"]
    out = np.empty((n, d), dtype=np.uint8 if cfg["dtype"] == "u8" else np.float32)
    for lo in range(0, n, CHUNK):
        hi = min(n, lo + CHUNK)
        b = hi - lo
        if name == "tiny":
            z = rng.integers(0, 16, size=b)
            out[lo:hi] = (centres[z] + rng.normal(0.0, 1.0, size=(b, d))).astype(np.float32)
        elif name == "sift":
            g = rng.gamma(0.6, 40.0, size=(b, d))
            out[lo:hi] = np.rint(np.minimum(255.0, g)).astype(np.uint8)
        elif name == "gist":
            g = np.abs(rng.normal(0.0, 1.0, size=(b, d))) * 0.05
            out[lo:hi] = _unit_rows_f32(g)
        elif name == "deep":
            z = rng.integers(0, 256, size=b)
            g = centres[z] + rng.normal(0.0, 1.0, size=(b, d)) * DEEP_SPREAD
            out[lo:hi] = _unit_rows_f32(g)
        else:
            raise KeyError(name)
    return out


def dataset(name: str, n: int | None = None) -> np.ndarray:
    """First ``n`` base vectors of workload ``name`` (all of them if ``n`` is None)."""
    cfg = CONFIGS[name]
    n = cfg["n"] if n is None else int(n)
    rng = _gen(1000 + cfg["index"])
    centres = None
    if name == "tiny":
        centres = _tiny_centres(rng)
    elif name == "deep":
        centres = _deep_centres(rng, cfg["d"])
    return _rows(name, n, rng, centres)


def queries(name: str, nq: int | None = None) -> np.ndarray:
    """First ``nq`` query vectors of workload ``name``, drawn from the base set's mixture."""
    cfg = CONFIGS[name]
    nq = cfg["nq"] if nq is None else int(nq)
    centres = None
    if name in ("tiny", "deep"):
        base_rng = _gen(1000 + cfg["index"])
        centres = _tiny_centres(base_rng) if name == "tiny" else _deep_centres(base_rng, cfg["d"])
    return _rows(name, nq, _gen(2000 + cfg["index"]), centres)


def random_graph(n: int, deg_lo: int, deg_hi: int, seed: int,
                 dup_frac: float = 0.0, self_frac: float = 0.0):
    """A random directed graph in CSR form (row_ptr int64[n+1], col int32[nnz]).

    Out-degrees are uniform on [deg_lo, deg_hi].  A fraction ``dup_frac`` of the
    entries repeat an earlier entry of the same row and ``self_frac`` of them
    are self loops, so that loaders can be tested on unclean input.
    """
    rng = _gen(seed)
    deg = rng.integers(deg_lo, deg_hi + 1, size=n)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(deg, out=row_ptr[1:])
    col = rng.integers(0, max(n, 1), size=int(row_ptr[-1])).astype(np.int32)
    if n > 0 and (dup_frac > 0 or self_frac > 0):
        u = rng.random(col.shape[0])
        for p in range(n):
            a, b = row_ptr[p], row_ptr[p + 1]
            for e in range(a, b):
                if u[e] < self_frac:
                    col[e] = p
                elif u[e] < self_frac + dup_frac and e > a:
                    col[e] = col[a + rng.integers(0, e - a)]
    return row_ptr, col


def poisson_stream(n_requests: int, rate_per_s: float, seed: int = 3004,
                   prune_frac: float = 0.10):
    """Arrival stream for the serving workload: Poisson arrivals, a mix of
    prune-to-(alpha, R) jobs and ragged query batches.

    Returns a list of dicts ordered by arrival time.  alpha ~ U[1.0, 1.2]
    rounded to 0.001, R ~ U{32, 48, 64}; query batches have 2^U{0..10} queries,
    L ~ U{64, 80, ..., 256}, k = 100, addressed to a resident graph slot drawn
    uniformly from the slots that exist at arrival.
    """
    rng = _gen(seed)
    t = 0.0
    out = []
    for i in range(n_requests):
        t += rng.exponential(1.0 / rate_per_s)
        if rng.random() < prune_frac:
            alpha = round(float(rng.uniform(1.0, 1.2)), 3)
            R = int(rng.choice([32, 48, 64]))
            out.append(dict(kind="tune", t=t, alpha=alpha, R=R, id=i))
        else:
            nq = int(2 ** rng.integers(0, 11))
            L = int(rng.choice(np.arange(64, 257, 16)))
            out.append(dict(kind="search", t=t, nq=nq, L=L, k=100,
                            slot_u=float(rng.random()), qseed=int(rng.integers(0, 2**31)), id=i))
    return out
