"""The seeded input generators that both the oracle and the CUDA path consume
(datagen): deterministic, of the documented shapes and types, with the value
recipes stated (sift ~8% zeros from rint(min(255, Gamma(0.6, 40))); gist and
deep rows of unit norm, gist's nonnegative), prefixes across a chunk boundary
for the single-distribution sets, and queries drawn apart from the base."""
import numpy as np
import pytest

import datagen


@pytest.mark.parametrize("name,d,dtype", [("tiny", 32, np.float32), ("sift", 128, np.uint8),
                                          ("gist", 960, np.float32), ("deep", 96, np.float32)])
def test_shapes_types_and_determinism(name, d, dtype):
    a = datagen.dataset(name, 300)
    b = datagen.dataset(name, 300)
    assert a.shape == (300, d) and a.dtype == dtype
    assert np.array_equal(a, b)
    q = datagen.queries(name, 20)
    assert q.shape == (20, d) and q.dtype == dtype and np.array_equal(q, datagen.queries(name, 20))
    assert not np.array_equal(q, a[:20])


def test_sift_values():
    X = datagen.dataset("sift", 20000)
    zeros = float(np.mean(X == 0))
    # P(rint(G) = 0) = P(G < 0.5) for G ~ Gamma(0.6, 40): 0.0807
    assert 0.075 < zeros < 0.087
    assert X.max() == 255  # the clip at 255 is reached


@pytest.mark.parametrize("name", ["gist", "deep"])
def test_unit_rows(name):
    X = datagen.dataset(name, 2000).astype(np.float64)
    np.testing.assert_allclose(np.linalg.norm(X, axis=1), 1.0, rtol=0, atol=1e-6)
    if name == "gist":
        assert X.min() >= 0.0


def test_prefix_across_a_chunk_boundary():
    big = datagen.dataset("sift", datagen.CHUNK + 100)
    assert np.array_equal(datagen.dataset("sift", 1000), big[:1000])
    assert np.array_equal(datagen.dataset("sift", datagen.CHUNK + 7), big[:datagen.CHUNK + 7])


def _lid_mle(X, nq=200, k=20):
    # Levina-Bickel maximum-likelihood estimate of the local intrinsic
    # dimension from k nearest neighbours, median over the first nq rows
    Q = X[:nq]
    d2 = np.einsum("ij,ij->i", Q, Q)[:, None] + np.einsum("ij,ij->i", X, X)[None, :] - 2.0 * Q @ X.T
    d2[np.arange(nq), np.arange(nq)] = np.inf  # not its own neighbour
    r = np.sqrt(np.maximum(np.sort(np.partition(d2, k, axis=1)[:, :k], axis=1), 1e-300))
    return float(np.median(-1.0 / np.mean(np.log(r[:, :-1] / r[:, -1:]), axis=1)))


def test_deep_intrinsic_dimension_is_low():
    # The deep mixture's components spread like PCA outputs (s_i = 1.5 i^-0.75),
    # so its local intrinsic dimension sits far below d = 96, and far below that
    # of isotropic components (sigma 0.5) around centres drawn the same way.
    n = 20000
    X = datagen.dataset("deep", n).astype(np.float64)
    rng = np.random.default_rng(5)
    Y = rng.normal(0.0, 1.0, (256, 96))[rng.integers(0, 256, n)] + 0.5 * rng.normal(0.0, 1.0, (n, 96))
    Y /= np.linalg.norm(Y, axis=1, keepdims=True)
    lx, ly = _lid_mle(X), _lid_mle(Y)
    assert 4.0 < lx < 12.0 and ly > 20.0 and lx < 0.5 * ly
