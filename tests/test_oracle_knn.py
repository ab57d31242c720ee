"""Pins for the oracle's exact k-NN (not gpu)."""
import itertools

import numpy as np
import pytest

import datagen
from oracle import knn as oknn


def brute_loops(X, k):
    """Tiny-n brute force with Python loops and a plain sort."""
    X = np.asarray(X, np.float64)
    n = len(X)
    out = []
    for i in range(n):
        cand = []
        for j in range(n):
            if j != i:
                cand.append((sum((X[i, c] - X[j, c]) ** 2 for c in range(X.shape[1])), j))
        cand.sort()
        out.append([j for _, j in cand[:k]])
    return np.array(out)


def test_matches_python_loops_tiny():
    X = np.random.default_rng(1).normal(size=(25, 4))
    idx, dist = oknn.knn(X, 6)
    assert np.array_equal(idx, brute_loops(X, 6))


@pytest.mark.parametrize("n,d,k", [(500, 50, 15), (1200, 3, 15), (300, 100, 7)])
def test_matches_sklearn_brute(n, d, k):
    NearestNeighbors = pytest.importorskip("sklearn.neighbors").NearestNeighbors
    X, _ = datagen.mixture(n, d, 10, seed=n)
    idx, dist = oknn.knn(X, k)
    nn = NearestNeighbors(n_neighbors=k + 1, algorithm="brute").fit(X.astype(np.float64))
    sd, si = nn.kneighbors(X.astype(np.float64))
    # drop self (always at distance 0 for distinct points)
    assert np.all(si[:, 0] == np.arange(n))
    np.testing.assert_allclose(dist, sd[:, 1:], rtol=1e-9, atol=1e-9)
    mism = idx != si[:, 1:]
    # any disagreement must be a distance tie
    assert np.allclose(dist[mism], sd[:, 1:][mism])


def test_duplicate_points_tie_by_index():
    g = np.random.default_rng(3)
    base = g.normal(size=(40, 8))
    X = np.concatenate([base, base[:10], base[:10]])  # points 40..59 duplicate 0..9
    idx, dist = oknn.knn(X, 5, margin=1)  # tiny shortlist forces the certificate path
    assert np.array_equal(idx, brute_loops(X, 5))
    # point 0 has duplicates 40 and 50 at distance 0, in index order
    assert list(idx[0, :2]) == [40, 50]
    assert dist[0, 0] == 0.0 and dist[0, 1] == 0.0


def test_knn_rows_with_database_chunks():
    X, _ = datagen.mixture(3000, 16, 5, seed=9)
    rows = np.array([0, 17, 2999, 1500])
    i1, d1 = oknn.knn_rows(X, rows, 15, db_chunk=700, q_chunk=3)
    i2, d2 = oknn.knn(X, 15)
    assert np.array_equal(i1, i2[rows])
    np.testing.assert_array_equal(d1, d2[rows])


def test_rejects_k_too_large():
    with pytest.raises(ValueError):
        oknn.knn(np.zeros((5, 2)), 5)
