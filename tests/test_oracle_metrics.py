"""Pins for the oracle's quality metrics (not gpu)."""
import numpy as np
import pytest

import datagen
from oracle import knn as oknn, metrics


@pytest.mark.parametrize("k", [5, 15])
def test_trustworthiness_matches_sklearn(k):
    sk_trust = pytest.importorskip("sklearn.manifold").trustworthiness
    X, _ = datagen.mixture(400, 20, 4, seed=1)
    Y = np.random.default_rng(2).normal(size=(400, 2)) + X[:, :2]
    ny = metrics.knn_2d(Y, k)
    ours = metrics.trustworthiness(X, ny)
    ref = sk_trust(X.astype(np.float64), Y, n_neighbors=k)
    assert ours == pytest.approx(ref, abs=1e-12)


def test_identity_embedding_is_perfect():
    X = np.random.default_rng(0).normal(size=(300, 2))
    nx = oknn.knn(X, 10)[0]
    ny = metrics.knn_2d(X, 10)
    assert metrics.recall(nx, ny) == 1.0
    assert metrics.trustworthiness(X, ny) == 1.0


def test_random_embedding_recall_near_chance():
    X, _ = datagen.mixture(2000, 50, 10, seed=3)
    Y = np.random.default_rng(4).normal(size=(2000, 2))
    r = metrics.recall(oknn.knn(X, 15)[0], metrics.knn_2d(Y, 15))
    assert r < 5 * 15 / 2000


def test_kdtree_path_matches_brute():
    Y = np.random.default_rng(8).normal(size=(6000, 2))
    rows = np.arange(0, 6000, 13)
    a = metrics.knn_2d(Y, 15, rows)                 # kd-tree shortlist
    b = oknn.knn_rows(Y, rows, 15)[0]               # brute force
    assert np.array_equal(a, b)


def test_sampled_trust_equals_full_on_all_rows():
    X, _ = datagen.mixture(300, 10, 3, seed=5)
    Y = np.random.default_rng(6).normal(size=(300, 2))
    ny = metrics.knn_2d(Y, 7)
    full = metrics.trustworthiness(X, ny)
    part = metrics.trustworthiness(X, ny, rows=np.arange(300))
    assert full == part
