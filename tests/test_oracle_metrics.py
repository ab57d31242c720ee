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


# ---------------------------------------------------------------- held-out recall
def _brute_heldout(Xt, Yt, Xn, Yn, k, rows):
    """Python loops over (squared distance, index) pairs in both spaces."""
    hits = 0
    for r in rows:
        dx = sorted((float(((Xt[j] - Xn[r]) ** 2).sum()), j) for j in range(len(Xt)))
        dy = sorted((float(((Yt[j] - Yn[r]) ** 2).sum()), j) for j in range(len(Yt)))
        hits += len({j for _, j in dx[:k]} & {j for _, j in dy[:k]})
    return hits / (k * len(rows))


def test_heldout_recall_matches_brute_force():
    g = np.random.default_rng(11)
    Xt, Xn = g.normal(size=(120, 6)), g.normal(size=(40, 6))
    # a lossy 2-D view: the first two coordinates plus noise
    Yt = Xt[:, :2] + 0.3 * g.normal(size=(120, 2))
    Yn = Xn[:, :2] + 0.3 * g.normal(size=(40, 2))
    for k, nq in [(5, 0), (10, 13)]:
        rows = metrics.strided_rows(40, nq)
        want = _brute_heldout(Xt, Yt, Xn, Yn, k, rows)
        assert metrics.heldout_recall(Xt, Yt, Xn, Yn, k, nq) == pytest.approx(want, abs=1e-12)
        assert 0.0 < want < 1.0


def test_heldout_recall_of_an_isometry_is_one():
    g = np.random.default_rng(12)
    Xt, Xn = g.normal(size=(500, 2)), g.normal(size=(100, 2))
    c, s_ = np.cos(0.7), np.sin(0.7)
    Rm = 3.0 * np.array([[c, -s_], [s_, c]])
    shift = np.array([5.0, -2.0])
    assert metrics.heldout_recall(Xt, Xt @ Rm + shift, Xn, Xn @ Rm + shift, 15) == 1.0


def test_heldout_recall_uses_the_training_points_as_reference():
    # the new points' neighbours are taken among the training points: a new
    # embedding that is right but a training embedding that is shuffled
    # scores near chance (k / n_train)
    g = np.random.default_rng(13)
    Xt, Xn = g.normal(size=(2000, 2)), g.normal(size=(300, 2))
    Yt = Xt[g.permutation(2000)]
    r = metrics.heldout_recall(Xt, Yt, Xn, Xn, 15)
    assert r < 5 * 15 / 2000


def test_strided_rows():
    assert list(metrics.strided_rows(10, 4)) == [0, 2, 5, 7]
    assert list(metrics.strided_rows(5, 0)) == [0, 1, 2, 3, 4]
    assert list(metrics.strided_rows(5, 9)) == [0, 1, 2, 3, 4]
