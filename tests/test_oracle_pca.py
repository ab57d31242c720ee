"""Pins for the oracle's PCA (not gpu)."""
import numpy as np
import pytest

from oracle import pca


def test_covariance_by_loops():
    g = np.random.default_rng(1)
    X = g.normal(size=(30, 5)) * [1, 2, 3, 4, 5] + 7.0
    mu, C = pca.covariance(X)
    for a in range(5):
        assert mu[a] == pytest.approx(sum(X[i, a] for i in range(30)) / 30)
        for b in range(5):
            want = sum((X[i, a] - mu[a]) * (X[i, b] - mu[b]) for i in range(30)) / 29
            assert C[a, b] == pytest.approx(want, rel=1e-12, abs=1e-12)
    assert np.allclose(C, np.cov(X, rowvar=False), rtol=1e-12)


def test_known_axes_and_variances():
    # independent coordinates with variances 9, 4, 1 along known orthonormal
    # axes: the components are those axes, the eigenvalues those variances
    g = np.random.default_rng(2)
    n = 200_000
    Q, _ = np.linalg.qr(g.normal(size=(6, 6)))
    S = g.normal(size=(n, 6)) * [3.0, 2.0, 1.0, 0.1, 0.1, 0.1]
    X = S @ Q.T + 5.0
    Z, V, mu, vals = pca.pca(X, 3)
    assert np.allclose(vals, [9.0, 4.0, 1.0], rtol=2e-2)
    for k in range(3):
        assert abs(abs(V[:, k] @ Q[:, k]) - 1.0) < 1e-3
    assert np.allclose(mu, 5.0, atol=2e-2)
    # the projection is the data in the component basis: its covariance is diag(vals)
    assert np.allclose(np.cov(Z, rowvar=False), np.diag(vals), atol=1e-8 * vals.max() + 1e-10)


def test_components_are_orthonormal_eigenvectors_with_signs():
    g = np.random.default_rng(3)
    X = g.normal(size=(500, 12)) @ g.normal(size=(12, 12))
    Z, V, mu, vals = pca.pca(X, 5)
    _, C = pca.covariance(X)
    assert np.allclose(V.T @ V, np.eye(5), atol=1e-12)
    assert np.all(np.diff(vals) <= 0)
    for k in range(5):
        assert np.linalg.norm(C @ V[:, k] - vals[k] * V[:, k]) < 1e-9 * vals[0]
        i = int(np.argmax(np.abs(V[:, k])))
        assert V[i, k] > 0
    assert np.allclose(Z, (X - mu) @ V)


def test_matches_the_svd_of_the_centred_data():
    # an independent route: Xc = U S W^T gives eigenvalues S^2 / (n - 1) and
    # components W, each up to its sign
    g = np.random.default_rng(4)
    X = g.normal(size=(400, 9)) @ g.normal(size=(9, 9)) + 3.0
    Z, V, mu, vals = pca.pca(X, 4)
    U, S, Wt = np.linalg.svd(X - X.mean(axis=0), full_matrices=False)
    assert np.allclose(vals, S[:4] ** 2 / (len(X) - 1), rtol=1e-10)
    for k in range(4):
        assert abs(abs(V[:, k] @ Wt[k]) - 1.0) < 1e-10
        assert np.allclose(np.abs(Z[:, k]), np.abs(U[:, k] * S[k]), atol=1e-9 * S[0])


def test_sign_rule_takes_the_lowest_index_among_equal_magnitudes():
    V = np.array([[-0.5, 0.6], [0.5, -0.6], [0.5, 0.2], [0.5, 0.1]])
    F = pca.fix_signs(V)
    assert np.array_equal(F[:, 0], -V[:, 0])   # |v| ties at 0.5: row 0 decides, and it is negative
    assert np.array_equal(F[:, 1], V[:, 1])    # |v| ties at 0.6: row 0 decides, and it is positive
