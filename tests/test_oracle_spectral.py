"""Pins for the oracle's spectral initial layout (not gpu).

Closed forms: the normalised adjacency of a path graph has the eigenvectors
D^1/2 cos(pi k i / (n - 1)) with eigenvalues cos(pi k / (n - 1)) (those of the
random walk D^-1 W of a path, carried over by D^1/2); a ring's leading
non-trivial eigenspace is spanned by cos and sin of 2 pi i / n; the top
eigenvector of any connected graph is D^1/2 1 / |D^1/2 1| with eigenvalue 1.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import datagen
from oracle import fuzzy, knn as oknn, spectral


def _csr_from_edges(n, edges, weights=None):
    i = np.array([a for a, b in edges] + [b for a, b in edges])
    j = np.array([b for a, b in edges] + [a for a, b in edges])
    w = np.ones(len(i)) if weights is None else np.concatenate([weights, weights])
    W = sp.csr_matrix((w, (i, j)), shape=(n, n))
    W.sort_indices()
    return W.indptr, W.indices, W.data


def test_path_graph_closed_form():
    n = 40
    rp, col, w = _csr_from_edges(n, [(i, i + 1) for i in range(n - 1)])
    M = spectral.normalized_adjacency(rp, col, w, n)
    vals, vecs = spectral.leading_eigenvectors(M, 3)
    d = np.full(n, 2.0)
    d[0] = d[-1] = 1.0
    i = np.arange(n)
    for k in range(3):
        assert vals[k] == pytest.approx(np.cos(np.pi * k / (n - 1)), abs=1e-10)
        v = np.sqrt(d) * np.cos(np.pi * k * i / (n - 1))
        v /= np.linalg.norm(v)
        assert abs(abs(v @ vecs[:, k]) - 1.0) < 1e-9
    # the layout: v2 with its largest entry positive, scaled to max |Y| = R
    Y, _ = spectral.spectral_init(rp, col, w, n, init_range=10.0, seed=3)
    v2 = np.sqrt(d) * np.cos(np.pi * i / (n - 1))
    v2 = spectral.fix_signs(v2[:, None])[:, 0]
    v3 = spectral.fix_signs((np.sqrt(d) * np.cos(2 * np.pi * i / (n - 1)))[:, None])[:, 0]
    V = np.stack([v2 / np.linalg.norm(v2), v3 / np.linalg.norm(v3)], axis=1)
    assert np.allclose(Y, 10.0 * V / np.abs(V).max(), atol=10.0 * spectral.JITTER * 1.0001)


def test_ring_leading_eigenspace_is_cos_sin():
    n = 64
    rp, col, w = _csr_from_edges(n, [(i, (i + 1) % n) for i in range(n)])
    M = spectral.normalized_adjacency(rp, col, w, n)
    vals, vecs = spectral.leading_eigenvectors(M, 3)
    assert vals[0] == pytest.approx(1.0, abs=1e-12)
    assert vals[1] == pytest.approx(np.cos(2 * np.pi / n), abs=1e-10)
    assert vals[2] == pytest.approx(np.cos(2 * np.pi / n), abs=1e-10)
    t = 2 * np.pi * np.arange(n) / n
    B = np.stack([np.cos(t), np.sin(t)], axis=1) / np.sqrt(n / 2)
    # principal angles between span(v2, v3) and span(cos, sin) are zero
    s = np.linalg.svd(B.T @ vecs[:, 1:3], compute_uv=False)
    assert np.allclose(s, 1.0, atol=1e-9)
    # so the layout puts the ring on a circle
    Y, _ = spectral.spectral_init(rp, col, w, n, init_range=10.0)
    r = np.linalg.norm(Y - Y.mean(axis=0), axis=1)
    assert r.std() / r.mean() < 1e-3


def test_trivial_eigenvector_and_residuals_on_a_knn_graph():
    X, _ = datagen.mixture(1500, 20, 1, seed=4)          # one cluster: a connected graph
    idx, dist = oknn.knn(X, 15)
    g = fuzzy.build_csr(idx, dist, 200, 15)
    n = len(X)
    M = spectral.normalized_adjacency(g["row_ptr"], g["col"], g["w"], n)
    assert abs(M - M.T).max() < 1e-15
    vals, vecs = spectral.leading_eigenvectors(M, 3)
    W = sp.csr_matrix((g["w"], g["col"], g["row_ptr"]), shape=(n, n))
    d = np.asarray(W.sum(axis=1)).ravel()
    u1 = np.sqrt(d) / np.linalg.norm(np.sqrt(d))
    assert vals[0] == pytest.approx(1.0, abs=1e-10)
    assert abs(abs(u1 @ vecs[:, 0]) - 1.0) < 1e-9
    for k in range(3):
        r = M @ vecs[:, k] - vals[k] * vecs[:, k]
        assert np.linalg.norm(r) < 1e-8
    assert np.allclose(vecs.T @ vecs, np.eye(3), atol=1e-10)
    assert vals[1] < 1.0 - 1e-6 and vals[1] >= vals[2]


def test_sign_convention_and_jitter():
    V = np.array([[0.1, -0.5], [-0.7, 0.2], [0.7, 0.5]])
    F = spectral.fix_signs(V)
    assert np.array_equal(F[:, 0], -V[:, 0])     # |-0.7| first at index 1: made positive
    assert np.array_equal(F[:, 1], -V[:, 1])     # |-0.5| at index 0 comes before |0.5| at index 2
    assert np.array_equal(spectral.fix_signs(F), F)
    j = spectral.jitter(10_000, 7)
    assert j.min() >= -1.0 and j.max() < 1.0 and abs(j.mean()) < 0.03


def test_sparse_path_residuals_beyond_the_dense_size():
    # beyond DENSE_MAX rows the Lanczos path runs: pinned by the closed-form
    # top eigenvector, residuals and orthogonality on a connected graph
    g0 = np.random.default_rng(5)
    U = g0.uniform(0, 1, size=(spectral.DENSE_MAX + 1000, 2)) * [3.0, 1.0]
    X = np.concatenate([U, 0.01 * g0.normal(size=(len(U), 8))], axis=1)
    idx, dist = oknn.knn(X, 10)
    g = fuzzy.build_csr(idx, dist, 200, 10)
    n = len(X)
    M = spectral.normalized_adjacency(g["row_ptr"], g["col"], g["w"], n)
    vals, vecs = spectral.leading_eigenvectors(M, 3, tol=1e-10)
    W = sp.csr_matrix((g["w"], g["col"], g["row_ptr"]), shape=(n, n))
    d = np.asarray(W.sum(axis=1)).ravel()
    u1 = np.sqrt(d) / np.linalg.norm(np.sqrt(d))
    assert vals[0] == pytest.approx(1.0, abs=1e-8)
    assert abs(abs(u1 @ vecs[:, 0]) - 1.0) < 1e-7
    for k in range(3):
        assert np.linalg.norm(M @ vecs[:, k] - vals[k] * vecs[:, k]) < 1e-6
    assert np.allclose(vecs.T @ vecs, np.eye(3), atol=1e-8)
