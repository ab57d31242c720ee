"""Spectral initialisation of the embedding (oracle side, FP64).

The UMAP optimisation the paper times starts from a spectral layout of the
fuzzy graph (the UMAP construction it cites; the paper names the method and
prints no formulas).  Restated here:

* W = the symmetric fuzzy-graph weights, as kept in the CSR (after the
  1/T pruning); d_i = sum_j W_ij.
* M = D^-1/2 W D^-1/2, the normalised adjacency (I - M is the normalised
  graph Laplacian, so the largest eigenvalues of M are the smallest of the
  Laplacian).  Its top eigenvector is D^1/2 1 / |D^1/2 1| with eigenvalue 1
  (trivial: it carries no layout).
* The layout is the next two eigenvectors v2, v3 (by decreasing eigenvalue),
  each with its sign fixed so that its entry of largest magnitude (lowest
  index among equals) is positive.
* Y0 = R [v2 v3] / max_ik |v_k(i)|  (so max |Y0| = R, the init range), plus a
  jitter of R 1e-5 (2u - 1) per coordinate, u = (Philox word >> 8) / 2^24 from
  words 2 and 3 of the initialisation stream (counter (i, 0, 0, 1), key =
  seed), so that coincident layouts do not stay coincident.

A disconnected graph has eigenvalue 1 once per component; v2 and v3 are then
some pair of vectors of that eigenspace (each component collapses towards a
segment), as in any solver that does not lay out components separately.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg
import scipy.sparse as sp
from scipy.sparse.linalg import eigsh

from . import philox

JITTER = 1e-5


def normalized_adjacency(row_ptr, col, w, n: int) -> sp.csr_matrix:
    """M = D^-1/2 W D^-1/2 of the CSR graph (rows with no entries keep 0)."""
    W = sp.csr_matrix((np.asarray(w, np.float64), np.asarray(col, np.int64), np.asarray(row_ptr, np.int64)),
                      shape=(n, n))
    d = np.asarray(W.sum(axis=1)).ravel()
    s = np.zeros(n)
    s[d > 0] = 1.0 / np.sqrt(d[d > 0])
    return (sp.diags(s) @ W @ sp.diags(s)).tocsr()


def fix_signs(V: np.ndarray) -> np.ndarray:
    """Each column with its largest-magnitude entry (lowest index among equal
    magnitudes) positive."""
    V = np.array(V, dtype=np.float64, copy=True)
    for k in range(V.shape[1]):
        i = int(np.argmax(np.abs(V[:, k])))   # first index of the maximum
        if V[i, k] < 0:
            V[:, k] = -V[:, k]
    return V


DENSE_MAX = 8000


def leading_eigenvectors(M: sp.csr_matrix, count: int = 3, tol: float = 1e-12):
    """The `count` largest eigenvalues of M (decreasing) and their unit
    eigenvectors (columns).  Up to DENSE_MAX rows a dense symmetric
    eigensolver, which resolves repeated eigenvalues; beyond, Lanczos
    (ARPACK), which may miss the second copy of an exactly repeated one."""
    n = M.shape[0]
    if n <= DENSE_MAX:
        vals, vecs = scipy.linalg.eigh(M.toarray(), subset_by_index=[n - count, n - 1])
    else:
        # a seeded Gaussian start: a symmetric one (all ones, say) has no
        # component along eigenvectors of a symmetric graph that are odd
        v0 = np.random.default_rng(0).standard_normal(n)
        vals, vecs = eigsh(M, k=count, which="LA", tol=tol, v0=v0)
    order = np.argsort(-vals, kind="stable")
    return vals[order], vecs[:, order]


def jitter(n: int, seed: int) -> np.ndarray:
    """Uniform values in [-1, 1) (n x 2) from words 2, 3 of the
    initialisation stream."""
    k0, k1 = philox.split_seed(seed)
    w = philox.philox4x32(np.arange(n, dtype=np.uint64), 0, 0, philox.TAG_INIT, k0, k1)
    u = np.stack([(w[2] >> np.uint64(8)).astype(np.float64),
                  (w[3] >> np.uint64(8)).astype(np.float64)], axis=1) * 2.0 ** -24
    return 2.0 * u - 1.0


def spectral_init(row_ptr, col, w, n: int, init_range: float = 10.0, seed: int = 1):
    """Y0 (n x 2, FP64) from the spectral layout (module docstring); also
    returns the three leading eigenvalues."""
    M = normalized_adjacency(row_ptr, col, w, n)
    vals, vecs = leading_eigenvectors(M, 3)
    V = fix_signs(vecs[:, 1:3])
    Y = init_range * V / np.abs(V).max()
    return Y + init_range * JITTER * jitter(n, seed), vals


__all__ = ["normalized_adjacency", "fix_signs", "leading_eigenvectors", "jitter", "spectral_init", "JITTER"]
