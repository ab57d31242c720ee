"""PCA preprocessing (oracle side, FP64).

The paper's timed pipeline starts with PCA of the raw features (Section 3,
the per-method timings include it) and exposes its target width as the
pca_dim knob (Section 3.3); it does not state the decomposition, so it is
restated here:

* mu = the column means of X (n x D); Xc = X - mu.
* C = Xc^T Xc / (n - 1), the sample covariance (D x D).
* V = the eigenvectors of C for its `dim` largest eigenvalues, in decreasing
  order of eigenvalue, each signed so that its entry of largest magnitude
  (lowest index among equals) is positive.
* Z = Xc V (n x dim), the projected data.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg


def covariance(X):
    X = np.asarray(X, np.float64)
    mu = X.mean(axis=0)
    Xc = X - mu
    return mu, (Xc.T @ Xc) / (len(X) - 1)


def fix_signs(V):
    """Each column with its largest-magnitude entry (lowest index among equal
    magnitudes) positive."""
    V = np.array(V, dtype=np.float64, copy=True)
    for k in range(V.shape[1]):
        i = int(np.argmax(np.abs(V[:, k])))
        if V[i, k] < 0:
            V[:, k] = -V[:, k]
    return V


def pca(X, dim: int = 50):
    """(Z, V, mu, eigenvalues) of the `dim` leading principal components."""
    mu, C = covariance(X)
    D = C.shape[0]
    vals, vecs = scipy.linalg.eigh(C, subset_by_index=[D - dim, D - 1])
    order = np.argsort(-vals, kind="stable")
    vals, V = vals[order], fix_signs(vecs[:, order])
    Z = (np.asarray(X, np.float64) - mu) @ V
    return Z, V, mu, vals


__all__ = ["covariance", "fix_signs", "pca"]
