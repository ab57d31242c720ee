"""Embedding-quality metrics (oracle side, FP64).

Section 3.2 of the paper reports k-NN preservation (the fraction of the k
high-dimensional neighbours that are also among the k nearest in 2-D) and
trustworthiness (Venna & Kaski 2006), computed from exact distances.

* recall(i) = |N_X(i) & N_Y(i)| / k, averaged over the (sampled) rows.
* trustworthiness T(k) = 1 - 2 / (m k (2n - 3k - 1)) * sum_i sum_{j in
  N_Y(i) \\ N_X(i)} (r_X(i, j) - k), with r_X(i, j) the rank (1 = nearest,
  self excluded, ties by index) of j among i's neighbours in X, and m the
  number of rows summed (m = n for the full metric; a seeded row sample
  otherwise).
* held-out recall (for embeddings of new points, which the paper does not
  evaluate; the k-NN-preservation measure above carried over to points
  outside the training set): for a new point p with 2-D position y_p,
  |N_X(p) & N_Y(p)| / k, where N_X(p) are the k nearest training points to
  x_p in the input space and N_Y(p) the k nearest training points to y_p in
  the method's own 2-D embedding of the training set; averaged over the
  evenly strided new points i_r = floor(r n_new / m).
"""
from __future__ import annotations

import numpy as np
from scipy.spatial import cKDTree

from .knn import knn_query, knn_rows


def knn_2d(Y: np.ndarray, k: int, rows=None, brute_max: int = 4096):
    """Exact k-NN in the 2-D embedding, self excluded, ties by index."""
    Y64 = np.asarray(Y, dtype=np.float64)
    n = Y64.shape[0]
    rows = np.arange(n) if rows is None else np.asarray(rows, dtype=np.int64)
    if n <= brute_max:
        return knn_rows(Y64, rows, k)[0]
    tree = cKDTree(Y64)
    extra = 8
    dd, jj = tree.query(Y64[rows], k=k + extra)
    out = np.empty((rows.size, k), dtype=np.int64)
    for t in range(rows.size):
        # re-sort the kd-tree's shortlist by (distance, index), drop self
        j = jj[t]
        d2 = ((Y64[j] - Y64[rows[t]]) ** 2).sum(axis=1)
        d2[j == rows[t]] = np.inf
        o = np.lexsort((j, d2))
        if not d2[o[k - 1]] < d2[o[-1]]:  # shortlist boundary tie: brute row
            out[t] = knn_rows(Y64, rows[t:t + 1], k)[0][0]
        else:
            out[t] = j[o[:k]]
    return out


def recall(nx: np.ndarray, ny: np.ndarray) -> float:
    """Mean |N_X(i) & N_Y(i)| / k over rows, from two (m x k) index arrays."""
    k = nx.shape[1]
    hits = sum(np.intersect1d(a, b, assume_unique=True).size for a, b in zip(nx, ny))
    return hits / (k * nx.shape[0])


def trustworthiness(X: np.ndarray, ny: np.ndarray, rows=None, n_total: int | None = None,
                    chunk: int = 32) -> float:
    """Trustworthiness from X and the 2-D neighbour lists ``ny`` of ``rows``.

    Ranks r_X(i, j) are counts of points strictly closer to i than j (ties
    broken by index), plus one, from FP64 expansion distances.
    """
    X64 = np.asarray(X, dtype=np.float64)
    n = X64.shape[0] if n_total is None else n_total
    rows = np.arange(X64.shape[0]) if rows is None else np.asarray(rows, dtype=np.int64)
    k = ny.shape[1]
    sq = (X64 ** 2).sum(axis=1)
    total = 0.0
    ar = np.arange(X64.shape[0])
    for s in range(0, rows.size, chunk):
        r = rows[s:s + chunk]
        D = sq[r, None] + sq[None, :] - 2.0 * (X64[r] @ X64.T)
        D[np.arange(r.size), r] = np.inf
        nyc = np.asarray(ny[s:s + r.size])
        dj = np.take_along_axis(D, nyc, axis=1)                      # (c, k)
        less = (D[:, None, :] < dj[:, :, None]).sum(axis=2)
        ties = ((D[:, None, :] == dj[:, :, None]) & (ar[None, None, :] < nyc[:, :, None])).sum(axis=2)
        rank = less + ties + 1
        total += float(np.where(rank > k, rank - k, 0).sum())
    m = rows.size
    return 1.0 - 2.0 / (m * k * (2.0 * n - 3.0 * k - 1.0)) * total


def quality(X, Y, k: int = 15, rows=None, knn_x=None):
    """(recall, trustworthiness) of embedding Y of X on the given rows."""
    X = np.asarray(X)
    rows = np.arange(X.shape[0]) if rows is None else np.asarray(rows)
    nx = knn_rows(X, rows, k)[0] if knn_x is None else knn_x
    ny = knn_2d(Y, k, rows)
    return recall(nx, ny), trustworthiness(X, ny, rows)


def strided_rows(n: int, m: int) -> np.ndarray:
    """The m evenly strided rows floor(r n / m), r = 0 .. m-1 (all rows when
    m <= 0 or m >= n)."""
    if m <= 0 or m >= n:
        return np.arange(n)
    return (np.arange(m, dtype=np.int64) * n) // m


def heldout_recall(X_train, Y_train, X_new, Y_new, k: int = 15, n_query: int = 0) -> float:
    """Held-out k-NN preservation of new points against the training set
    (module docstring): exact neighbour sets in both spaces, ties by index."""
    rows = strided_rows(len(X_new), n_query)
    nx = knn_query(np.asarray(X_new)[rows], X_train, k)[0]
    ny = knn_query(np.asarray(Y_new)[rows], Y_train, k)[0]
    return recall(nx, ny)
