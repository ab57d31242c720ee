"""Exact k-nearest neighbours in FP64 (oracle side).

Definition followed: for each query point i, the k other points j (self
excluded) with the smallest squared Euclidean distance sum_c (x_ic - x_jc)^2,
ordered lexicographically by (distance, index), lower index first on ties.
Distances are returned as Euclidean distances (square roots).

Section 2.2 of the paper computes distances with the expansion
|a|^2 + |b|^2 - 2 a.b on the GPU.  Here that expansion (FP64 matrix product)
only shortlists k + 16 candidates per row; their squared distances are then
recomputed directly, and a row whose shortlist cannot be proven to contain the
true k nearest (the shortlist margin is smaller than the expansion's rounding
bound, e.g. many duplicate points) is recomputed directly over all points.
"""
from __future__ import annotations

import numpy as np

_EPS64 = 2.0 ** -52


def _direct_row(X64: np.ndarray, i: int, k: int):
    dd = ((X64 - X64[i]) ** 2).sum(axis=1)
    dd[i] = np.inf
    order = np.lexsort((np.arange(X64.shape[0]), dd))[:k]
    return order, dd[order]


def knn_rows(X: np.ndarray, rows: np.ndarray, k: int, margin: int = 16,
             q_chunk: int = 512, db_chunk: int = 1 << 20):
    """Exact k-NN of the given rows of X against all of X (self excluded).

    Returns (idx int64 len(rows) x k, dist FP64 Euclidean len(rows) x k).
    """
    X64 = np.asarray(X, dtype=np.float64)
    n, d = X64.shape
    rows = np.asarray(rows, dtype=np.int64)
    if k < 1 or k > n - 1:
        raise ValueError("k must satisfy 1 <= k <= n - 1")
    m = min(n - 1, k + margin)
    sq = (X64 ** 2).sum(axis=1)
    sq_max = float(sq.max())
    out_idx = np.empty((rows.size, k), dtype=np.int64)
    out_d2 = np.empty((rows.size, k), dtype=np.float64)
    for s in range(0, rows.size, q_chunk):
        r = rows[s:s + q_chunk]
        Q = X64[r]
        best_d = np.full((r.size, 0), np.inf)
        best_j = np.empty((r.size, 0), dtype=np.int64)
        for b0 in range(0, n, db_chunk):
            B = X64[b0:b0 + db_chunk]
            D = sq[r, None] + sq[None, b0:b0 + B.shape[0]] - 2.0 * (Q @ B.T)
            inblk = (r >= b0) & (r < b0 + B.shape[0])
            D[np.nonzero(inblk)[0], r[inblk] - b0] = np.inf
            mm = min(m, B.shape[0])
            part = np.argpartition(D, mm - 1, axis=1)[:, :mm] if mm < B.shape[0] else \
                np.broadcast_to(np.arange(B.shape[0]), D.shape)
            cand_d = np.take_along_axis(D, part, axis=1)
            best_d = np.concatenate([best_d, cand_d], axis=1)
            best_j = np.concatenate([best_j, part + b0], axis=1)
            if best_d.shape[1] > m:
                sel = np.argpartition(best_d, m - 1, axis=1)[:, :m]
                best_d = np.take_along_axis(best_d, sel, axis=1)
                best_j = np.take_along_axis(best_j, sel, axis=1)
        # direct recomputation of the shortlisted squared distances
        dd = ((X64[best_j] - Q[:, None, :]) ** 2).sum(axis=2)
        dd[best_j == r[:, None]] = np.inf
        order = np.lexsort((best_j, dd), axis=1)[:, :k]
        sel_j = np.take_along_axis(best_j, order, axis=1)
        sel_d = np.take_along_axis(dd, order, axis=1)
        # certificate: every point outside the shortlist has an expansion value
        # >= the largest shortlisted one; the expansion is within `bound` of the
        # true squared distance.
        if m < n - 1:
            bound = 8.0 * (d + 2) * _EPS64 * 2.0 * (sq[r] + sq_max)
            worst_in = best_d.max(axis=1)
            ok = (worst_in - bound) > sel_d[:, -1]
        else:
            ok = np.ones(r.size, dtype=bool)
        for t in np.nonzero(~ok)[0]:
            sel_j[t], sel_d[t] = _direct_row(X64, int(r[t]), k)
        out_idx[s:s + r.size] = sel_j
        out_d2[s:s + r.size] = sel_d
    return out_idx, np.sqrt(out_d2)


def knn(X: np.ndarray, k: int, **kw):
    """Exact k-NN graph of all points: (idx int64 n x k, dist FP64 n x k)."""
    return knn_rows(X, np.arange(np.asarray(X).shape[0]), k, **kw)


def sq_dist_rows(X: np.ndarray, rows: np.ndarray, cols: np.ndarray) -> np.ndarray:
    """Direct FP64 squared distances between X[rows[a]] and X[cols[a, b]]."""
    X64 = np.asarray(X, dtype=np.float64)
    return ((X64[cols] - X64[rows][:, None, :]) ** 2).sum(axis=2)


def knn_query(Q: np.ndarray, X: np.ndarray, k: int, chunk: int = 256):
    """Exact k nearest rows of X for each row of Q (no self exclusion): the
    FP64 expansion shortlists k + 16 candidates, whose squared distances are
    recomputed directly; (distance, index) order.  Returns (idx, dist)."""
    Q64 = np.asarray(Q, dtype=np.float64)
    X64 = np.asarray(X, dtype=np.float64)
    n = X64.shape[0]
    m = min(n, k + 16)
    sqx = (X64 ** 2).sum(axis=1)
    out_i = np.empty((len(Q64), k), dtype=np.int64)
    out_d = np.empty((len(Q64), k))
    for s in range(0, len(Q64), chunk):
        q = Q64[s:s + chunk]
        D = (q ** 2).sum(axis=1)[:, None] + sqx[None, :] - 2.0 * (q @ X64.T)
        cand = np.argpartition(D, m - 1, axis=1)[:, :m] if m < n else np.broadcast_to(np.arange(n), D.shape)
        dd = ((X64[cand] - q[:, None, :]) ** 2).sum(axis=2)
        order = np.lexsort((cand, dd), axis=1)[:, :k]
        out_i[s:s + len(q)] = np.take_along_axis(cand, order, axis=1)
        out_d[s:s + len(q)] = np.sqrt(np.take_along_axis(dd, order, axis=1))
    return out_i, out_d
