"""Fuzzy simplicial-set graph of the k-NN graph (oracle side).

The paper times the construction of UMAP's fuzzy simplicial-set graph
(Section 3, the MLX vs PyTorch/MPS study) and cites UMAP (McInnes et al. 2018)
for it without printing the construction.  The construction followed here, in FP64:

1. rho_i = distance from i to its nearest neighbour.
2. sigma_i solves  sum_{j in kNN(i)} exp(-max(0, d_ij - rho_i) / sigma) = log2 k
   by bisection: lo = 0, hi = +inf, sigma = 1; each of 64 steps compares the
   sum with the target, moves hi (sum too large) or lo, then doubles sigma
   while hi is unbounded, else takes the midpoint.  Afterwards sigma_i is
   floored at 1e-3 * mean_j d_ij.
3. Directed membership w_{j|i} = exp(-max(0, d_ij - rho_i) / sigma_i)
   (exactly 1 where d_ij = rho_i).
4. Fuzzy union over both directions:
   w_ij = w_{j|i} + w_{i|j} - w_{j|i} w_{i|j}  (a missing direction counts 0).
5. Both (i, j) and (j, i) are stored, sorted by (head, tail).  Schedule word
   q_e = round(2^24 * w_e / w_max).  An entry is dropped when it would fire in
   none of the T epochs, i.e. when T * q_e < 2^24 (the integer form of
   "w / w_max < 1 / T").
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

Q_ONE = 1 << 24


def smooth_knn(dist: np.ndarray, k: int | None = None, n_iter: int = 64,
               min_scale: float = 1e-3):
    """(rho, sigma) per row of a (n x k) ascending Euclidean distance matrix."""
    dist = np.asarray(dist, dtype=np.float64)
    n, kk = dist.shape
    k = kk if k is None else k
    target = np.log2(k)
    rho = dist[:, 0].copy()
    excess = np.maximum(0.0, dist - rho[:, None])
    lo = np.zeros(n)
    hi = np.full(n, np.inf)
    mid = np.ones(n)
    for _ in range(n_iter):
        psum = np.exp(-excess / mid[:, None]).sum(axis=1)
        above = psum > target
        hi = np.where(above, mid, hi)
        lo = np.where(above, lo, mid)
        mid = np.where(np.isinf(hi), mid * 2.0, 0.5 * (lo + hi))
    sigma = np.maximum(mid, min_scale * dist.mean(axis=1))
    return rho, sigma


def directed_weights(dist: np.ndarray, rho: np.ndarray, sigma: np.ndarray) -> np.ndarray:
    dist = np.asarray(dist, dtype=np.float64)
    excess = dist - rho[:, None]
    with np.errstate(divide="ignore", invalid="ignore"):
        w = np.exp(-excess / sigma[:, None])
    return np.where(excess > 0.0, w, 1.0)


def union_matrix(idx: np.ndarray, w_dir: np.ndarray, n: int) -> sp.csr_matrix:
    """Symmetric FP64 sparse matrix of fuzzy-union weights."""
    k = idx.shape[1]
    heads = np.repeat(np.arange(n), k)
    P = sp.csr_matrix((np.asarray(w_dir, np.float64).ravel(), (heads, np.asarray(idx).ravel())),
                      shape=(n, n))
    S = (P + P.T - P.multiply(P.T)).tocsr()
    S.sum_duplicates()
    S.sort_indices()
    return S


def schedule_words(w: np.ndarray, w_max: float):
    """Unrounded and rounded (round half to even) schedule words 2^24 w / w_max."""
    q_exact = Q_ONE * (np.asarray(w, np.float64) / w_max)
    return q_exact, np.rint(q_exact).astype(np.uint64)


def build_csr(idx: np.ndarray, dist: np.ndarray, n_epochs: int, k: int | None = None):
    """Full graph construction: returns a dict of CSR arrays and diagnostics.

    Keys: row_ptr (int64 n+1), col (int64), w (FP64), q (uint64), q_exact
    (FP64, before rounding), rho, sigma, w_dir (n x k), w_max.
    """
    idx = np.asarray(idx, dtype=np.int64)
    n = idx.shape[0]
    rho, sigma = smooth_knn(dist, k)
    w_dir = directed_weights(dist, rho, sigma)
    S = union_matrix(idx, w_dir, n)
    w_max = float(S.data.max())
    q_exact, q = schedule_words(S.data, w_max)
    keep = (np.uint64(n_epochs) * q) >= np.uint64(Q_ONE)
    heads = np.repeat(np.arange(n), np.diff(S.indptr))
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(row_ptr, heads[keep] + 1, 1)
    row_ptr = np.cumsum(row_ptr)
    return dict(row_ptr=row_ptr, col=S.indices[keep].astype(np.int64), w=S.data[keep],
                q=q[keep], q_exact=q_exact[keep], rho=rho, sigma=sigma, w_dir=w_dir,
                w_max=w_max, union=S)
