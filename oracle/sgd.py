"""Initialisation, synchronous SGD epoch and full fit (oracle side, FP64).

The paper's UMAP optimiser (Section 2.5, its SGD step; Section 3, 500
epochs, negative-sample rate, gradient expression; Section 4.1, scatter-add on
sampled edges) follows UMAP.  Its per-epoch step, as restated here:

With d = |Y_i - Y_j|^2 (squared distance) and the fitted a, b:

* attraction along an active CSR entry e = (i, j):
      c_att = -2 a b d^(b-1) / (1 + a d^b)        (0 when d = 0)
      g    += clip(c_att (Y_i - Y_j), -4, 4)
  which is -grad_{Y_i} of log(1 + a d^b) = -log Phi(d).
* for each of ``neg`` negatives m of that entry (m = i contributes nothing):
      c_rep = 2 b / ((eps + d) (1 + a d^b)),  eps = 0.001
      g    += clip(c_rep (Y_i - Y_m), -4, 4)
  which, for eps = 0, is -grad_{Y_i} of -log(1 - Phi(d)).
* Y'_i = Y_i + lr * g_i for every row i, all gradients taken at Y^(t)
  (synchronous update; only the head i of an entry moves, and the symmetric
  CSR holds both (i, j) and (j, i)).

Schedule: entry e with schedule word q_e (2^24 fixed point) is active at
epoch t iff floor((t+1) q_e / 2^24) > floor(t q_e / 2^24), so it fires
floor(T q_e / 2^24) times in T epochs.  Negative j' of entry e at epoch t is
floor(u n / 2^32) with u = word (j' mod 4) of Philox4x32-10 at counter
(e, t, j' div 4, 0).  Learning rate lr_t = lr0 (1 - t / T).
"""
from __future__ import annotations

import numpy as np

from . import philox
from .curve import find_ab
from .fuzzy import Q_ONE, build_csr
from .knn import knn

INIT_SCALE = 2.0 ** -24


def init_embedding(n: int, seed: int, init_range: float = 10.0) -> np.ndarray:
    """Y0 ~ U[-R, R]^2: words 0, 1 of Philox at counter (i, 0, 0, 1), top 24 bits.

    Returned in FP64, where u * 2R - R (u a 24-bit integer over 2^24) is
    exact; a single-precision implementation that rounds once (a fused
    multiply-add) yields exactly the FP32 rounding of this value.
    """
    k0, k1 = philox.split_seed(seed)
    w = philox.philox4x32(np.arange(n, dtype=np.uint64), 0, 0, philox.TAG_INIT, k0, k1)
    u = np.stack([(w[0] >> np.uint64(8)).astype(np.float64),
                  (w[1] >> np.uint64(8)).astype(np.float64)], axis=1) * INIT_SCALE
    return u * (2.0 * init_range) - init_range


def active_mask(q: np.ndarray, t: int) -> np.ndarray:
    q = np.asarray(q, dtype=np.uint64)
    s = np.uint64(24)
    return ((np.uint64(t + 1) * q) >> s) > ((np.uint64(t) * q) >> s)


def _clip(v, c):
    return v if c is None else np.clip(v, -c, c)


def attraction_coeff(d, a, b):
    with np.errstate(divide="ignore", invalid="ignore"):
        c = -2.0 * a * b * np.power(d, b - 1.0) / (1.0 + a * np.power(d, b))
    return np.where(d > 0.0, c, 0.0)


def repulsion_coeff(d, a, b, eps=1e-3):
    with np.errstate(divide="ignore", invalid="ignore"):
        return 2.0 * b / ((eps + d) * (1.0 + a * np.power(d, b)))


def epoch(Y, row_ptr, col, q, a, b, lr, neg, t, seed, eps=1e-3, clip=4.0,
          return_parts=False):
    """One synchronous epoch; returns Y^(t+1) in FP64 (n x 2).

    With ``return_parts`` also returns the per-row force g (n x 2) and the
    per-row sum of |term| (n x 2), which bounds how much rounding the force can
    carry.
    """
    Y64 = np.asarray(Y, dtype=np.float64)
    n = Y64.shape[0]
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    heads = np.repeat(np.arange(n), np.diff(row_ptr))
    e_act = np.nonzero(active_mask(q, t))[0]
    i = heads[e_act]
    j = np.asarray(col, dtype=np.int64)[e_act]
    G = np.zeros((n, 2))
    A = np.zeros((n, 2))

    diff = Y64[i] - Y64[j]
    d = (diff ** 2).sum(axis=1)
    term = _clip(attraction_coeff(d, a, b)[:, None] * diff, clip)
    for c in range(2):
        G[:, c] += np.bincount(i, weights=term[:, c], minlength=n)
        A[:, c] += np.bincount(i, weights=np.abs(term[:, c]), minlength=n)

    if neg > 0 and e_act.size:
        words = philox.negative_words(e_act, t, neg, seed)
        for jj in range(neg):
            m = philox.negative_index(words[:, jj], n)
            keep = m != i
            diff = Y64[i[keep]] - Y64[m[keep]]
            d = (diff ** 2).sum(axis=1)
            term = _clip(repulsion_coeff(d, a, b, eps)[:, None] * diff, clip)
            for c in range(2):
                G[:, c] += np.bincount(i[keep], weights=term[:, c], minlength=n)
                A[:, c] += np.bincount(i[keep], weights=np.abs(term[:, c]), minlength=n)
    Y_next = Y64 + lr * G
    if return_parts:
        return Y_next, G, A
    return Y_next


def epoch_rows(Y, row_ptr, col, q, rows, a, b, lr, neg, t, seed, eps=1e-3, clip=4.0):
    """The epoch update of selected rows only (same arithmetic as ``epoch``);
    returns their new coordinates (len(rows) x 2).  For checks on large graphs
    where a full FP64 epoch is too costly."""
    Y64 = np.asarray(Y, dtype=np.float64)
    n = Y64.shape[0]
    row_ptr = np.asarray(row_ptr, np.int64)
    out = np.empty((len(rows), 2))
    for r, i in enumerate(np.asarray(rows, np.int64)):
        e = np.arange(row_ptr[i], row_ptr[i + 1])
        e = e[active_mask(np.asarray(q)[e], t)]
        g = np.zeros(2)
        if e.size:
            j = np.asarray(col, np.int64)[e]
            diff = Y64[i] - Y64[j]
            d = (diff ** 2).sum(axis=1)
            g += _clip(attraction_coeff(d, a, b)[:, None] * diff, clip).sum(axis=0)
            if neg > 0:
                words = philox.negative_words(e, t, neg, seed)
                for jj in range(neg):
                    m = philox.negative_index(words[:, jj], n)
                    keep = m != i
                    diff = Y64[i] - Y64[m[keep]]
                    d = (diff ** 2).sum(axis=1)
                    g += _clip(repulsion_coeff(d, a, b, eps)[:, None] * diff, clip).sum(axis=0)
        out[r] = Y64[i] + lr * g
    return out


def anchored_epoch(Y_train, Y_new, row_ptr, col, q, a, b, lr, neg, t, seed, eps=1e-3, clip=4.0):
    """One epoch that moves only new points: row i of the CSR is new point i,
    its entries point into the fixed training embedding, negatives are drawn
    from the training points (m = floor(u n_train / 2^32), Philox counter
    (e, t, j' div 4, 0) with e the entry index of the new points' CSR).
    Returns the new points' coordinates (FP64)."""
    Yt = np.asarray(Y_train, dtype=np.float64)
    Yn = np.asarray(Y_new, dtype=np.float64)
    n_train, n_new = Yt.shape[0], Yn.shape[0]
    heads = np.repeat(np.arange(n_new), np.diff(np.asarray(row_ptr, np.int64)))
    e_act = np.nonzero(active_mask(q, t))[0]
    i = heads[e_act]
    j = np.asarray(col, np.int64)[e_act]
    G = np.zeros((n_new, 2))
    diff = Yn[i] - Yt[j]
    d = (diff ** 2).sum(axis=1)
    term = _clip(attraction_coeff(d, a, b)[:, None] * diff, clip)
    for c in range(2):
        G[:, c] += np.bincount(i, weights=term[:, c], minlength=n_new)
    if neg > 0 and e_act.size:
        words = philox.negative_words(e_act, t, neg, seed)
        for jj in range(neg):
            m = philox.negative_index(words[:, jj], n_train)
            diff = Yn[i] - Yt[m]
            d = (diff ** 2).sum(axis=1)
            term = _clip(repulsion_coeff(d, a, b, eps)[:, None] * diff, clip)
            for c in range(2):
                G[:, c] += np.bincount(i, weights=term[:, c], minlength=n_new)
    return Yn + lr * G


def transform(X_train, Y_train, X_new, k=15, n_epochs=200, min_dist=0.1, spread=1.0, neg=5, lr0=1.0,
              seed_neg=2, ab=None):
    """New points against a fixed training embedding: exact k nearest training
    points, directed memberships (rho, sigma as in the fuzzy graph), start at
    the membership-weighted mean of the neighbours' coordinates, then
    ceil(T / 3) anchored epochs with lr0 (1 - t / T')."""
    from .fuzzy import directed_weights, smooth_knn
    from .knn import knn_query
    a, b = find_ab(spread, min_dist) if ab is None else ab
    idx, dist = knn_query(X_new, X_train, k)
    rho, sigma = smooth_knn(dist, k)
    w = directed_weights(dist, rho, sigma)
    order = np.argsort(idx, axis=1, kind="stable")
    col = np.take_along_axis(idx, order, axis=1)
    w = np.take_along_axis(w, order, axis=1)
    Yt = np.asarray(Y_train, np.float64)
    Y = (w[:, :, None] * Yt[col]).sum(axis=1) / w.sum(axis=1)[:, None]
    q = np.rint(Q_ONE * w).astype(np.uint64).ravel()
    row_ptr = np.arange(len(X_new) + 1) * k
    T3 = (n_epochs + 2) // 3
    for t in range(T3):
        Y = anchored_epoch(Yt, Y, row_ptr, col.ravel(), q, a, b, lr0 * (1.0 - t / T3), neg, t, seed_neg)
    return Y


def active_count(q, t_total: int) -> np.ndarray:
    """Times each entry fires over epochs 0..T-1: floor(T q / 2^24)."""
    return (np.uint64(t_total) * np.asarray(q, np.uint64)) >> np.uint64(24)


def fit(X, k: int = 15, n_epochs: int = 200, min_dist: float = 0.1, spread: float = 1.0,
        neg: int = 5, lr0: float = 1.0, init_range: float = 10.0, seed_init: int = 1,
        seed_neg: int = 2, graph=None, ab=None, callback=None):
    """k-NN -> fuzzy graph -> a, b -> init -> T synchronous epochs.

    Returns (Y FP64 n x 2, graph dict).  ``graph`` and ``ab`` may be passed in
    to reuse a precomputed graph or fixed kernel parameters.
    """
    X = np.asarray(X)
    n = X.shape[0]
    if graph is None:
        idx, dist = knn(X, k)
        graph = build_csr(idx, dist, n_epochs, k)
        graph["knn_idx"], graph["knn_dist"] = idx, dist
    a, b = find_ab(spread, min_dist) if ab is None else ab
    Y = init_embedding(n, seed_init, init_range)
    for t in range(n_epochs):
        lr = lr0 * (1.0 - t / n_epochs)
        Y = epoch(Y, graph["row_ptr"], graph["col"], graph["q"], a, b, lr, neg, t, seed_neg)
        if callback is not None:
            callback(t, Y)
    return Y, graph


__all__ = ["init_embedding", "active_mask", "attraction_coeff", "repulsion_coeff", "epoch",
           "epoch_rows", "anchored_epoch", "transform", "active_count", "fit", "Q_ONE"]
