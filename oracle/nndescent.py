"""NNDescent approximate k-NN graph (oracle side, FP64).

Test infrastructure: imported only by tests, the smoke check and the bench's
CPU baseline, never by the product path.

The paper (Section 2.2) builds its k-NN graph by NNDescent (Dong et al.
2011): every point starts with k random neighbours, the graph is refined by
exploring neighbours of neighbours, the k nearest candidates are kept by a
top-k selection, and the loop ends early once the update rate falls below
delta = 0.015.  It does not spell out the candidate set, the random draw or
the update rate, so this restatement fixes them (the same readings bind the
CUDA path):

* start: point i draws words from Philox4x32-10 with key = (seed lo, seed
  hi) at counters (i, r, 0, 5), r = 0, 1, ..., 15, the four words of each
  counter in order; a word u proposes m = floor(u n / 2^32), accepted when
  m != i and m is not yet in the list, until k are accepted.  If the 64
  words do not give k (only possible when k is close to n - 1), the list is
  completed by the smallest indices not yet in it.
* one iteration (synchronous: every list read is the previous iteration's):
  the candidates of i are C(i) = G(i) united with G(j) for every j in G(i),
  without i; the new G(i) is the k candidates with the smallest (squared
  distance, index), in that order.
* with reverse = True (the basic algorithm of Dong et al., which Section 2.2
  cites: the join runs over each point's general neighbours, its own list
  and the points whose lists hold it): R(i) = up to k of the points j with i
  in G(j), the k with the smallest (squared distance, j); B(i) = G(i) united
  with R(i); C(i) = B(i) united with B(u) for every u in B(i), without i.
* updates u_t = sum_i |G_{t+1}(i) minus G_t(i)| (new neighbours entering the
  lists); rate_t = u_t / (n k).  The loop stops after the first iteration
  whose rate is below delta, or after max_iter iterations.
* output: the lists in (distance, index) order, Euclidean distances.
"""
from __future__ import annotations

import numpy as np

from . import philox

TAG_NND = 5
WORDS = 64          # Philox words a point may use for its random start
DELTA = 0.015       # the paper's early-termination update rate
MAX_ITER = 30


def init_graph(n: int, k: int, seed: int) -> np.ndarray:
    """The random start: int64 n x k, point i's k distinct random neighbours."""
    if k < 1 or n < k + 1:
        raise ValueError("need 1 <= k <= n - 1")
    k0, k1 = philox.split_seed(seed)
    rows = np.arange(n, dtype=np.uint64)[:, None]
    ctr = np.arange(WORDS // 4, dtype=np.uint64)[None, :]
    w = philox.philox4x32(rows, ctr, 0, TAG_NND, k0, k1)
    words = np.stack(w, axis=2).reshape(n, WORDS)          # counter r, then word 0..3
    prop = philox.negative_index(words, n)                  # floor(u n / 2^32)
    G = np.empty((n, k), dtype=np.int64)
    for i in range(n):
        taken: list[int] = []
        for m in prop[i]:
            if len(taken) == k:
                break
            m = int(m)
            if m != i and m not in taken:
                taken.append(m)
        c = 0
        while len(taken) < k:
            if c != i and c not in taken:
                taken.append(c)
            c += 1
        G[i] = taken
    return G


def reverse_lists(G: np.ndarray, d2: np.ndarray, k: int) -> np.ndarray:
    """R(i) for every i (int64 n x k, -1 where fewer): the points j whose list
    G(j) holds i, the k with the smallest (d2 of that entry, j)."""
    n, kk = G.shape
    owner = np.repeat(np.arange(n), kk)
    tgt = G.ravel()
    order = np.lexsort((owner, d2.ravel(), tgt))       # by target, then distance, then owner
    tgt_s, own_s = tgt[order], owner[order]
    lo = np.searchsorted(tgt_s, np.arange(n), side="left")
    hi = np.searchsorted(tgt_s, np.arange(n), side="right")
    R = np.full((n, k), -1, dtype=np.int64)
    for i in range(n):
        m = min(k, hi[i] - lo[i])
        R[i, :m] = own_s[lo[i]:lo[i] + m]
    return R


def candidates(G: np.ndarray, i: int) -> np.ndarray:
    """C(i): G(i) and the lists of its members, without i, as a sorted set."""
    c = np.unique(np.concatenate([G[i], G[G[i]].ravel()]))
    return c[c != i]


def iterate(X, G: np.ndarray, reverse: bool = False):
    """One synchronous iteration: (new lists, their squared distances, updates)."""
    X64 = np.asarray(X, dtype=np.float64)
    n, k = G.shape
    new = np.empty_like(G)
    new_d2 = np.empty((n, k))
    updates = 0
    if reverse:
        R = reverse_lists(G, ((X64[G] - X64[:, None, :]) ** 2).sum(axis=2), k)
        B = [np.unique(np.concatenate([G[i], R[i][R[i] >= 0]])) for i in range(n)]
    for i in range(n):
        if reverse:
            c = np.unique(np.concatenate([B[i]] + [B[u] for u in B[i]]))
            c = c[c != i]
        else:
            c = candidates(G, i)
        d2 = ((X64[c] - X64[i]) ** 2).sum(axis=1)
        order = np.lexsort((c, d2))[:k]
        new[i] = c[order]
        new_d2[i] = d2[order]
        updates += np.setdiff1d(new[i], G[i], assume_unique=True).size
    return new, new_d2, updates


def nndescent(X, k: int, seed: int, delta: float = DELTA, max_iter: int = MAX_ITER, G0=None,
              reverse: bool = False):
    """(idx n x k, Euclidean dist n x k, iterations run, rate of each iteration).

    G0 replaces the random start when given (for tests)."""
    X64 = np.asarray(X, dtype=np.float64)
    n = X64.shape[0]
    G = init_graph(n, k, seed) if G0 is None else np.asarray(G0, dtype=np.int64)
    rates: list[float] = []
    d2 = None
    for _ in range(max_iter):
        G, d2, u = iterate(X64, G, reverse)
        rates.append(u / (n * k))
        if rates[-1] < delta:
            break
    return G, np.sqrt(d2), len(rates), rates


__all__ = ["init_graph", "reverse_lists", "candidates", "iterate", "nndescent", "TAG_NND", "DELTA", "MAX_ITER"]
