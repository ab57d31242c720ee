"""Philox4x32-10 counter-based generator (oracle side).

Written from the published description of the Philox family (J. Salmon,
M. Moraes, R. Dror, D. Shaw, "Parallel random numbers: as easy as 1, 2, 3",
SC'11, Section 3.3 / Table 2): a 4-word counter is passed through R rounds of
two multiply-high/low S-boxes and a word permutation, the key is bumped by the
Weyl constants between rounds.  The same construction with 64-bit words and
the 64-bit constants is Philox4x64-10, which ``philox_generic`` also covers so
that the round structure can be checked against numpy's Philox bit generator.

How the method consumes it:

* negative sample j' of CSR entry e at epoch t (a stream keyed by seed,
  epoch, edge and sample number): key = (seed lo, seed hi), counter
  = (e, t, j' // 4, 0), word j' % 4 -> u; the sampled point is (u * n) >> 32.
* initial coordinates of point i: key = (seed lo, seed hi), counter =
  (i, 0, 0, 1); words 0 and 1 give x and y.
* the random start of NNDescent: counters (i, r, 0, 5), r = 0..15
  (``nndescent.init_graph``).
"""
from __future__ import annotations

import numpy as np

M4x32 = (0xD2511F53, 0xCD9E8D57)
W4x32 = (0x9E3779B9, 0xBB67AE85)
M4x64 = (0xD2E7470EE14C6C93, 0xCA5A826395121157)
W4x64 = (0x9E3779B97F4A7C15, 0xBB67AE8584CAA73B)

TAG_NEGATIVE = 0
TAG_INIT = 1
TAG_MLP = 2


def philox_generic(ctr, key, width: int = 32, rounds: int = 10):
    """One Philox4xW block with Python integers (W = 32 or 64)."""
    mask = (1 << width) - 1
    M0, M1 = M4x32 if width == 32 else M4x64
    W0, W1 = W4x32 if width == 32 else W4x64
    c0, c1, c2, c3 = (int(v) & mask for v in ctr)
    k0, k1 = (int(v) & mask for v in key)
    for r in range(rounds):
        if r:
            k0 = (k0 + W0) & mask
            k1 = (k1 + W1) & mask
        p0 = M0 * c0
        p1 = M1 * c2
        hi0, lo0 = p0 >> width, p0 & mask
        hi1, lo1 = p1 >> width, p1 & mask
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def philox4x32(c0, c1, c2, c3, k0, k1, rounds: int = 10):
    """Vectorised Philox4x32-10; all arguments broadcast, values < 2^32.

    Products of two 32-bit words are formed exactly in uint64.
    Returns four uint64 arrays holding 32-bit words.
    """
    mask = np.uint64(0xFFFFFFFF)
    s32 = np.uint64(32)
    c0, c1, c2, c3 = (np.asarray(v, dtype=np.uint64) & mask for v in (c0, c1, c2, c3))
    c0, c1, c2, c3 = np.broadcast_arrays(c0, c1, c2, c3)
    k0 = np.uint64(int(k0) & 0xFFFFFFFF)
    k1 = np.uint64(int(k1) & 0xFFFFFFFF)
    M0, M1 = np.uint64(M4x32[0]), np.uint64(M4x32[1])
    W0, W1 = np.uint64(W4x32[0]), np.uint64(W4x32[1])
    for r in range(rounds):
        if r:
            k0 = (k0 + W0) & mask
            k1 = (k1 + W1) & mask
        p0 = M0 * c0
        p1 = M1 * c2
        c0, c1, c2, c3 = ((p1 >> s32) ^ c1 ^ k0, p1 & mask, (p0 >> s32) ^ c3 ^ k1, p0 & mask)
    return c0, c1, c2, c3


def split_seed(seed: int):
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return seed & 0xFFFFFFFF, seed >> 32


def negative_words(e, t: int, neg: int, seed: int) -> np.ndarray:
    """uint64 array (len(e), neg) of the 32-bit words drawn for negatives."""
    e = np.asarray(e, dtype=np.uint64)
    k0, k1 = split_seed(seed)
    out = np.empty((e.shape[0], neg), dtype=np.uint64)
    for blk in range((neg + 3) // 4):
        words = philox4x32(e, np.uint64(t), np.uint64(blk), np.uint64(TAG_NEGATIVE), k0, k1)
        for w in range(4):
            jj = 4 * blk + w
            if jj < neg:
                out[:, jj] = words[w]
    return out


def negative_index(u: np.ndarray, n: int) -> np.ndarray:
    """Multiply-shift map of a 32-bit word onto [0, n): floor(u * n / 2^32)."""
    return ((u.astype(np.uint64) * np.uint64(n)) >> np.uint64(32)).astype(np.int64)
