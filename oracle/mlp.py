"""Learned parametric embedder (oracle side, FP64).

An MLP d -> h -> h -> 2 (h = 256 for the product; any h here) with exact-erf
GELU, trained on the UMAP cross-entropy of edges of the fuzzy graph.  This is
a project addition: the paper has no learned embedder.  The loss of one edge
(i, j) with negatives m_1..m_neg, on embedded points z:

    L = -log Phi(|z_i - z_j|^2) - sum_t log(1 - Phi(|z_i - z_m_t|^2)),
    Phi(d) = 1 / (1 + a d^b), clamped to [1e-4, 1 - 1e-4] (zero gradient
    where the clamp is active); negatives equal to the head are skipped;
    the batch loss is the mean over edges.

Parameter vector layout (FP32 in the CUDA path, FP64 here):
W1 [h][64] (input columns >= d are zero), b1 [h], W2 [h][h], b2 [h],
W3 [2][h], b3 [2]; weights (out, in) row-major.

``emulate=True`` rounds to BF16 (round to nearest even, from FP32) at the
points where the CUDA path stores BF16: the gathered inputs, the weights
(W3 is used as its BF16-rounded value), both hidden activations, and the
back-propagated pre-activation gradients that enter the weight-gradient and
input-gradient products; bias gradients use the unrounded values.  Sums are
FP64 here and FP32 on the GPU.

Edge sampling (``sample``): for slot s, Philox4x32-10 with key = seed at
counter (step, s, try, 2) gives words (u0, u1); entry e = (u0 * nnz) >> 32 is
accepted when (u1 >> 8) < q_e (so edges are drawn proportional to the
schedule words q = round(2^24 w)); at most 64 tries, the last one is kept.
Negative t of slot s is (u * n) >> 32 with u = word (t mod 4) at counter
(step, s, 64 + t div 4, 2).
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf

from . import philox

IN = 64
OUT = 2
PHI_LO, PHI_HI = 1e-4, 1.0 - 1e-4


def param_count(h: int = 256) -> int:
    return h * IN + h + h * h + h + OUT * h + OUT


def unpack(P: np.ndarray, h: int = 256):
    P = np.asarray(P, dtype=np.float64)
    o = 0
    W1 = P[o:o + h * IN].reshape(h, IN); o += h * IN
    b1 = P[o:o + h]; o += h
    W2 = P[o:o + h * h].reshape(h, h); o += h * h
    b2 = P[o:o + h]; o += h
    W3 = P[o:o + OUT * h].reshape(OUT, h); o += OUT * h
    b3 = P[o:o + OUT]
    return W1, b1, W2, b2, W3, b3


def pack(parts) -> np.ndarray:
    return np.concatenate([np.asarray(p, np.float64).ravel() for p in parts])


def bf16(x) -> np.ndarray:
    """Round to BF16 (nearest even) from FP32; returned as FP64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + np.uint64(0x7FFF) + ((u >> np.uint64(16)) & np.uint64(1))) & np.uint64(0xFFFF0000)
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def gelu(x):
    return 0.5 * x * (1.0 + erf(x / np.sqrt(2.0)))


def gelu_grad(x):
    return 0.5 * (1.0 + erf(x / np.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / np.sqrt(2.0 * np.pi)


def _r(x, emulate):
    return bf16(x) if emulate else np.asarray(x, np.float64)


def forward(P, X, rows, d, h=256, emulate=True):
    """Cache of the forward pass for the given rows of X (FP64)."""
    W1, b1, W2, b2, W3, b3 = unpack(P, h)
    Xr = np.zeros((len(rows), IN))
    Xr[:, :d] = np.asarray(X, np.float64)[np.asarray(rows)]
    Xb = _r(Xr, emulate)
    W1b, W2b, W3b = _r(W1, emulate), _r(W2, emulate), _r(W3, emulate)
    pre1 = Xb @ W1b.T + b1
    H1 = _r(gelu(pre1), emulate)
    pre2 = H1 @ W2b.T + b2
    H2 = _r(gelu(pre2), emulate)
    z = H2 @ W3b.T + b3
    return dict(Xb=Xb, W1b=W1b, W2b=W2b, W3b=W3b, pre1=pre1, H1=H1, pre2=pre2, H2=H2, z=z)


def loss_and_dz(z, rows, n_edges, neg, a, b):
    """Mean batch loss and its gradient with respect to z (rows of 2 + neg)."""
    R = 2 + neg
    z = np.asarray(z, np.float64)
    rows = np.asarray(rows)
    dz = np.zeros_like(z)
    L = 0.0
    for s in range(n_edges):
        i = s * R
        for t in range(1, R):
            r = i + t
            if t >= 2 and rows[r] == rows[i]:
                continue
            diff = z[i] - z[r]
            dd = float(diff @ diff)
            adb = a * dd ** b if dd > 0 else 0.0
            phi = 1.0 / (1.0 + adb)
            inside = PHI_LO < phi < PHI_HI
            pc = min(max(phi, PHI_LO), PHI_HI)
            if t == 1:
                L -= np.log(pc)
                dLdd = b * adb / (dd * (1.0 + adb)) if inside else 0.0
            else:
                L -= np.log(1.0 - pc)
                dLdd = -b / (dd * (1.0 + adb)) if inside else 0.0
            g = dLdd * 2.0 * diff / n_edges
            dz[i] += g
            dz[r] -= g
    return L / n_edges, dz


def backward(cache, dz, h=256, emulate=True):
    """Gradient of the batch loss with respect to the parameter vector."""
    dpre2 = (dz @ cache["W3b"]) * gelu_grad(cache["pre2"])
    D2 = _r(dpre2, emulate)
    dW3 = dz.T @ cache["H2"]
    db3 = dz.sum(axis=0)
    db2 = dpre2.sum(axis=0)
    dW2 = D2.T @ cache["H1"]
    dpre1 = (D2 @ cache["W2b"]) * gelu_grad(cache["pre1"])
    D1 = _r(dpre1, emulate)
    db1 = dpre1.sum(axis=0)
    dW1 = D1.T @ cache["Xb"]
    return pack([dW1, db1, dW2, db2, dW3, db3])


def grad(P, X, rows, d, n_edges, neg, a, b, h=256, emulate=True):
    """(loss, gradient vector) of one batch with explicit rows."""
    cache = forward(P, X, rows, d, h, emulate)
    L, dz = loss_and_dz(cache["z"], rows, n_edges, neg, a, b)
    return L, backward(cache, dz, h, emulate)


def sample(row_ptr, col, q, n, n_edges, neg, step, seed):
    """Rows (int64, n_edges * (2 + neg)) of one sampled batch."""
    R = 2 + neg
    k0, k1 = philox.split_seed(seed)
    row_ptr = np.asarray(row_ptr, np.int64)
    col = np.asarray(col, np.int64)
    q = np.asarray(q, np.uint64)
    nnz = len(col)
    out = np.empty(n_edges * R, dtype=np.int64)
    for s in range(n_edges):
        e = 0
        for r in range(64):
            u = philox.philox_generic((step, s, r, philox.TAG_MLP), (k0, k1), 32)
            e = (u[0] * nnz) >> 32
            if (u[1] >> 8) < int(q[e]):
                break
        head = int(np.searchsorted(row_ptr, e, side="right") - 1)
        out[s * R] = head
        out[s * R + 1] = col[e]
        for t in range(neg):
            u = philox.philox_generic((step, s, 64 + t // 4, philox.TAG_MLP), (k0, k1), 32)
            out[s * R + 2 + t] = (u[t % 4] * n) >> 32
    return out


def adam_step(P, m, v, g, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (t counts from 1); returns new (P, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    P = P - lr * (m / (1 - b1 ** t)) / (np.sqrt(v / (1 - b2 ** t)) + eps)
    return P, m, v


def embed(P, X, d, h=256, emulate=True):
    return forward(P, X, np.arange(len(X)), d, h, emulate)["z"]
