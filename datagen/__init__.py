"""Seeded synthetic inputs for the neighbour-embedding workloads.

This module is shared by the CUDA path's tests and benchmark and by the CPU
oracle.  It holds no arithmetic of the embedding method itself: it only draws
input point clouds (and the PCA projection that turns the synthetic images into
50-d vectors, which is preprocessing of the input, not a step of the method).

The paper measures on Fashion-MNIST 70K x 784 (Section 3), MNIST, CIFAR-10 and
GloVe-Twitter subsamples up to 10M points (Section 3.3, Figure 3, Table 5).
None of those datasets is available, so the generators below stand in for them
with the same shapes and sizes:

* ``mixture``        n points in d dims from isotropic Gaussians with centres
                     N(0, 5^2 I) and unit within-cluster sigma, label i mod c.
* ``blob_images``    28x28 uint8 "images": 10 class prototypes, each a sum of
                     3-6 smooth Gaussian blobs (width 2-6 px) scaled to
                     [0, 255], plus N(0, 25^2) pixel noise, clipped and rounded.
* ``pca_basis``      centring + top-50 eigenvectors of the FP64 covariance.
* ``aniso_mixture``  100 anisotropic Gaussians, covariance Q diag(L) Q^T with Q
                     Haar-orthogonal and L ~ U[0.2, 2]; a chunked torch version
                     draws 10M points directly on a CUDA device.
* ``batched``        256 instances with n_b = floor(exp(U[ln 1e3, ln 5e4])),
                     5-20 isotropic clusters each, concatenated with offsets.

Every generator is a pure function of its seed.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "mixture",
    "blob_prototypes",
    "blob_images",
    "pca_basis",
    "pca_project",
    "images_config",
    "images_heldout",
    "aniso_params",
    "aniso_mixture",
    "aniso_mixture_torch",
    "batched",
    "batched_sizes",
    "config_small",
    "config_70k",
]


def _rng(seed: int, stream: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64([int(seed) & 0xFFFFFFFF, stream]))


def mixture(n: int, d: int = 50, n_clusters: int = 10, seed: int = 0,
            center_scale: float = 5.0, sigma: float = 1.0):
    """Isotropic Gaussian mixture; returns (X float32 n x d, labels int32)."""
    g = _rng(seed, 1)
    centres = g.normal(0.0, center_scale, size=(n_clusters, d))
    labels = (np.arange(n) % n_clusters).astype(np.int32)
    X = centres[labels] + g.normal(0.0, sigma, size=(n, d))
    return X.astype(np.float32), labels


def blob_prototypes(seed: int = 0, n_classes: int = 10, side: int = 28) -> np.ndarray:
    """Class prototypes: each a sum of 3-6 Gaussian blobs, scaled to [0, 255]."""
    g = _rng(seed, 2)
    yy, xx = np.mgrid[0:side, 0:side].astype(np.float64)
    protos = np.zeros((n_classes, side, side))
    for c in range(n_classes):
        for _ in range(int(g.integers(3, 7))):
            cy, cx = g.uniform(3.0, side - 4.0, size=2)
            width = g.uniform(2.0, 6.0)
            amp = g.uniform(0.3, 1.0)
            protos[c] += amp * np.exp(-((yy - cy) ** 2 + (xx - cx) ** 2) / (2.0 * width ** 2))
        protos[c] *= 255.0 / protos[c].max()
    return protos.reshape(n_classes, side * side)


def blob_images(n: int, seed: int = 0, stream: int = 3, noise: float = 25.0,
                start: int = 0):
    """n noisy prototype images (uint8 n x 784) and labels (i mod 10).

    ``stream`` selects an independent noise stream over the same prototypes
    (3 = training set, 4 = held-out set); ``start`` offsets the labels so that
    chunks of one stream can be drawn separately.
    """
    protos = blob_prototypes(seed)
    g = _rng(seed, stream * 1_000_003 + start)
    labels = ((np.arange(n) + start) % protos.shape[0]).astype(np.int32)
    img = protos[labels] + g.normal(0.0, noise, size=(n, protos.shape[1]))
    return np.clip(np.rint(img), 0, 255).astype(np.uint8), labels


def pca_basis(images: np.ndarray, dim: int = 50):
    """Mean (FP64) and top-``dim`` principal axes (784 x dim, FP64) of the images.

    The covariance is formed and diagonalised in FP64; each axis is signed so
    that its largest-magnitude entry is positive, which makes the basis a pure
    function of the data.
    """
    Z = images.astype(np.float64)
    mean = Z.mean(axis=0)
    Z -= mean
    cov = (Z.T @ Z) / max(1, Z.shape[0] - 1)
    evals, evecs = np.linalg.eigh(cov)
    order = np.argsort(evals)[::-1][:dim]
    V = evecs[:, order]
    flip = np.sign(V[np.abs(V).argmax(axis=0), np.arange(dim)])
    return mean, V * flip


def pca_project(images: np.ndarray, mean: np.ndarray, V: np.ndarray) -> np.ndarray:
    """FP32 projection (images - mean) @ V."""
    Z = images.astype(np.float32) - mean.astype(np.float32)
    return np.ascontiguousarray(Z @ V.astype(np.float32), dtype=np.float32)


def images_config(n: int = 70_000, seed: int = 0, dim: int = 50):
    """70K-style workload: images -> centred FP32 PCA to ``dim``.

    Returns (X float32 n x dim, labels, mean, V) so that held-out points can be
    projected with the same basis.
    """
    imgs, labels = blob_images(n, seed)
    mean, V = pca_basis(imgs, dim)
    return pca_project(imgs, mean, V), labels, mean, V


def images_heldout(n: int, mean: np.ndarray, V: np.ndarray, seed: int = 0, chunk: int = 100_000):
    """n further images of the 70K-style generator (its held-out noise stream),
    projected with the training basis (mean, V); generated in chunks."""
    out = np.empty((n, V.shape[1]), dtype=np.float32)
    for s in range(0, n, chunk):
        m = min(chunk, n - s)
        imgs, _ = blob_images(m, seed, stream=4, start=s)
        out[s:s + m] = pca_project(imgs, mean, V)
    return out


def aniso_params(d: int = 50, n_clusters: int = 100, seed: int = 0,
                 center_scale: float = 5.0, lam_lo: float = 0.2, lam_hi: float = 2.0):
    """Centres (c x d) and per-cluster transforms T_c = Q_c diag(sqrt(L_c))."""
    g = _rng(seed, 5)
    centres = g.normal(0.0, center_scale, size=(n_clusters, d))
    T = np.empty((n_clusters, d, d))
    for c in range(n_clusters):
        Q, R = np.linalg.qr(g.normal(size=(d, d)))
        Q *= np.sign(np.diag(R))  # Haar-distributed orthogonal matrix
        lam = g.uniform(lam_lo, lam_hi, size=d)
        T[c] = Q * np.sqrt(lam)
    return centres, T


def aniso_mixture(n: int, d: int = 50, n_clusters: int = 100, seed: int = 0):
    """Anisotropic mixture on the host (small n); label i mod c."""
    centres, T = aniso_params(d, n_clusters, seed)
    g = _rng(seed, 6)
    labels = (np.arange(n) % n_clusters).astype(np.int32)
    z = g.normal(size=(n, d))
    X = centres[labels] + np.einsum("nij,nj->ni", T[labels], z)
    return X.astype(np.float32), labels


def aniso_mixture_torch(n: int, d: int = 50, n_clusters: int = 100, seed: int = 0,
                        device: str = "cuda", chunk: int = 1 << 20):
    """Anisotropic mixture drawn on ``device`` in chunks (used for 10M points).

    Returns a contiguous float32 torch tensor n x d.  The parameters come from
    ``aniso_params``; the Gaussian draws come from a seeded torch generator on
    the device, so the result is a pure function of (n, seed) on one device
    type.
    """
    import torch

    centres, T = aniso_params(d, n_clusters, seed)
    C = torch.as_tensor(centres, dtype=torch.float32, device=device)
    Tt = torch.as_tensor(T, dtype=torch.float32, device=device)
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed) * 7919 + 17)
    X = torch.empty((n, d), dtype=torch.float32, device=device)
    for s in range(0, n, chunk):
        m = min(chunk, n - s)
        z = torch.randn((m, d), generator=gen, device=device, dtype=torch.float32)
        for c in range(n_clusters):  # rows with label c: s + r, (s + r) mod n_clusters = c
            first = (c - s) % n_clusters
            if first < m:
                X[s + first:s + m:n_clusters] = C[c] + z[first::n_clusters] @ Tt[c].T
    return X


def batched_sizes(count: int = 256, seed: int = 0, lo: float = 1e3, hi: float = 5e4):
    g = _rng(seed, 7)
    return np.floor(np.exp(g.uniform(math.log(lo), math.log(hi), size=count))).astype(np.int64)


def batched(count: int = 256, d: int = 50, seed: int = 0, lo: float = 1e3, hi: float = 5e4):
    """Uneven instances; returns (X_cat float32 (sum n) x d, offsets int64 count+1)."""
    sizes = batched_sizes(count, seed, lo, hi)
    g = _rng(seed, 8)
    clusters = g.integers(5, 21, size=count)
    parts = [mixture(int(sizes[b]), d, int(clusters[b]), seed=seed * 100_003 + b + 1)[0]
             for b in range(count)]
    offsets = np.zeros(count + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(sizes)
    return np.ascontiguousarray(np.concatenate(parts, axis=0)), offsets


def sheet(n: int, d: int = 50, seed: int = 0, aspect: float = 3.0, noise: float = 0.01):
    """Points on a flat 2-D sheet [0, aspect] x [0, 1] placed in d dimensions
    by a random orthonormal map, plus isotropic Gaussian noise: a connected
    k-NN graph with a known low-dimensional structure.  Returns (X, uv)."""
    g = _rng(seed, 7)
    uv = g.uniform(0.0, 1.0, size=(n, 2)) * np.array([aspect, 1.0])
    Q, _ = np.linalg.qr(g.normal(size=(d, 2)))
    X = uv @ Q.T + noise * g.normal(size=(n, d))
    return X.astype(np.float32), uv


def config_small(seed: int = 0):
    """The 2,000-point, 50-d, 10-cluster workload."""
    return mixture(2000, 50, 10, seed)


def config_70k(seed: int = 0):
    """The 70,000-point workload (synthetic images, PCA to 50)."""
    X, labels, _, _ = images_config(70_000, seed)
    return X, labels
