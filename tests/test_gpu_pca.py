"""PCA on the GPU against the FP64 oracle (gpu).

The GPU forms the covariance from a two-term BF16 split of the centred data
(about 16 significant bits per value, FP32 accumulation) and finds its
eigenvectors by FP32 subspace iteration until each of the dim leading pairs
has |C v - theta v| <= 1e-5 theta_1.  Against the exact covariance that
gives a residual budget r = 2e-5 lambda_1 (the stopping rule plus the
rounding of C), so:

* each eigenvalue is within r of the oracle's;
* a component is compared only where it is unique to that accuracy: by
  Davis-Kahan its angle to the exact eigenvector is at most r / gap_k, gap_k
  the distance from lambda_k to the other eigenvalues, and it is checked
  where that bound is below 0.05 (with its sign, fixed by the convention);
* where eigenvalues are too close for that, the subspace properties are
  checked instead: orthonormal components, Z = (X - mu) V, and cov(Z) =
  diag(theta) to within r.
"""
import numpy as np
import pytest

import datagen
from gpu_util import drgb_module
from oracle import pca as opca

pytestmark = pytest.mark.gpu

R_BUDGET = 2e-5


@pytest.fixture(scope="module")
def drgb():
    return drgb_module()


def _run(drgb, X, dim):
    import torch
    Z, comps, mu, ev = drgb.pca(torch.from_numpy(np.ascontiguousarray(X, np.float32)).cuda(), dim)
    return (Z.cpu().numpy().astype(np.float64), comps.cpu().numpy().astype(np.float64).T,
            mu.cpu().numpy().astype(np.float64), np.array(ev))


def _check(X, dim, Zg, Vg, mug, evg, min_unique):
    Xd = np.asarray(X, np.float64)
    n, D = Xd.shape
    Zo, Vo, muo, evo = opca.pca(Xd, dim)
    all_ev = np.linalg.eigvalsh(opca.covariance(Xd)[1])[::-1]
    lam1 = all_ev[0]
    r = R_BUDGET * lam1
    # mean: FP64 sums rounded to FP32
    assert np.abs(mug - muo).max() <= 1e-6 * np.abs(Xd).max() + 1e-7
    # eigenvalues within the residual budget
    assert np.abs(evg - evo).max() <= r, (np.abs(evg - evo).max(), r)
    # components: orthonormal
    assert np.abs(Vg.T @ Vg - np.eye(dim)).max() < 1e-5
    # unique components agree with the oracle, sign included
    unique = 0
    for k in range(dim):
        others = np.delete(all_ev, k)
        gap = np.abs(others - all_ev[k]).min()
        bound = r / gap
        if bound >= 0.05:
            continue
        unique += 1
        cos = float(Vg[:, k] @ Vo[:, k])
        # the sine from the part orthogonal to the exact vector (1 - cos^2
        # would lose it to the rounding of |v| = 1)
        sin = np.linalg.norm(Vg[:, k] - cos * Vo[:, k]) / np.linalg.norm(Vg[:, k])
        assert cos > 0, (k, cos)
        assert sin <= bound + 1e-5, (k, sin, bound)
        # the projection onto it as well
        scale = np.linalg.norm(Xd - muo, axis=1).max()
        assert np.abs(Zg[:, k] - Zo[:, k]).max() <= (bound + 1e-5) * scale, k
    assert unique >= min_unique, unique
    # Z is the centred data in the GPU's own basis (FP32 product)
    Zc = (Xd - mug) @ Vg
    rown = np.linalg.norm(Xd - mug, axis=1)
    assert np.all(np.abs(Zg - Zc).max(axis=1) <= 1e-5 * rown + 1e-6)
    # cov(Z) = V^T C V = diag(theta) up to the residuals
    cz = np.cov(Zg, rowvar=False)
    assert np.abs(cz - np.diag(evg)).max() <= 1.5 * r, (np.abs(cz - np.diag(evg)).max(), r)


def test_distinct_spectrum_matches_oracle(drgb):
    # rank-60 signal with geometric variances plus isotropic noise, rotated,
    # off-centre; n and D ragged against the 64-row and 128-column tiles
    g = np.random.default_rng(5)
    n, D = 30_011, 200
    Q, _ = np.linalg.qr(g.normal(size=(D, D)))
    sd = np.concatenate([10 * 0.93 ** np.arange(60), np.zeros(D - 60)]) + 0.05
    X = ((g.normal(size=(n, D)) * sd) @ Q.T + 3.0).astype(np.float32)
    Zg, Vg, mug, evg = _run(drgb, X, 50)
    _check(X, 50, Zg, Vg, mug, evg, min_unique=40)


def test_images_match_oracle(drgb):
    # the 70K-style image generator: ten class prototypes over N(0, 25^2)
    # pixel noise: nine large eigenvalues, then a dense noise floor whose
    # eigenvectors are not unique to the residual budget
    imgs, _ = datagen.blob_images(20_000, 0)
    X = imgs.astype(np.float32)
    Zg, Vg, mug, evg = _run(drgb, X, 50)
    _check(X, 50, Zg, Vg, mug, evg, min_unique=9)


def test_small_d_host_path(drgb):
    # D <= 64: the covariance is diagonalised whole on the host
    g = np.random.default_rng(6)
    n, D = 5_000, 40
    X = (g.normal(size=(n, D)) * np.linspace(3.0, 0.5, D) @ np.linalg.qr(g.normal(size=(D, D)))[0]).astype(np.float32)
    Zg, Vg, mug, evg = _run(drgb, X, 12)
    _check(X, 12, Zg, Vg, mug, evg, min_unique=12)


def test_rank_deficient_and_tiny(drgb):
    # exact rank 20 in 100 dimensions: the null space must not break the
    # block; dim 1 with n = 2 is the smallest case
    g = np.random.default_rng(7)
    X = (g.normal(size=(4_000, 20)) * np.linspace(4.0, 1.0, 20) @ g.normal(size=(20, 100))).astype(np.float32)
    Zg, Vg, mug, evg = _run(drgb, X, 10)
    _check(X, 10, Zg, Vg, mug, evg, min_unique=10)
    X2 = np.array([[1.0, 2.0, 3.0], [3.0, 2.0, 0.0]], np.float32)
    Zg, Vg, mug, evg = _run(drgb, X2, 1)
    Zo, Vo, muo, evo = opca.pca(X2, 1)
    assert np.allclose(evg, evo, rtol=1e-5) and np.allclose(Vg, Vo, atol=1e-5) and np.allclose(Zg, Zo, atol=1e-5)


def test_rejects_bad_sizes(drgb):
    import torch
    X = torch.zeros((100, 80), dtype=torch.float32, device="cuda")
    for dim in (0, 57, 81):
        with pytest.raises(drgb.DrgbError):
            drgb.pca(X, dim)
    with pytest.raises(drgb.DrgbError):
        drgb.pca(torch.zeros((1, 80), dtype=torch.float32, device="cuda"), 2)
    with pytest.raises(drgb.DrgbError):
        drgb.pca(torch.zeros((10, 1025), dtype=torch.float32, device="cuda"), 2)


def test_fit_with_pca_dim_equals_fit_on_the_projection(drgb):
    # fit_transform(X, pca_dim=50) is PCA then the fit on the projection; both
    # paths run the same fixed-order kernels, so the embeddings are identical
    import torch
    imgs, _ = datagen.blob_images(6_000, 1)
    X = torch.from_numpy(imgs.astype(np.float32)).cuda()
    Y_raw = drgb.fit_transform(X, n_epochs=60, pca_dim=50)
    Z = drgb.pca(X, 50)[0]
    Y_z = drgb.fit_transform(Z, n_epochs=60)
    assert torch.equal(Y_raw, Y_z)
    # pca_dim >= d is no PCA
    assert torch.equal(drgb.fit_transform(Z, n_epochs=60, pca_dim=50), Y_z)
    with pytest.raises(drgb.DrgbError):
        drgb.fit_transform(X, n_epochs=5, pca_dim=57)
    with pytest.raises(drgb.DrgbError):
        drgb.fit_transform_batched(X, [0, 3000, 6000], n_epochs=5, pca_dim=50)
