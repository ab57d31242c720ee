"""Spectral initial layout on the GPU against the FP64 oracle (gpu).

The eigen-solver differs (FP32 Chebyshev-filtered subspace iteration on the
GPU, a dense FP64 eigensolver in the oracle), so vectors are compared where
they are unique: on a connected graph with distinct leading eigenvalues each
layout column is one eigenvector up to sign, and the sign convention (largest
entry positive) makes it unique.  The GPU stops at a residual of 1e-5, so a
vector may differ from the exact one by about 1e-5 / gap in angle.
"""
import numpy as np
import pytest

import datagen
from gpu_util import drgb_module
from oracle import fuzzy as ofuzzy, knn as oknn, metrics as omet, sgd as osgd, spectral as ospec

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def drgb():
    return drgb_module()


def _graph(drgb, g):
    import torch
    return drgb.Graph(torch.from_numpy(g["row_ptr"].astype(np.int32)).cuda(),
                      torch.from_numpy(g["col"].astype(np.int32)).cuda(),
                      torch.from_numpy(g["w"].astype(np.float32)).cuda(),
                      torch.from_numpy(g["q"].astype(np.int32)).cuda())


@pytest.fixture(scope="module")
def sheet_graph():
    X, _ = datagen.sheet(3000, 50, seed=1)
    idx, dist = oknn.knn(X, 15)
    return X, ofuzzy.build_csr(idx, dist, 200, 15)


def test_layout_matches_oracle_on_a_connected_graph(drgb, sheet_graph):
    X, g = sheet_graph
    n = len(X)
    Yg, ev = drgb.spectral_init(_graph(drgb, g), 10.0, seed=4)
    Yg = Yg.cpu().numpy().astype(np.float64)
    Yo, vals = ospec.spectral_init(g["row_ptr"], g["col"], g["w"], n, 10.0, seed=4)
    assert np.allclose(ev, vals, atol=2e-5), (ev, vals)
    gap = min(vals[1] - vals[2], vals[2] - ospec.leading_eigenvectors(
        ospec.normalized_adjacency(g["row_ptr"], g["col"], g["w"], n), 4)[0][3])
    assert gap > 1e-3                     # distinct eigenvalues: each column is unique up to sign
    for k in range(2):
        cos = Yg[:, k] @ Yo[:, k] / (np.linalg.norm(Yg[:, k]) * np.linalg.norm(Yo[:, k]))
        assert cos > 0.999, (k, cos)      # same vector, same sign
    assert abs(np.abs(Yg).max() - 10.0) < 1e-3
    assert np.abs(Yg - Yo).max() < 0.05 * 10.0


def test_ring_layout_is_a_circle(drgb):
    import torch
    # gap to the next eigenvalue cos(2 pi / n) - cos(4 pi / n) = 1.5e-3; at a
    # residual of 1e-5 the layout's angle to span(cos, sin) is below 1e-2
    n = 200
    heads = np.concatenate([np.arange(n), np.arange(n)])
    tails = np.concatenate([(np.arange(n) + 1) % n, (np.arange(n) - 1) % n])
    order = np.lexsort((tails, heads))
    heads, tails = heads[order], tails[order]
    rp = np.zeros(n + 1, np.int64)
    np.add.at(rp, heads + 1, 1)
    rp = np.cumsum(rp)
    g = drgb.Graph(torch.from_numpy(rp.astype(np.int32)).cuda(), torch.from_numpy(tails.astype(np.int32)).cuda(),
                   torch.ones(len(tails), device="cuda"), torch.full((len(tails),), 1 << 24, dtype=torch.int32,
                                                                     device="cuda"))
    Y, ev = drgb.spectral_init(g, 10.0)
    Y = Y.cpu().numpy().astype(np.float64)
    assert ev[0] == pytest.approx(1.0, abs=1e-5)
    assert ev[1] == pytest.approx(np.cos(2 * np.pi / n), abs=1e-5)
    r = np.linalg.norm(Y - Y.mean(axis=0), axis=1)
    assert r.std() / r.mean() < 2e-2


def test_fit_from_spectral_layout_matches_oracle_quality(drgb):
    import torch
    X, _ = datagen.sheet(2000, 50, seed=2)
    rows = np.arange(len(X))
    gq, oq = [], []
    graph = None
    for s in range(3):
        Yg = drgb.fit_transform(torch.from_numpy(X).cuda(), n_epochs=200, init="spectral",
                                seed_init=10 * s + 1, seed_neg=10 * s + 2).cpu().numpy()
        if graph is None:
            idx, dist = oknn.knn(X, 15)
            graph = ofuzzy.build_csr(idx, dist, 200, 15)
            graph["knn_idx"] = idx
        Y0, _ = ospec.spectral_init(graph["row_ptr"], graph["col"], graph["w"], len(X), 10.0, seed=10 * s + 1)
        Yo = Y0
        for t in range(200):
            Yo = osgd.epoch(Yo, graph["row_ptr"], graph["col"], graph["q"], *drgb.find_ab(), 1.0 - t / 200, 5, t,
                            10 * s + 2)
        gq.append(omet.quality(X, Yg, 15, rows, knn_x=graph["knn_idx"]))
        oq.append(omet.quality(X, Yo, 15, rows, knn_x=graph["knn_idx"]))
    gq, oq = np.mean(gq, axis=0), np.mean(oq, axis=0)
    print("spectral-init fit quality gpu", gq, "oracle", oq)
    assert abs(gq[0] - oq[0]) < 0.005 and abs(gq[1] - oq[1]) < 0.005, (gq, oq)
    assert gq[1] > 0.95
