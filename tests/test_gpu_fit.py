"""fit_transform and metric parity against the oracle (gpu).

A fit is a chaotic iteration, so trajectories are not compared; the embeddings
are judged by 15-NN recall and trustworthiness, which must agree with the
oracle's own fit (same graph definition, seeds and schedule) within 0.005.
At n = 2,000 the oracle's seed-to-seed spread of recall is about 0.003, so
the comparison averages several seeds on each side.
"""
import numpy as np
import pytest

import datagen
from gpu_util import drgb_module
from oracle import metrics as omet, sgd as osgd

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def drgb():
    return drgb_module()


def _gpu_fit(drgb, X, **kw):
    import torch
    Y = drgb.fit_transform(torch.from_numpy(X).cuda(), **kw)
    return Y.cpu().numpy()


def test_fit_small_quality_matches_oracle(drgb):
    X, _ = datagen.config_small(seed=0)
    rows = np.arange(len(X))
    seeds = range(6)
    gq, oq = [], []
    graph = None
    for s in seeds:
        Yg = _gpu_fit(drgb, X, n_epochs=200, seed_init=10 * s + 1, seed_neg=10 * s + 2)
        Yo, graph = osgd.fit(X, n_epochs=200, seed_init=10 * s + 1, seed_neg=10 * s + 2, graph=graph)
        gq.append(omet.quality(X, Yg, 15, rows, knn_x=graph["knn_idx"]))
        oq.append(omet.quality(X, Yo, 15, rows, knn_x=graph["knn_idx"]))
    gq, oq = np.mean(gq, axis=0), np.mean(oq, axis=0)
    assert abs(gq[0] - oq[0]) < 0.005, (gq, oq)
    assert abs(gq[1] - oq[1]) < 0.005, (gq, oq)
    assert gq[0] > 10 * 15 / len(X) and gq[1] > 0.9


def test_fit_70k_quality_matches_oracle(drgb):
    X, _ = datagen.config_70k(seed=0)
    rows = np.linspace(0, len(X) - 1, 3000).astype(np.int64)
    Yg = _gpu_fit(drgb, X, n_epochs=500, seed_init=1, seed_neg=2)
    Yo, graph = osgd.fit(X, n_epochs=500, seed_init=1, seed_neg=2)
    kx = graph["knn_idx"][rows]
    rg, tg = omet.quality(X, Yg, 15, rows, knn_x=kx)
    ro, to = omet.quality(X, Yo, 15, rows, knn_x=kx)
    assert abs(rg - ro) < 0.005 and abs(tg - to) < 0.005, (rg, tg, ro, to)


def test_metrics_match_oracle(drgb):
    import torch
    X, _ = datagen.mixture(3000, 50, 10, seed=2)
    Y = _gpu_fit(drgb, X, n_epochs=100)
    Xd, Yd = torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()
    for n_query, rows in [(0, np.arange(3000)), (700, (np.arange(700) * 3000) // 700)]:
        r = drgb.eval_recall(Xd, Yd, 15, n_query)
        t = drgb.eval_trust(Xd, Yd, 15, n_query)
        ro, to = omet.quality(X, Y, 15, rows)
        assert abs(r - ro) < 2e-3 and abs(t - to) < 1e-4, (r, ro, t, to)


@pytest.mark.parametrize("n_query", [0, 333])
def test_heldout_recall_matches_oracle(drgb, n_query):
    import torch
    X, _ = datagen.mixture(3500, 50, 10, seed=5)
    Xt, Xn = X[:3000], X[3000:]
    Yt = _gpu_fit(drgb, np.ascontiguousarray(Xt), n_epochs=100)
    # new points placed near their first training neighbour's position, with noise
    near = np.argmin(((Xn[:, None, :5] - Xt[None, :, :5]) ** 2).sum(-1), axis=1)
    Yn = (Yt[near] + np.random.default_rng(1).normal(scale=0.5, size=(500, 2))).astype(np.float32)
    d = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (Xt, Yt, Xn, Yn)]
    r = drgb.eval_recall_heldout(*d, 15, n_query)
    ro = omet.heldout_recall(Xt, Yt, Xn, Yn, 15, n_query)
    # exact neighbour sets on both sides; only FP32/FP64 distance ties may differ
    assert abs(r - ro) < 2e-3, (r, ro)
    assert 0.01 < ro < 0.99


def test_epoch_callback_sees_every_epoch(drgb):
    import torch
    X, _ = datagen.mixture(500, 20, 5, seed=1)
    seen = []

    def cb(t, Y):
        seen.append((t, float(Y.abs().sum())))
        return t == 9   # stop after epoch 9

    drgb.fit_transform(torch.from_numpy(X).cuda(), n_epochs=50, epoch_callback=cb)
    assert [t for t, _ in seen] == list(range(10))


def test_fit_rejects_nonfinite_input(drgb):
    import torch
    X = torch.randn(200, 10, device="cuda")
    X[17, 3] = float("nan")
    with pytest.raises(drgb.DrgbError) as e:
        drgb.fit_transform(X, n_epochs=5)
    assert e.value.code == -5
    # the context stays usable
    Y = drgb.fit_transform(torch.randn(200, 10, device="cuda"), n_epochs=5)
    assert torch.isfinite(Y).all()


def test_umap_class_front_end(drgb):
    X, _ = datagen.mixture(400, 16, 4, seed=3)
    Y = drgb.UMAP(n_epochs=30, seed=4).fit_transform(X)
    assert tuple(Y.shape) == (400, 2)


def test_stage_times_split_the_knn_stage(drgb):
    # the tensor-core k-NN's sub-stages (ordering and staging, GEMM, re-rank,
    # re-scan) are recorded inside the k-NN stage and add up to at most it
    import torch
    X = torch.from_numpy(datagen.mixture(5000, 50, 10, 1)[0]).cuda()
    drgb.set_profiling(True)
    try:
        drgb.fit_transform(X, n_epochs=20, knn_mode=3)
        st = drgb.stage_times()
        drgb.fit_transform(X, n_epochs=20, knn_mode=1)
        st1 = drgb.stage_times()
    finally:
        drgb.set_profiling(False)
    parts = ("knn_gemm", "knn_prep", "knn_rerank", "knn_rescan")
    assert set(parts) <= set(st), st
    assert all(st[p] > 0 for p in parts[:3]) and st["knn_rescan"] >= 0
    assert sum(st[p] for p in parts) <= st["knn"] * 1.001 + 1e-3, st
    # the exact scan records no sub-stage
    assert all(st1[p] == 0 for p in parts), st1
