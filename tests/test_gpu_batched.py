"""Batched form and schedule autotuner (gpu).

Each instance of a batched fit must be bit-identical to fitting that instance
alone with the same seeds, whatever the instance sizes (some take the exact
FP32 k-NN scan, some the tensor-core path), and whatever epoch schedule the
autotuner picks.
"""
import numpy as np
import pytest

import datagen
from gpu_util import drgb_module

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def drgb():
    return drgb_module()


def _instances(sizes, seed=0):
    parts = [datagen.mixture(int(nb), 50, 5 + b % 16, seed=seed * 1000 + b)[0] for b, nb in enumerate(sizes)]
    off = np.zeros(len(sizes) + 1, np.int64)
    off[1:] = np.cumsum(sizes)
    return np.ascontiguousarray(np.concatenate(parts)), off


@pytest.mark.parametrize("autotune", [False, True])
def test_batched_equals_sequential_plain_runs(drgb, autotune):
    import torch
    sizes = [500, 1200, 4500, 60, 2000, 5000, 16]
    X, off = _instances(sizes, seed=3)
    si = [11 + 7 * b for b in range(len(sizes))]
    sn = [101 + 13 * b for b in range(len(sizes))]
    Xd = torch.from_numpy(X).cuda()
    Yb = drgb.fit_transform_batched(Xd, off, si, sn, autotune=autotune, n_epochs=120).cpu()
    for b in range(len(sizes)):
        Yp = drgb.fit_transform(Xd[off[b]:off[b + 1]].contiguous(), n_epochs=120, seed_init=si[b],
                                seed_neg=sn[b]).cpu()
        assert torch.equal(Yb[off[b]:off[b + 1]], Yp), f"instance {b} (n={sizes[b]}) differs"


def test_batched_default_seeds_and_quality(drgb):
    import torch
    from oracle import metrics as omet
    sizes = [800, 1500]
    X, off = _instances(sizes, seed=5)
    Y = drgb.fit_transform_batched(torch.from_numpy(X).cuda(), off, n_epochs=200).cpu().numpy()
    for b in range(len(sizes)):
        Xb, Yb = X[off[b]:off[b + 1]], Y[off[b]:off[b + 1]]
        r, t = omet.quality(Xb, Yb, 15)
        assert r > 10 * 15 / len(Xb) and t > 0.9


def test_batched_rejects_small_instance(drgb):
    import torch
    X, off = _instances([100, 10, 100])
    with pytest.raises(drgb.DrgbError):
        drgb.fit_transform_batched(torch.from_numpy(X).cuda(), off, n_epochs=5)


def test_autotune_returns_a_supported_choice(drgb):
    import torch
    X, _ = datagen.mixture(5000, 50, 10, seed=1)
    idx, dist = drgb.knn_graph(torch.from_numpy(X).cuda(), 15)
    g = drgb.fuzzy_weights(idx, dist, 200)
    Y = drgb.init_embedding(5000, 10.0, 1)
    Y0 = Y.clone()
    choice, us = drgb.autotune_epoch(Y, g, 1.577, 0.895, trials=2)
    assert choice[0] in (4, 8) and choice[1] in (0, 1)
    assert us > 0 and torch.equal(Y, Y0)   # the caller's embedding is untouched


def test_fit_is_deterministic_from_a_fresh_context(drgb):
    # the first fit on a new context grows the scratch; the k-NN scratch must
    # not overlap the fit's own buffers (tensor-core path at this size)
    import torch
    X, _ = datagen.mixture(9000, 50, 10, seed=4)
    Xd = torch.from_numpy(X).cuda()
    drgb._destroy_all()
    Y1 = drgb.fit_transform(Xd, n_epochs=60)
    drgb._destroy_all()
    drgb.context()
    Y2 = drgb.fit_transform(Xd, n_epochs=60)
    Y3 = drgb.fit_transform(Xd, n_epochs=60)
    assert torch.equal(Y1, Y2) and torch.equal(Y2, Y3)


def test_autotune_uses_and_fills_the_tuning_cache(drgb, tmp_path):
    import json
    import torch
    from paper_2603_04035_gb300 import _lib
    sizes = [1500, 3000, 800, 2500]
    X, off = _instances(sizes, seed=9)
    Xd = torch.from_numpy(X).cuda()
    path = str(tmp_path / "tune.json")
    drgb.set_tuning_cache(path)
    try:
        Y0 = drgb.fit_transform_batched(Xd, off, autotune=True, n_epochs=60).cpu()   # times and records
        with open(path) as f:
            entries = json.load(f)
        assert len(entries) == 1
        key, val = next(iter(entries.items()))
        assert key.endswith(f"|rows 2^{int(np.log2(sum(sizes)))}|instances 2^2|k 15")
        assert val["epoch_warps"] == drgb.get_tuning(_lib.TUNE_EPOCH_WARPS)
        assert val["epoch_pipe"] == drgb.get_tuning(_lib.TUNE_EPOCH_PIPE)
        other = (4 if val["epoch_warps"] == 8 else 8, 1 - val["epoch_pipe"])
        drgb.tuning_cache_store(path, key, *other)
        Y1 = drgb.fit_transform_batched(Xd, off, autotune=True, n_epochs=60).cpu()   # takes the stored setting
        assert (drgb.get_tuning(_lib.TUNE_EPOCH_WARPS), drgb.get_tuning(_lib.TUNE_EPOCH_PIPE)) == other
        assert torch.equal(Y0, Y1)
    finally:
        drgb.set_tuning_cache(None)
