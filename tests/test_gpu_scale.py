"""The 10-million-point workload (gpu): sampled outputs against the oracle and
properties that hold at any size.  Runs about a minute."""
import numpy as np
import pytest

import datagen
from gpu_util import check_knn, drgb_module, epoch_tolerance
from oracle import knn as oknn, sgd as osgd

pytestmark = pytest.mark.gpu

N = 10_000_000


@pytest.fixture(scope="module")
def drgb():
    return drgb_module()


@pytest.fixture(scope="module")
def big(drgb):
    import torch
    X = datagen.aniso_mixture_torch(N, 50, 100, seed=0, device="cuda")
    idx, dist = drgb.knn_graph(X, 15)
    unc = drgb.knn_uncertified()
    g = drgb.fuzzy_weights(idx, dist, 200)
    torch.cuda.synchronize()
    return X, idx, dist, g, unc


def test_knn_sampled_rows(drgb, big):
    X, idx, dist, g, unc = big
    Xh = X.cpu().numpy()
    rows = np.random.default_rng(0).choice(N, 48, replace=False)
    rows = np.concatenate([rows, [0, N - 1]])
    oi, od = oknn.knn_rows(Xh, rows, 15)
    check_knn(Xh, rows, idx[rows].cpu().numpy(), dist[rows].cpu().numpy(), oi, od, 15)
    assert unc < 0.01 * N


def test_graph_symmetric_and_schedule_consistent(drgb, big):
    import torch
    X, idx, dist, g, unc = big
    rp = g.row_ptr.long()
    heads = torch.repeat_interleave(torch.arange(N, device="cuda"), rp[1:] - rp[:-1])
    key = heads * N + g.col.long()
    rkey = g.col.long() * N + heads
    order = torch.argsort(key)
    pos = torch.searchsorted(key[order], rkey)
    assert torch.equal(key[order][pos], rkey)              # every (i, j) has its (j, i)
    assert torch.equal(g.w[order][pos], g.w)                # with the same weight
    assert torch.equal(g.q, torch.round(g.w.double() * (1 << 24)).int())
    assert bool((200 * g.q.long() >= (1 << 24)).all())


def test_epoch_sampled_rows(drgb, big):
    import torch
    X, idx, dist, g, unc = big
    a, b = drgb.find_ab()
    Y = drgb.init_embedding(N, 10.0, 1)
    Y1 = drgb.embed_epoch(Y, g, a, b, 0.9, 5, 3, 2)
    rows = np.random.default_rng(1).choice(N, 200, replace=False)
    ref = osgd.epoch_rows(Y.cpu().numpy(), g.row_ptr.cpu().numpy(), g.col.cpu().numpy(),
                          g.q.cpu().numpy().astype(np.uint64), rows, a, b, float(np.float32(0.9)), 5, 3, 2)
    got = Y1[rows].cpu().numpy()
    assert np.all(np.abs(got - ref) <= epoch_tolerance(ref))


def test_fit_quality_at_scale(drgb, big):
    X = big[0]
    Y = drgb.fit_transform(X, n_epochs=200)
    r = drgb.eval_recall(X, Y, 15, 10_000)
    t = drgb.eval_trust(X, Y, 15, 10_000)
    # Measured on GB300 (seeds 0 and 1 of this workload, 10K sampled rows):
    # recall 1.7e-4 and 2.5e-4 (110-170x chance: inside a 100,000-point
    # Gaussian cluster a point's 15 nearest neighbours are set by noise that
    # no 2-D map keeps), trustworthiness 0.9950 both.  The floors sit below
    # half the measured recall and 0.005 below the measured trust, and at
    # least at the 0.9 trust floor of the smaller fits.
    assert r > 50 * 15 / N and t > 0.99, (r, t)
