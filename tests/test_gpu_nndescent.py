"""NNDescent on the GPU against the FP64 oracle (gpu).

The iteration is synchronous and its start is a counter-based draw, so both
sides compute the same graph; the only difference is the precision of the
distances (FP32 direct sums on the GPU, FP64 in the oracle), which can order
two candidates differently only where their distances agree to about 1e-6.
Each comparison therefore asks for identical lists except on a few rows,
and on those rows for sorted distance lists equal to 1e-5 (a near-tie swap);
distances of shared entries agree to FP32 accumulation error (rtol 4e-6 for
d <= 50 positive terms)."""
import numpy as np
import pytest

from gpu_util import drgb_module
from oracle import knn as oknn, nndescent as onnd

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def drgb():
    return drgb_module()


def _mixture(n, d, seed, clusters=6, spread=4.0):
    g = np.random.default_rng(seed)
    centres = g.normal(size=(clusters, d)) * spread
    return (centres[np.arange(n) % clusters] + g.normal(size=(n, d))).astype(np.float32)


def _gpu(drgb, X, k, seed, delta, max_iter, reverse=False):
    import torch
    idx, dist, rates = drgb.knn_nndescent(torch.from_numpy(X).cuda(), k, seed=seed, delta=delta, max_iter=max_iter,
                                          reverse=reverse)
    return idx.cpu().numpy().astype(np.int64), dist.cpu().numpy().astype(np.float64), rates


def _compare(X, gi, gd, oi, od, max_rows):
    same = np.all(gi == oi, axis=1)
    bad = np.nonzero(~same)[0]
    assert bad.size <= max_rows, (bad.size, bad[:10])
    for r in bad:   # a near-tie swap: the two sorted distance lists agree
        assert np.allclose(np.sort(gd[r]), np.sort(od[r]), rtol=1e-5), r
    assert np.allclose(gd[same], od[same], rtol=4e-6, atol=1e-6)


@pytest.mark.parametrize("d,k", [(20, 15), (7, 10), (50, 15)])
def test_iterations_match_oracle(drgb, d, k):
    # odd d takes the scalar distance loop, even d the paired loads
    X = _mixture(2500, d, seed=d)
    for t in (1, 2, 4):
        gi, gd, grates = _gpu(drgb, X, k, seed=3, delta=0.0, max_iter=t)
        oi, od, oit, orates = onnd.nndescent(X, k, seed=3, delta=0.0, max_iter=t)
        assert len(grates) == oit == t
        _compare(X, gi, gd, oi, od, max_rows=5)
        assert np.allclose(grates, orates, atol=5 * 1.0 / (len(X) * k) + 1e-12)


@pytest.mark.parametrize("d,k", [(20, 15), (7, 16), (50, 4)])
def test_reverse_form_iterations_match_oracle(drgb, d, k):
    # the reverse lists are chosen by (distance, owner) too, so an FP32/FP64
    # near-tie there can also move a few rows; the same bounds apply
    X = _mixture(2500, d, seed=d + 100)
    for t in (1, 3):
        gi, gd, grates = _gpu(drgb, X, k, seed=5, delta=0.0, max_iter=t, reverse=True)
        oi, od, oit, orates = onnd.nndescent(X, k, seed=5, delta=0.0, max_iter=t, reverse=True)
        assert len(grates) == oit == t
        _compare(X, gi, gd, oi, od, max_rows=10)
        assert np.allclose(grates, orates, atol=10 * 1.0 / (len(X) * k) + 1e-12)


def test_converged_graph_matches_oracle_and_recall(drgb):
    X = _mixture(3000, 24, seed=5)
    gi, gd, grates = _gpu(drgb, X, 15, seed=1, delta=0.015, max_iter=30)
    oi, od, oit, orates = onnd.nndescent(X, 15, seed=1)
    assert abs(len(grates) - oit) <= 1
    if len(grates) == oit:
        _compare(X, gi, gd, oi, od, max_rows=10)
    assert grates[-1] < 0.015 and all(r >= 0.015 for r in grates[:-1])
    ref, _ = oknn.knn(X, 15)
    recall = np.mean([len(set(a) & set(b)) / 15 for a, b in zip(gi.tolist(), ref.tolist())])
    o_recall = np.mean([len(set(a) & set(b)) / 15 for a, b in zip(oi.tolist(), ref.tolist())])
    # the method's own quality at d = 24 (no reverse neighbours): about 0.93
    assert recall > 0.9 and abs(recall - o_recall) < 0.002, (recall, o_recall)


def test_edge_cases(drgb):
    g = np.random.default_rng(8)
    # complete graph: k = n - 1 gives the exact lists after one iteration
    X = g.normal(size=(33, 5)).astype(np.float32)
    gi, gd, rates = _gpu(drgb, X, 32, seed=2, delta=0.015, max_iter=30)
    ref, refd = oknn.knn(X, 32)
    assert np.array_equal(gi, ref) and rates == [0.0]
    assert np.allclose(gd, refd, rtol=4e-6)
    # k = 1, and duplicated points: equal distances are ordered by index on both sides
    X2 = np.repeat(g.normal(size=(300, 6)), 2, axis=0).astype(np.float32)
    for k in (1, 4):
        gi, gd, rates = _gpu(drgb, X2, k, seed=4, delta=0.0, max_iter=3)
        oi, od, _, orates = onnd.nndescent(X2, k, seed=4, delta=0.0, max_iter=3)
        _compare(X2, gi, gd, oi, od, max_rows=3)
    # every run is deterministic
    a = _gpu(drgb, X2, 4, seed=4, delta=0.0, max_iter=3)
    b = _gpu(drgb, X2, 4, seed=4, delta=0.0, max_iter=3)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and a[2] == b[2]


def test_rejects_bad_arguments(drgb):
    import torch
    X = torch.zeros((100, 8), dtype=torch.float32, device="cuda")
    with pytest.raises(drgb.DrgbError):
        drgb.knn_nndescent(X, 17, reverse=True)
    for kw in (dict(delta=-0.1), dict(delta=1.5), dict(max_iter=0), dict(max_iter=1001)):
        with pytest.raises(drgb.DrgbError):
            drgb.knn_nndescent(X, 5, **kw)
    with pytest.raises(drgb.DrgbError):
        drgb.knn_nndescent(torch.zeros((100, 1025), dtype=torch.float32, device="cuda"), 5)
    with pytest.raises(drgb.DrgbError):
        drgb.knn_nndescent(X, 100)
    Xn = X.clone()
    Xn[3, 2] = float("nan")
    with pytest.raises(drgb.DrgbError):
        drgb.knn_nndescent(Xn, 5)


def test_70k_recall_against_the_exact_graph(drgb):
    import torch
    import datagen
    X, _ = datagen.config_70k(seed=0)
    Xd = torch.from_numpy(X).cuda()
    gi, gd, rates = drgb.knn_nndescent(Xd, 15, seed=1)
    ei, ed = drgb.knn_graph(Xd, 15, mode=1)
    same = (gi.unsqueeze(2) == ei.unsqueeze(1)).any(dim=2).float().mean().item()
    # measured 0.595: the images are noise-dominated in 50-d, where a point's
    # nearest neighbours are scattered over its class of 7,000 and the
    # neighbours-of-neighbours search (no reverse neighbours) stalls early;
    # the floor guards against a regression, not the method's ceiling
    assert same > 0.55, same
    assert rates[-1] < 0.015 and len(rates) < 30
    # the reverse form (the basic algorithm of the method the paper cites)
    # finds more of the exact neighbours
    ri, rd, rrates = drgb.knn_nndescent(Xd, 15, seed=1, reverse=True)
    same_rev = (ri.unsqueeze(2) == ei.unsqueeze(1)).any(dim=2).float().mean().item()
    assert same_rev > same + 0.1, (same_rev, same)
    # every kept distance is the FP32 distance of its pair, and no list holds its own point
    rows = torch.arange(len(X), device="cuda").unsqueeze(1)
    assert not (gi == rows).any()
    direct = ((Xd[gi.long()] - Xd.unsqueeze(1)) ** 2).sum(2).sqrt()
    assert torch.allclose(gd, direct, rtol=1e-5, atol=1e-5)


def test_fit_with_nndescent(drgb):
    import torch
    X = _mixture(4000, 30, seed=9, clusters=10)
    Xd = torch.from_numpy(X).cuda()
    Y4 = drgb.fit_transform(Xd, n_epochs=200, knn_mode=4)
    Y4b = drgb.fit_transform(Xd, n_epochs=200, knn_mode=4)
    assert torch.equal(Y4, Y4b)
    Y1 = drgb.fit_transform(Xd, n_epochs=200, knn_mode=1)
    r4, r1 = drgb.eval_recall(Xd, Y4, 15), drgb.eval_recall(Xd, Y1, 15)
    t4, t1 = drgb.eval_trust(Xd, Y4, 15), drgb.eval_trust(Xd, Y1, 15)
    assert abs(r4 - r1) < 0.02 and abs(t4 - t1) < 0.01, (r4, r1, t4, t1)
    with pytest.raises(drgb.DrgbError):
        drgb.knn_graph(Xd, 15, mode=4)
