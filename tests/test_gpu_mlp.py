"""Learned embedder against the FP64 oracle with BF16 rounding emulated (gpu)."""
import numpy as np
import pytest

import datagen
from gpu_util import drgb_module
from oracle import fuzzy as ofuzzy, knn as oknn, mlp as omlp

pytestmark = pytest.mark.gpu

A_, B_ = 1.577, 0.895
BLOCKS = ["W1", "b1", "W2", "b2", "W3", "b3"]


@pytest.fixture(scope="module")
def drgb():
    return drgb_module()


@pytest.fixture(scope="module")
def problem():
    X, _ = datagen.mixture(2000, 50, 10, seed=7)
    oi, od = oknn.knn(X, 15)
    g = ofuzzy.build_csr(oi, od, 200, 15)
    return X, g


def _graph(drgb, g):
    import torch
    return drgb.Graph(torch.from_numpy(g["row_ptr"].astype(np.int32)).cuda(),
                      torch.from_numpy(g["col"].astype(np.int32)).cuda(),
                      torch.from_numpy(g["w"].astype(np.float32)).cuda(),
                      torch.from_numpy(g["q"].astype(np.int32)).cuda())


def _blocks(v, h=256):
    sizes = [h * omlp.IN, h, h * h, h, 2 * h, 2]
    out, o = {}, 0
    for name, s in zip(BLOCKS, sizes):
        out[name] = v[o:o + s]
        o += s
    return out


@pytest.mark.parametrize("neg,step,seed", [(5, 0, 0), (5, 17, 123), (3, 2, 9), (8, 1, 4)])
def test_sampler_bit_exact(drgb, problem, neg, step, seed):
    X, g = problem
    rows = drgb.mlp_sample(_graph(drgb, g), 300, neg, step, seed).cpu().numpy()
    ref = omlp.sample(g["row_ptr"], g["col"], g["q"], len(X), 300, neg, step, seed)
    assert np.array_equal(rows, ref)


@pytest.mark.parametrize("n_edges,neg", [(4096, 5), (100, 5), (37, 2)])
def test_gradient_matches_oracle(drgb, problem, n_edges, neg):
    import torch
    X, g = problem
    Xd = torch.from_numpy(X).cuda()
    P = drgb.mlp_init(50, seed=3)
    rows = drgb.mlp_sample(_graph(drgb, g), n_edges, neg, 0, 5)
    grad, loss = drgb.mlp_grad(P, Xd, rows, n_edges, neg, A_, B_)
    Lo, go = omlp.grad(P.cpu().numpy().astype(np.float64), X, rows.cpu().numpy(), 50, n_edges, neg, A_, B_)
    assert loss == pytest.approx(Lo, rel=1e-3)
    gg, oo = _blocks(grad.cpu().numpy().astype(np.float64)), _blocks(go)
    scale = np.linalg.norm(go)
    for name in BLOCKS:
        # relative per block; b3 = sum of dL/dz is exactly 0 (each pair's two
        # forces cancel), so it is held to the gradient's overall scale
        err = np.linalg.norm(gg[name] - oo[name])
        assert err <= 2e-2 * np.linalg.norm(oo[name]) + 1e-6 * scale, (name, err, np.linalg.norm(oo[name]))
    # padded input columns of W1 get exactly zero gradient
    assert np.all(gg["W1"].reshape(256, 64)[:, 50:] == 0)


def test_forward_matches_oracle(drgb, problem):
    import torch
    X, g = problem
    P = drgb.mlp_init(50, seed=8)
    Y = drgb.mlp_embed(P, torch.from_numpy(X[:777]).cuda()).cpu().numpy()   # ragged chunk of rows
    z = omlp.embed(P.cpu().numpy().astype(np.float64), X[:777], 50)
    err = np.abs(Y - z)
    assert np.all(err <= 1e-2 * (np.abs(z).max() + 1.0)), err.max()


def test_training_step_matches_oracle_adam(drgb, problem):
    import torch
    X, g = problem
    Xd = torch.from_numpy(X).cuda()
    gd = _graph(drgb, g)
    P = drgb.mlp_init(50, seed=2)
    P0 = P.cpu().numpy().astype(np.float64)
    m, v = torch.zeros_like(P), torch.zeros_like(P)
    losses = drgb.mlp_train(Xd, gd, A_, B_, P, m, v, steps=1, batch_edges=512, neg=5, seed=11)
    rows = omlp.sample(g["row_ptr"], g["col"], g["q"], len(X), 512, 5, 0, 11)
    Lo, go = omlp.grad(P0, X, rows, 50, 512, 5, A_, B_)
    P1, _, _ = omlp.adam_step(P0, np.zeros_like(P0), np.zeros_like(P0), go, 1)
    assert float(losses[0]) == pytest.approx(Lo, rel=1e-3)
    # first Adam step moves each weight by about lr * sign(g): compare directions
    dg = P.cpu().numpy() - P0
    do = P1 - P0
    big = np.abs(do) > 5e-4
    assert np.mean(np.sign(dg[big]) == np.sign(do[big])) > 0.97


def test_training_reduces_loss_and_embeds_held_out(drgb, problem):
    import torch
    from oracle import metrics as omet
    X, g = problem
    Xd = torch.from_numpy(X).cuda()
    P = drgb.mlp_init(50, seed=1)
    m, v = torch.zeros_like(P), torch.zeros_like(P)
    losses = drgb.mlp_train(Xd, _graph(drgb, g), A_, B_, P, m, v, steps=400, batch_edges=1024, neg=5,
                            seed=2).cpu().numpy()
    assert losses[-20:].mean() < 0.8 * losses[:20].mean()
    Xn, _ = datagen.mixture(3000, 50, 10, seed=7)  # same centres, later draws
    Xn = Xn[2000:]
    Yn = drgb.mlp_embed(P, torch.from_numpy(np.ascontiguousarray(Xn)).cuda()).cpu().numpy()
    r, t = omet.quality(Xn, Yn, 15)
    assert r > 10 * 15 / len(Xn) and t > 0.85


def test_transform_matches_oracle(drgb, problem):
    import torch
    from oracle import sgd as osgd
    X, g = problem
    from oracle import knn as oknn2, fuzzy as ofz
    Xn, _ = datagen.mixture(2300, 50, 10, seed=7)
    Xn = np.ascontiguousarray(Xn[2000:])
    ab = drgb.find_ab(1.0, 0.1)
    Yt, _ = osgd.fit(X, n_epochs=60, graph=g, ab=ab)       # the oracle's own training embedding
    Yt = Yt.astype(np.float32)
    # a small learning rate keeps the anchored epochs from amplifying the
    # start difference (near-coincident pairs have a steep attraction force)
    Y = drgb.transform(torch.from_numpy(X).cuda(), torch.from_numpy(Yt).cuda(), torch.from_numpy(Xn).cuda(),
                       n_epochs=6, seed_neg=5, lr0=0.01).cpu().numpy()
    ref = osgd.transform(X, Yt, Xn, k=15, n_epochs=6, neg=5, seed_neg=5, ab=ab, lr0=0.01)
    # The start is a membership-weighted mean; memberships carry the fuzzy-graph
    # tolerance (1e-5, FP32 sigma bisection), which moves the start by at most
    # 1e-5 * sum_j |y_j - y0| / sum_j w_j; the epochs then add the epoch tolerance.
    idx, dist = oknn2.knn_query(Xn, X, 15)
    rho, sig = ofz.smooth_knn(dist, 15)
    w = ofz.directed_weights(dist, rho, sig)
    y0 = (w[:, :, None] * Yt[idx]).sum(1) / w.sum(1)[:, None]
    spread = (np.abs(Yt[idx] - y0[:, None, :])).sum(1) / w.sum(1)[:, None]
    bound = 2e-5 * spread + 3e-5 * np.maximum(np.abs(ref), 1.0)
    err = np.abs(Y - ref)
    assert np.all(err <= bound), (err.max(), (err / bound).max())


def test_learned_embedder_gain_over_plain_transform(drgb):
    """What the trained network buys: new points embedded by one forward pass
    instead of a k-NN search and an optimisation, at the same held-out 15-NN
    recall.  Held-out recall compares each new point's 15 nearest training
    points in X with its 15 nearest training points in 2-D (the network's own
    image of the training set for the MLP, the fitted embedding for the
    transform); 15-NN recall among the new points themselves cannot separate
    the two here, because within a Gaussian cluster the neighbours in 50-d
    are set by noise that no 2-D map keeps."""
    import time
    import torch
    X, _ = datagen.mixture(12_000, 50, 10, seed=7)
    Xd = torch.from_numpy(np.ascontiguousarray(X[:10_000])).cuda()
    Xn = torch.from_numpy(np.ascontiguousarray(X[10_000:])).cuda()
    idx, dist = drgb.knn_graph(Xd, 15)
    g = drgb.fuzzy_weights(idx, dist, 200)
    P = drgb.mlp_init(50, seed=0)
    m, v = torch.zeros_like(P), torch.zeros_like(P)
    drgb.mlp_train(Xd, g, A_, B_, P, m, v, steps=int(50 * g.nnz / 4096), batch_edges=4096, neg=5, seed=1)
    Yt = drgb.fit_transform(Xd, n_epochs=200)
    for _ in range(2):
        drgb.mlp_embed(P, Xn)
        drgb.transform(Xd, Yt, Xn, n_epochs=200)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    Ym = drgb.mlp_embed(P, Xn)
    torch.cuda.synchronize()
    t_mlp = time.perf_counter() - t0
    t0 = time.perf_counter()
    Yp = drgb.transform(Xd, Yt, Xn, n_epochs=200)
    torch.cuda.synchronize()
    t_plain = time.perf_counter() - t0
    rm = drgb.eval_recall_heldout(Xd, drgb.mlp_embed(P, Xd), Xn, Ym, 15)
    rp = drgb.eval_recall_heldout(Xd, Yt, Xn, Yp, 15)
    print(f"mlp {len(Xn) / t_mlp:.3g} pts/s held-out recall {rm:.4f}; "
          f"transform {len(Xn) / t_plain:.3g} pts/s held-out recall {rp:.4f}")
    chance = 15 / len(Xd)
    assert rm > 10 * chance and rp > 10 * chance
    assert abs(rm - rp) <= 0.01, (rm, rp)
    assert t_plain > 5 * t_mlp
