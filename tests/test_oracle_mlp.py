"""Pins for the oracle's learned embedder (not gpu)."""
import numpy as np
import pytest

from oracle import mlp, philox


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    x = np.random.default_rng(0).normal(scale=100, size=10000).astype(np.float32)
    x[:4] = [1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -0.0, 65504.0]      # ties and edge values
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16(x), ref)


def test_gelu_matches_torch_exact_form():
    torch = pytest.importorskip("torch")
    x = np.linspace(-8, 8, 2001)
    t = torch.from_numpy(x).requires_grad_(True)
    y = torch.nn.functional.gelu(t, approximate="none")
    y.sum().backward()
    np.testing.assert_allclose(mlp.gelu(x), y.detach().numpy(), rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(mlp.gelu_grad(x), t.grad.numpy(), rtol=1e-12, atol=1e-14)


def _tiny_problem(h=8, d=5, n=40, n_edges=3, neg=2, seed=0):
    g = np.random.default_rng(seed)
    P = g.normal(scale=0.5, size=mlp.param_count(h))
    W1 = P[:h * mlp.IN].reshape(h, mlp.IN)
    W1[:, d:] = 0.0
    X = g.normal(size=(n, d))
    rows = g.integers(0, n, size=n_edges * (2 + neg))
    return P, X, rows


def test_backward_matches_central_differences():
    h, d, n_edges, neg, a, b = 8, 5, 3, 2, 1.577, 0.895
    P, X, rows = _tiny_problem(h, d, n_edges=n_edges, neg=neg)
    L, g = mlp.grad(P, X, rows, d, n_edges, neg, a, b, h=h, emulate=False)
    eps = 1e-6
    for p in range(0, len(P), 7):
        if p < h * mlp.IN and (p % mlp.IN) >= d:
            continue  # padded input columns do not exist
        Pp, Pm = P.copy(), P.copy()
        Pp[p] += eps
        Pm[p] -= eps
        fd = (mlp.grad(Pp, X, rows, d, n_edges, neg, a, b, h=h, emulate=False)[0]
              - mlp.grad(Pm, X, rows, d, n_edges, neg, a, b, h=h, emulate=False)[0]) / (2 * eps)
        assert abs(fd - g[p]) <= 1e-6 * max(1.0, abs(fd)), p


def test_adam_matches_torch():
    torch = pytest.importorskip("torch")
    g = np.random.default_rng(1)
    P0 = g.normal(size=50)
    grads = g.normal(size=(4, 50))
    t = torch.tensor(P0, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([t], lr=1e-3, betas=(0.9, 0.999), eps=1e-8)
    P, m, v = P0.copy(), np.zeros(50), np.zeros(50)
    for s in range(4):
        opt.zero_grad()
        t.grad = torch.tensor(grads[s])
        opt.step()
        P, m, v = mlp.adam_step(P, m, v, grads[s], s + 1)
    np.testing.assert_allclose(P, t.detach().numpy(), rtol=1e-13, atol=1e-15)


def test_sampler_heads_and_proportionality():
    # 3 rows; entries with schedule words 2^24, 2^23, 2^22, 2^24 (weights 1, .5, .25, 1)
    row_ptr = np.array([0, 2, 3, 4])
    col = np.array([1, 2, 0, 0])
    q = np.array([1 << 24, 1 << 23, 1 << 22, 1 << 24], np.uint64)
    rows = mlp.sample(row_ptr, col, q, 3, 4000, 1, step=5, seed=9).reshape(-1, 3)
    heads, tails = rows[:, 0], rows[:, 1]
    # map (head, tail) back to the entry and count
    ent = {(0, 1): 0, (0, 2): 1, (1, 0): 2, (2, 0): 3}
    counts = np.bincount([ent[(h_, t_)] for h_, t_ in zip(heads, tails)], minlength=4)
    expect = 4000 * np.array([1, 0.5, 0.25, 1]) / 2.75
    assert np.all(np.abs(counts - expect) < 5 * np.sqrt(expect))
    assert rows[:, 2].min() >= 0 and rows[:, 2].max() < 3


def test_sampler_uses_documented_counters():
    row_ptr = np.array([0, 1, 2])
    col = np.array([1, 0])
    q = np.array([1 << 24, 1 << 24], np.uint64)  # always accepted at the first try
    r = mlp.sample(row_ptr, col, q, 2, 2, 3, step=7, seed=3)
    u = philox.philox_generic((7, 1, 0, philox.TAG_MLP), (3, 0), 32)
    e = (u[0] * 2) >> 32
    assert r[5] == e and r[6] == col[e]
    un = philox.philox_generic((7, 1, 64, philox.TAG_MLP), (3, 0), 32)
    assert list(r[7:10]) == [(un[t] * 2) >> 32 for t in range(3)]


def test_knn_query_matches_brute_force():
    from oracle import knn as oknn
    g = np.random.default_rng(4)
    X, Q = g.normal(size=(300, 6)), g.normal(size=(40, 6))
    idx, dist = oknn.knn_query(Q, X, 9)
    D = ((Q[:, None, :] - X[None, :, :]) ** 2).sum(-1)
    ref = np.argsort(D, axis=1, kind="stable")[:, :9]
    assert np.array_equal(idx, ref)
    np.testing.assert_allclose(dist, np.sqrt(np.take_along_axis(D, ref, axis=1)), rtol=1e-12)


def test_anchored_epoch_equals_full_epoch_on_joined_graph():
    # moving only the new rows equals a full epoch on [train; new] whose training
    # rows have no entries, with the new rows' negatives restricted to the training set
    from oracle import sgd
    g = np.random.default_rng(5)
    n_t, n_n, k = 50, 7, 4
    Yt, Yn = g.normal(size=(n_t, 2)), g.normal(size=(n_n, 2))
    col = np.sort(g.choice(n_t, size=(n_n, k)), axis=1)
    q = g.integers(1 << 20, 1 << 24, size=n_n * k).astype(np.uint64)
    rp = np.arange(n_n + 1) * k
    Y1 = sgd.anchored_epoch(Yt, Yn, rp, col.ravel(), q, 1.5, 0.9, 0.7, 0, 3, 11)
    # with no negatives the joined-graph epoch is a plain epoch on n_t + n_n rows
    rp_all = np.concatenate([np.zeros(n_t, np.int64), rp])
    Y2 = sgd.epoch(np.concatenate([Yt, Yn]), rp_all, col.ravel(), q, 1.5, 0.9, 0.7, 0, 3, 11)
    np.testing.assert_allclose(Y1, Y2[n_t:], rtol=1e-14)
    np.testing.assert_array_equal(Y2[:n_t], Yt)
