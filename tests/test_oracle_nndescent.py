"""Pins for the oracle's NNDescent (not gpu).

The graph it reaches is approximate, so it is pinned by what must hold for
any correct run: the random start's structure, a hand-worked iteration, the
exact k-NN graph as a fixed point, monotone neighbour distances, the complete
graph when k = n - 1, the stopping rule, and a recall floor against the
brute-force graph."""
import numpy as np
import pytest

from oracle import knn, nndescent as nnd, philox


def test_start_is_k_distinct_other_points_and_seeded():
    G = nnd.init_graph(500, 15, seed=3)
    assert G.shape == (500, 15)
    for i, row in enumerate(G):
        assert len(set(row.tolist())) == 15 and i not in row and row.min() >= 0 and row.max() < 500
    assert np.array_equal(G, nnd.init_graph(500, 15, seed=3))
    assert not np.array_equal(G, nnd.init_graph(500, 15, seed=4))


def test_start_takes_the_first_accepted_words_in_counter_order():
    # row 7: its proposals in (counter, word) order, self and repeats skipped
    n, k, seed = 40, 6, 11
    k0, k1 = philox.split_seed(seed)
    props = []
    for r in range(16):
        w = philox.philox4x32(7, r, 0, 5, k0, k1)
        props += [int((int(x) * n) >> 32) for x in w]
    want = []
    for m in props:
        if m != 7 and m not in want:
            want.append(m)
    assert nnd.init_graph(n, k, seed)[7].tolist() == want[:k]


def test_start_is_uniform_over_the_other_points():
    n, k = 50, 5
    G = nnd.init_graph(n, k, seed=1)
    counts = np.bincount(G.ravel(), minlength=n)
    for s in range(2, 41):
        counts += np.bincount(nnd.init_graph(n, k, seed=s).ravel(), minlength=n)
    expected = 40 * n * k / n
    chi2 = ((counts - expected) ** 2 / expected).sum()
    assert chi2 < 2.0 * (n - 1)          # about n - 1 for a uniform draw


def test_complete_graph_when_k_is_n_minus_1():
    n = 9
    G = nnd.init_graph(n, n - 1, seed=5)
    for i in range(n):
        assert sorted(G[i].tolist()) == [j for j in range(n) if j != i]
    X = np.random.default_rng(0).normal(size=(n, 3))
    idx, dist, iters, rates = nnd.nndescent(X, n - 1, seed=5)
    ref_i, ref_d = knn.knn(X, n - 1)
    assert np.array_equal(idx, ref_i) and np.allclose(dist, ref_d, rtol=1e-12)
    assert iters == 1 and rates == [0.0]


def test_one_iteration_by_hand():
    # points 0, 1, 2, 10 on a line, k = 1, start [3], [3], [3], [2]:
    # C(0) = {3, 2} -> 2; C(1) = {3, 2} -> 2; C(2) = {3}; C(3) = {2}
    X = np.array([[0.0], [1.0], [2.0], [10.0]])
    G0 = np.array([[3], [3], [3], [2]])
    G, d2, u = nnd.iterate(X, G0)
    assert G[:, 0].tolist() == [2, 2, 3, 2]
    assert d2[:, 0].tolist() == [4.0, 1.0, 64.0, 64.0]
    assert u == 2


def test_exact_graph_is_a_fixed_point():
    X = np.random.default_rng(1).normal(size=(300, 8))
    ref_i, ref_d = knn.knn(X, 10)
    G, d2, u = nnd.iterate(X, ref_i)
    assert u == 0 and np.array_equal(G, ref_i) and np.allclose(np.sqrt(d2), ref_d, rtol=1e-12)


def test_distances_never_grow_and_the_loop_stops_by_its_rule():
    g = np.random.default_rng(2)
    X = np.concatenate([g.normal(size=(150, 6)) + 6 * c for c in range(4)])
    G = nnd.init_graph(len(X), 8, seed=9)
    prev = np.sort(((X[G] - X[:, None, :]) ** 2).sum(axis=2), axis=1)
    for _ in range(4):
        G, d2, u = nnd.iterate(X, G)
        # G(i) is among the candidates, so the j-th smallest distance of
        # every list can only fall, for every j
        assert np.all(d2 <= prev + 1e-12)
        prev = d2
    idx, dist, iters, rates = nnd.nndescent(X, 8, seed=9, delta=0.015, max_iter=30)
    assert iters == len(rates) and all(r >= 0.015 for r in rates[:-1])
    assert rates[-1] < 0.015 or iters == 30
    idx1, _, iters1, rates1 = nnd.nndescent(X, 8, seed=9, delta=0.015, max_iter=1)
    assert iters1 == 1 and rates1 == rates[:1]


def test_recall_against_brute_force():
    g = np.random.default_rng(3)
    X = np.concatenate([g.normal(size=(200, 10)) + 5 * c for c in range(5)])
    idx, dist, iters, rates = nnd.nndescent(X, 15, seed=2)
    ref_i, ref_d = knn.knn(X, 15)
    recall = np.mean([len(set(a) & set(b)) / 15 for a, b in zip(idx.tolist(), ref_i.tolist())])
    assert recall > 0.95, recall
    # the lists are sorted by (distance, index) with the direct distances
    assert np.all(np.diff(dist, axis=1) >= 0)
    assert np.allclose(dist, np.sqrt(((X[idx] - X[:, None, :]) ** 2).sum(axis=2)), rtol=1e-12)


def test_reverse_lists_by_hand():
    # points 0, 1, 2, 10 on a line, k = 1, lists [1], [0], [1], [2]:
    # 0 is held by 1; 1 by 0 and 2 (equal distance 1: the lower index wins);
    # 2 by 3; nobody holds 3
    X = np.array([[0.0], [1.0], [2.0], [10.0]])
    G = np.array([[1], [0], [1], [2]])
    d2 = ((X[G] - X[:, None, :]) ** 2).sum(axis=2)
    assert nnd.reverse_lists(G, d2, 1)[:, 0].tolist() == [1, 0, 3, -1]
    R2 = nnd.reverse_lists(G, d2, 2)
    assert R2[1].tolist() == [0, 2] and R2[3].tolist() == [-1, -1]


def test_one_iteration_with_reverse_neighbours_by_hand():
    # points 0, 1, 3, 10, k = 1, start [3], [3], [3], [0]: R = [3], [], [], [2]
    # (3 is held by 0, 1, 2 at squared distances 100, 81, 49); B = {3}, {3},
    # {3}, {0, 2}; the candidates give new lists 2, 0, 0, 2 (4 updates), where
    # the forward-only iteration gives 3, 0, 0, 0 (2 updates)
    X = np.array([[0.0], [1.0], [3.0], [10.0]])
    G0 = np.array([[3], [3], [3], [0]])
    G, d2, u = nnd.iterate(X, G0, reverse=True)
    assert G[:, 0].tolist() == [2, 0, 0, 2] and u == 4
    assert d2[:, 0].tolist() == [9.0, 1.0, 9.0, 49.0]
    Gf, _, uf = nnd.iterate(X, G0)
    assert Gf[:, 0].tolist() == [3, 0, 0, 0] and uf == 2


def test_reverse_form_keeps_the_fixed_point_and_is_not_worse():
    g = np.random.default_rng(4)
    X = np.concatenate([g.normal(size=(150, 12)) + 4 * c for c in range(4)])
    ref, ref_d = knn.knn(X, 10)
    G, d2, u = nnd.iterate(X, ref, reverse=True)
    assert u == 0 and np.array_equal(G, ref)
    G = nnd.init_graph(len(X), 10, seed=7)
    prev = np.sort(((X[G] - X[:, None, :]) ** 2).sum(axis=2), axis=1)
    for _ in range(3):
        G, d2, u = nnd.iterate(X, G, reverse=True)
        assert np.all(d2 <= prev + 1e-12)
        prev = d2
    rec = lambda idx: np.mean([len(set(a) & set(b)) / 10 for a, b in zip(idx.tolist(), ref.tolist())])
    f = nnd.nndescent(X, 10, seed=7)[0]
    r = nnd.nndescent(X, 10, seed=7, reverse=True)[0]
    assert rec(r) >= rec(f) - 0.005 and rec(r) > 0.95
