"""Pins for the oracle's fuzzy simplicial-set graph (not gpu)."""
import numpy as np
import pytest

import datagen
from oracle import fuzzy, knn as oknn
from oracle.fuzzy import Q_ONE


@pytest.fixture(scope="module")
def graph():
    X, _ = datagen.mixture(800, 50, 10, seed=4)
    idx, dist = oknn.knn(X, 15)
    return idx, dist, fuzzy.build_csr(idx, dist, n_epochs=200)


def test_row_sums_equal_log2k(graph):
    idx, dist, g = graph
    floor = 1e-3 * dist.mean(axis=1)
    free = g["sigma"] > floor
    sums = g["w_dir"].sum(axis=1)
    assert free.mean() > 0.99
    np.testing.assert_allclose(sums[free], np.log2(15), atol=1e-9)


def test_nearest_weight_one_and_range(graph):
    _, _, g = graph
    assert np.all(g["w_dir"][:, 0] == 1.0)
    assert np.all((g["w_dir"] > 0) & (g["w_dir"] <= 1))
    assert np.all((g["w"] > 0) & (g["w"] <= 1))


def test_union_symmetric_and_dominates(graph):
    idx, _, g = graph
    S = g["union"]
    assert (abs(S - S.T) > 0).nnz == 0
    n = idx.shape[0]
    for i in range(0, n, 37):
        for jj, j in enumerate(idx[i]):
            assert S[i, j] >= g["w_dir"][i, jj] - 1e-15


def test_csr_sorted_and_pruned(graph):
    _, _, g = graph
    rp, col, q = g["row_ptr"], g["col"], g["q"]
    for i in range(len(rp) - 1):
        assert np.all(np.diff(col[rp[i]:rp[i + 1]]) > 0)
    assert np.all(200 * q.astype(np.int64) >= Q_ONE)
    # pruned entries are exactly those with T q < 2^24
    S = g["union"]
    qa = np.rint(Q_ONE * S.data / S.data.max())
    assert len(col) == int(np.count_nonzero(200 * qa >= Q_ONE))
    assert g["w_max"] == 1.0


def test_hand_sigma_closed_form():
    # row distances (rho, rho+s, ..., rho+s) with k entries: the sum is
    # 1 + (k-1) exp(-s/sigma) = log2 k  =>  sigma = s / ln((k-1)/(log2 k - 1))
    for k, rho, s in [(4, 1.0, 0.5), (8, 2.0, 0.25), (15, 0.3, 1.7)]:
        dist = np.array([[rho] + [rho + s] * (k - 1)])
        _, sigma = fuzzy.smooth_knn(dist, k)
        expect = s / np.log((k - 1) / (np.log2(k) - 1))
        np.testing.assert_allclose(sigma[0], expect, rtol=1e-12)


def test_sigma_floor_when_unsolvable():
    # three points tied at rho already exceed log2 4 = 2: sigma -> floor
    dist = np.array([[1.0, 1.0, 1.0, 3.0]])
    _, sigma = fuzzy.smooth_knn(dist, 4)
    assert sigma[0] == pytest.approx(1e-3 * dist.mean())
    w = fuzzy.directed_weights(dist, np.array([1.0]), sigma)
    np.testing.assert_allclose(w[0], [1, 1, 1, np.exp(-2.0 / sigma[0])])


def test_three_point_union_by_hand():
    # points 0, 1, 2 on a line at 0, 1, 3; k = 1: each point's nearest neighbour
    # gets weight 1; kNN: 0->1, 1->0, 2->1.  Union: (0,1)=1+1-1=1, (1,2)=1.
    idx = np.array([[1], [0], [1]])
    dist = np.array([[1.0], [1.0], [2.0]])
    g = fuzzy.build_csr(idx, dist, n_epochs=10, k=2)
    assert list(g["row_ptr"]) == [0, 1, 3, 4]
    assert list(g["col"]) == [1, 0, 2, 1]
    assert np.all(g["w"] == 1.0) and np.all(g["q"] == Q_ONE)


def test_union_formula_two_directions():
    # k = 2 on 3 points; directed weights chosen directly
    idx = np.array([[1, 2], [0, 2], [1, 0]])
    w_dir = np.array([[1.0, 0.3], [1.0, 0.6], [1.0, 0.2]])
    S = fuzzy.union_matrix(idx, w_dir, 3).toarray()
    expect = np.array([[0, 1.0, 0.3 + 0.2 - 0.06],
                       [1.0, 0, 0.6 + 1.0 - 0.6],
                       [0.3 + 0.2 - 0.06, 1.0, 0]])
    np.testing.assert_allclose(S, expect, rtol=1e-15)
