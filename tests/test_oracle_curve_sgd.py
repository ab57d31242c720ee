"""Pins for the oracle's a,b fit, initialisation and SGD epoch (not gpu)."""
import numpy as np
import pytest
from scipy.optimize import curve_fit

import datagen
from conftest import golden_rows
from oracle import curve, fuzzy, knn as oknn, philox, sgd
from oracle.fuzzy import Q_ONE


# ---------------------------------------------------------------- a, b fit
@pytest.mark.parametrize("spread,min_dist", [(1.0, 0.1), (1.0, 0.5), (2.0, 0.25), (1.0, 0.01)])
def test_find_ab_matches_scipy_curve_fit(spread, min_dist):
    x, y = curve.target_curve(spread, min_dist)
    (a_ref, b_ref), _ = curve_fit(lambda xx, a, b: 1.0 / (1.0 + a * xx ** (2 * b)), x, y,
                                  p0=(1.0, 1.0), maxfev=20000)
    a, b = curve.find_ab(spread, min_dist)
    assert a == pytest.approx(a_ref, rel=1e-4)
    assert b == pytest.approx(b_ref, rel=1e-4)


@pytest.mark.parametrize("row", golden_rows("umap_ab.txt"))
def test_find_ab_quoted_values(row):
    spread, min_dist, a_q, b_q, tol = map(float, row)
    a, b = curve.find_ab(spread, min_dist)
    assert abs(a - a_q) < tol and abs(b - b_q) < tol


# ---------------------------------------------------------------- init
def test_init_range_uniform_and_fp32_exact():
    Y = sgd.init_embedding(100_000, seed=11, init_range=10.0)
    assert Y.min() >= -10.0 and Y.max() < 10.0
    # Y = u * 2R / 2^24 - R exactly, with u a 24-bit integer
    u = (Y + 10.0) * 2.0 ** 24 / 20.0
    assert np.all(u == np.rint(u)) and u.min() >= 0 and u.max() < 2 ** 24
    counts = np.histogram(Y[:, 0], bins=50, range=(-10, 10))[0]
    assert counts.min() > 0.85 * counts.mean()
    assert abs(np.corrcoef(Y[:, 0], Y[:, 1])[0, 1]) < 0.02


# ---------------------------------------------------------------- epoch
def _small_graph(n=40, k=6, T=50, seed=0):
    X, _ = datagen.mixture(n, 5, 3, seed=seed)
    idx, dist = oknn.knn(X, k)
    return fuzzy.build_csr(idx, dist, T, k)


def _row_loss(Yi, i, others_att, others_rep, a, b):
    """Cross-entropy terms of row i as a function of Y_i alone (eps = 0)."""
    L = 0.0
    for yj in others_att:
        d = ((Yi - yj) ** 2).sum()
        L += np.log1p(a * d ** b)                      # -log Phi
    for ym in others_rep:
        d = ((Yi - ym) ** 2).sum()
        L += -np.log(1.0 - 1.0 / (1.0 + a * d ** b))   # -log(1 - Phi)
    return L


def test_epoch_force_matches_central_differences():
    g = _small_graph()
    n = len(g["row_ptr"]) - 1
    a, b = 1.577, 0.895
    Y = np.random.default_rng(5).uniform(-3, 3, size=(n, 2))
    t, neg, seed = 0, 5, 99
    Y1 = sgd.epoch(Y, g["row_ptr"], g["col"], g["q"], a, b, 1.0, neg, t, seed, eps=0.0, clip=None)
    G = Y1 - Y
    act = sgd.active_mask(g["q"], t)
    heads = np.repeat(np.arange(n), np.diff(g["row_ptr"]))
    h = 1e-6
    checked = 0
    for i in range(n):
        es = np.nonzero(act & (heads == i))[0]
        att = [Y[g["col"][e]] for e in es]
        rep = []
        for e in es:
            for u in philox.negative_words(np.array([e]), t, neg, seed)[0]:
                m = int(philox.negative_index(np.array([u]), n)[0])
                if m != i:
                    rep.append(Y[m])
        fd = np.zeros(2)
        for c in range(2):
            Yp, Ym = Y[i].copy(), Y[i].copy()
            Yp[c] += h
            Ym[c] -= h
            fd[c] = -(_row_loss(Yp, i, att, rep, a, b) - _row_loss(Ym, i, att, rep, a, b)) / (2 * h)
        np.testing.assert_allclose(G[i], fd, rtol=1e-6, atol=1e-7)
        checked += len(es)
    assert checked > n  # plenty of active entries were exercised


def test_coefficients_equal_symbolic_gradient():
    sympy = pytest.importorskip("sympy")
    a, b = sympy.Rational(1577, 1000), sympy.Rational(895, 1000)
    x, y = sympy.symbols("x y", real=True)
    d = x ** 2 + y ** 2  # Y_i - Y_j = (x, y)
    att = sympy.log(1 + a * d ** b)
    rep = -sympy.log(1 - 1 / (1 + a * d ** b))
    for (xv, yv) in [(0.3, -1.2), (2.0, 0.5), (-0.01, 0.02)]:
        dv = xv * xv + yv * yv
        ga = [-float(sympy.diff(att, s).subs({x: xv, y: yv})) for s in (x, y)]
        gr = [-float(sympy.diff(rep, s).subs({x: xv, y: yv})) for s in (x, y)]
        ca = sgd.attraction_coeff(np.array(dv), 1.577, 0.895)
        cr = sgd.repulsion_coeff(np.array(dv), 1.577, 0.895, eps=0.0)
        np.testing.assert_allclose([ca * xv, ca * yv], ga, rtol=1e-12)
        np.testing.assert_allclose([cr * xv, cr * yv], gr, rtol=1e-12)


def test_clip_bounds_each_term():
    g = _small_graph(60, 8, 20, seed=2)
    n = len(g["row_ptr"]) - 1
    Y = np.random.default_rng(1).uniform(-0.05, 0.05, size=(n, 2))  # tiny d: huge raw forces
    Y1, G, A = sgd.epoch(Y, g["row_ptr"], g["col"], g["q"], 1.577, 0.895, 1.0, 5, 0, 3,
                         return_parts=True)
    act = sgd.active_mask(g["q"], 0)
    heads = np.repeat(np.arange(n), np.diff(g["row_ptr"]))
    terms = np.bincount(heads[act], minlength=n) * 6
    assert np.all(np.abs(G) <= 4.0 * terms[:, None] + 1e-12)
    assert np.abs(G).max() > 4.0  # clipping was actually exercised on sums


def test_coincident_points_contribute_nothing():
    # two coincident points joined by an always-active edge, no negatives
    rp = np.array([0, 1, 2])
    col = np.array([1, 0])
    q = np.array([Q_ONE, Q_ONE], dtype=np.uint64)
    Y = np.array([[1.0, 2.0], [1.0, 2.0]])
    Y1 = sgd.epoch(Y, rp, col, q, 1.5, 0.9, 1.0, 0, 0, 0)
    assert np.array_equal(Y1, Y)


def test_activation_count_closed_form():
    q = np.array([0, 1, 83886, 83887, 1 << 23, (1 << 24) - 1, 1 << 24, 12345678], np.uint64)
    T = 200
    fired = sum(sgd.active_mask(q, t).astype(int) for t in range(T))
    assert np.array_equal(fired, sgd.active_count(q, T).astype(int))
    assert fired[-2] == T and fired[0] == 0 and fired[2] == 0 and fired[3] == 1


def test_self_negative_skipped():
    # one point: every negative maps to itself and must be skipped
    rp = np.array([0, 1, 1])
    col = np.array([1])
    q = np.array([Q_ONE], np.uint64)
    Y = np.array([[0.0, 0.0], [3.0, 4.0]])
    # n = 2: negatives are 0 or 1; compare against explicit enumeration
    Y1 = sgd.epoch(Y, rp, col, q, 1.0, 1.0, 0.5, 8, 0, 7)
    u = philox.negative_words(np.array([0]), 0, 8, 7)[0]
    m = philox.negative_index(u, 2)
    n_rep = int(np.count_nonzero(m == 1))
    d = 25.0
    att = -2 * 1 * 1 * d ** 0 / (1 + d) * np.array([-3.0, -4.0])
    rep = 2 / ((1e-3 + d) * (1 + d)) * np.array([-3.0, -4.0])
    expect = 0.5 * (np.clip(att, -4, 4) + n_rep * np.clip(rep, -4, 4))
    np.testing.assert_allclose(Y1[0], expect, rtol=1e-14)
    assert 0 < n_rep < 8


def test_fit_small_mixture_quality():
    from oracle import metrics
    X, _ = datagen.mixture(1000, 50, 10, seed=0)
    Y, graph = sgd.fit(X, k=15, n_epochs=100)
    rows = np.arange(0, 1000, 5)
    r, tw = metrics.quality(X, Y, 15, rows, knn_x=graph["knn_idx"][rows])
    assert r > 10 * 15 / 1000  # an order of magnitude above a random embedding
    assert tw > 0.9


def test_epoch_rows_equals_full_epoch():
    g = _small_graph(200, 8, 50, seed=3)
    n = len(g["row_ptr"]) - 1
    Y = np.random.default_rng(9).uniform(-5, 5, size=(n, 2))
    full = sgd.epoch(Y, g["row_ptr"], g["col"], g["q"], 1.577, 0.895, 0.8, 5, 4, 21)
    rows = np.array([0, 3, 77, n - 1])
    part = sgd.epoch_rows(Y, g["row_ptr"], g["col"], g["q"], rows, 1.577, 0.895, 0.8, 5, 4, 21)
    np.testing.assert_allclose(part, full[rows], rtol=1e-13, atol=1e-13)
