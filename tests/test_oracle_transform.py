"""Pins for the oracle's transform of new points (not gpu).

The transform places each new point at the membership-weighted mean of its
training neighbours' coordinates, then runs ceil(T / 3) anchored epochs with
lr0 (1 - t / T').  Its parts (k-NN query, rho/sigma, directed weights, the
anchored epoch) are pinned elsewhere; these tests pin the two steps of its
own: the start, against weights that are known in closed form, and the
schedule, by recording the calls it makes.
"""
import math

import numpy as np
import pytest

from oracle import sgd


def _star(dists, idx, n_train=12, d=3, seed=0):
    """Training set with the points `idx` at Euclidean distances `dists` from
    the origin (each along its own axis direction, rotated), the rest far
    away; the single new point is the origin."""
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(n_train, d))
    X = 50.0 + X / np.linalg.norm(X, axis=1, keepdims=True)     # far from the origin
    for r, i in zip(dists, idx):
        v = rng.normal(size=d)
        X[i] = r * v / np.linalg.norm(v)
    Yt = rng.uniform(-7.0, 7.0, size=(n_train, 2))
    return X, Yt, np.zeros((1, d))


def test_start_is_the_closed_form_weighted_mean():
    # k = 4 with distances (rho, rho + s, rho + s, rho + s): the row sum
    # 1 + 3 exp(-s / sigma) = log2 4 = 2 gives exp(-s / sigma) = 1/3 exactly,
    # so the weights are (1, 1/3, 1/3, 1/3).  The nearest point has the
    # highest index, so the index sort inside the transform moves it.
    X, Yt, Xn = _star([1.0, 1.5, 1.5, 1.5], [9, 2, 4, 7])
    Y0 = sgd.transform(X, Yt, Xn, k=4, n_epochs=0, ab=(1.577, 0.895))
    want = (1.0 * Yt[9] + (Yt[2] + Yt[4] + Yt[7]) / 3.0) / (1.0 + 3.0 / 3.0)
    assert np.allclose(Y0[0], want, rtol=0, atol=1e-12)
    # an unnormalised sum, or the weights on the wrong neighbours, is far off
    assert not np.allclose(Y0[0], Yt[9] + (Yt[2] + Yt[4] + Yt[7]) / 3.0, atol=1e-3)
    assert not np.allclose(Y0[0], (Yt[2] + (Yt[9] + Yt[4] + Yt[7]) / 3.0) / 2.0, atol=1e-3)


def test_start_with_unit_weights_is_the_plain_mean():
    # k = 2 at equal distances: both excesses are 0, so both weights are 1
    X, Yt, Xn = _star([2.0, 2.0], [3, 8])
    Y0 = sgd.transform(X, Yt, Xn, k=2, n_epochs=0, ab=(1.577, 0.895))
    assert np.allclose(Y0[0], 0.5 * (Yt[3] + Yt[8]), rtol=0, atol=1e-12)


@pytest.mark.parametrize("T", [1, 2, 3, 4, 200])
def test_anchored_schedule(monkeypatch, T):
    X, Yt, Xn = _star([1.0, 1.5, 1.5, 1.5], [9, 2, 4, 7])
    start = sgd.transform(X, Yt, Xn, k=4, n_epochs=0, ab=(1.577, 0.895))
    calls = []

    def record(Y_train, Y_new, row_ptr, col, q, a, b, lr, neg, t, seed, **kw):
        calls.append((t, lr, neg, seed, np.array(Y_new, copy=True)))
        # the new point's entries: its neighbours in index order, with
        # schedule words round(2^24 w) of the closed-form weights
        assert list(np.asarray(row_ptr)) == [0, 4]
        assert list(np.asarray(col)) == [2, 4, 7, 9]
        assert list(np.asarray(q)) == [5592405, 5592405, 5592405, 1 << 24]
        return np.asarray(Y_new) + 1.0          # a marker the next call must see

    monkeypatch.setattr(sgd, "anchored_epoch", record)
    lr0 = 0.75
    Y = sgd.transform(X, Yt, Xn, k=4, n_epochs=T, ab=(1.577, 0.895), lr0=lr0, neg=3, seed_neg=17)
    Tp = math.ceil(T / 3)
    assert [c[0] for c in calls] == list(range(Tp))
    for t, lr, neg, seed, _ in calls:
        assert lr == pytest.approx(lr0 * (1.0 - t / Tp), rel=0, abs=1e-15)
        assert (neg, seed) == (3, 17)
    # the first epoch starts from the weighted mean; each later one from the
    # previous epoch's output; the result is the last output
    expect = np.array(start, copy=True)
    for _, _, _, _, y_in in calls:
        assert np.array_equal(y_in, expect)
        expect = expect + 1.0
    assert np.array_equal(Y, expect)
