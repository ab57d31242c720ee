"""Pins for the oracle's circle-splatting renderer (not gpu)."""
import math

import numpy as np
import pytest

from oracle import render


def test_single_splat_weights_by_hand():
    # a point at the centre of pixel (10, 7): weights 1 - r / R at the
    # neighbouring centres
    Y = np.array([[10.5, 7.5]])
    A, C = render.accumulate(Y, [[1.0, 0.0, 0.0]], 20, 15, radius=3.0, alpha=1.0, view=(0.0, 0.0, 1.0))
    assert A[7, 10] == pytest.approx(1.0)
    assert A[7, 11] == pytest.approx(2.0 / 3.0)
    assert A[8, 11] == pytest.approx(1.0 - math.sqrt(2.0) / 3.0)
    assert A[9, 12] == pytest.approx(1.0 - math.sqrt(8.0) / 3.0)
    assert A[7, 13] == 0.0 and A[10, 10] == 0.0          # r = 3 = R: weight 0
    assert np.array_equal(C[:, :, 0], A) and not C[:, :, 1:].any()
    assert A[7, 9] == A[7, 11] and A[6, 10] == A[8, 10]  # symmetric about the centre


def test_total_weight_is_the_cone_volume():
    R = 40.0
    Y = np.array([[60.5, 60.5]])
    A, _ = render.accumulate(Y, [[1.0, 1.0, 1.0]], 121, 121, radius=R, alpha=1.0, view=(0.0, 0.0, 1.0))
    assert A.sum() == pytest.approx(math.pi * R * R / 3.0, rel=2e-3)


def test_premultiplied_mean_colour_and_coverage():
    Y = np.array([[5.5, 5.5], [5.5, 5.5]])
    rgb = np.array([[1.0, 0.0, 0.0], [0.0, 0.0, 1.0]])
    bg = (0.2, 0.3, 0.4)
    A, C = render.accumulate(Y, rgb, 12, 12, radius=4.0, alpha=0.5, view=(0.0, 0.0, 1.0))
    img = render.resolve(A, C, bg)
    m = A > 0
    assert np.allclose(C[m] / A[m][:, None], [0.5, 0.0, 0.5])
    # centre: A = 1, full coverage; a pixel at r = 3: A = 1/4, a quarter of the
    # mean colour over three quarters of the background
    assert np.allclose(img[5, 5], [0.5, 0.0, 0.5])
    assert A[5, 8] == pytest.approx(0.25)
    assert np.allclose(img[5, 8], 0.25 * np.array([0.5, 0.0, 0.5]) + 0.75 * np.array(bg))
    assert np.allclose(img[0, 0], bg)                   # uncovered: the background


def test_fit_view_frames_the_points():
    g = np.random.default_rng(3)
    Y = g.normal(size=(500, 2)) * [3.0, 1.0] + [10.0, -4.0]
    x0, y0, s = render.fit_view(Y, 400, 300)
    P = (Y - [x0, y0]) * s
    assert P.min() > 0 and P[:, 0].max() < 400 and P[:, 1].max() < 300
    ext = (Y.max(0) - Y.min(0)) * s
    assert ext[0] == pytest.approx(400 / 1.1)           # the wider extent fills the frame, 5% margins
    lo, hi = P.min(0), P.max(0)
    assert (lo + hi)[0] / 2 == pytest.approx(200) and (lo + hi)[1] / 2 == pytest.approx(150)


def test_store_rounds_halves_up_and_clamps():
    v = np.array([0.5 / 255, 1.5 / 255, -0.1, 1.2, 254.49 / 255])
    assert list(render.to_u8(v)) == [1, 2, 0, 255, 254]
