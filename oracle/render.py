"""Circle-splatting renderer of an embedding (oracle side, FP64).

The paper (Section 2.4, its GPU rendering pipeline) renders each frame by
splatting every point as a disc of radius R with a linear falloff, adding
premultiplied colour into a framebuffer by scatter-add, then dividing the
colour by the accumulated alpha and compositing over the background.
Restated here:

* pixel space: px = (x - x0) s, py = (y - y0) s; pixel (u, v) (column u, row
  v, row v growing with y) has its centre at (u + 1/2, v + 1/2).
* each point i with colour c_i (RGB in [0, 1]) and opacity alpha adds, to
  every pixel whose centre lies at distance r < R from (px_i, py_i),
      A(u, v) += alpha w,   C(u, v) += alpha w c_i,   w = max(0, 1 - r / R).
* resolve: where A > 0, colour = C / A and coverage = min(1, A); the pixel is
  coverage * colour + (1 - coverage) * background; elsewhere the background.
  Channels are stored as round(255 * clamp(value, 0, 1)) (half up).
* view: (x0, y0, s) given, or fitted to the points' bounding box with a 5%
  margin on each side, the larger extent filling the frame, the box centred.
"""
from __future__ import annotations

import numpy as np


def fit_view(Y: np.ndarray, width: int, height: int, margin: float = 0.05):
    """(x0, y0, s) placing the points' bounding box, grown by `margin` of its
    extent on each side, in a width x height frame, centred."""
    Y = np.asarray(Y, np.float64)
    lo, hi = Y.min(axis=0), Y.max(axis=0)
    ext = np.maximum(hi - lo, 1e-12) * (1.0 + 2.0 * margin)
    s = min(width / ext[0], height / ext[1])
    cx, cy = 0.5 * (lo + hi)
    return cx - 0.5 * width / s, cy - 0.5 * height / s, s


def accumulate(Y, rgb, width: int, height: int, radius: float, alpha: float, view):
    """The premultiplied accumulators A (H x W) and C (H x W x 3)."""
    Y = np.asarray(Y, np.float64)
    rgb = np.asarray(rgb, np.float64)
    x0, y0, s = view
    A = np.zeros((height, width))
    C = np.zeros((height, width, 3))
    px, py = (Y[:, 0] - x0) * s, (Y[:, 1] - y0) * s
    for i in range(len(Y)):
        u_lo, u_hi = int(np.floor(px[i] - radius)), int(np.ceil(px[i] + radius))
        v_lo, v_hi = int(np.floor(py[i] - radius)), int(np.ceil(py[i] + radius))
        for v in range(max(v_lo, 0), min(v_hi, height - 1) + 1):
            for u in range(max(u_lo, 0), min(u_hi, width - 1) + 1):
                r = np.hypot(u + 0.5 - px[i], v + 0.5 - py[i])
                w = max(0.0, 1.0 - r / radius)
                if w > 0.0:
                    A[v, u] += alpha * w
                    C[v, u] += alpha * w * rgb[i]
    return A, C


def resolve(A, C, background):
    """Colour / alpha, composited over the background; FP64 image H x W x 3."""
    bg = np.asarray(background, np.float64)
    out = np.broadcast_to(bg, C.shape).copy()
    m = A > 0.0
    col = C[m] / A[m][:, None]
    cov = np.minimum(1.0, A[m])[:, None]
    out[m] = cov * col + (1.0 - cov) * bg
    return out


def to_u8(img):
    """round(255 * clamp(value, 0, 1)), halves rounded up."""
    return np.floor(255.0 * np.clip(img, 0.0, 1.0) + 0.5).astype(np.uint8)


def render(Y, rgb, width: int, height: int, radius: float = 2.0, alpha: float = 1.0,
           background=(1.0, 1.0, 1.0), view=None):
    """The frame as uint8 H x W x 3, plus the FP64 image before storing."""
    view = fit_view(Y, width, height) if view is None else view
    A, C = accumulate(Y, rgb, width, height, radius, alpha, view)
    img = resolve(A, C, background)
    return to_u8(img), img


__all__ = ["fit_view", "accumulate", "resolve", "to_u8", "render"]
