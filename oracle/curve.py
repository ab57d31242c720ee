"""Fit of the low-dimensional similarity curve (oracle side).

Section 2.3 states that UMAP fits its output-kernel parameters by Gauss-Newton
instead of SciPy's curve fitting.  The curve is Phi(x) = 1 / (1 + a x^(2b))
and the target, for the given min_dist and spread, is
psi(x) = 1 for x < min_dist and exp(-(x - min_dist) / spread) otherwise,
sampled at 300 equally spaced x in [0, 3 * spread] (UMAP's grid).
The least-squares problem in (a, b) is solved by Gauss-Newton steps on the
normal equations, each step halved until the residual norm decreases.
"""
from __future__ import annotations

import numpy as np


def target_curve(spread: float, min_dist: float, n_grid: int = 300):
    x = np.linspace(0.0, 3.0 * spread, n_grid)
    y = np.where(x < min_dist, 1.0, np.exp(-(x - min_dist) / spread))
    return x, y


def phi(x, a, b):
    x = np.asarray(x, dtype=np.float64)
    x2b = np.where(x > 0.0, np.power(np.where(x > 0.0, x, 1.0), 2.0 * b), 0.0)
    return 1.0 / (1.0 + a * x2b)


def find_ab(spread: float = 1.0, min_dist: float = 0.1, n_grid: int = 300,
            max_iter: int = 200, tol: float = 1e-14):
    x, y = target_curve(spread, min_dist, n_grid)
    pos = x > 0.0
    lnx = np.where(pos, np.log(np.where(pos, x, 1.0)), 0.0)

    def resid(a, b):
        return phi(x, a, b) - y

    a, b = 1.0, 1.0
    r = resid(a, b)
    cost = float(r @ r)
    for _ in range(max_iter):
        x2b = np.where(pos, np.exp(2.0 * b * lnx), 0.0)
        den = 1.0 + a * x2b
        Ja = -x2b / den ** 2
        Jb = -a * x2b * 2.0 * lnx / den ** 2
        J = np.stack([Ja, Jb], axis=1)
        step = np.linalg.solve(J.T @ J, -(J.T @ r))
        lam = 1.0
        while lam > 1e-12:
            a_new, b_new = a + lam * step[0], b + lam * step[1]
            if a_new > 0.0 and b_new > 0.0:
                r_new = resid(a_new, b_new)
                c_new = float(r_new @ r_new)
                if c_new < cost:
                    break
            lam *= 0.5
        else:
            break
        done = cost - c_new <= tol * max(cost, 1e-300)
        a, b, r, cost = a_new, b_new, r_new, c_new
        if done:
            break
    return a, b
