"""Independent checkers used to pin the oracle (test-side only).

Nothing here calls the oracle or the CUDA path.  Each routine solves a piece
of problem (2) by a different, textbook method:
  - dense grid search + Newton polish for one quartic on an interval;
  - a log-barrier interior-point method (Boyd and Vandenberghe, Convex
    Optimization, Sec. 11.3) for whole small instances of eq. (2);
  - closed-form solutions of special cases of eq. (2).
"""
from __future__ import annotations

import math

import numpy as np


def quartic_value(A, B, C, D, x):
    return (((A * x + B) * x + C) * x + D) * x


def quartic_argmin_grid(A, B, C, D, lo, hi, pts=100_001):
    """Minimiser of A x^4 + B x^3 + C x^2 + D x on [lo, hi] by a dense grid and
    a safeguarded Newton polish on the derivative around the best grid
    points.  Returns (x, value, second_best_gap) where the gap is the value
    difference to the best point of the other basin (for near-tie checks)."""
    xs = np.linspace(lo, hi, pts)
    fv = quartic_value(A, B, C, D, xs)
    cand = [lo, hi]
    # local minima of the sampled values
    idx = np.where((fv[1:-1] <= fv[:-2]) & (fv[1:-1] <= fv[2:]))[0] + 1
    h = (hi - lo) / (pts - 1)
    for i in idx:
        a, b = max(lo, xs[i] - h), min(hi, xs[i] + h)
        x = xs[i]
        for _ in range(100):
            g = ((4 * A * x + 3 * B) * x + 2 * C) * x + D
            gg = (12 * A * x + 6 * B) * x + 2 * C
            if gg <= 0:
                break
            xn = x - g / gg
            if not (a <= xn <= b):
                break
            if abs(xn - x) <= 1e-16 * max(1.0, abs(x)):
                x = xn
                break
            x = xn
        cand.append(x)
    cand = np.array(cand)
    vals = quartic_value(A, B, C, D, cand)
    o = np.argsort(vals, kind="stable")
    best = cand[o[0]]
    gap = math.inf
    for j in o[1:]:
        if abs(cand[j] - best) > 1e-6 * max(1.0, abs(best)):
            gap = vals[j] - vals[o[0]]
            break
    return best, vals[o[0]], gap


# ---------------------------------------------------------------------------
# log-barrier interior point for eq. (2)
# ---------------------------------------------------------------------------
class _Layout:
    """Variables of eq. (2) with the copy constraint eliminated: x_1^(i) once
    per source, then x_k^(i,j) for k >= 2."""

    def __init__(self, n, m, q):
        self.n, self.m, self.q = n, m, q
        self.nv = m + m * q * (n - 1)

    def expand(self, v):
        n, m, q = self.n, self.m, self.q
        x = np.empty((m, q, n))
        x[:, :, 0] = v[:m][:, None]
        x[:, :, 1:] = v[m:].reshape(m, q, n - 1)
        return x

    def jac(self):
        """Sparse-ish map: dx[i,j,k]/dv as a dense (m*q*n, nv) matrix."""
        n, m, q = self.n, self.m, self.q
        J = np.zeros((m * q * n, self.nv))
        for i in range(m):
            for j in range(q):
                J[(i * q + j) * n + 0, i] = 1.0
                for k in range(1, n):
                    J[(i * q + j) * n + k, m + (i * q + j) * (n - 1) + (k - 1)] = 1.0
        return J


def barrier_solve(prob, t_final=1e13, x0=None):
    """Solves eq. (2) by the barrier method: minimise t f(x) - sum log(-h(x))
    for t = 1, 10, 100, ... with damped Newton steps.  Returns x [m, q, n]."""
    n, m, q = prob.n, prob.m, prob.q
    L = _Layout(n, m, q)
    J = L.jac()
    f2, f1 = prob.f2.reshape(-1), prob.f1.reshape(-1)
    g2, g1, g0 = prob.g2.reshape(-1), prob.g1.reshape(-1), prob.g0.reshape(-1)
    lo = np.broadcast_to(prob.lo[:, None, :], (m, q, n)).reshape(-1)
    hi = np.broadcast_to(prob.hi[:, None, :], (m, q, n)).reshape(-1)
    y = prob.y
    capped = [i for i in range(m) if np.isfinite(prob.c[i])]

    if x0 is None:
        v = np.empty(L.nv)
        v[:m] = y[:, 0].max() / m + 0.05
        v[m:] = (np.broadcast_to(y[None, :, 1:], (m, q, n - 1)) / m + 0.05).reshape(-1)
    else:
        v = x0.copy()

    def parts(v):
        x = J @ v
        X = x.reshape(m, q, n)
        dem = X.sum(axis=0) - y                     # > 0
        gx = (g2 * x * x + g1 * x + g0).reshape(m, q, n)
        cap = np.array([[prob.c[i] - gx[i, j].sum() for j in range(q)] for i in capped]).reshape(len(capped), q)
        return x, dem, cap

    def feasible(v):
        x, dem, cap = parts(v)
        return np.all(x > lo) and np.all(x < hi) and np.all(dem > 0) and np.all(cap > 0)

    def phi(v, t):
        x, dem, cap = parts(v)
        if not (np.all(x > lo) and np.all(x < hi) and np.all(dem > 0) and np.all(cap > 0)):
            return math.inf
        obj = (f2 * x * x + f1 * x).sum() / q
        return t * obj - np.log(x - lo).sum() - np.log(hi - x).sum() - np.log(dem).sum() - np.log(cap).sum()

    assert feasible(v), "barrier: start point not strictly feasible"
    t = 1.0
    while True:
        for _ in range(200):
            x, dem, cap = parts(v)
            # gradient / Hessian in x-space, then chain to v
            gr = t * (2 * f2 * x + f1) / q + 1.0 / (hi - x) - 1.0 / (x - lo)
            hd = t * 2 * f2 / q + 1.0 / (hi - x) ** 2 + 1.0 / (x - lo) ** 2
            H = np.diag(hd)
            # demand: -log(sum_i x - y) per (j, k)
            for j in range(q):
                for k in range(n):
                    ids = [(i * q + j) * n + k for i in range(m)]
                    d = dem[j, k]
                    gr[ids] -= 1.0 / d
                    H[np.ix_(ids, ids)] += 1.0 / d ** 2
            # capacity: -log(c - sum_k g) per (i, j)
            for a, i in enumerate(capped):
                for j in range(q):
                    ids = [(i * q + j) * n + k for k in range(n)]
                    cc = cap[a, j]
                    gp = 2 * g2[ids] * x[ids] + g1[ids]
                    gr[ids] += gp / cc
                    H[np.ix_(ids, ids)] += np.outer(gp, gp) / cc ** 2
                    H[ids, ids] += 2 * g2[ids] / cc
            gv = J.T @ gr
            Hv = J.T @ H @ J
            dv = -np.linalg.solve(Hv, gv)
            lam2 = -gv @ dv
            if lam2 / 2 <= 1e-14:
                break
            s, f0 = 1.0, phi(v, t)
            while phi(v + s * dv, t) > f0 + 0.25 * s * gv @ dv:
                s *= 0.5
                if s < 1e-20:
                    break
            v = v + s * dv
        if t >= t_final:
            break
        t *= 10.0
    return L.expand(v)


# ---------------------------------------------------------------------------
# closed forms
# ---------------------------------------------------------------------------
def waterfill_linear_capacity(f2, f1, g1, lo, hi, c, q):
    """Minimiser of (1/q) sum_k (f2 x^2 + f1 x) s.t. sum_k g1 x <= c, x in
    [lo, hi] (one source and scenario; g linear, g1 > 0).  KKT: x(gamma) =
    clamp(-(f1/q + gamma g1) / (2 f2/q)); gamma >= 0 by bisection."""
    def xg(gm):
        return np.clip(-(f1 / q + gm * g1) / (2 * f2 / q), lo, hi)
    if (g1 * xg(0.0)).sum() <= c:
        return xg(0.0), 0.0
    a, b = 0.0, 1.0
    while (g1 * xg(b)).sum() > c:
        b *= 2.0
    for _ in range(200):
        mid = 0.5 * (a + b)
        if (g1 * xg(mid)).sum() > c:
            a = mid
        else:
            b = mid
    return xg(b), b
