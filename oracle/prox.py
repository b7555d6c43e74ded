"""Scalar and set operators by their definitions, in FP64 (test infrastructure).

ORACLE: test infrastructure only (``tests/``, ``smoke()``, the bench's CPU
baseline); shares no code with the CUDA solver.

* ``prox_cost``: the proximal map of the per-asset trading cost of Eq. 1,
  gamma * (c1 |z| + c2 |z|^d), computed from its optimality condition by
  bisection (not by a closed form).
* ``project_l1``: Euclidean projection onto the budget set ||w||_1 <= r of
  Eq. 3 by sorting (Duchi, Shalev-Shwartz, Singer, Chandra, ICML 2008).
* ``prox_joint``: the proximal map of the trading cost of Eq. 1 and the
  budget set of Eq. 3 together (the joint primal prox), by bisection on the
  coordinate problems' right derivatives and on the budget multiplier.
"""
from __future__ import annotations

import numpy as np


def prox_cost(v, gamma, c1, c2, d):
    """argmin_z 0.5 (z - v)^2 + gamma (c1 |z| + c2 |z|^d), elementwise.

    The minimiser has the sign of v.  With r = |z| it is 0 when
    |v| <= gamma c1; otherwise r is the root of the increasing function
    r + gamma c2 d r^(d-1) - (|v| - gamma c1) on [0, |v| - gamma c1],
    found here by bisection to the last bit.
    """
    v = np.asarray(v, dtype=np.float64)
    gamma, c1, c2 = (np.broadcast_to(np.asarray(a, dtype=np.float64), v.shape)
                     for a in (gamma, c1, c2))
    a = np.abs(v) - gamma * c1
    out = np.zeros_like(v)
    act = a > 0
    lo = np.zeros(int(act.sum()))
    hi = a[act].copy()
    gc = (gamma * c2)[act]
    tgt = a[act]
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        val = mid + gc * d * np.power(mid, d - 1.0) - tgt
        pos = val > 0
        hi = np.where(pos, mid, hi)
        lo = np.where(pos, lo, mid)
        if np.all(hi - lo <= 0.0 + 1e-300):
            break
    r = 0.5 * (lo + hi)
    out[act] = np.sign(v[act]) * r
    return out


def project_l1(v, radius: float = 1.0):
    """Euclidean projection of v onto {w : ||w||_1 <= radius} (sort based)."""
    v = np.asarray(v, dtype=np.float64)
    a = np.abs(v)
    if a.sum() <= radius:
        return v.copy()
    u = np.sort(a)[::-1]
    css = np.cumsum(u)
    j = np.arange(1, u.size + 1)
    cond = u - (css - radius) / j > 0
    rho = int(np.nonzero(cond)[0][-1])
    theta = (css[rho] - radius) / (rho + 1.0)
    return np.sign(v) * np.maximum(a - theta, 0.0)


def l1_threshold(v, radius: float = 1.0) -> float:
    """The shrinkage theta of ``project_l1`` (0 when v is inside the ball)."""
    v = np.asarray(v, dtype=np.float64)
    a = np.abs(v)
    if a.sum() <= radius:
        return 0.0
    u = np.sort(a)[::-1]
    css = np.cumsum(u)
    j = np.arange(1, u.size + 1)
    rho = int(np.nonzero(u - (css - radius) / j > 0)[0][-1])
    return float((css[rho] - radius) / (rho + 1.0))


def cost_conjugate(y, c1, c2, d):
    """phi*(y) for phi(z) = c1 |z| + c2 |z|^d, elementwise (Fenchel conjugate).

    0 when |y| <= c1; otherwise (|y| - c1) r (1 - 1/d) with
    r = ((|y| - c1) / (d c2))^(1/(d-1)); +inf when c2 = 0 and |y| > c1.
    """
    y = np.asarray(y, dtype=np.float64)
    c1 = np.broadcast_to(np.asarray(c1, dtype=np.float64), y.shape)
    c2 = np.broadcast_to(np.asarray(c2, dtype=np.float64), y.shape)
    a = np.abs(y) - c1
    out = np.zeros_like(y)
    act = a > 0
    with np.errstate(divide="ignore", invalid="ignore"):
        r = np.where(act & (c2 > 0), np.power(np.where(act, a, 0.0) / np.where(c2 > 0, d * c2, 1.0),
                                               1.0 / (d - 1.0)), 0.0)
    out[act] = a[act] * r[act] * (1.0 - 1.0 / d)
    out[act & (c2 <= 0)] = np.inf
    return out


def _cost_right_derivative(z, c1, c2, d):
    """Right derivative of c1 |z| + c2 |z|^d at z (elementwise)."""
    s = np.where(z >= 0.0, 1.0, -1.0)
    return c1 * s + c2 * d * np.power(np.abs(z), d - 1.0) * np.sign(z)


def prox_joint_coord(v, a, mu, gamma, c1, c2, d):
    """argmin_w 0.5 (w - v)^2 + gamma (c1 |w - a| + c2 |w - a|^d) + mu |w|,
    elementwise (the coordinate problem of the joint primal prox).

    The objective is strictly convex in w, so its minimiser is the smallest w
    whose right derivative
        (w - v) + gamma * phi'_+(w - a) + mu * sgn_+(w)      (sgn_+(0) = 1)
    is >= 0; found by bisection to the last bit on a bracket that holds v,
    a and 0 widened by the largest subgradient magnitude.
    """
    v, a, mu, gamma, c1, c2 = np.broadcast_arrays(*(np.asarray(x, dtype=np.float64)
                                                     for x in (v, a, mu, gamma, c1, c2)))
    span = np.abs(v) + np.abs(a) + gamma * (c1 + c2 * d * np.power(np.abs(v) + 2.0 * np.abs(a) + 1.0, d - 1.0)) \
        + mu + 1.0
    lo = np.minimum(np.minimum(v, a), 0.0) - span
    hi = np.maximum(np.maximum(v, a), 0.0) + span

    def rd(w):
        return (w - v) + gamma * _cost_right_derivative(w - a, c1, c2, d) + mu * np.where(w >= 0.0, 1.0, -1.0)

    for _ in range(400):
        mid = 0.5 * (lo + hi)
        pos = rd(mid) >= 0.0
        hi = np.where(pos, mid, hi)
        lo = np.where(pos, lo, mid)
        if np.all(np.nextafter(lo, np.inf) >= hi):
            break
    # the minimiser lies in (lo, hi]; a kink (0 or a) inside that interval is
    # the minimiser itself (the bisection toward 0 stops short of the subnormals)
    w = hi.copy()
    for k in (np.zeros_like(w), a):
        w = np.where((lo <= k) & (k <= hi), k, w)
    return w


def prox_joint(v, a, gamma, c1, c2, d, radius: float = 1.0):
    """Proximal map of gamma * sum_i phi_i(w_i - a_i) + indicator{||w||_1 <= radius}
    (the joint primal prox of the single-period model: trading cost of Eq. 1
    around w0 = a and the budget set of Eq. 3 in one operator).

    With mu >= 0 the multiplier of the budget constraint, the minimiser is
    w(mu) of ``prox_joint_coord``; mu = 0 when ||w(0)||_1 <= radius, else the
    root of the non-increasing function ||w(mu)||_1 - radius, found by
    bisection.  Returns (w, mu).
    """
    v = np.asarray(v, dtype=np.float64)
    a = np.broadcast_to(np.asarray(a, dtype=np.float64), v.shape)
    w = prox_joint_coord(v, a, 0.0, gamma, c1, c2, d)
    if np.abs(w).sum() <= radius:
        return w, 0.0
    # at mu_hi every coordinate is 0: |v - gamma phi'(-a)| <= mu_hi for every
    # element of the subdifferential
    c1b, c2b = (np.broadcast_to(np.asarray(x, dtype=np.float64), v.shape) for x in (c1, c2))
    mu_lo, mu_hi = 0.0, float(np.max(np.abs(v) + gamma * (c1b + c2b * d * np.power(np.abs(a), d - 1.0)))) + 1.0
    for _ in range(200):
        mid = 0.5 * (mu_lo + mu_hi)
        if np.abs(prox_joint_coord(v, a, mid, gamma, c1, c2, d)).sum() > radius:
            mu_lo = mid
        else:
            mu_hi = mid
        if mu_hi - mu_lo <= 1e-17 * max(mu_hi, 1e-300):
            break
    mu = 0.5 * (mu_lo + mu_hi)
    return prox_joint_coord(v, a, mu, gamma, c1, c2, d), mu
