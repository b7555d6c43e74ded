"""Scalar and set operators by their definitions, in FP64 (test infrastructure).

ORACLE: test infrastructure only (``tests/``, ``smoke()``, the bench's CPU
baseline); shares no code with the CUDA solver.

* ``prox_cost``: the proximal map of the per-asset trading cost of Eq. 1,
  gamma * (c1 |z| + c2 |z|^d), computed from its optimality condition by
  bisection (not by a closed form).
* ``project_l1``: Euclidean projection onto the budget set ||w||_1 <= r of
  Eq. 3 by sorting (Duchi, Shalev-Shwartz, Singer, Chandra, ICML 2008).
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
