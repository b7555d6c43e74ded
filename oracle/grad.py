"""Derivatives of the optimal portfolio with respect to the problem data, FP64
(test infrastructure).

ORACLE: test infrastructure only; shares no code with the CUDA solver.

At the optimum x*(theta) of the scaled model (``oracle.model``) the active
pieces (dead trades, zero holdings, active budget rows, active exposure rows)
are fixed in a neighbourhood of theta when strict complementarity holds, and
x* is the solution of the smooth, equality-constrained reduced problem of
``oracle.active``:  x = S v + x_fix(theta),  r(v, theta) + E^T nu = 0,
E v = e(theta), with r the gradient of the smooth reduced objective.  The
implicit function theorem then gives the directional derivative
    [H  E^T] [dv ]   [-(d/dt) r(v*, theta + t delta)]
    [E   0 ] [dnu] = [ (d/dt) e(theta + t delta)    ],   dx = S dv + (d/dt) x_fix,
with H the Hessian of the reduced objective, the dense KKT matrix solved by
LAPACK.  The t-derivatives of r, e and x_fix at fixed v are taken by central
differences of those functions themselves (they are polynomial in alpha, F,
D, s, q, so the differences are exact up to rounding; smooth in w0 and w_T on
live trades): no hand-derived partial derivative enters, so this oracle is
independent of the adjoint formulas of the CUDA path.
"""
from __future__ import annotations

from dataclasses import replace

import numpy as np

from .active import hessian_grad
from .model import Scaled

PARAMS = ("alpha", "F", "D", "s", "q", "w0")
MULTI_PARAMS = PARAMS + ("wT",)   # the fixed final portfolio of Eq. 4 (multi-period only)


def _fixed_sources(sc: Scaled, red):
    """Which parameter each fixed holding equals: 1 = w0, 2 = w_T, 0 = zero."""
    src = np.zeros(red.x_fix.shape, dtype=np.int8)
    fixed = ~red.free_mask
    nz = fixed & (red.x_fix != 0)
    w0b = np.broadcast_to(sc.w0, red.x_fix.shape)
    src[nz & (red.x_fix == w0b)] = 1
    if sc.multi:
        wTb = np.broadcast_to(sc.wT, red.x_fix.shape)
        src[nz & (src == 0) & (red.x_fix == wTb)] = 2
    return src


def _x_fix(sc: Scaled, src):
    xf = np.zeros(src.shape)
    xf[src == 1] = np.broadcast_to(sc.w0, src.shape)[src == 1]
    if sc.multi:
        xf[src == 2] = np.broadcast_to(sc.wT, src.shape)[src == 2]
    return xf


def _rhs_e(sc: Scaled, red, x_fix):
    """Right-hand sides of the reduced equalities, in the row order of red.E."""
    e = []
    for p in range(sc.P):
        if red.budget[p]:
            e.append(1.0 - float(np.sum(np.abs(x_fix[p]))))
    for (p, j, bound, side) in red.box:
        e.append(bound - float(sc.A[j] @ x_fix[p]))
    return np.array(e)


def jvp(prob, sol, name: str, delta, h: float = None) -> np.ndarray:
    """dx*/dtheta applied to the direction ``delta`` of parameter ``name``
    (one of alpha, F, D, s, q, w0, and wT for a multi-period problem),
    shape (P, n).  ``sol`` is a polished ``oracle.solve`` result (it carries
    the reduced problem)."""
    if name not in (MULTI_PARAMS if int(getattr(prob, "T", 0)) >= 2 else PARAMS):
        raise ValueError(name)
    red = sol.reduced
    if red is None:
        raise ValueError("the solution has no active-set reduction (polish failed)")
    sc = Scaled(prob)
    src = _fixed_sources(sc, red)
    x = sol.x
    cnt = np.asarray(red.S.sum(axis=0)).ravel()
    v = np.asarray(red.S.T @ x.ravel()).ravel() / np.maximum(cnt, 1.0)
    _, H, _, _ = hessian_grad(sc, red, v)
    base = np.asarray(getattr(prob, name), dtype=np.float64)
    delta = np.asarray(delta, dtype=np.float64).reshape(base.shape)
    if h is None:
        scale = max(float(np.max(np.abs(base))), 1e-12) / max(float(np.max(np.abs(delta))), 1e-300)
        if name in ("w0", "wT"):
            z = sc.trades(x)
            live = np.abs(z[red.live]) if np.any(red.live) else np.array([1.0])
            h = 1e-4 * float(np.min(live)) / max(float(np.max(np.abs(delta))), 1e-300)
        else:
            h = 1e-3 * scale

    def at(t):
        p2 = replace(prob, **{name: base + t * delta})
        sc2 = Scaled(p2)
        xf = _x_fix(sc2, src)
        red2 = replace(red, x_fix=xf)
        r = hessian_grad(sc2, red2, v)[0]
        return r, _rhs_e(sc2, red2, xf), xf

    rp, ep, xp = at(h)
    rm, em, xm = at(-h)
    G = H.shape[0]
    E = red.E
    neq = E.shape[0]
    K = np.zeros((G + neq, G + neq))
    K[:G, :G] = H
    K[:G, G:] = E.T
    K[G:, :G] = E
    rhs = np.concatenate([-(rp - rm) / (2 * h), (ep - em) / (2 * h)])
    s = np.linalg.solve(K, rhs)
    dv = s[:G]
    return (red.S @ dv).reshape(sc.P, sc.n) + (xp - xm) / (2 * h)


def directional_vjp(prob, sol, g, name: str, delta) -> float:
    """<g, dx*/dtheta [delta]>: the directional derivative of L = <g, x*>."""
    return float(np.sum(np.asarray(g, dtype=np.float64).reshape(sol.x.shape) * jvp(prob, sol, name, delta)))
