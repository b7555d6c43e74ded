"""Active-set refinement of the interior-point solution (test infrastructure).

ORACLE: test infrastructure only; shares no code with the CUDA solver.

At the optimum of the scaled model (``oracle.model``) each piece of the
nonsmooth structure is either "on a kink" or smooth:
  * a trade z_{r,i} is zero (dead zone of the spread cost, Eq. 1 / Eq. 4) or
    has a fixed sign, so c1 |z| + c2 |z|^d is smooth in it;
  * a holding x_{p,i} is zero or has a fixed sign, so the budget
    ||x_p||_1 <= 1 (Eq. 3 / Eq. 6) is linear once the signs are known;
  * an exposure row (Eq. 2 / Eq. 5) is at U, at L, or inactive.
Given these sets (read from the interior-point multipliers) the optimum is
the minimiser of a smooth convex function under linear equalities. Dead
trades tie x_{r-1,i} = x_{r,i} (or x_1 = w0, x_{T-1} = w_T), zero holdings fix
x = 0; the remaining free groups v are found by Newton's method on the
equality-constrained KKT system (dense). The result is accepted only if the
independently evaluated relative KKT residual (``oracle.kkt``) certifies it.

The same reduced system gives the implicit-function derivatives used by
``oracle.grad``.
"""
from __future__ import annotations

import time
from dataclasses import dataclass
from typing import Optional

import numpy as np
import scipy.sparse as sp

from .kkt import evaluate
from .model import Scaled

ZFLOOR = 1e-14   # |z| used for the cost derivatives of a trade that is live but still at 0


@dataclass
class Reduced:
    """Reduced smooth problem: x = S v + x_fix, equalities E v = e."""
    S: sp.csr_matrix          # (P n, G) selection of free groups
    x_fix: np.ndarray         # (P, n) values of fixed holdings (0, w0 or w_T), 0 on free ones
    free_mask: np.ndarray     # (P, n) True where x_{p,i} is a free group member
    group: np.ndarray         # (P, n) group index (-1 if fixed)
    live: np.ndarray          # (R, n) True where the trade is nonzero
    sz: np.ndarray            # (R, n) trade signs (0 on dead)
    sx: np.ndarray            # (P, n) holding signs (0 on zero holdings)
    budget: np.ndarray        # (P,) budget active
    box: list                 # [(p, j, bound, side)] active exposure rows, side=+1 upper, -1 lower
    E: np.ndarray             # (neq, G)
    e: np.ndarray             # (neq,)


def _identify(sc: Scaled, x, st) -> Reduced:
    """Reduced problem for the activity state ``st`` (zero, dead, budget, upper,
    lower masks and forced signs sx_force / sz_force for newly freed pieces)."""
    P, R, n = sc.P, sc.R, sc.n
    zero, dead = st["zero"], st["dead"]
    sx = np.where(zero, 0.0, np.where(st["sx_force"] != 0, st["sx_force"], np.sign(x)))
    z = sc.trades(x)
    sz = np.where(dead, 0.0, np.where(st["sz_force"] != 0, st["sz_force"], np.sign(z)))
    group = -np.ones((P, n), dtype=np.int64)
    x_fix = np.zeros((P, n))
    free_mask = np.zeros((P, n), dtype=bool)
    G = 0
    for i in range(n):
        p = 0
        while p < P:
            q = p
            while q + 1 < P and dead[q + 1, i]:   # trade r = q+1 links x_q and x_{q+1}
                q += 1
            fixv = None
            if p == 0 and dead[0, i]:
                fixv = sc.w0[i]
            if sc.multi and q == P - 1 and dead[R - 1, i]:
                fixv = sc.wT[i] if fixv is None else fixv
            if np.any(zero[p:q + 1, i]):
                fixv = 0.0 if fixv is None else fixv
            if fixv is None:
                group[p:q + 1, i] = G
                free_mask[p:q + 1, i] = True
                G += 1
            else:
                x_fix[p:q + 1, i] = fixv
            p = q + 1
    rows, cols = np.nonzero(free_mask)
    S = sp.csr_matrix((np.ones(rows.size), (rows * n + cols, group[rows, cols])), shape=(P * n, G))
    # fixed holdings carry their sign into the budget; a free group shares one sign
    sx = np.where(free_mask, sx, np.sign(x_fix))
    for p in range(P):
        for i in np.nonzero(free_mask[p])[0]:
            if sx[p, i] == 0:
                sx[p, i] = 1.0 if x[p, i] >= 0 else -1.0
    box = []
    Erows, evals = [], []
    for p in range(P):
        if st["budget"][p]:
            row = S[p * n:(p + 1) * n].T @ sx[p]
            Erows.append(np.asarray(row).ravel())
            evals.append(1.0 - float(np.sum(np.abs(x_fix[p]))))
    for p in range(P):
        for j in range(sc.m):
            for side, flag, bound in ((1.0, st["upper"][p, j], sc.U[j]), (-1.0, st["lower"][p, j], sc.L[j])):
                if flag:
                    row = S[p * n:(p + 1) * n].T @ sc.A[j]
                    Erows.append(np.asarray(row).ravel())
                    evals.append(bound - float(sc.A[j] @ x_fix[p]))
                    box.append((p, j, bound, side))
    E = np.array(Erows).reshape(len(Erows), G)
    return Reduced(S=S, x_fix=x_fix, free_mask=free_mask, group=group, live=~dead, sz=sz, sx=sx,
                   budget=np.asarray(st["budget"]).copy(), box=box, E=E, e=np.array(evals))


def _x_of(sc, red, v):
    return (red.S @ v).reshape(sc.P, sc.n) + red.x_fix


def trade_jacobian(sc: Scaled, red: Reduced) -> sp.csr_matrix:
    """dz/dv for all (R n) trades (rows of dead trades are structurally zero)."""
    Dk = sp.kron(sp.csr_matrix(sc.Delta), sp.identity(sc.n, format="csr"), format="csr")
    return (Dk @ red.S).tocsr()


def hessian_grad(sc: Scaled, red: Reduced, v):
    """Gradient and Hessian of the smooth reduced objective in v."""
    x = _x_of(sc, red, v)
    G = red.S.shape[1]
    gx = sc.grad_f(x)                                  # (P, n)
    z = sc.trades(x)
    az = np.maximum(np.abs(z), ZFLOOR)
    live = red.live
    d = sc.d
    with np.errstate(divide="ignore", invalid="ignore"):
        gz = np.where(live, red.sz * (sc.c1 + d * sc.c2 * np.power(az, d - 1.0)), 0.0)
        hz = np.where(live, sc.c2 * d * (d - 1.0) * np.power(az, d - 2.0), 0.0)
    Jz = trade_jacobian(sc, red)
    grad = red.S.T @ gx.ravel() + Jz.T @ gz.ravel()
    H = np.zeros((G, G))
    for p in range(sc.P):
        Sp = red.S[p * sc.n:(p + 1) * sc.n]            # (n, G)
        Fsel = np.asarray((Sp.T @ sc.F))              # (G, k)
        H += 2.0 * sc.kappa * (Fsel @ sc.Omega @ Fsel.T)
        H += np.diag(np.asarray(Sp.T @ (2.0 * sc.kappa * sc.Dp[p])).ravel())
    H += (Jz.T @ sp.diags(hz.ravel()) @ Jz).toarray()
    return np.asarray(grad).ravel(), H, x, z


def _dual_from_chain(sc: Scaled, x, yA, nu_b, red: Reduced):
    """Trade multipliers y_D from stationarity
        g_p + y_{D,p} - y_{D,p+1} + n_p = 0,  g = grad f + A^T y_A,
    (y_{D,P} = 0 past the single period), with y_D on live trades fixed by the
    cost derivative, |y_D| <= c1 on dead trades, n_p = nu_b sx on nonzero
    holdings and |n_p| <= nu_b on zero holdings.  Feasible ranges are
    propagated forward per asset; where a range is empty the activity guess is
    wrong, and the returned flips say which piece to free:
    ("trade", r, i, sign) or ("hold", p, i, sign)."""
    P, R, n = sc.P, sc.R, sc.n
    g = sc.grad_f(x) + yA @ sc.A                     # (P, n)
    z = sc.trades(x)
    d = sc.d
    # the subdifferential is read off the point itself: a trade or holding that
    # sits on its kink gets the whole interval, whatever the activity guess said
    ztol = 1e-14 * max(1e-3, float(np.max(np.abs(z))))
    xtol = 1e-14 * max(1e-3, float(np.max(np.abs(x))))
    on_kink_z = (~red.live) | (np.abs(z) <= ztol)
    zero_x = (red.sx == 0) | (np.abs(x) <= xtol)
    sgz = np.where(red.sz != 0, red.sz, np.sign(z))
    ylive = sgz * (sc.c1 + d * sc.c2 * np.power(np.maximum(np.abs(z), ZFLOOR), d - 1.0))
    nb = np.array([nu_b[p] if red.budget[p] else 0.0 for p in range(P)])
    lo = np.where(on_kink_z, -sc.c1, ylive)
    hi = np.where(on_kink_z, sc.c1, ylive)
    nlo = np.where(zero_x, -nb[:, None], nb[:, None] * red.sx)
    nhi = np.where(zero_x, nb[:, None], nb[:, None] * red.sx)
    Ylo = np.zeros((P + 1, n))
    Yhi = np.zeros((P + 1, n))
    Ylo[0], Yhi[0] = lo[0], hi[0]
    flips = {}
    tol = 1e-13 * max(1.0, float(np.max(np.abs(g))))
    for p in range(P):
        a = Ylo[p] + g[p] + nlo[p]
        b = Yhi[p] + g[p] + nhi[p]
        if p + 1 < R:
            tlo, thi = lo[p + 1], hi[p + 1]
        else:
            tlo, thi = np.zeros(n), np.zeros(n)
        nlo_, nhi_ = np.maximum(a, tlo), np.minimum(b, thi)
        bad = nlo_ > nhi_ + tol
        for i in np.nonzero(bad)[0]:
            if i in flips:
                continue
            up = a[i] > thi[i]           # range lies above the target: y_{p+1} must grow
            if p + 1 < R and on_kink_z[p + 1, i]:
                flips[i] = ("trade", p + 1, i, 1.0 if up else -1.0)
            elif zero_x[p, i] and nb[p] > 0:
                flips[i] = ("hold", p, i, -1.0 if up else 1.0)
            elif on_kink_z[p, i]:
                flips[i] = ("trade", p, i, -1.0 if up else 1.0)
            elif zero_x[p, i]:
                flips[i] = ("hold", p, i, -1.0 if up else 1.0)
        # clamp so the propagation continues
        Ylo[p + 1] = np.where(bad, np.where(a > thi, thi, tlo), np.minimum(nlo_, nhi_))
        Yhi[p + 1] = np.where(bad, np.where(a > thi, thi, tlo), np.maximum(nlo_, nhi_))
    yD = np.zeros((P + 1, n))
    yD[P] = 0.0 if R == P else 0.5 * (Ylo[P] + Yhi[P])
    for p in range(P - 1, -1, -1):
        want_lo = yD[p + 1] - g[p] - nhi[p]
        want_hi = yD[p + 1] - g[p] - nlo[p]
        lo_p = np.maximum(want_lo, Ylo[p])
        hi_p = np.minimum(want_hi, Yhi[p])
        yD[p] = np.where(lo_p <= hi_p, 0.5 * (lo_p + hi_p), np.where(Ylo[p] > want_hi, Ylo[p], Yhi[p]))
    return yD[:R], list(flips.values())


def _newton(sc: Scaled, red: Reduced, x0, max_newton: int):
    """Newton's method on the equality-constrained reduced problem.  A step
    that would carry a live trade or a nonzero holding through its kink is cut
    at the kink and the piece is returned as blocking (primal active-set step).
    Returns (x, nu, blocked_trades (R, n) bool, blocked_holdings (P, n) bool)."""
    G = red.S.shape[1]
    v = np.asarray(red.S.T @ x0.ravel()).ravel()
    cnt = np.asarray(red.S.sum(axis=0)).ravel()
    v = v / np.maximum(cnt, 1.0)
    neq = red.E.shape[0]
    nu = np.zeros(neq)
    hold_live = red.free_mask & (red.sx != 0)
    nob_t = np.zeros((sc.R, sc.n), dtype=bool)
    nob_x = np.zeros((sc.P, sc.n), dtype=bool)
    for _ in range(max_newton):
        grad, H, x, z = hessian_grad(sc, red, v)
        K = np.zeros((G + neq, G + neq))
        K[:G, :G] = H
        K[:G, G:] = red.E.T
        K[G:, :G] = red.E
        rhs = np.concatenate([-grad, red.e - red.E @ v])
        sol = np.linalg.lstsq(K, rhs, rcond=None)[0] if neq > G else np.linalg.solve(K, rhs)
        dv, nu = sol[:G], sol[G:]
        dx = (red.S @ dv).reshape(sc.P, sc.n)
        dz = sc.Delta @ dx
        step = 1.0
        blocks = []
        for val, dval, mask, sg, kind in ((z, dz, red.live, red.sz, "t"), (x, dx, hold_live, red.sx, "x")):
            cross = mask & (sg * (val + dval) < 0)
            if np.any(cross):
                ratio = np.full(val.shape, np.inf)
                ratio[cross] = np.maximum(sg[cross] * val[cross], 0.0) / np.abs(dval[cross])
                rmin = float(ratio.min())
                if rmin < step:
                    step = rmin
                blocks.append((kind, ratio))
        if step < 1.0:
            for kind, ratio in blocks:
                hit = ratio <= step * (1.0 + 1e-12) + 1e-300
                (nob_t if kind == "t" else nob_x)[...] |= hit
            v = v + step * dv
            return _x_of(sc, red, v), nu, nob_t, nob_x
        v = v + dv
        if dv.size == 0 or np.max(np.abs(dv)) <= 1e-15 * max(1e-3, np.max(np.abs(v), initial=0.0)):
            break
    return _x_of(sc, red, v), nu, nob_t, nob_x


def refine(prob, ipm_sol, max_newton: int = 60, rounds: int = 40, accept: float = 1e-12,
           fallback: float = 1e-9, max_groups: int = 6000, seconds: Optional[float] = None):
    """Polish an interior-point solution.  Returns (x, yA, yD, kkt, red) for the
    first activity guess certified to ``accept``, else the best one found if it
    is certified to ``fallback``, else None.  ``seconds``: wall-clock budget;
    no new round starts after it (None: rounds only)."""
    t_start = time.perf_counter()
    sc = Scaled(prob)
    act = ipm_sol.active
    # kinks: a trade is dead when its interior-point multiplier lies inside the
    # spread cost's dead zone (|y_D| < c1, Eq. 1 / Eq. 4) or its value is zero
    # to 1e-9 of the largest trade (the interior point exits near 1e-6 relative
    # KKT on large multi-period instances, where the primal threshold alone
    # leaves hundreds of dead trades to be found one Newton step at a time); a
    # holding is zero to 1e-9 of the largest holding; rows from the
    # slack/multiplier ratio.  A wrong guess only costs rounds: every result is
    # accepted only when the independent KKT evaluation certifies it.
    xi = ipm_sol.x
    zi = sc.trades(xi)
    tx = 1e-9 * max(1e-3, float(np.max(np.abs(xi))))
    tz = 1e-9 * max(1e-3, float(np.max(np.abs(zi))))
    dead = np.abs(zi) <= tz
    if getattr(ipm_sol, "yD", None) is not None:
        dead |= np.abs(np.asarray(ipm_sol.yD).reshape(zi.shape)) < sc.c1 * (1.0 - 1e-4)
    st = dict(zero=np.abs(xi) <= tx, dead=dead,
              budget=np.asarray(act["budget"]).copy(), upper=act["upper"].copy(),
              lower=act["lower"].copy(), sx_force=np.zeros((sc.P, sc.n)),
              sz_force=np.zeros((sc.R, sc.n)))
    x = ipm_sol.x.copy()
    best = None
    for _ in range(rounds):
        if seconds is not None and time.perf_counter() - t_start > seconds:
            break
        red = _identify(sc, x, st)
        if red.S.shape[1] > max_groups:
            return None
        try:
            x, nu, blk_t, blk_x = _newton(sc, red, x, max_newton)
        except np.linalg.LinAlgError:
            return None
        if np.any(blk_t) or np.any(blk_x):
            st["dead"] |= blk_t
            st["zero"] |= blk_x
            st["sx_force"][:] = 0.0
            st["sz_force"][:] = 0.0
            continue
        yA = np.zeros((sc.P, sc.m))
        nb = np.zeros(sc.P)
        k = 0
        for p in range(sc.P):
            if red.budget[p]:
                nb[p] = nu[k]
                k += 1
        for (p, j, bound, side) in red.box:
            yA[p, j] = nu[k]
            k += 1
        yD, flips = _dual_from_chain(sc, x, yA, nb, red)
        res = evaluate(sc, x, yA, yD)
        if np.isfinite(res.rel_kkt) and (best is None or res.rel_kkt < best[3].rel_kkt):
            best = (x.copy(), yA, yD, res, red)
        if np.isfinite(res.rel_kkt) and res.rel_kkt <= accept:
            return best
        changed = False
        st["sx_force"][:] = 0.0
        st["sz_force"][:] = 0.0
        # primal side: collapsed pieces become kinks, violated rows become active
        z = sc.trades(x)
        zs = 1e-11 * max(1e-3, float(np.max(np.abs(z))))
        coll = red.live & (np.abs(z) <= zs)
        if np.any(coll & ~st["dead"]):
            st["dead"] |= coll
            changed = True
        xs_ = 1e-13 * max(1e-3, float(np.max(np.abs(x))))
        collx = red.free_mask & (red.sx != 0) & (np.abs(x) <= xs_)
        if np.any(collx & ~st["zero"]):
            st["zero"] |= collx
            changed = True
        for p in range(sc.P):
            if st["budget"][p] and nb[p] < 0:
                st["budget"][p] = False
                changed = True
            elif not st["budget"][p] and np.abs(x[p]).sum() > 1.0 + 1e-14:
                st["budget"][p] = True
                changed = True
        Ax = x @ sc.A.T
        for (p, j, bound, side) in red.box:
            if side * yA[p, j] < 0:
                (st["upper"] if side > 0 else st["lower"])[p, j] = False
                changed = True
        viol_u = (Ax > sc.U[None, :] + 1e-14) & ~st["upper"]
        viol_l = (Ax < sc.L[None, :] - 1e-14) & ~st["lower"]
        if np.any(viol_u) or np.any(viol_l):
            st["upper"] |= viol_u
            st["lower"] |= viol_l
            changed = True
        # dual side: free the kinks whose multiplier left its range
        for kind, a, i, sign in flips:
            if kind == "trade" and st["dead"][a, i]:
                st["dead"][a, i] = False
                st["sz_force"][a, i] = sign
                changed = True
            elif kind == "hold" and st["zero"][a, i]:
                st["zero"][a, i] = False
                st["sx_force"][a, i] = sign
                changed = True
        if not changed:
            break
    if best is not None and best[3].rel_kkt <= fallback:
        return best
    return None
