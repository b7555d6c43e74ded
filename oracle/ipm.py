"""FP64 primal-dual interior-point solver for the portfolio models (test infrastructure).

ORACLE: test infrastructure only (``tests/``, ``smoke()``, the bench's CPU
baseline). It shares no code with the CUDA solver, which is a first-order
method; this is a second-order method for the same convex program.

What it computes: the unique minimiser of the scaled form (``oracle.model``)
of the single-period model (Sec. 2.1, Eqs. 1-3) or the multi-period model
(Sec. 2.2, Eqs. 4-6), with Lagrange multipliers of the exposure rows and of
the trades. Uniqueness: with lambda1 > 0 and D > 0 the objective is strictly
convex in x.

Epigraph form (all constraints linear):
    variables: x (P, n) holdings, t (R, n) >= |z| with z = Delta x + b,
               e (P, n) >= |x|
    min  f(x) + sum c1 t + sum c2 t^d
    s.t. t - z >= 0, t + z >= 0                (trade epigraph, Eq. 1 / Eq. 4)
         e - x >= 0, e + x >= 0                (abs epigraph)
         1 - sum_i e_{p,i} >= 0                (Eq. 3 / Eq. 6)
         U - A x_p >= 0, A x_p - L >= 0        (Eq. 2 / Eq. 5)
Since c1, c2 >= 0 the objective increases in t, so t = |z| at the optimum.

Method: Mehrotra predictor-corrector on grad f - G^T lam = 0, G x - h = s,
s o lam = sigma mu, one common primal/dual step (the objective is
nonlinear in t). Newton matrix H + G^T W G, W = lam / s:
  * t_r and e_p are eliminated per asset in closed form. The resulting
    weights are written without differences of large numbers:
      trade r:  omega = (4 W1 W2 + (W1 + W2) H_t) / (W1 + W2 + H_t)
      abs p:    4 W3 W4 / (W3 + W4)
  * what is left per asset is a P x P tridiagonal matrix: a path with link
    weights omega_r (trade r joins x_{r-1} and x_r) and positive "ground"
    terms. It is factored by series-conductance recursions in which every
    operation adds positive numbers.
  * the couplings across assets (2 kappa F Omega F^T and A^T W A on every
    x_p, W_b 1 1^T on every e_p) have rank P (k + m + 1) and are applied with
    the Sherman-Morrison-Woodbury identity in its C^{-1} + V^T M^{-1} V form.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import warnings

import numpy as np
import scipy.linalg as sla

from .model import Scaled

TINY = 1e-300


@dataclass
class IPMSolution:
    x: np.ndarray          # (P, n) optimal holdings
    yA: np.ndarray         # (P, m) exposure-row multipliers (upper minus lower)
    yD: np.ndarray         # (R, n) trade multipliers (a subgradient of the cost at z*)
    obj: float             # scaled minimisation objective
    paper_obj: float       # Eq. 1 / Eq. 4 objective in paper units
    iters: int
    status: str
    history: list = field(default_factory=list)
    active: dict = field(default_factory=dict)

    @property
    def w(self) -> np.ndarray:
        return self.x[0] if self.x.shape[0] == 1 else self.x


def _series(a, b):
    """Series combination a b / (a + b) of two nonnegative conductances."""
    s = a + b
    return np.where(s > 0, a * (b / np.where(s > 0, s, 1.0)), 0.0)


class _PathFactor:
    """Factor of the per-asset P x P matrix  diag(ground) + sum_r omega_r g_r g_r^T
    where the middle trades r = 1..P-1 join x_{r-1} and x_r."""

    def __init__(self, ground, link):
        # ground (P, n) > 0; link (P, n): link[r] joins r-1 and r (link[0] unused)
        P = ground.shape[0]
        self.P = P
        self.link = link
        Lc = np.empty_like(ground)
        Lc[0] = ground[0]
        for p in range(1, P):
            Lc[p] = ground[p] + _series(Lc[p - 1], link[p])
        piv = Lc.copy()
        piv[:-1] += link[1:]
        self.piv = piv

    def solve(self, r):
        """r: (P, n, ...) -> S^{-1} r."""
        P, piv, link = self.P, self.piv, self.link
        ext = (slice(None),) + (None,) * (r.ndim - 2)
        y = np.empty_like(r)
        y[0] = r[0]
        for p in range(1, P):
            y[p] = r[p] + (link[p] / piv[p - 1])[ext] * y[p - 1]
        x = np.empty_like(r)
        x[P - 1] = y[P - 1] / piv[P - 1][ext]
        for p in range(P - 2, -1, -1):
            x[p] = (y[p] + link[p + 1][ext] * x[p + 1]) / piv[p][ext]
        return x

    def inverse(self):
        """Full inverse, shape (P, P, n)."""
        P = self.P
        n = self.piv.shape[1]
        eye = np.zeros((P, n, P))
        for p in range(P):
            eye[p, :, p] = 1.0
        inv = self.solve(eye)            # (P, n, P): inv[p, i, q] = S_i^{-1}[p, q]
        return np.transpose(inv, (0, 2, 1))


def solve(prob, tol: float = 1e-11, max_iter: int = 150, verbose: bool = False) -> IPMSolution:
    with np.errstate(all="ignore"), warnings.catch_warnings():
        warnings.simplefilter("ignore")
        return _solve(prob, tol, max_iter, verbose)


def _solve(prob, tol, max_iter, verbose) -> IPMSolution:
    sc = Scaled(prob)
    P, R, n, m, k = sc.P, sc.R, sc.n, sc.m, sc.k
    kap, d = sc.kappa, sc.d
    A, Dl, b = sc.A, sc.Delta, sc.b
    fin_u = np.isfinite(sc.U)
    fin_l = np.isfinite(sc.L)
    Uf = np.where(fin_u, sc.U, 0.0)
    Lf = np.where(fin_l, sc.L, 0.0)
    mu_ = np.broadcast_to(fin_u[None, :], (P, m))
    ml_ = np.broadcast_to(fin_l[None, :], (P, m))
    box_cols = np.nonzero(fin_u | fin_l)[0]
    Ab = A[box_cols]                                   # rows with at least one finite bound
    mb = Ab.shape[0]
    use_fac = kap > 0
    kf = k if use_fac else 0
    Cfac_inv = np.linalg.inv(2.0 * kap * sc.Omega) if use_fac else np.zeros((0, 0))
    B = kf + mb + 1
    ncomp = 2 * R * n + 2 * P * n + P + int(mu_.sum()) + int(ml_.sum())

    # ---- constraint map and its adjoint ------------------------------------
    def g_all(x, t, e):
        z = Dl @ x + b
        Ax = x @ A.T
        return dict(tm=t - z, tp=t + z, am=e - x, ap=e + x, bud=1.0 - e.sum(axis=1),
                    up=np.where(mu_, Uf - Ax, 1.0), lo=np.where(ml_, Ax - Lf, 1.0))

    def G_lin(dx, dt, de):
        dz = Dl @ dx
        dAx = dx @ A.T
        return dict(tm=dt - dz, tp=dt + dz, am=de - dx, ap=de + dx, bud=-de.sum(axis=1),
                    up=np.where(mu_, -dAx, 0.0), lo=np.where(ml_, dAx, 0.0))

    def G_T(v):
        gx = -Dl.T @ v["tm"] + Dl.T @ v["tp"] - v["am"] + v["ap"] + (np.where(ml_, v["lo"], 0.0)
                                                                     - np.where(mu_, v["up"], 0.0)) @ A
        gt = v["tm"] + v["tp"]
        ge = v["am"] + v["ap"] - v["bud"][:, None]
        return gx, gt, ge

    def grad_obj(x, t):
        gx = sc.grad_f(x)
        gt = sc.c1 + d * sc.c2 * np.power(t, d - 1.0)
        return gx, gt, np.zeros((P, n))

    def obj_val(x, t):
        return sc.f(x) + float(np.sum(sc.c1 * t) + np.sum(sc.c2 * np.power(t, d)))

    keys = ("tm", "tp", "am", "ap", "bud", "up", "lo")
    masks = dict(tm=None, tp=None, am=None, ap=None, bud=None, up=mu_, lo=ml_)

    def msk(key, a, fill):
        mk = masks[key]
        return a if mk is None else np.where(mk, a, fill)

    # ---- initial point ---------------------------------------------------------
    x = np.zeros((P, n))
    t = np.abs(b) + 1.0
    e = np.full((P, n), 0.5 / n)
    g0 = g_all(x, t, e)
    s = {kk: msk(kk, np.maximum(g0[kk], 1e-2), 1.0) for kk in keys}
    mu0 = 1e-4
    lam = {kk: msk(kk, mu0 / s[kk], 0.0) for kk in keys}

    history = []
    status = "max_iter"
    best = None
    it_count = 0
    for it_count in range(1, max_iter + 1):
        gv = g_all(x, t, e)
        rp = {kk: msk(kk, gv[kk] - s[kk], 0.0) for kk in keys}
        grx, grt, gre = grad_obj(x, t)
        Gx, Gt, Ge = G_T(lam)
        rdx, rdt, rde = grx - Gx, grt - Gt, gre - Ge
        comp = float(sum(np.sum(msk(kk, s[kk] * lam[kk], 0.0)) for kk in keys))
        mu = comp / ncomp
        fval = obj_val(x, t)
        pres = max(float(np.abs(rp[kk]).max(initial=0.0)) for kk in keys)
        dscale = max(np.abs(grx).max(), np.abs(grt).max(), np.abs(Gx).max(), np.abs(Gt).max(),
                     np.abs(Ge).max(), TINY)
        dres = max(np.abs(rdx).max(), np.abs(rdt).max(), np.abs(rde).max()) / dscale
        crel = comp / max(abs(fval), TINY)
        history.append((fval, pres, dres, crel))
        if verbose:
            print(f"ipm {it_count:3d} f={fval:.12e} pres={pres:.2e} dres={dres:.2e} comp={crel:.2e}")
        merit = max(pres, crel, min(dres, 1.0) * 1e-3)
        if best is None or merit < best[0]:
            best = (merit, x.copy(), t.copy(), e.copy(), {kk: s[kk].copy() for kk in keys},
                    {kk: lam[kk].copy() for kk in keys}, it_count)
        if pres < tol and crel < tol and dres < 1e-6:
            status = "optimal"
            break
        if (best[0] < 1e-6 and it_count - best[6] > 10) or (best[0] < 1e-8 and (merit > 1e3 * best[0] or it_count - best[6] > 6)):
            status = "stalled"
            break

        # ---- Newton matrix, factored -----------------------------------------
        W = {kk: msk(kk, lam[kk] / s[kk], 0.0) for kk in keys}
        Ht = sc.c2 * d * (d - 1.0) * np.power(t, d - 2.0)
        W1, W2, W3, W4 = W["tm"], W["tp"], W["am"], W["ap"]
        Dt = W1 + W2 + Ht
        omega = (4.0 * W1 * W2 + (W1 + W2) * Ht) / Dt
        delta = (W2 - W1) / Dt
        De = W3 + W4
        beta = (W4 - W3) / De
        ground = 2.0 * kap * sc.Dp + 4.0 * W3 * (W4 / De)
        ground[0] += omega[0]
        link = np.zeros((P, n))
        for r in range(1, P):
            link[r] = omega[r]
        if sc.multi:
            ground[P - 1] += omega[R - 1]
        fac = _PathFactor(ground, link)
        Sinv = fac.inverse()                           # (P, P, n)
        Wbox = (W["up"] + W["lo"])[:, box_cols]         # (P, mb)
        Wb = W["bud"]

        def Mloc_solve(rx, rt, re):
            rxp = rx - Dl.T @ (delta * rt) - beta * re
            xx = fac.solve(rxp)
            tt = rt / Dt - delta * (Dl @ xx)
            ee = re / De - beta * xx
            return xx, tt, ee

        # capacitance C^{-1} + V^T Mloc^{-1} V,  V_p = [F | Ab^T] on x_p, [1] on e_p
        Vx = np.hstack([sc.F, Ab.T]) if use_fac else Ab.T.copy()     # (n, kf + mb)
        cap = np.zeros((P, B, P, B))
        for p in range(P):
            for q in range(P):
                nxx = Sinv[p, q]
                nxe = -Sinv[p, q] * beta[q]
                nex = -beta[p] * Sinv[p, q]
                nee = beta[p] * Sinv[p, q] * beta[q] + (1.0 / De[p] if p == q else 0.0)
                cap[p, :B - 1, q, :B - 1] = Vx.T @ (nxx[:, None] * Vx)
                cap[p, :B - 1, q, B - 1] = Vx.T @ nxe
                cap[p, B - 1, q, :B - 1] = nex @ Vx
                cap[p, B - 1, q, B - 1] = nee.sum()
            cap[p, :kf, p, :kf] += Cfac_inv
            cap[p, kf + np.arange(mb), p, kf + np.arange(mb)] += 1.0 / np.maximum(Wbox[p], TINY)
            cap[p, B - 1, p, B - 1] += 1.0 / max(Wb[p], TINY)
        cap = cap.reshape(P * B, P * B)
        if not np.all(np.isfinite(cap)):
            status = "numerical"
            break
        try:
            cfac = sla.cho_factor(cap)
        except np.linalg.LinAlgError:
            status = "numerical"
            break

        def V_T(xx, ee):
            out = np.empty((P, B))
            out[:, :B - 1] = xx @ Vx
            out[:, B - 1] = ee.sum(axis=1)
            return out.reshape(-1)

        def V_apply(yv):
            yv = yv.reshape(P, B)
            return yv[:, :B - 1] @ Vx.T, yv[:, B - 1][:, None] * np.ones((1, n))

        def M_solve(rx, rt, re):
            xx, tt, ee = Mloc_solve(rx, rt, re)
            yv = sla.cho_solve(cfac, V_T(xx, ee))
            vx, ve = V_apply(yv)
            cx, ct, ce = Mloc_solve(vx, np.zeros_like(rt), ve)
            return xx - cx, tt - ct, ee - ce

        def direction(rc):
            v = {kk: msk(kk, (rc[kk] + lam[kk] * rp[kk]) / s[kk], 0.0) for kk in keys}
            gx_, gt_, ge_ = G_T(v)
            dx, dt, de = M_solve(-rdx - gx_, -rdt - gt_, -rde - ge_)
            dg = G_lin(dx, dt, de)
            ds = {kk: msk(kk, dg[kk] + rp[kk], 0.0) for kk in keys}
            dl = {kk: msk(kk, -(rc[kk] + lam[kk] * ds[kk]) / s[kk], 0.0) for kk in keys}
            return (dx, dt, de), ds, dl

        def max_step(dt, ds, dl):
            a = 1.0
            for kk in keys:
                for v_, dv in ((s[kk], ds[kk]), (lam[kk], dl[kk])):
                    neg = dv < 0
                    if np.any(neg):
                        a = min(a, float(np.min(-v_[neg] / dv[neg])))
            neg = dt < 0
            if np.any(neg):
                a = min(a, float(np.min(-t[neg] / dt[neg])))
            return a

        rc_aff = {kk: msk(kk, s[kk] * lam[kk], 0.0) for kk in keys}
        da, dsa, dla = direction(rc_aff)
        aa = max_step(da[1], dsa, dla)
        comp_aff = float(sum(np.sum(msk(kk, (s[kk] + aa * dsa[kk]) * (lam[kk] + aa * dla[kk]), 0.0))
                             for kk in keys))
        sigma = (comp_aff / max(comp, TINY)) ** 3
        rc = {kk: msk(kk, s[kk] * lam[kk] + dsa[kk] * dla[kk] - sigma * mu, 0.0) for kk in keys}
        (dx, dt, de), ds, dl = direction(rc)
        a = min(1.0, 0.995 * max_step(dt, ds, dl))
        if not (np.all(np.isfinite(dx)) and all(np.all(np.isfinite(dl[kk])) for kk in keys)):
            status = "numerical"
            break
        x, t, e = x + a * dx, t + a * dt, e + a * de
        for kk in keys:
            s[kk] = msk(kk, s[kk] + a * ds[kk], 1.0)
            lam[kk] = msk(kk, lam[kk] + a * dl[kk], 0.0)

    _, x, t, e, s, lam, _ = best
    yA = np.where(mu_, lam["up"], 0.0) - np.where(ml_, lam["lo"], 0.0)
    yD = lam["tm"] - lam["tp"]
    sol = IPMSolution(x=x.copy(), yA=yA, yD=yD, obj=sc.objective(x), paper_obj=sc.paper_objective(x),
                      iters=it_count, status=status, history=history)
    sol.active = dict(trade_pos=s["tm"] < lam["tm"], trade_neg=s["tp"] < lam["tp"],
                      abs_pos=s["am"] < lam["am"], abs_neg=s["ap"] < lam["ap"],
                      budget=s["bud"] < lam["bud"], upper=mu_ & (s["up"] < lam["up"]),
                      lower=ml_ & (s["lo"] < lam["lo"]))
    return sol
