"""Scaled form of the portfolio models, written out in FP64 (test infrastructure).

ORACLE: this package is test infrastructure. Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may import it.
It shares no code with the CUDA solver.

Both models are put in one minimisation form over P free portfolios
x_1..x_P (P = 1 for the single-period model of Sec. 2.1, P = T - 1 for the
multi-period model of Sec. 2.2), by dividing the maximised objective of
Eq. 1 / Eq. 4 by -GMV:

    min  sum_p [ -alpha_p^T x_p + kappa (x_p - c)^T Sigma_p (x_p - c) ]
       + sum_r phi_r(z_r),       z = Delta x + b,
    s.t. L <= A x_p <= U,  ||x_p||_1 <= 1          (Eqs. 2-3 / Eqs. 5-6)

with kappa = lambda1 * GMV, Sigma_p = F Omega F^T + diag(D_p) (Sec. 3.2),
phi_r(z) = sum_i c1_{r,i} |z_i| + c2_{r,i} |z_i|^d, c1 = lambda2 s, c2 = lambda3 q.

Trades (Eq. 1: w - w0; Eq. 4: w_t - w_{t-1}, t = 1..T):
    single: R = 1, z_1 = x_1 - w0, c = 0.
    multi:  R = T, z_1 = x_1 - w0, z_r = x_r - x_{r-1} (2 <= r <= T-1),
            z_T = w_T - x_{T-1}, c = w_T.
So Delta is the R x P matrix with +1 on the diagonal and -1 on the first
subdiagonal, b_1 = -w0 and (multi) b_T = +w_T.

In Eq. 4 the t = T return term alpha_T^T w_T is a constant and the t = T
risk term is zero, so both are dropped from the minimisation; the t = T
trading cost is kept. ``paper_objective`` restores the constant.
"""
from __future__ import annotations

import numpy as np


class Scaled:
    """FP64 arrays of the scaled problem built from a ``Problem``-like object."""

    def __init__(self, prob):
        self.n = int(prob.F.shape[0])
        self.k = int(prob.F.shape[1])
        self.m = int(prob.A.shape[0])
        self.multi = int(getattr(prob, "T", 0)) >= 2
        T = int(prob.T) if self.multi else 0
        self.T = T
        self.P = T - 1 if self.multi else 1
        self.R = T if self.multi else 1
        f64 = lambda a: np.asarray(a, dtype=np.float64)
        self.F = f64(prob.F)
        self.Omega = f64(prob.Omega)
        self.A = f64(prob.A).reshape(self.m, self.n)
        self.L = f64(prob.L).reshape(self.m)
        self.U = f64(prob.U).reshape(self.m)
        self.GMV = float(prob.GMV)
        self.kappa = float(prob.lam1) * self.GMV
        self.d = float(prob.d)
        n, P, R = self.n, self.P, self.R
        if self.multi:
            self.alpha = f64(prob.alpha)[:P].copy()
            self.alpha_T = f64(prob.alpha)[T - 1].copy()
            self.Dp = f64(prob.D)[:P].copy()
            self.c1 = float(prob.lam2) * f64(prob.s)[:R]
            self.c2 = float(prob.lam3) * f64(prob.q)[:R]
            self.center = f64(prob.wT).copy()
            self.wT = self.center
        else:
            self.alpha = f64(prob.alpha).reshape(1, n).copy()
            self.alpha_T = None
            self.Dp = f64(prob.D).reshape(1, n).copy()
            self.c1 = float(prob.lam2) * f64(prob.s).reshape(1, n)
            self.c2 = float(prob.lam3) * f64(prob.q).reshape(1, n)
            self.center = np.zeros(n)
            self.wT = None
        self.w0 = f64(prob.w0).copy()
        self.b = np.zeros((R, n))
        self.b[0] -= self.w0
        if self.multi:
            self.b[R - 1] += self.wT
        self.Delta = np.zeros((R, P))
        for r in range(R):
            if r < P:
                self.Delta[r, r] = 1.0
            if 1 <= r <= P:
                self.Delta[r, r - 1] = -1.0

    # ---- linear maps -------------------------------------------------
    def Sigma_apply(self, v: np.ndarray, p: int) -> np.ndarray:
        """Sigma_p v = F (Omega (F^T v)) + D_p v  (Sec. 3.2 factor form)."""
        return self.F @ (self.Omega @ (self.F.T @ v)) + self.Dp[p] * v

    def trades(self, x: np.ndarray) -> np.ndarray:
        """z = Delta x + b, shape (R, n)."""
        return self.Delta @ x + self.b

    def delta_T(self, y: np.ndarray) -> np.ndarray:
        """Delta^T y, shape (P, n)."""
        return self.Delta.T @ y

    # ---- objective pieces -------------------------------------------
    def f(self, x: np.ndarray) -> float:
        tot = 0.0
        for p in range(self.P):
            dx = x[p] - self.center
            tot += -self.alpha[p] @ x[p] + self.kappa * (dx @ self.Sigma_apply(dx, p))
        return float(tot)

    def grad_f(self, x: np.ndarray) -> np.ndarray:
        g = np.empty_like(x)
        for p in range(self.P):
            g[p] = -self.alpha[p] + 2.0 * self.kappa * self.Sigma_apply(x[p] - self.center, p)
        return g

    def phi(self, z: np.ndarray) -> float:
        a = np.abs(z)
        return float(np.sum(self.c1 * a) + np.sum(self.c2 * a ** self.d))

    def objective(self, x: np.ndarray) -> float:
        """Scaled minimisation objective (no feasibility terms)."""
        return self.f(x) + self.phi(self.trades(x))

    def paper_objective(self, x: np.ndarray) -> float:
        """Eq. 1 / Eq. 4 in the paper's units (maximised), constants included."""
        val = -self.objective(x)
        if self.multi:
            val += float(self.alpha_T @ self.wT)
        return self.GMV * val


def as_periods(sc: Scaled, w) -> np.ndarray:
    """Reshape a single-period vector (n,) or a stack (P, n) to (P, n)."""
    w = np.asarray(w, dtype=np.float64)
    return w.reshape(sc.P, sc.n)
