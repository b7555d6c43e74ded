"""Optimality measures of a candidate (x, y) in FP64 (test infrastructure).

ORACLE: test infrastructure only; shares no code with the CUDA solver.

The splitting used to state the dual is min f(x) + g(x) + h(Kx) with
    f(x)  = sum_p -alpha_p^T x_p + kappa (x_p - c)^T Sigma_p (x_p - c)   (smooth),
    g(x)  = sum_p indicator{||x_p||_1 <= 1}                               (Eq. 3 / Eq. 6),
    K x   = (A x_1, ..., A x_P ; Delta x),
    h_A   = indicator of [L, U] per row                                   (Eq. 2 / Eq. 5),
    h_D(v)= phi(v + b)  (spread + impact cost on the trades, Eq. 1 / Eq. 4).
Dual variables: y_A (P, m) for the exposure rows and y_D (R, n) for the
trades.  The paper stops on a "fixed-point residual" whose norm it does not
state (Sec. 4.1); the measures below are the relative KKT residuals this
project reports instead:

    r_p   = ||Ax - clip(Ax, L, U)|| / (||Ax|| + ||clip(Ax, L, U)||)
    r_d   = ||x - Proj_B1(x - (grad f(x) + K^T y))|| / (||x|| + ||grad f(x)|| + ||K^T y||)
    r_gap = |P(x) - D(y; x)| / (|P(x)| + |D(y; x)|)
(purely relative, with no "1 +": the scaled objectives are of order 1e-4 to
1e-3, so an absolute floor would hide the gap).  Reported beside it, not part
of rel_kkt: r_gap_terms = |P - D| / max(|P| + |D|, Phi(x)) with
Phi(x) = sum |alpha_i x_i| + kappa sum_p (x_p - c)^T Sigma_p (x_p - c) + phi(Delta x + b),
the magnitude of the objective's terms; with the weak-duality bound (valid for
every x, y)
    D(y; x) = f(x) - <grad f(x), x> - g*(-grad f(x) - K^T y) - h_A*(y_A) - h_D*(y_D),
    g*(v) = sum_p ||v_p||_inf,  h_A*(y) = sum U y^+ - L y^-,
    h_D*(y) = -<y, b> + sum phi*(y).
All norms are Euclidean over every period.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .model import Scaled
from .prox import cost_conjugate, project_l1

TINY = 1e-30


@dataclass
class KKT:
    primal_obj: float      # P(x), scaled minimisation form
    dual_obj: float        # D(y; x)
    r_primal: float
    r_dual: float
    r_gap: float
    r_gap_terms: float = float("nan")   # |P - D| / max(|P| + |D|, Phi): not part of rel_kkt
    term_scale: float = float("nan")    # Phi(x)

    @property
    def rel_kkt(self) -> float:
        return max(self.r_primal, self.r_dual, self.r_gap)


def K_T_apply(sc: Scaled, yA: np.ndarray, yD: np.ndarray) -> np.ndarray:
    """K^T y = (A^T yA_p + (Delta^T yD)_p)_p, shape (P, n)."""
    return yA @ sc.A + sc.delta_T(yD)


def hA_conj(sc: Scaled, yA: np.ndarray) -> float:
    pos = np.maximum(yA, 0.0)
    neg = np.maximum(-yA, 0.0)
    with np.errstate(invalid="ignore"):
        up = np.where(pos > 0, sc.U[None, :] * pos, 0.0)
        lo = np.where(neg > 0, sc.L[None, :] * neg, 0.0)
    return float(np.sum(up) - np.sum(lo))


def hD_conj(sc: Scaled, yD: np.ndarray) -> float:
    return float(-np.sum(yD * sc.b) + np.sum(cost_conjugate(yD, sc.c1, sc.c2, sc.d)))


def dual_bound(sc: Scaled, x: np.ndarray, yA: np.ndarray, yD: np.ndarray) -> float:
    g = sc.grad_f(x)
    v = -g - K_T_apply(sc, yA, yD)
    gstar = float(np.sum(np.max(np.abs(v), axis=1)))
    return sc.f(x) - float(np.sum(g * x)) - gstar - hA_conj(sc, yA) - hD_conj(sc, yD)


def term_scale(sc: Scaled, x: np.ndarray) -> float:
    """Phi(x): sum of |alpha_{p,i} x_{p,i}|, the risk terms and the trading cost."""
    ret = float(np.sum(np.abs(sc.alpha * x)))
    risk = 0.0
    for p in range(sc.P):
        dx = x[p] - sc.center
        risk += sc.kappa * float(dx @ sc.Sigma_apply(dx, p))
    return ret + risk + sc.phi(sc.trades(x))


def evaluate(sc: Scaled, x, yA, yD) -> KKT:
    """Relative KKT residuals of (x, yA, yD) for the scaled problem ``sc``."""
    x = np.asarray(x, dtype=np.float64).reshape(sc.P, sc.n)
    yA = np.asarray(yA, dtype=np.float64).reshape(sc.P, sc.m)
    yD = np.asarray(yD, dtype=np.float64).reshape(sc.R, sc.n)
    Ax = x @ sc.A.T
    cl = np.clip(Ax, sc.L[None, :], sc.U[None, :])
    r_p = np.linalg.norm(Ax - cl) / (np.linalg.norm(Ax) + np.linalg.norm(cl) + TINY)
    g = sc.grad_f(x)
    Kty = K_T_apply(sc, yA, yD)
    step = x - (g + Kty)
    proj = np.stack([project_l1(step[p]) for p in range(sc.P)])
    r_d = np.linalg.norm(x - proj) / (np.linalg.norm(x) + np.linalg.norm(g) + np.linalg.norm(Kty) + TINY)
    P_ = sc.objective(x)
    D_ = dual_bound(sc, x, yA, yD)
    r_gap = abs(P_ - D_) / (abs(P_) + abs(D_) + TINY)
    phi = term_scale(sc, x)
    r_gap_terms = abs(P_ - D_) / (max(abs(P_) + abs(D_), phi) + TINY)
    return KKT(P_, D_, float(r_p), float(r_d), float(r_gap), float(r_gap_terms), float(phi))


def strong_convexity_modulus(sc: Scaled) -> float:
    """mu with P(x') >= P(x*) + mu/2 ||x' - x*||^2 on the feasible set:
    2 kappa lambda_min(Sigma_p) >= 2 kappa min D."""
    return 2.0 * sc.kappa * float(np.min(sc.Dp))


def distance_bound(sc: Scaled, x, yA, yD) -> float:
    """Certified ||x - x*||_2 <= sqrt(2 (P(x) - D(y; x)) / mu) for a feasible x."""
    x = np.asarray(x, dtype=np.float64).reshape(sc.P, sc.n)
    gap = sc.objective(x) - dual_bound(sc, x, yA, yD)
    return float(np.sqrt(max(gap, 0.0) * 2.0 / strong_convexity_modulus(sc)))
