"""Pins of the FP64 oracle solve against facts fixed by the models of Sec. 2.

Each pin comes from something other than the oracle itself:
  * brute-force search over the feasible set on tiny instances (Eqs. 1-6);
  * closed form w* = Sigma^{-1} alpha / (2 lambda1 GMV) when costs and
    exposure rows are off and the budget is slack (first-order condition of Eq. 1);
    for the multi-period model w_t* = w_T + Sigma_t^{-1} alpha_t / (2 lambda1 GMV);
  * the separable case F = 0, no exposure rows: one 1-D convex problem per
    asset (slack budget) or a 1-D search on the budget multiplier (tight budget),
    both by golden-section search;
  * the multi-period model with T = 2, w_T = 0 and no cost at t = 2 is the
    single-period model (Eq. 4 reduces to Eq. 1);
  * weak duality of the dual bound and the optimality certificate.
"""
import numpy as np
import pytest

import oracle
from oracle import Scaled
from oracle.kkt import dual_bound, distance_bound, evaluate
from paper_2604_22625_gb300 import synthetic as S


def _tiny_single(n, m, seed, lam2=1.0, lam3=1.0, alpha_scale=2e-3, bound=0.05):
    rng = np.random.default_rng(seed)
    k = 2
    F = rng.normal(0, 1, (n, k))
    p = S.Problem(F=F, Omega=np.diag(rng.uniform(1e-5, 1e-4, k)), D=rng.uniform(1e-4, 9e-4, n),
                  alpha=rng.normal(0, alpha_scale, n), s=rng.uniform(2e-4, 2e-3, n),
                  q=rng.uniform(1e-3, 1e-2, n), w0=S._signed_l1(rng, n, 0.9),
                  A=rng.normal(0, 1, (m, n)), L=np.full(m, -bound), U=np.full(m, bound),
                  lam1=10.0 / 1e9, lam2=lam2, lam3=lam3)
    return p


def _brute(obj, feasible, lo, hi, levels=16, pts=41):
    """Nested grid search with zoom over a box; returns the best feasible point."""
    lo = np.asarray(lo, float)
    hi = np.asarray(hi, float)
    best = None
    for _ in range(levels):
        axes = [np.linspace(a, b, pts) for a, b in zip(lo, hi)]
        grid = np.stack(np.meshgrid(*axes, indexing="ij"), -1).reshape(-1, lo.size)
        ok = feasible(grid)
        if not np.any(ok):
            break
        vals = obj(grid[ok])
        j = int(np.argmin(vals))
        c = grid[ok][j]
        if best is None or vals[j] < best[1]:
            best = (c, vals[j])
        span = (hi - lo) / (pts - 1) * 20
        lo, hi = best[0] - span, best[0] + span
    return best


@pytest.mark.parametrize("seed", range(4))
def test_single_brute_force(seed):
    n, m = (2, 1) if seed % 2 == 0 else (3, 1)
    p = _tiny_single(n, m, seed, alpha_scale=2e-2)
    sc = Scaled(p)
    sol = oracle.solve(p)
    assert sol.kkt.rel_kkt < 1e-10

    Sigma = p.F @ p.Omega @ p.F.T + np.diag(p.D)

    def obj(W):
        # Eq. 1 in paper units, negated and divided by GMV
        tr = np.abs(W - p.w0)
        val = (p.GMV * W @ p.alpha - p.lam1 * p.GMV ** 2 * np.einsum("bi,ij,bj->b", W, Sigma, W)
               - p.lam2 * p.GMV * tr @ p.s - p.lam3 * p.GMV * (tr ** p.d) @ p.q)
        return -val / p.GMV

    def feas(W):
        return (np.abs(W).sum(1) <= 1) & np.all(W @ p.A.T <= p.U, 1) & np.all(W @ p.A.T >= p.L, 1)

    c, val = _brute(obj, feas, -np.ones(n), np.ones(n), levels=18, pts=301 if n == 2 else 101)
    assert sol.obj <= val + 1e-12
    assert val - sol.obj <= 1e-7 * abs(sol.obj)
    assert np.max(np.abs(c - sol.w)) < 1e-4


def test_multi_brute_force():
    rng = np.random.default_rng(21)
    n, T = 1, 3
    p = S.Problem(F=np.zeros((n, 1)), Omega=np.eye(1) * 5e-5, D=rng.uniform(1e-4, 9e-4, (T, n)),
                  alpha=rng.normal(0, 2e-2, (T, n)), s=rng.uniform(2e-4, 2e-3, (T, n)),
                  q=rng.uniform(1e-3, 1e-2, (T, n)), w0=np.array([0.6]), A=np.ones((1, n)),
                  L=np.array([-0.7]), U=np.array([0.7]), T=T, wT=np.array([-0.5]))
    sc = Scaled(p)
    sol = oracle.solve(p)
    assert sol.kkt.rel_kkt < 1e-10

    Sig = [p.F @ p.Omega @ p.F.T + np.diag(p.D[t]) for t in range(T)]

    def obj(W):
        # Eq. 4 in paper units (t = 1..T, w_0 and w_T fixed), negated and divided by GMV
        path = [np.full(len(W), p.w0[0]), W[:, 0], W[:, 1], np.full(len(W), p.wT[0])]
        val = 0.0
        for t in range(1, T + 1):
            dev = path[t] - p.wT[0]
            tr = np.abs(path[t] - path[t - 1])
            val = val + (p.GMV * p.alpha[t - 1, 0] * path[t] - p.lam1 * p.GMV ** 2 * Sig[t - 1][0, 0] * dev ** 2
                         - p.lam2 * p.GMV * p.s[t - 1, 0] * tr - p.lam3 * p.GMV * p.q[t - 1, 0] * tr ** p.d)
        return -val / p.GMV + p.alpha[T - 1, 0] * p.wT[0]

    def feas(W):
        return np.all(np.abs(W) <= 0.7, 1)

    c, val = _brute(obj, feas, -np.ones(2), np.ones(2), levels=18, pts=301)
    assert sol.obj <= val + 1e-12
    assert np.max(np.abs(c - sol.x.ravel())) < 1e-4


def test_closed_form_single():
    """lambda2 = lambda3 = 0, no rows, slack budget: Sigma w = alpha / (2 kappa)."""
    p = S.make_single(120, 8, 5, n_onehot=3, lam2=0.0, lam3=0.0)
    p.alpha = p.alpha * 1e-3
    p.A = np.zeros((0, p.n))
    p.L = np.zeros(0)
    p.U = np.zeros(0)
    sol = oracle.solve(p)
    Sigma = p.F @ p.Omega @ p.F.T + np.diag(p.D)
    w = np.linalg.solve(Sigma, p.alpha) / (2 * p.lam1 * p.GMV)
    assert np.abs(w).sum() < 1
    np.testing.assert_allclose(sol.w, w, rtol=1e-9, atol=1e-13)


def test_closed_form_multi():
    p = S.make_multi(4, 60, 6, 9, n_onehot=2, lam2=0.0, lam3=0.0)
    p.alpha = p.alpha * 1e-3
    p.wT = p.wT * 0.1
    p.A = np.zeros((0, p.n))
    p.L = np.zeros(0)
    p.U = np.zeros(0)
    sol = oracle.solve(p)
    for t in range(p.T - 1):
        Sigma = p.F @ p.Omega @ p.F.T + np.diag(p.D[t])
        w = p.wT + np.linalg.solve(Sigma, p.alpha[t]) / (2 * p.lam1 * p.GMV)
        np.testing.assert_allclose(sol.x[t], w, rtol=1e-9, atol=1e-13)


def _golden(fun, lo, hi, iters=300):
    g = (np.sqrt(5.0) - 1.0) / 2.0
    a, b = lo, hi
    for _ in range(iters):
        c, d = b - g * (b - a), a + g * (b - a)
        if fun(c) < fun(d):
            b = d
        else:
            a = c
    return 0.5 * (a + b)


@pytest.mark.parametrize("tight,dexp", [(False, 1.5), (True, 1.5), (False, 2.0), (True, 2.0), (False, 1.3)])
def test_separable_single(tight, dexp):
    """F = 0 and no rows: each asset solves
    min_w -alpha w + kappa D w^2 + c1 |w - w0| + c2 |w - w0|^d + mu |w|,
    with mu = 0 (slack budget) or mu found by bisection so that ||w||_1 = 1,
    for the paper's d = 1.5, the quadratic-impact end d = 2 and an exponent
    without a closed-form prox (d = 1.3)."""
    rng = np.random.default_rng(2)
    n = 40
    p = S.Problem(F=np.zeros((n, 1)), Omega=np.eye(1) * 1e-5, D=rng.uniform(1e-4, 9e-4, n),
                  alpha=rng.normal(0, 1e-4 if not tight else 4e-2, n), s=rng.uniform(2e-4, 2e-3, n),
                  q=rng.uniform(1e-3, 1e-2, n), w0=S._signed_l1(rng, n, 0.9 if tight else 0.5),
                  A=np.zeros((0, n)), L=np.zeros(0), U=np.zeros(0), d=dexp)
    sc = Scaled(p)
    kap, c1, c2, d = sc.kappa, sc.c1[0], sc.c2[0], sc.d

    def coord(mu):
        out = np.empty(n)
        for i in range(n):
            f = lambda w: (-p.alpha[i] * w + kap * p.D[i] * w * w + c1[i] * abs(w - p.w0[i])
                           + c2[i] * abs(w - p.w0[i]) ** d + mu * abs(w))
            out[i] = _golden(f, -1.5, 1.5)
        return out

    w = coord(0.0)
    if np.abs(w).sum() > 1:
        assert tight
        lo, hi = 0.0, 1.0
        for _ in range(80):
            mid = 0.5 * (lo + hi)
            if np.abs(coord(mid)).sum() > 1:
                lo = mid
            else:
                hi = mid
        w = coord(hi)
    sol = oracle.solve(p)
    np.testing.assert_allclose(sol.w, w, atol=1e-7)


def test_multi_T2_reduces_to_single():
    ps = S.make_single(150, 9, 13, n_onehot=3)
    pm = S.Problem(F=ps.F, Omega=ps.Omega, D=np.stack([ps.D, ps.D]), alpha=np.stack([ps.alpha, ps.alpha]),
                   s=np.stack([ps.s, 0 * ps.s]), q=np.stack([ps.q, 0 * ps.q]), w0=ps.w0, A=ps.A,
                   L=ps.L, U=ps.U, T=2, wT=np.zeros(ps.n))
    a = oracle.solve(ps)
    b = oracle.solve(pm)
    np.testing.assert_allclose(a.w, b.x[0], atol=1e-10)
    assert abs(a.obj - b.obj) <= 1e-12 * abs(a.obj)


@pytest.mark.parametrize("maker", ["single", "multi"])
def test_invariants_and_weak_duality(maker):
    p = S.make_single(400, 16, 3, n_onehot=6) if maker == "single" else S.make_multi(6, 120, 10, 4, n_onehot=4)
    sc = Scaled(p)
    sol = oracle.solve(p)
    x = sol.x
    # the polish certifies 1e-12; if a degenerate kink defeats it the interior
    # point result must still be certified to 1e-5 and within its distance bound
    assert sol.kkt.rel_kkt < (1e-12 if sol.polished else 1e-5)
    assert np.all(np.abs(x).sum(1) <= 1 + 1e-12)
    Ax = x @ p.A.T
    assert np.all(Ax <= p.U + 1e-12) and np.all(Ax >= p.L - 1e-12)
    assert distance_bound(sc, x, sol.yA, sol.yD) < (1e-5 if sol.polished else 1e-2)
    rng = np.random.default_rng(0)
    for _ in range(20):
        # weak duality: D(y; x') <= P(x*) for any y and any x'
        yA = rng.normal(0, 1e-3, sol.yA.shape)
        yD = sol.yD + rng.normal(0, 1e-4, sol.yD.shape)
        xp = x + rng.normal(0, 1e-3, x.shape)
        assert dual_bound(sc, xp, yA, yD) <= sol.obj + 1e-15
        # a feasible perturbation never improves the objective
        xq = x + rng.normal(0, 1e-4, x.shape)
        xq /= np.maximum(1.0, np.abs(xq).sum(1, keepdims=True))
        if np.all(xq @ p.A.T <= p.U) and np.all(xq @ p.A.T >= p.L):
            assert sc.objective(xq) >= sol.obj - 1e-15


def test_paper_objective_units():
    p = S.make_single(80, 5, 17, n_onehot=2)
    sol = oracle.solve(p)
    w = sol.w
    Sigma = p.F @ p.Omega @ p.F.T + np.diag(p.D)
    tr = np.abs(w - p.w0)
    direct = (p.GMV * p.alpha @ w - p.lam1 * p.GMV ** 2 * w @ Sigma @ w
              - p.lam2 * p.GMV * p.s @ tr - p.lam3 * p.GMV * p.q @ tr ** p.d)
    assert abs(direct - sol.paper_obj) <= 1e-9 * abs(direct)


def test_polish_budget_and_certificate():
    """The polish either certifies its point (relative KKT <= 1e-12 by the
    independent evaluation) or the interior-point point comes back unpolished;
    with no time budget left no polish round starts."""
    prob = S.make_multi(4, 60, 3, 71, n_onehot=1)
    full = oracle.solve(prob)
    assert full.polished and full.kkt.rel_kkt <= 1e-12
    none = oracle.solve(prob, polish_seconds=0.0)
    assert not none.polished
    assert float(np.max(np.abs(none.x - full.x))) <= 1e-5
