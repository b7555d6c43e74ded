"""Properties of the oracle's KKT measures (oracle/kkt.py).

* Phi(x) (the magnitude of the objective's terms) is the sum of |alpha_i x_i|,
  the risk and the trading cost: pinned to a value worked out by hand on a
  2-asset instance, and it bounds |P(x)| from above;
* r_gap is the purely relative gap |P - D| / (|P| + |D|) (the relative KKT
  definition of the hot-path scope); the gap against max(|P| + |D|, Phi),
  reported beside it, never exceeds it and equals it when |P| + |D| >= Phi;
* at the oracle optimum every measure is at rounding level, and a feasible
  perturbation of the optimum raises the gap.
"""
import numpy as np

import oracle
from oracle import Scaled
from oracle.kkt import dual_bound, evaluate, term_scale
from paper_2604_22625_gb300 import synthetic as S


def _two_assets():
    """n = 2, k = 1, m = 0, GMV = 1 (kappa = lambda1 = 2), d = 2."""
    return S.Problem(F=np.array([[1.0], [2.0]]), Omega=np.array([[0.5]]), D=np.array([0.1, 0.2]),
                     alpha=np.array([0.3, -0.4]), s=np.array([0.01, 0.02]), q=np.array([0.03, 0.04]),
                     w0=np.array([0.1, -0.2]), A=np.zeros((0, 2)), L=np.zeros(0), U=np.zeros(0),
                     GMV=1.0, lam1=2.0, lam2=1.0, lam3=1.0, d=2.0)


def test_term_scale_hand_value():
    """At x = (0.2, 0.3): Sigma = 0.5 F F^T + diag(0.1, 0.2) = [[0.6, 1.0], [1.0, 2.2]],
    x^T Sigma x = 0.024 + 0.12 + 0.198 = 0.342, kappa x^T Sigma x = 0.684;
    |alpha_1 x_1| + |alpha_2 x_2| = 0.06 + 0.12 = 0.18; trades z = x - w0 = (0.1, 0.5),
    cost = 0.01*0.1 + 0.03*0.1^2 + 0.02*0.5 + 0.04*0.5^2 = 0.0213.
    Phi = 0.18 + 0.684 + 0.0213 = 0.8853 and P(x) = 0.06 + 0.684 + 0.0213 = 0.7653."""
    sc = Scaled(_two_assets())
    x = np.array([[0.2, 0.3]])
    assert abs(term_scale(sc, x) - 0.8853) <= 1e-14
    assert abs(sc.objective(x) - 0.7653) <= 1e-14


def test_term_scale_bounds_objective():
    for prob in (S.make_single(60, 6, 1, n_onehot=2), S.make_multi(4, 30, 4, 2, n_onehot=2)):
        sc = Scaled(prob)
        rng = np.random.default_rng(0)
        for _ in range(5):
            x = rng.normal(0, 1e-2, (sc.P, sc.n))
            phi = term_scale(sc, x)
            assert phi >= 0
            assert abs(sc.objective(x)) <= phi * (1 + 1e-12)


def test_gap_normalisation():
    prob = S.make_single(60, 6, 3, n_onehot=2)
    sc = Scaled(prob)
    sol = oracle.solve(prob)
    rng = np.random.default_rng(1)
    for scale in (1e-6, 1e-4, 1e-2):
        x = sol.x + rng.normal(0, scale, sol.x.shape)
        x /= max(1.0, np.abs(x).sum())                 # stay in the l1 ball
        k = evaluate(sc, x, sol.yA, sol.yD)
        P_, D_ = sc.objective(x), dual_bound(sc, x, sol.yA, sol.yD)
        plain = abs(P_ - D_) / (abs(P_) + abs(D_))
        assert abs(k.r_gap - plain) <= 1e-12 * plain
        assert k.r_gap_terms <= plain * (1 + 1e-12)
        assert abs(k.term_scale - term_scale(sc, x)) <= 1e-15 * k.term_scale
        if abs(P_) + abs(D_) >= term_scale(sc, x):
            assert abs(k.r_gap_terms - plain) <= 1e-12 * plain
        assert k.r_gap >= evaluate(sc, sol.x, sol.yA, sol.yD).r_gap


def test_optimum_is_at_rounding_level():
    sol = oracle.solve(S.make_multi(3, 25, 3, 5, n_onehot=1))
    assert sol.kkt.rel_kkt <= 1e-10
