"""Properties of the oracle's KKT measures (oracle/kkt.py).

* Phi(x) (the magnitude of the objective's terms) is the sum of |alpha_i x_i|,
  the risk and the trading cost, so it bounds |P(x)| from above;
* the relative gap with the max(|P| + |D|, Phi) denominator never exceeds the
  purely relative gap and equals it when |P| + |D| >= Phi;
* at the oracle optimum every measure is at rounding level, and a feasible
  perturbation of the optimum raises the gap.
"""
import numpy as np

import oracle
from oracle import Scaled
from oracle.kkt import dual_bound, evaluate, term_scale
from paper_2604_22625_gb300 import synthetic as S


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
        assert k.r_gap <= plain * (1 + 1e-12)
        if abs(P_) + abs(D_) >= term_scale(sc, x):
            assert abs(k.r_gap - plain) <= 1e-12 * plain
        assert k.r_gap >= evaluate(sc, sol.x, sol.yA, sol.yD).r_gap


def test_optimum_is_at_rounding_level():
    sol = oracle.solve(S.make_multi(3, 25, 3, 5, n_onehot=1))
    assert sol.kkt.rel_kkt <= 1e-10
