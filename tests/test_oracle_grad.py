"""Pins of the oracle's implicit-function derivative (oracle/grad.py).

The directional derivative dx*/dtheta [delta] from the reduced KKT system is
checked against central differences of complete oracle solves at
theta +- h delta (h = 1e-5, FP64; the rounding of the perturbed solves rules
out much smaller steps): an independent route to the same number through the
optimality conditions of the perturbed problems, not through the
linearisation.  Cases: dead trades with active exposure rows (single period),
an active budget with zero holdings (single period), a multi-period
trajectory whose dead trades tie periods together (also differentiated in
the fixed final portfolio w_T), quadratic impact (d = 2) and a full factor
covariance.
"""
from dataclasses import replace

import numpy as np
import pytest

import oracle
from oracle import grad as OG
from paper_2604_22625_gb300 import synthetic as S


def _budget_case():
    p = S.make_single(40, 6, 13, n_onehot=2, lam1=1e-11, lam2=0.3, lam3=0.3)
    return p


def _full_omega_case():
    p = S.make_single(40, 5, 41, n_onehot=1)
    rng = np.random.default_rng(41)
    Q, _ = np.linalg.qr(rng.standard_normal((5, 5)))
    p.Omega = Q @ np.diag(rng.uniform(1e-5, 1e-4, 5)) @ Q.T
    p.Omega = 0.5 * (p.Omega + p.Omega.T)
    return p


CASES = {
    "single_dead_rows": lambda: S.make_single(40, 6, 11, n_onehot=2),
    "single_budget_zeros": _budget_case,
    "multi_T4": lambda: S.make_multi(4, 20, 4, 12, n_onehot=2),
    "single_quadratic_impact": lambda: S.make_single(40, 6, 17, n_onehot=2, d=2.0),
    "single_full_omega": _full_omega_case,
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_jvp_matches_central_differences_of_solves(case):
    prob = CASES[case]()
    sol = oracle.solve(prob)
    assert sol.polished and sol.reduced is not None
    red = sol.reduced
    if case == "single_budget_zeros":
        assert red.budget[0] and int((red.sx == 0).sum()) > 0
    elif case in ("single_dead_rows", "multi_T4"):
        assert int((~red.live).sum()) > 0 and len(red.box) > 0
    rng = np.random.default_rng(7)
    h = 1e-5
    names = OG.MULTI_PARAMS if case.startswith("multi") else OG.PARAMS
    for name in names:
        base = np.asarray(getattr(prob, name))
        delta = rng.standard_normal(base.shape) * np.abs(base).mean()
        dx = OG.jvp(prob, sol, name, delta)
        xp = oracle.solve(replace(prob, **{name: base + h * delta})).x
        xm = oracle.solve(replace(prob, **{name: base - h * delta})).x
        fd = (xp - xm) / (2 * h)
        scale = max(float(np.max(np.abs(dx))), 1e-12)
        assert float(np.max(np.abs(fd - dx))) <= 5e-6 * scale, (name, case)


def test_directional_vjp_is_linear_in_delta():
    prob = CASES["single_dead_rows"]()
    sol = oracle.solve(prob)
    rng = np.random.default_rng(3)
    g = rng.standard_normal(sol.x.shape)
    d1 = rng.standard_normal(prob.F.shape)
    d2 = rng.standard_normal(prob.F.shape)
    a = OG.directional_vjp(prob, sol, g, "F", d1)
    b = OG.directional_vjp(prob, sol, g, "F", d2)
    c = OG.directional_vjp(prob, sol, g, "F", 2.0 * d1 - 3.0 * d2)
    assert abs(c - (2.0 * a - 3.0 * b)) <= 1e-8 * (abs(a) + abs(b))
