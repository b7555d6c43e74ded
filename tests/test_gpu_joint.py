"""GPU parity of the joint primal prox variant (ff_solve_joint_batch).

The variant solves the same single-period problem (Eqs. 1-3) with the trading
cost and the budget set in one primal prox, so its solution is compared with
the FP64 oracle's solution of the same instance, with the bars of the plain
solver's parity tests: converged at TOL_SOLVE, the kernel's relative KKT <=
1e-6, |w - w*|_inf <= 1e-5, relative objective gap <= 1e-6, and the oracle's
own KKT evaluation at the returned (w, y_A, y_D) -- y_D the trade multiplier
the kernel recovers from the prox's optimality condition -- <= 1e-6.  The
plain FP64 solver runs the same instances, and both must agree.
"""
import numpy as np
import pytest

import oracle
from oracle import Scaled
from oracle.kkt import evaluate
from paper_2604_22625_gb300 import synthetic as S

pytestmark = pytest.mark.gpu

TOL_W = 1e-5
TOL_OBJ = 1e-6
TOL_KKT = 1e-6
TOL_SOLVE = 2e-7


@pytest.fixture(scope="module")
def api():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2604_22625_gb300 import api as _api
    from paper_2604_22625_gb300.build import build
    build()
    return _api


def _no_rows(p):
    p.A = np.zeros((0, p.n))
    p.L = np.zeros(0)
    p.U = np.zeros(0)
    return p


def _tight_budget(p):
    # a strong signal against a start on the budget's boundary: the l1 ball binds
    p.alpha = p.alpha * 20.0
    p.w0 = p.w0 / np.abs(p.w0).sum()
    return p


CASES = {
    "small_rows": lambda: S.config_single_small(),
    "ragged_33": lambda: S.make_single(33, 3, 2, n_onehot=1),
    "ragged_1000": lambda: S.make_single(1000, 24, 4, n_onehot=8),
    "no_rows": lambda: _no_rows(S.make_single(400, 8, 7, n_onehot=2)),
    "budget_binds": lambda: _tight_budget(S.make_single(600, 10, 8, n_onehot=3)),
    "impact_d2": lambda: S.make_single(500, 12, 9, n_onehot=4, d=2.0),
    "impact_d13": lambda: S.make_single(500, 12, 10, n_onehot=4, d=1.3),
    "spread_only": lambda: S.make_single(500, 12, 11, n_onehot=4, lam3=0.0),
}


def _check(prob, sol, ref):
    sc = Scaled(prob)
    info = sol.info
    assert info["status_name"] == "converged", info
    assert info["rel_kkt"] <= TOL_KKT, info
    err = float(np.max(np.abs(sol.x - ref.x)))
    pobj = sc.objective(sol.x)
    gap = abs(pobj - ref.obj) / abs(ref.obj)
    assert err <= TOL_W, (err, info)
    assert gap <= TOL_OBJ, (gap, info)
    assert abs(info["primal_obj"] - pobj) <= 1e-9 * abs(pobj) + 1e-14
    k = evaluate(sc, sol.x, sol.yA, sol.yD)
    assert k.rel_kkt <= TOL_KKT, k
    assert np.abs(sol.x).sum() <= 1.0 + 1e-12


@pytest.mark.parametrize("name", list(CASES))
def test_joint_matches_oracle(api, name):
    prob = CASES[name]()
    sol = api.solve_joint([prob], tol=TOL_SOLVE)[0]
    _check(prob, sol, oracle.solve(prob))


def test_joint_batch_matches_plain_split(api):
    """A batch of mixed sizes in one launch; every instance matches the oracle,
    and the plain FP64 split reaches the same point."""
    probs = [S.make_single(n, k, 200 + i, n_onehot=max(1, k // 3)) for i, (n, k) in
             enumerate([(300, 9), (1200, 20), (77, 4), (2500, 30)])]
    sols = api.solve_joint(probs, tol=TOL_SOLVE)
    for p, s in zip(probs, sols):
        _check(p, s, oracle.solve(p))
        plain = api.solve(p, precision="f64", tol=TOL_SOLVE)
        assert float(np.max(np.abs(plain.x - s.x))) <= 2 * TOL_W


def test_joint_max_iter_and_time_limit(api):
    """The stops of the plain solver: max_iter gives FF_MAX_ITER after exactly
    that many iterations, a 1 us device time limit FF_TIME_LIMIT at the first
    check; a multi-period instance is refused (FF_ERR_UNSUPPORTED)."""
    from paper_2604_22625_gb300 import _lib as L
    prob = S.make_single(300, 6, 12, n_onehot=2)
    s = api.solve_joint([prob], max_iter=5)[0]
    assert s.info["status"] == L.FF_MAX_ITER and s.info["iterations"] == 5, s.info
    s = api.solve_joint([prob], time_limit=1e-6)[0]
    assert s.info["status"] == L.FF_TIME_LIMIT, s.info
    with pytest.raises(ValueError):
        api.solve_joint([S.make_multi(3, 50, 4, 13, n_onehot=2)])
