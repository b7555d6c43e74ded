"""GPU adjoint (ff_backward_single through FlashFolioFn) against the oracle's
implicit-function derivative (oracle/grad.py, itself pinned by central
differences of complete solves in test_oracle_grad.py).

For L = <g, w*> with a random g, and for every parameter block theta in
(alpha, F, D, s, q, w0), the GPU gradient contracted with a random direction
delta must match the oracle's directional derivative to 1e-4 relative (the
differentiation bar).  A second test differentiates the scaled return-minus-
risk objective alpha^T w* - kappa w*^T Sigma w* through torch autograd (its
explicit dependence on alpha, F, D plus the implicit one through w*).
"""
import numpy as np
import pytest

import oracle
from oracle import grad as OG
from paper_2604_22625_gb300 import synthetic as S

pytestmark = pytest.mark.gpu

TOL_GRAD = 1e-4


@pytest.fixture(scope="module")
def torch_mod():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2604_22625_gb300.build import build
    build()
    return torch


def _full_omega_case():
    p = S.make_single(120, 5, 41, n_onehot=1)
    rng = np.random.default_rng(41)
    Q, _ = np.linalg.qr(rng.standard_normal((5, 5)))
    p.Omega = Q @ np.diag(rng.uniform(1e-5, 1e-4, 5)) @ Q.T
    p.Omega = 0.5 * (p.Omega + p.Omega.T)
    return p


CASES = {
    "dead_rows_f64": (lambda: S.make_single(40, 6, 11, n_onehot=2), "f64", 1e-10),
    "budget_zeros_f64": (lambda: S.make_single(40, 6, 13, n_onehot=2, lam1=1e-11, lam2=0.3, lam3=0.3), "f64", 1e-10),
    "full_omega_f64": (_full_omega_case, "f64", 1e-10),
    "diff_config_f32": (lambda: S.config_diff(n_single=1, n_multi=0)[0], "f32", 1e-7),
}


def _tensors(torch, prob, dtype, dev):
    Om = np.asarray(prob.Omega)
    if np.count_nonzero(Om - np.diag(np.diag(Om))) == 0:
        Om = np.diag(Om)
    t = {}
    for nm in ("alpha", "F", "D", "s", "q", "w0", "A", "L", "U"):
        t[nm] = torch.tensor(np.asarray(getattr(prob, nm), dtype=np.float64), dtype=dtype, device=dev)
    t["Omega"] = torch.tensor(np.asarray(Om, dtype=np.float64), dtype=dtype, device=dev)
    return t


def _solve_diff(torch, prob, prec, tol):
    from paper_2604_22625_gb300.autograd import SolveParams, solve_diff
    dtype = torch.float64 if prec == "f64" else torch.float32
    t = _tensors(torch, prob, dtype, "cuda")
    for nm in OG.PARAMS:
        t[nm].requires_grad_(True)
    prm = SolveParams(GMV=prob.GMV, lam1=prob.lam1, lam2=prob.lam2, lam3=prob.lam3, d=prob.d, precision=prec, tol=tol)
    w = solve_diff(t["alpha"], t["F"], t["D"], t["s"], t["q"], t["w0"], t["Omega"], t["A"], t["L"], t["U"], prm)
    return t, w


@pytest.mark.parametrize("case", sorted(CASES))
def test_vjp_matches_oracle(torch_mod, case):
    torch = torch_mod
    make, prec, tol = CASES[case]
    prob = make()
    if prec == "f32":
        prob = prob.rounded(np.float32)
    sol = oracle.solve(prob)
    assert sol.polished
    t, w = _solve_diff(torch, prob, prec, tol)
    rng = np.random.default_rng(5)
    g = rng.standard_normal(prob.n)
    (w * torch.tensor(g, dtype=w.dtype, device=w.device)).sum().backward()
    torch.cuda.synchronize()
    assert float(np.max(np.abs(w.detach().cpu().numpy() - sol.w))) <= 1e-5
    for nm in OG.PARAMS:
        grad = t[nm].grad.detach().cpu().numpy().astype(np.float64).reshape(np.shape(getattr(prob, nm)))
        delta = rng.standard_normal(grad.shape)
        a = float(np.sum(grad * delta))
        b = OG.directional_vjp(prob, sol, g, nm, delta)
        scale = float(np.linalg.norm(grad) * np.linalg.norm(delta))
        assert abs(a - b) <= TOL_GRAD * abs(b) + 1e-7 * scale, (case, nm, a, b)


def test_autograd_return_minus_risk(torch_mod):
    """d(alpha^T w* - kappa w*^T Sigma w*)/d theta through torch autograd."""
    torch = torch_mod
    prob = S.make_single(40, 6, 11, n_onehot=2)
    sol = oracle.solve(prob)
    t, w = _solve_diff(torch, prob, "f64", 1e-10)
    kap = prob.lam1 * prob.GMV
    Fw = t["F"].T @ w
    Sw = t["F"] @ (t["Omega"] * Fw) + t["D"] * w
    ell = t["alpha"] @ w - kap * (w @ Sw)
    ell.backward()
    x = sol.w
    Om = np.diag(prob.Omega)
    Sigx = prob.F @ (Om * (prob.F.T @ x)) + prob.D * x
    g = prob.alpha - 2.0 * kap * Sigx                     # d ell / d w at fixed data
    explicit = {"alpha": x, "D": -kap * x * x, "F": -2.0 * kap * np.outer(x, Om * (prob.F.T @ x)),
                "s": np.zeros_like(x), "q": np.zeros_like(x), "w0": np.zeros_like(x)}
    rng = np.random.default_rng(9)
    for nm in OG.PARAMS:
        grad = t[nm].grad.detach().cpu().numpy().reshape(np.shape(getattr(prob, nm)))
        delta = rng.standard_normal(grad.shape)
        a = float(np.sum(grad * delta))
        b = float(np.sum(explicit[nm] * delta)) + OG.directional_vjp(prob, sol, g, nm, delta)
        scale = float(np.linalg.norm(grad) * np.linalg.norm(delta))
        assert abs(a - b) <= TOL_GRAD * abs(b) + 1e-7 * scale, (nm, a, b)


def test_batched_backward_matches_oracle(torch_mod):
    """ff_backward_batch over several instances in one launch (through
    BatchRunner with duals) gives each instance's oracle derivative."""
    torch = torch_mod
    from paper_2604_22625_gb300 import api
    probs = [CASES["dead_rows_f64"][0](), CASES["budget_zeros_f64"][0](), S.make_single(300, 12, 44, n_onehot=4)]
    br = api.BatchRunner(probs, precision="f64", duals=True, tol=1e-10)
    br.prepare_backward()
    rng = np.random.default_rng(21)
    gs = [rng.standard_normal(p.n) for p in probs]
    for i, g in enumerate(gs):
        o = int(br.w_off[i])
        br.g_dev[o:o + probs[i].n] = torch.tensor(g, dtype=br.g_dev.dtype, device=br.g_dev.device)
    br.run()
    br.backward()
    torch.cuda.synchronize()
    assert all(i["status_name"] == "converged" for i in br.results())
    assert int(br.bstatus.abs().sum().item()) == 0
    for i, p in enumerate(probs):
        sol = oracle.solve(p)
        for nm in OG.PARAMS:
            grad = br.gradient(i, nm)
            delta = rng.standard_normal(grad.shape)
            a = float(np.sum(grad * delta))
            b = OG.directional_vjp(p, sol, gs[i], nm, delta)
            scale = float(np.linalg.norm(grad) * np.linalg.norm(delta))
            assert abs(a - b) <= TOL_GRAD * abs(b) + 1e-7 * scale, (i, nm, a, b)


def test_autograd_raises_on_unconverged_forward():
    """Implicit differentiation is only valid at a solution: a forward solve
    stopped by max_iter raises SolveError unless check_status is False."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2604_22625_gb300.autograd import SolveError, SolveParams, solve_diff
    from paper_2604_22625_gb300.build import build
    build()
    prob = S.make_single(200, 8, 71, n_onehot=2)
    t = {nm: torch.tensor(np.asarray(getattr(prob, nm), dtype=np.float64), device="cuda")
         for nm in ("alpha", "F", "D", "s", "q", "w0", "A", "L", "U")}
    t["Omega"] = torch.tensor(np.diag(prob.Omega).copy(), device="cuda")
    t["alpha"].requires_grad_(True)
    args = (t["alpha"], t["F"], t["D"], t["s"], t["q"], t["w0"], t["Omega"], t["A"], t["L"], t["U"])
    with pytest.raises(SolveError):
        solve_diff(*args, SolveParams(precision="f64", max_iter=1))
    w = solve_diff(*args, SolveParams(precision="f64", max_iter=1, check_status=False))
    assert w.shape == (200,)
