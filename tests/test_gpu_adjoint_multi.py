"""GPU multi-period adjoint (ff_backward_multi_batch through BatchRunner)
against the oracle's implicit-function derivative (oracle/grad.py, pinned by
central differences of complete solves in test_oracle_grad.py, w_T included).

For L = <g, x*> with a random g over the T-1 free periods, and for every
parameter block theta in (alpha, F, D, s, q, w0, w_T), the GPU gradient
contracted with a random direction must match the oracle's directional
derivative to 1e-4 relative (the differentiation bar).  Cases: dead trades
that tie periods to w0 and w_T with active exposure rows, many zero holdings
with active budgets, quadratic impact (d = 2), FP32 data, and a batch that
mixes single- and multi-period instances.  At the largest differentiation
size (T = 50, n = 2000, k = 60) the oracle cannot polish, so the check there
is a property: the VJP along alpha equals central differences of GPU solves.
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


CASES = {
    "ties_w0_wT_f64": (lambda: S.make_multi(4, 20, 4, 12, n_onehot=2), "f64"),
    "zeros_budget_f64": (lambda: S.make_multi(6, 200, 12, 1), "f64"),
    "quadratic_impact_f64": (lambda: S.make_multi(5, 60, 6, 3, n_onehot=2, d=2.0), "f64"),
    "rounded_f32": (lambda: S.make_multi(5, 60, 6, 3, n_onehot=2).rounded(np.float32), "f32"),
}


def _check(br, i, prob, sol, g, rng, names):
    for nm in names:
        grad = br.gradient(i, nm)
        delta = rng.standard_normal(grad.shape)
        a = float(np.sum(grad * delta))
        b = OG.directional_vjp(prob, sol, g, nm, delta)
        scale = float(np.linalg.norm(grad) * np.linalg.norm(delta))
        assert abs(a - b) <= TOL_GRAD * abs(b) + 1e-7 * scale, (i, nm, a, b)


def _run(torch, probs, precision, tol, seed):
    from paper_2604_22625_gb300 import api
    br = api.BatchRunner(probs, precision=precision, duals=True, tol=tol)
    br.prepare_backward()
    rng = np.random.default_rng(seed)
    gs = []
    for i, p in enumerate(probs):
        P = int(p.T) - 1 if int(p.T) >= 2 else 1
        g = rng.standard_normal(P * p.F.shape[0])
        o = int(br.w_off[i])
        br.g_dev[o:o + g.size] = torch.tensor(g, dtype=br.g_dev.dtype, device=br.g_dev.device)
        gs.append(g.reshape(P, -1) if int(p.T) >= 2 else g)
    br.run()
    br.backward()
    torch.cuda.synchronize()
    assert all(r["status_name"] == "converged" for r in br.results())
    assert int(br.bstatus.abs().sum().item()) == 0
    return br, gs, rng


@pytest.mark.parametrize("case", sorted(CASES))
def test_multi_vjp_matches_oracle(torch_mod, case):
    make, prec = CASES[case]
    prob = make()
    sol = oracle.solve(prob)
    assert sol.polished
    br, gs, rng = _run(torch_mod, [prob], prec, 1e-10 if prec == "f64" else 1e-7, 5)
    assert float(np.max(np.abs(br.portfolios()[0] - sol.x))) <= 1e-5
    _check(br, 0, prob, sol, gs[0], rng, OG.MULTI_PARAMS)


def test_mixed_batch_backward(torch_mod):
    """Single- and multi-period instances in one BatchRunner: each kind goes to
    its own adjoint call, every instance matches its oracle derivative."""
    probs = [S.make_single(40, 6, 11, n_onehot=2), S.make_multi(4, 20, 4, 12, n_onehot=2),
             S.make_single(300, 12, 44, n_onehot=4), S.make_multi(5, 60, 6, 3, n_onehot=2)]
    br, gs, rng = _run(torch_mod, probs, "f64", 1e-10, 21)
    for i, p in enumerate(probs):
        sol = oracle.solve(p)
        _check(br, i, p, sol, gs[i], rng, OG.MULTI_PARAMS if int(p.T) >= 2 else OG.PARAMS)


def test_full_size_vjp_alpha_matches_solve_differences(torch_mod):
    """T = 50, n = 2000, k = 60: <dL/dalpha, delta> against central differences
    of two GPU solves at alpha +- h delta (L = <g, x*>)."""
    torch = torch_mod
    from dataclasses import replace

    from paper_2604_22625_gb300 import api
    prob = S.make_multi(50, 2000, 60, 4 * 10 ** 6 + 64)
    br, gs, rng = _run(torch, [prob], "f64", 1e-10, 3)
    grad = br.gradient(0, "alpha")
    delta = rng.standard_normal(grad.shape) * 2e-3
    a = float(np.sum(grad * delta))
    h = 1e-3
    vals = []
    for sgn_ in (1.0, -1.0):
        pp = replace(prob, alpha=prob.alpha + sgn_ * h * delta)
        b2 = api.BatchRunner([pp], precision="f64", tol=1e-10)
        b2.run()
        torch.cuda.synchronize()
        vals.append(float(np.sum(gs[0] * b2.portfolios()[0])))
    fd = (vals[0] - vals[1]) / (2 * h)
    assert abs(a - fd) <= 1e-2 * abs(fd), (a, fd)


def test_autograd_multi_matches_oracle(torch_mod):
    """solve_diff_multi: L = <g, x*> back-propagated through torch autograd
    gives the oracle's derivative for every parameter block, w_T included."""
    torch = torch_mod
    from paper_2604_22625_gb300.autograd import SolveParams, solve_diff_multi
    prob = CASES["ties_w0_wT_f64"][0]()
    sol = oracle.solve(prob)
    dev = "cuda"
    t = {nm: torch.tensor(np.asarray(getattr(prob, nm), dtype=np.float64), device=dev)
         for nm in ("alpha", "F", "D", "s", "q", "w0", "wT", "A", "L", "U")}
    t["Omega"] = torch.tensor(np.diag(prob.Omega).copy(), device=dev)
    for nm in OG.MULTI_PARAMS:
        t[nm].requires_grad_(True)
    prm = SolveParams(GMV=prob.GMV, lam1=prob.lam1, lam2=prob.lam2, lam3=prob.lam3, d=prob.d, precision="f64",
                      tol=1e-10)
    x = solve_diff_multi(t["alpha"], t["F"], t["D"], t["s"], t["q"], t["w0"], t["wT"], t["Omega"], t["A"],
                         t["L"], t["U"], prm)
    rng = np.random.default_rng(8)
    g = rng.standard_normal(sol.x.shape)
    (x * torch.tensor(g, device=dev)).sum().backward()
    torch.cuda.synchronize()
    assert float(np.max(np.abs(x.detach().cpu().numpy() - sol.x))) <= 1e-5
    for nm in OG.MULTI_PARAMS:
        grad = t[nm].grad.detach().cpu().numpy()
        delta = rng.standard_normal(grad.shape)
        a = float(np.sum(grad * delta))
        b = OG.directional_vjp(prob, sol, g, nm, delta)
        scale = float(np.linalg.norm(grad) * np.linalg.norm(delta))
        assert abs(a - b) <= TOL_GRAD * abs(b) + 1e-7 * scale, (nm, a, b)
