"""Failure paths of the solver on the GPU, none of which faults or hangs it.

Every stop other than convergence ends the instance with a status in
ff_result (Sec. 4.1's solver has a 360 s limit; the library reports the
reason of every stop):

* max_iter = 1                      -> FF_MAX_ITER
* a device time limit of 1 us       -> FF_TIME_LIMIT (checked at the first KKT check)
* a NaN in alpha (host-side data)   -> FF_NUMERICAL: the host does not read device
                                       arrays, so the NaN reaches the kernel, which
                                       detects it in its FP64 KKT evaluation
* test_expire_first_wait = 1        -> FF_STALLED: the first wait of each instance
                                       for a panel-tile copy counts as expired while
                                       the copy itself is valid; the ring freezes and
                                       is drained before the team moves on

After each failed solve, the next solve on the same workspace (and, for the
batch, the same launch configuration) must converge: nothing of the failure
survives in the workspace or the device.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2604_22625_gb300 import _lib as L
from paper_2604_22625_gb300 import synthetic as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2604_22625_gb300 import api
    from paper_2604_22625_gb300.build import build
    build()
    return torch, api


def _solve(torch, api, prob, precision, ws=None, **kw):
    """One solve through the C ABI on workspace ws (allocated when None);
    returns (status, result record, ws)."""
    dtype = torch.float64 if precision == "f64" else torch.float32
    dp = api.to_device(prob, dtype=dtype)
    opts = api.options(precision, **kw)
    nb = L.ff_workspace_size(C.byref(dp.struct), 1, opts)
    assert nb > 0
    if ws is None:
        ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    assert ws.numel() >= nb
    res = torch.zeros(L.RESULT_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    w = torch.empty(dp.P * dp.n, dtype=dtype, device="cuda")
    fn = L.ff_solve_multi if int(prob.T) >= 2 else L.ff_solve_single
    s = torch.cuda.current_stream()
    rc = fn(dp.struct, opts, ws.data_ptr(), ws.numel(), res.data_ptr(), w.data_ptr(), 0, 0, s.cuda_stream)
    assert rc == L.FF_OK, L.ff_last_error()
    s.synchronize()
    rec = res.cpu().numpy().view(L.RESULT_DTYPE)[0]
    return int(rec["status"]), rec, ws


CASES = [
    ("single_f64", lambda: S.make_single(600, 12, 41, n_onehot=4), "f64", {}),
    ("single_f32_cluster4", lambda: S.make_single(3000, 20, 42, n_onehot=5).rounded(np.float32), "f32",
     {"cluster_size": 4}),
    ("multi_f32", lambda: S.make_multi(6, 400, 10, 43, n_onehot=3).rounded(np.float32), "f32", {}),
]


@pytest.mark.parametrize("name,make,prec,kw", CASES, ids=[c[0] for c in CASES])
def test_max_iter_then_converge(env, name, make, prec, kw):
    torch, api = env
    prob = make()
    st, rec, ws = _solve(torch, api, prob, prec, max_iter=1, **kw)
    assert st == L.FF_MAX_ITER and rec["iterations"] == 1, rec
    st, rec, _ = _solve(torch, api, prob, prec, ws=ws, tol=1e-6, **kw)
    assert st == L.FF_CONVERGED and rec["rel_kkt"] <= 1e-6, rec


@pytest.mark.parametrize("name,make,prec,kw", CASES, ids=[c[0] for c in CASES])
def test_time_limit_then_converge(env, name, make, prec, kw):
    torch, api = env
    prob = make()
    st, rec, ws = _solve(torch, api, prob, prec, time_limit=1e-6, **kw)
    assert st == L.FF_TIME_LIMIT, rec
    st, rec, _ = _solve(torch, api, prob, prec, ws=ws, tol=1e-6, **kw)
    assert st == L.FF_CONVERGED, rec


@pytest.mark.parametrize("name,make,prec,kw", CASES, ids=[c[0] for c in CASES])
def test_nan_input_then_converge(env, name, make, prec, kw):
    torch, api = env
    prob = make()
    bad = prob.rounded(np.float64)
    bad.alpha = np.array(bad.alpha, copy=True)
    bad.alpha.reshape(-1)[7] = np.nan
    st, rec, ws = _solve(torch, api, bad, prec, **kw)
    assert st == L.FF_NUMERICAL, rec
    st, rec, _ = _solve(torch, api, prob, prec, ws=ws, tol=1e-6, **kw)
    assert st == L.FF_CONVERGED, rec


@pytest.mark.parametrize("name,make,prec,kw", CASES, ids=[c[0] for c in CASES])
def test_expired_wait_then_converge(env, name, make, prec, kw):
    torch, api = env
    prob = make()
    st, rec, ws = _solve(torch, api, prob, prec, test_expire_first_wait=1, **kw)
    assert st == L.FF_STALLED, rec
    st, rec, _ = _solve(torch, api, prob, prec, ws=ws, tol=1e-6, **kw)
    assert st == L.FF_CONVERGED and rec["rel_kkt"] <= 1e-6, rec


def test_batch_mixed_statuses(env):
    """A batch in which every team stalls on its first copy: every instance
    reports FF_STALLED, and the same batch solved again converges."""
    torch, api = env
    probs = [S.make_single(n, 16, 50 + i, n_onehot=4).rounded(np.float32) for i, n in enumerate([300, 1200, 90])]
    probs += [S.make_multi(4, 200, 8, 60, n_onehot=2).rounded(np.float32)]
    br = api.BatchRunner(probs, precision="f32", test_expire_first_wait=1)
    br.run()
    torch.cuda.synchronize()
    assert all(i["status"] == L.FF_STALLED for i in br.results())
    br.opts.test_expire_first_wait = 0
    br.opts.tol = 1e-6
    br.run()
    torch.cuda.synchronize()
    assert all(i["status"] == L.FF_CONVERGED for i in br.results())


def test_precision_floor_then_fp64(env):
    """FF_PRECISION: with stall_checks = 1 an FP32 solve to 1e-9 stops at the
    first check that does not halve the relative KKT residual; the API then
    solves the instance again in FP64 on the same device data, and the result
    matches the oracle."""
    torch, api = env
    import oracle
    prob = S.make_single(400, 10, 44, n_onehot=3).rounded(np.float32)
    sol = api.solve(prob, precision="f32", tol=1e-9, stall_checks=1, escalate=False)
    assert sol.info["status"] == L.FF_PRECISION, sol.info
    sol = api.solve(prob, precision="f32", tol=1e-9, stall_checks=1)
    assert sol.info["escalated"] and sol.info["status"] == L.FF_CONVERGED, sol.info
    ref = oracle.solve(prob)
    assert float(np.max(np.abs(sol.x - ref.x))) <= 1e-5


def test_batch_bf16_precision_floor_then_fp64(env):
    """The batched form: instances stopped by FF_PRECISION in the BF16 mode are
    solved again in FP64 with F and A rounded to bfloat16 in the repack, so
    they solve exactly the data of the BF16 solve (checked against the oracle
    on the BF16-rounded data)."""
    torch, api = env
    import oracle
    probs = [S.make_single(n, 16, 70 + i, n_onehot=4) for i, n in enumerate([500, 900])]
    probs += [S.make_multi(4, 300, 8, 72, n_onehot=2)]
    br = api.BatchRunner(probs, precision="bf16", tol=1e-9, stall_checks=1)
    br.run()
    assert br.finish() == len(probs)
    infos = br.results()
    assert all(i["status"] == L.FF_CONVERGED and i["escalated"] for i in infos), infos
    for p, w in zip(probs, br.portfolios()):
        pr = p.with_F_rounded_bf16()
        ref = oracle.solve(pr)
        assert float(np.max(np.abs(np.asarray(w).reshape(ref.x.shape) - ref.x))) <= 1e-5


def test_warm_start(env):
    """ff_options.warm_start: started from its own solution an instance needs
    fewer iterations than from w0 (the returned point, rounded to the output
    type, is near the fixed point, and the restarts re-certify it); started
    from the solution of a neighbouring lambda it converges to the oracle's
    solution of its own problem.  Whether the neighbour's start also saves
    iterations depends on where the restarts fall (one case here took 5,633
    warm against 5,057 cold), so only convergence and parity are required."""
    torch, api = env
    import oracle
    for make, prec in ((lambda lam: S.make_single(800, 12, 91, n_onehot=4, lam2=lam, lam3=lam), "f64"),
                       (lambda lam: S.make_multi(6, 300, 8, 92, n_onehot=2, lam2=lam, lam3=lam).rounded(np.float32),
                        "f32")):
        p1, p2 = make(1.0), make(1.3)
        cold1 = api.solve(p1, precision=prec, return_duals=True, tol=1e-7)
        again = api.solve(p1, precision=prec, return_duals=True, tol=1e-7, warm=cold1)
        assert again.info["status"] == 0 and again.info["iterations"] < cold1.info["iterations"], \
            (again.info["iterations"], cold1.info["iterations"])
        assert float(np.max(np.abs(again.x - oracle.solve(p1).x))) <= 1e-5
        cold2 = api.solve(p2, precision=prec, return_duals=True, tol=1e-7)
        warm2 = api.solve(p2, precision=prec, return_duals=True, tol=1e-7, warm=cold1)
        assert cold2.info["status"] == 0 and warm2.info["status"] == 0, (cold2.info, warm2.info)
        ref = oracle.solve(p2)
        assert float(np.max(np.abs(warm2.x - ref.x))) <= 1e-5
