"""ff_solve_single_static: the single-period solve that allocates nothing.

Some callers cannot allocate device memory when they solve (an application
or plugin host that reserved all device memory up front, or a loop that
cannot afford the device synchronisation of cudaMalloc).  For them the
library solves on its own fixed device array instead of a caller workspace.
These tests call it through the C ABI and check it against ff_solve_single
(caller workspace) on the same device inputs, over two calls in a row, so
that whatever the first call leaves in the shared array cannot change the
second call's result.  The file is named to be collected last.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2604_22625_gb300 import _lib as L
from paper_2604_22625_gb300 import synthetic as S

TOL_W = 1e-5      # the parity tests' bound on |w - w*|_inf
TOL_KKT = 1e-6


def test_static_rejects_oversize_problem_on_host():
    """A problem whose workspace exceeds the fixed array is refused before any
    CUDA call (runs without a GPU: the pointers are never dereferenced)."""
    L.load()
    p = L.ff_problem()
    p.n, p.k, p.m, p.T, p.dtype, p.omega_diag = 2_000_000, 20, 20, 0, L.FF_F32, 1
    for nm in ("F", "Omega", "D", "alpha", "s", "q", "w0", "A", "L", "U"):
        setattr(p, nm, 4096)
    p.GMV, p.lambda1, p.lambda2, p.lambda3, p.d = 1e9, 1e-8, 1.0, 1.0, 1.5
    o = L.default_options()
    rc = L.ff_solve_single_static(p, o, 4096, 4096)
    assert rc == L.FF_ERR_WORKSPACE
    msg = L.ff_last_error()
    assert "static workspace" in msg and str(L.FF_STATIC_WORKSPACE_BYTES) in msg


@pytest.mark.gpu
def test_static_matches_workspace_entry_two_calls():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2604_22625_gb300 import api
    from paper_2604_22625_gb300.build import build
    build()
    L.load()
    dev = "cuda:0"
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream(dev)
    # the last case needs about 28.6 MiB of the 32 MiB array and, with n > 6144,
    # gets 16-CTA clusters (a non-portable cluster size)
    cases = [(S.make_single(2500, 24, 31, n_onehot=8).rounded(np.float32), "f32"),
             (S.make_single(700, 12, 32, n_onehot=4), "f64"),
             (S.make_single(8000, 110, 33, n_onehot=10), "f64")]
    prepared = []
    for prob, prec in cases:
        dtype = torch.float64 if prec == "f64" else torch.float32
        dp = api.to_device(prob, dtype=dtype, device=dev)
        opts = api.options(prec)
        ws_bytes = L.ff_workspace_size(C.byref(dp.struct), 1, opts)
        assert 0 < ws_bytes <= L.FF_STATIC_WORKSPACE_BYTES
        prepared.append((prob, dp, opts, ws_bytes, dtype))
    clusters, _ = L.ff_batch_plan(C.byref(prepared[-1][1].struct), 1, prepared[-1][2])
    assert clusters[0] == 16

    def fresh(dp, dtype):
        res = torch.zeros(L.RESULT_DTYPE.itemsize, dtype=torch.uint8, device=dev)
        w = torch.full((dp.n,), float("nan"), dtype=dtype, device=dev)
        yA = torch.full((max(dp.m, 1),), float("nan"), dtype=dtype, device=dev)
        yD = torch.full((dp.n,), float("nan"), dtype=dtype, device=dev)
        return res, w, yA, yD

    def host(res, w, yA, yD, m):
        return (res.cpu().numpy().view(L.RESULT_DTYPE)[0], w.cpu().numpy().astype(np.float64),
                yA.cpu().numpy().astype(np.float64)[:m], yD.cpu().numpy().astype(np.float64))

    # reference results through the caller-workspace entry point
    refs = []
    for prob, dp, opts, ws_bytes, dtype in prepared:
        ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
        out = fresh(dp, dtype)
        rc = L.ff_solve_single(dp.struct, opts, ws.data_ptr(), ws_bytes, *[t.data_ptr() for t in out],
                               stream.cuda_stream)
        assert rc == L.FF_OK, L.ff_last_error()
        stream.synchronize()
        refs.append(host(*out, dp.m))

    # two static calls in a row (the second reuses what the first left behind)
    outs = []
    for prob, dp, opts, ws_bytes, dtype in prepared:
        out = fresh(dp, dtype)
        rc = L.ff_solve_single_static(dp.struct, opts, *[t.data_ptr() for t in out], stream.cuda_stream)
        assert rc == L.FF_OK, L.ff_last_error()
        outs.append((out, dp.m))
    stream.synchronize()
    for (rref, wref, yAref, yDref), (out, m) in zip(refs, outs):
        rec, wv, yA, yD = host(*out, m)
        assert rref["status"] == L.FF_CONVERGED and rec["status"] == L.FF_CONVERGED, (rref, rec)
        assert rec["rel_kkt"] <= TOL_KKT
        assert np.all(np.isfinite(wv)) and np.all(np.isfinite(yA)) and np.all(np.isfinite(yD))
        assert float(np.max(np.abs(wv - wref))) <= TOL_W
        # the multipliers, relative to the largest of each kind
        for a, b in ((yA, yAref), (yD, yDref)):
            if b.size:
                assert float(np.max(np.abs(a - b))) <= TOL_W * float(np.max(np.abs(b))) + 1e-12
        assert abs(rec["primal_obj"] - rref["primal_obj"]) <= 1e-6 * abs(rref["primal_obj"])
