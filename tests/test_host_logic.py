"""Host-side logic without a GPU: the synthetic input recipe, the packed batch
layout, the benchmark's algorithmic-byte count, the adjoint dispatch of
BatchRunner and the argument checks of the differentiable solves."""
import os
import sys

import numpy as np
import pytest

from paper_2604_22625_gb300 import api, synthetic as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_single_recipe():
    p = S.config_single_small()
    n, k = p.F.shape
    assert (n, k, p.A.shape[0]) == (500, 20, 20)
    assert np.allclose(p.A, p.F.T)                        # A = F^T
    onehot = p.F[:, 10:]
    assert np.all(onehot.sum(axis=1) == 1.0) and set(np.unique(onehot)) == {0.0, 1.0}
    om = np.diag(p.Omega)
    assert np.count_nonzero(p.Omega - np.diag(om)) == 0 and om.min() >= 1e-5 and om.max() <= 1e-4
    assert p.D.min() >= 1e-4 and p.D.max() <= 9e-4
    assert p.s.min() >= 2e-4 and p.s.max() <= 2e-3 and p.q.min() >= 1e-3 and p.q.max() <= 1e-2
    assert abs(np.abs(p.w0).sum() - 0.9) < 1e-12
    assert abs(p.alpha.std() - 2e-3) < 3e-4
    assert np.all(p.L == -0.05) and np.all(p.U == 0.05)
    assert (p.GMV, p.lam1 * p.GMV, p.lam2, p.lam3, p.d) == (1e9, 10.0, 1.0, 1.0, 1.5)
    q = S.config_single_small()
    assert np.array_equal(p.F, q.F) and np.array_equal(p.alpha, q.alpha)   # seeded


def test_large_single_recipe():
    p = S.config_single_large()
    assert p.F.shape == (10000, 100) and p.A.shape == (160, 10000)
    H = p.A[100:]
    assert np.all(H.sum(axis=0) == 1.0)                   # one industry per asset
    assert np.all(p.U == 0.02) and np.all(p.L == -0.02)


def test_multi_recipe():
    p = S.make_multi(40, 3000, 20, 5)
    assert p.alpha.shape == (40, 3000) and p.D.shape == (40, 3000)
    a0, a1 = p.alpha[:-1].ravel(), p.alpha[1:].ravel()
    corr = np.corrcoef(a0, a1)[0, 1]
    assert abs(corr - 0.8) < 0.02                        # AR(1) correlation across t
    ratio = p.D / p.D[0]
    assert ratio.min() >= 0.8 / 1.2 - 1e-12 and ratio.max() <= 1.2 / 0.8 + 1e-12
    assert np.all(p.s == p.s[0]) and np.all(p.q == p.q[0])
    assert abs(np.abs(p.wT).sum() - 0.9) < 1e-12


def test_batch_recipe():
    b = S.config_batch(n_single=40, n_multi=10)
    singles, multis = b[:40], b[40:]
    assert all(p.T == 0 and 500 <= p.n <= 8000 and p.k in (40, 80) for p in singles)
    assert all(5 <= p.T <= 40 and 1000 <= p.n <= 4000 and p.k in (40, 80) for p in multis)


def test_pack_layout():
    probs = [S.make_single(37, 5, 1, n_onehot=2), S.make_multi(3, 20, 4, 2, n_onehot=1)]
    flat, lay = api.pack(probs, np.float32)
    for p, ent in zip(probs, lay):
        for nm in ("F", "Omega", "D", "alpha", "s", "q", "w0", "A", "L", "U"):
            off, size = ent[nm]
            assert off % 64 == 0                           # 256-byte aligned in FP32
            ref = np.asarray(getattr(p, nm) if nm != "Omega" else np.diag(p.Omega), dtype=np.float32).ravel()
            assert size == ref.size and np.array_equal(flat[off:off + size], ref)
        assert ent["omega_diag"] == 1
    assert "wT" in lay[1] and "wT" not in lay[0]


def test_algorithmic_bytes_formula():
    sys.path.insert(0, ROOT)
    import bench
    p = S.make_multi(4, 100, 8, 3, n_onehot=2)             # P = 3, R = 4, m = 8
    n, k, m, P, R = 100, 8, 8, 3, 4
    want = 2 * (n * k + m * n) * 2 + ((2 * P + 2 * R + 2) * n + 2 * m) * 4 + 3 * (P * n + P * m + R * n) * 4
    assert bench.algorithmic_bytes_per_iter(p, "bf16") == want
    s = S.make_single(100, 8, 3, n_onehot=2)
    want_f64 = 2 * (n * k + m * n) * 8 + ((2 + 2 + 2) * n + 2 * m) * 8 + 3 * (n + m + n) * 8
    assert bench.algorithmic_bytes_per_iter(s, "f64") == want_f64


def test_batchrunner_backward_dispatch(monkeypatch):
    """BatchRunner sends single-period instances to ff_backward_batch and
    multi-period ones to ff_backward_multi_batch, each with its own pointers,
    gradients (w_T for multi-period only), workspace and status slots, and
    reports the statuses in instance order (host logic; the C calls are
    recorded, not run)."""
    import torch

    from paper_2604_22625_gb300 import _lib as L
    from paper_2604_22625_gb300 import api
    from paper_2604_22625_gb300.build import build
    build()
    probs = [S.make_single(30, 4, 1, n_onehot=2), S.make_multi(3, 20, 4, 2, n_onehot=2),
             S.make_single(50, 4, 3, n_onehot=2), S.make_multi(4, 25, 4, 4, n_onehot=2)]
    calls = []

    def rec(kind):
        def f(structs, count, w, yA, yD, g, grads, ws, nb, status, stream):
            calls.append(dict(kind=kind, T=[structs[t].T for t in range(count)], count=count, w=list(w),
                              yA=list(yA), yD=list(yD), g=list(g), wT=[gr.wT for gr in grads],
                              alpha=[gr.alpha for gr in grads], nb=nb, status=status))
            return L.FF_OK
        return f

    monkeypatch.setattr(L, "ff_backward_batch", rec("single"))
    monkeypatch.setattr(L, "ff_backward_multi_batch", rec("multi"))
    br = api.BatchRunner(probs, precision="f64", device="cpu", duals=True)
    br.prepare_backward()

    class _Stream:
        cuda_stream = 0

    br.backward(_Stream())
    assert [c["kind"] for c in calls] == ["single", "multi"]
    single, multi = calls
    assert single["count"] == 2 and single["T"] == [0, 0]
    assert multi["count"] == 2 and multi["T"] == [3, 4]
    for c, idx in ((single, [0, 2]), (multi, [1, 3])):
        assert c["w"] == [br.w_ptrs[i] for i in idx]
        assert c["yA"] == [br.yA_ptrs[i] for i in idx] and c["yD"] == [br.yD_ptrs[i] for i in idx]
        assert c["g"] == [br.g_ptrs[i] for i in idx]
        assert c["alpha"] == [br.grads[i].alpha for i in idx]
    assert single["wT"] == [None, None] and all(v for v in multi["wT"])
    assert single["nb"] == L.ff_backward_batch_workspace_size(
        (L.ff_problem * 2)(br.structs[0], br.structs[2]), 2)
    base = br._bstatus_sub.data_ptr()
    assert single["status"] == base and multi["status"] == base + 8
    br._bstatus_sub.copy_(torch.tensor([10, 12, 11, 13], dtype=torch.int32))
    assert br.bstatus.tolist() == [10, 11, 12, 13]
    # one single-period launch and one cooperative multi-period launch
    assert br.backward_launches() == 2


def test_multi_autograd_rejects_a_single_period_shape():
    """FlashFolioMultiFn checks the T x n shape of alpha before any library call."""
    import torch

    from paper_2604_22625_gb300.autograd import SolveParams, solve_diff_multi
    n, k = 5, 2
    z = torch.zeros
    with pytest.raises(ValueError):
        solve_diff_multi(z(n), z(n, k), z(n), z(n), z(n), z(n), z(n), z(k), z(0, n), z(0), z(0), SolveParams())
