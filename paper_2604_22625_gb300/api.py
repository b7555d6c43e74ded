"""Python entry points over the C ABI, with PyTorch owning device memory.

``solve`` / ``solve_batch`` move a ``synthetic.Problem`` (or any object with
the same fields) to the GPU, size and allocate the workspace, call the C entry
point and read back the portfolio and the per-instance ``ff_result``.  No
arithmetic of the method happens here.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass
from typing import List, Optional, Sequence

import numpy as np
import torch

from . import _lib as L

PRECISIONS = {"f64": L.FF_PREC_F64, "f32": L.FF_PREC_F32, "bf16": L.FF_PREC_BF16}


@dataclass
class DeviceProblem:
    """Device copies of one instance and the ff_problem that points at them."""
    struct: L.ff_problem
    tensors: dict
    P: int
    R: int
    n: int
    m: int
    dtype: torch.dtype


def to_device(prob, dtype: torch.dtype = torch.float64, device: str = "cuda",
              pinned_host: Optional[dict] = None, stream: Optional[torch.cuda.Stream] = None) -> DeviceProblem:
    """Copy the arrays of ``prob`` to ``device`` as ``dtype`` (float64 or float32)."""
    multi = int(prob.T) >= 2
    names = ["F", "Omega", "D", "alpha", "s", "q", "w0", "A", "L", "U"] + (["wT"] if multi else [])
    t = {}
    for nm in names:
        a = getattr(prob, nm)
        if pinned_host is not None and nm in pinned_host:
            t[nm] = pinned_host[nm].to(device=device, non_blocking=True)
        else:
            t[nm] = torch.as_tensor(np.array(a, dtype=np.float64, copy=True), dtype=dtype).to(device)
    omega_diag = 0
    Om = np.asarray(prob.Omega)
    if Om.ndim == 2 and np.count_nonzero(Om - np.diag(np.diag(Om))) == 0:
        t["Omega"] = torch.as_tensor(np.array(np.diag(Om), dtype=np.float64, copy=True), dtype=dtype).to(device)
        omega_diag = 1
    n, k = prob.F.shape
    m = prob.A.shape[0]
    st = L.ff_problem()
    st.n, st.k, st.m = n, k, m
    st.T = int(prob.T) if multi else 0
    st.dtype = L.FF_F64 if dtype == torch.float64 else L.FF_F32
    st.omega_diag = omega_diag
    for nm in names:
        setattr(st, nm, t[nm].data_ptr() if t[nm].numel() > 0 else None)
    if not multi:
        st.wT = None
    st.GMV, st.lambda1, st.lambda2, st.lambda3, st.d = (float(prob.GMV), float(prob.lam1), float(prob.lam2),
                                                         float(prob.lam3), float(prob.d))
    P = int(prob.T) - 1 if multi else 1
    R = int(prob.T) if multi else 1
    return DeviceProblem(st, t, P, R, n, m, dtype)


@dataclass
class Solution:
    w: np.ndarray            # (n,) single, (T-1, n) multi
    yA: Optional[np.ndarray]
    yD: Optional[np.ndarray]
    info: dict

    @property
    def x(self) -> np.ndarray:
        return self.w.reshape(-1, self.w.shape[-1])


def _info(rec) -> dict:
    d = {name: (rec[name].tolist() if rec[name].ndim else rec[name].item()) for name in L.RESULT_DTYPE.names}
    d["status_name"] = L.STATUS_NAMES.get(d["status"], str(d["status"]))
    return d


def options(precision: str = "f32", **kw) -> L.ff_options:
    """ff_options with the library defaults, except a 60 s device time limit
    unless ``time_limit`` is given."""
    kw.setdefault("time_limit", 60.0)
    return L.default_options(precision=PRECISIONS[precision], **kw)


def solve(prob, precision: str = "f32", device: str = "cuda", return_duals: bool = False,
          stream: Optional[torch.cuda.Stream] = None, **opt_kw) -> Solution:
    """Solve one instance on the GPU; returns host copies of the results."""
    dtype = torch.float64 if precision == "f64" else torch.float32
    dp = to_device(prob, dtype=dtype, device=device)
    opts = options(precision, **opt_kw)
    ws_bytes = L.ff_workspace_size(C.byref(dp.struct), 1, opts)
    if ws_bytes == 0:
        raise ValueError("invalid problem or options")
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device=device)
    res = torch.zeros(L.RESULT_DTYPE.itemsize, dtype=torch.uint8, device=device)
    w = torch.empty(dp.P * dp.n, dtype=dtype, device=device)
    yA = torch.empty(max(dp.P * dp.m, 1), dtype=dtype, device=device) if return_duals else None
    yD = torch.empty(dp.R * dp.n, dtype=dtype, device=device) if return_duals else None
    s = stream if stream is not None else torch.cuda.current_stream(device)
    fn = L.ff_solve_multi if dp.P > 1 or int(prob.T) >= 2 else L.ff_solve_single
    rc = fn(dp.struct, opts, ws.data_ptr(), ws_bytes, res.data_ptr(), w.data_ptr(),
            yA.data_ptr() if yA is not None else 0, yD.data_ptr() if yD is not None else 0, s.cuda_stream)
    if rc != L.FF_OK:
        raise RuntimeError(f"solve failed: {L.ff_status_string(rc)} ({rc})")
    s.synchronize()
    rec = res.cpu().numpy().view(L.RESULT_DTYPE)[0]
    wn = w.cpu().numpy().astype(np.float64)
    if int(prob.T) >= 2:
        wn = wn.reshape(dp.P, dp.n)
    return Solution(wn, yA.cpu().numpy().astype(np.float64)[:dp.P * dp.m].reshape(dp.P, dp.m) if yA is not None else None,
                    yD.cpu().numpy().astype(np.float64).reshape(dp.R, dp.n) if yD is not None else None,
                    _info(rec))


class BatchRunner:
    """Device-resident batch: inputs copied once, ``run()`` re-solves them all
    in one persistent launch (what the throughput benchmark times)."""

    def __init__(self, problems: Sequence, precision: str = "bf16", device: str = "cuda", **opt_kw):
        self.precision = precision
        self.dtype = torch.float64 if precision == "f64" else torch.float32
        self.dps: List[DeviceProblem] = [to_device(p, dtype=self.dtype, device=device) for p in problems]
        self.count = len(self.dps)
        self.structs = (L.ff_problem * self.count)(*[d.struct for d in self.dps])
        self.opts = options(precision, **opt_kw)
        self.ws_bytes = L.ff_workspace_size(self.structs, self.count, self.opts)
        if self.ws_bytes == 0:
            raise ValueError("invalid problem or options")
        self.ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device=device)
        self.res = torch.zeros(L.RESULT_DTYPE.itemsize * self.count, dtype=torch.uint8, device=device)
        self.w = [torch.empty(d.P * d.n, dtype=self.dtype, device=device) for d in self.dps]
        self.w_ptrs = [t.data_ptr() for t in self.w]

    def run(self, stream: Optional[torch.cuda.Stream] = None) -> None:
        s = stream if stream is not None else torch.cuda.current_stream()
        rc = L.ff_solve_batch(self.structs, self.count, self.opts, self.ws.data_ptr(), self.ws_bytes,
                              self.res.data_ptr(), self.w_ptrs, s.cuda_stream)
        if rc != L.FF_OK:
            raise RuntimeError(f"batch solve failed: {L.ff_status_string(rc)} ({rc})")

    def results(self) -> List[dict]:
        recs = self.res.cpu().numpy().view(L.RESULT_DTYPE)
        return [_info(r) for r in recs]

    def portfolios(self) -> List[np.ndarray]:
        out = []
        for d, t in zip(self.dps, self.w):
            a = t.cpu().numpy().astype(np.float64)
            out.append(a.reshape(d.P, d.n) if d.P > 1 or d.struct.T >= 2 else a)
        return out


def solve_batch(problems: Sequence, precision: str = "bf16", device: str = "cuda", **opt_kw):
    """Solve many instances in one persistent launch; returns (portfolios, infos)."""
    br = BatchRunner(problems, precision=precision, device=device, **opt_kw)
    br.run()
    torch.cuda.synchronize()
    return br.portfolios(), br.results()
