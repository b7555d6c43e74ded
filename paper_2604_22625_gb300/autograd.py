"""Differentiable solves: ``torch.autograd.Function`` over the C ABI.

``FlashFolioFn.apply(alpha, F, D, s, q, w0, Omega, A, L, U, params)`` returns
the optimal portfolio w* of the single-period model (Sec. 2.1, Eqs. 1-3) and
back-propagates through it with ``ff_backward_single`` (implicit
differentiation of the optimality conditions on the GPU).  Gradients flow to
alpha, F, D, s, q and w0; Omega, A, L and U are data without gradients.

``FlashFolioMultiFn.apply(alpha, F, D, s, q, w0, wT, Omega, A, L, U, params)``
does the same for the multi-period model (Sec. 2.2, Eqs. 4-6): alpha, D, s, q
are T x n, the result is the (T-1) x n trajectory w_1..w_{T-1}, and the
backward pass (``ff_backward``, multi-period adjoint) also returns the
gradient for w_T.

All tensors live on one CUDA device with one floating dtype (float32 or
float64); no arithmetic of the method runs in Python.

Implicit differentiation is valid only at a solution: unless
``SolveParams.check_status`` is False, the forward pass reads the solve's
ff_result.status (one device-to-host read) and raises ``SolveError`` unless
it is FF_CONVERGED, and the backward pass raises ``SolveError`` when the
adjoint reports a degenerate active set (non-positive pivot or curvature) or
an iteration limit.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import torch

from . import _lib as L


@dataclass(frozen=True)
class SolveParams:
    GMV: float = 1e9
    lam1: float = 10.0 / 1e9
    lam2: float = 1.0
    lam3: float = 1.0
    d: float = 1.5
    precision: str = "f32"
    tol: float = 1e-7
    max_iter: int = 400000
    time_limit: float = 360.0
    check_status: bool = True


class SolveError(RuntimeError):
    """A forward solve that did not converge, or an adjoint that failed."""


def _forward_status(res: torch.Tensor) -> int:
    return int(res[:4].view(torch.int32).item())


def _check_forward(res: torch.Tensor, prm: SolveParams, what: str) -> int:
    st = _forward_status(res)
    if prm.check_status and st != L.FF_CONVERGED:
        raise SolveError(f"{what}: the solve stopped with status {L.STATUS_NAMES.get(st, st)} "
                         f"(implicit differentiation needs a converged solution)")
    return st


def _check_backward(status: torch.Tensor, prm: SolveParams, what: str) -> None:
    if not prm.check_status:
        return
    st = int(status.abs().max().item())
    if st != 0:
        raise SolveError(f"{what}: adjoint status {st} (1/2: non-positive pivot, 3: iteration limit, "
                         f"4: non-positive curvature; a degenerate active set)")


_PREC = {"f64": L.FF_PREC_F64, "f32": L.FF_PREC_F32, "bf16": L.FF_PREC_BF16}


def _problem(t: dict, prm: SolveParams) -> L.ff_problem:
    p = L.ff_problem()
    n, k = t["F"].shape
    m = t["A"].shape[0]
    multi = "wT" in t
    p.n, p.k, p.m, p.T = n, k, m, (t["alpha"].shape[0] if multi else 0)
    p.dtype = L.FF_F64 if t["F"].dtype == torch.float64 else L.FF_F32
    p.omega_diag = 1 if t["Omega"].dim() == 1 else 0
    for nm in ("F", "Omega", "D", "alpha", "s", "q", "w0", "A", "L", "U"):
        setattr(p, nm, t[nm].data_ptr() if t[nm].numel() > 0 else None)
    p.wT = t["wT"].data_ptr() if multi else None
    p.GMV, p.lambda1, p.lambda2, p.lambda3, p.d = prm.GMV, prm.lam1, prm.lam2, prm.lam3, prm.d
    return p


class FlashFolioFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, alpha, F, D, s, q, w0, Omega, A, Lb, Ub, prm: SolveParams):
        t = {"alpha": alpha, "F": F, "D": D, "s": s, "q": q, "w0": w0, "Omega": Omega, "A": A, "L": Lb, "U": Ub}
        t = {k_: v.detach().contiguous() for k_, v in t.items()}
        dev = F.device
        dtype = F.dtype
        p = _problem(t, prm)
        opts = L.default_options(precision=_PREC[prm.precision], tol=prm.tol, max_iter=prm.max_iter,
                                 time_limit=prm.time_limit)
        ws_bytes = L.ff_workspace_size(C.byref(p), 1, opts)
        if ws_bytes == 0:
            raise ValueError("invalid problem or options")
        ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
        res = torch.zeros(L.RESULT_DTYPE.itemsize, dtype=torch.uint8, device=dev)
        n, m = p.n, p.m
        w = torch.empty(n, dtype=dtype, device=dev)
        yA = torch.empty(max(m, 1), dtype=dtype, device=dev)
        yD = torch.empty(n, dtype=dtype, device=dev)
        stream = torch.cuda.current_stream(dev)
        rc = L.ff_solve_single(p, opts, ws.data_ptr(), ws_bytes, res.data_ptr(), w.data_ptr(), yA.data_ptr(),
                               yD.data_ptr(), stream.cuda_stream)
        if rc != L.FF_OK:
            raise RuntimeError(f"ff_solve_single: {L.ff_status_string(rc)} {L.ff_last_error()}")
        ctx.prm = prm
        ctx.result = res
        ctx.status = _check_forward(res, prm, "ff_solve_single")
        ctx.save_for_backward(t["alpha"], t["F"], t["D"], t["s"], t["q"], t["w0"], t["Omega"], t["A"], t["L"],
                              t["U"], w, yA, yD)
        return w

    @staticmethod
    def backward(ctx, grad_w):
        alpha, F, D, s, q, w0, Omega, A, Lb, Ub, w, yA, yD = ctx.saved_tensors
        t = {"alpha": alpha, "F": F, "D": D, "s": s, "q": q, "w0": w0, "Omega": Omega, "A": A, "L": Lb, "U": Ub}
        p = _problem(t, ctx.prm)
        dev = F.device
        g = grad_w.detach().to(F.dtype).contiguous()
        need = ctx.needs_input_grad
        outs = {nm: (torch.empty_like(t[nm]) if need[i] else None)
                for i, nm in enumerate(("alpha", "F", "D", "s", "q", "w0"))}
        gr = L.ff_grads()
        for nm, tt in outs.items():
            setattr(gr, nm, tt.data_ptr() if tt is not None else None)
        ws_bytes = L.ff_backward_workspace_size(p)
        ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
        status = torch.zeros(1, dtype=torch.int32, device=dev)
        stream = torch.cuda.current_stream(dev)
        rc = L.ff_backward_single(p, w.data_ptr(), yA.data_ptr() if p.m > 0 else 0, yD.data_ptr(), g.data_ptr(), gr,
                                  ws.data_ptr(), ws_bytes, status.data_ptr(), stream.cuda_stream)
        if rc != L.FF_OK:
            raise RuntimeError(f"ff_backward_single: {L.ff_status_string(rc)} {L.ff_last_error()}")
        _check_backward(status, ctx.prm, "ff_backward_single")
        return (outs["alpha"], outs["F"], outs["D"], outs["s"], outs["q"], outs["w0"], None, None, None, None, None)


_MULTI_IN = ("alpha", "F", "D", "s", "q", "w0", "wT", "Omega", "A", "L", "U")
_MULTI_GRAD = ("alpha", "F", "D", "s", "q", "w0", "wT")


class FlashFolioMultiFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, alpha, F, D, s, q, w0, wT, Omega, A, Lb, Ub, prm: SolveParams):
        vals = (alpha, F, D, s, q, w0, wT, Omega, A, Lb, Ub)
        t = {nm: v.detach().contiguous() for nm, v in zip(_MULTI_IN, vals)}
        if t["alpha"].dim() != 2 or t["alpha"].shape[0] < 2:
            raise ValueError("alpha must be T x n with T >= 2")
        dev, dtype = F.device, F.dtype
        p = _problem(t, prm)
        opts = L.default_options(precision=_PREC[prm.precision], tol=prm.tol, max_iter=prm.max_iter,
                                 time_limit=prm.time_limit)
        ws_bytes = L.ff_workspace_size(C.byref(p), 1, opts)
        if ws_bytes == 0:
            raise ValueError("invalid problem or options")
        ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
        res = torch.zeros(L.RESULT_DTYPE.itemsize, dtype=torch.uint8, device=dev)
        P, n, m = p.T - 1, p.n, p.m
        w = torch.empty(P, n, dtype=dtype, device=dev)
        yA = torch.empty(max(P * m, 1), dtype=dtype, device=dev)
        yD = torch.empty(p.T, n, dtype=dtype, device=dev)
        stream = torch.cuda.current_stream(dev)
        rc = L.ff_solve_multi(p, opts, ws.data_ptr(), ws_bytes, res.data_ptr(), w.data_ptr(), yA.data_ptr(),
                              yD.data_ptr(), stream.cuda_stream)
        if rc != L.FF_OK:
            raise RuntimeError(f"ff_solve_multi: {L.ff_status_string(rc)} {L.ff_last_error()}")
        ctx.prm = prm
        ctx.result = res
        ctx.status = _check_forward(res, prm, "ff_solve_multi")
        ctx.save_for_backward(*[t[nm] for nm in _MULTI_IN], w, yA, yD)
        return w

    @staticmethod
    def backward(ctx, grad_w):
        saved = ctx.saved_tensors
        t = dict(zip(_MULTI_IN, saved[:len(_MULTI_IN)]))
        w, yA, yD = saved[len(_MULTI_IN):]
        p = _problem(t, ctx.prm)
        dev = t["F"].device
        g = grad_w.detach().to(t["F"].dtype).contiguous()
        need = ctx.needs_input_grad
        outs = {nm: (torch.empty_like(t[nm]) if need[i] else None) for i, nm in enumerate(_MULTI_GRAD)}
        gr = L.ff_grads()
        for nm, tt in outs.items():
            setattr(gr, nm, tt.data_ptr() if tt is not None else None)
        ws_bytes = L.ff_backward_workspace_size(p)
        ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
        status = torch.zeros(1, dtype=torch.int32, device=dev)
        stream = torch.cuda.current_stream(dev)
        rc = L.ff_backward(p, w.data_ptr(), yA.data_ptr() if p.m > 0 else 0, yD.data_ptr(), g.data_ptr(), gr,
                           ws.data_ptr(), ws_bytes, status.data_ptr(), stream.cuda_stream)
        if rc != L.FF_OK:
            raise RuntimeError(f"ff_backward: {L.ff_status_string(rc)} {L.ff_last_error()}")
        _check_backward(status, ctx.prm, "ff_backward")
        return tuple(outs[nm] for nm in _MULTI_GRAD) + (None, None, None, None, None)


def solve_diff_multi(alpha, F, D, s, q, w0, wT, Omega, A, Lb, Ub, prm: SolveParams = SolveParams()):
    """x* = (w_1..w_{T-1}) of the multi-period model, differentiable in alpha, F,
    D, s, q (T x n), w0 and w_T."""
    return FlashFolioMultiFn.apply(alpha, F, D, s, q, w0, wT, Omega, A, Lb, Ub, prm)


def solve_diff(alpha, F, D, s, q, w0, Omega, A, Lb, Ub, prm: SolveParams = SolveParams()):
    """w* of the single-period model, differentiable in alpha, F, D, s, q, w0."""
    return FlashFolioFn.apply(alpha, F, D, s, q, w0, Omega, A, Lb, Ub, prm)
