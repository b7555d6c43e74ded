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


def escalation_options(opts: L.ff_options) -> L.ff_options:
    """Options of the FP64 re-solve of an instance that ended with
    FF_PRECISION in the FP32 or BF16 mode: the same tolerances and limits in
    FF_PREC_F64, with F and A rounded to bfloat16 in the repack when the first
    solve was BF16 (so both solves see the same data), warm-started from the
    point the FP32 solve returned (its output buffers)."""
    o = L.ff_options()
    C.pointer(o)[0] = opts
    o.round_panels_bf16 = 1 if opts.precision == L.FF_PREC_BF16 else 0
    o.precision = L.FF_PREC_F64
    o.reuse_workspace = 0
    o.warm_start = 1
    return o


def solve(prob, precision: str = "f32", device: str = "cuda", return_duals: bool = False,
          stream: Optional[torch.cuda.Stream] = None, escalate: bool = True, warm: Optional[Solution] = None,
          **opt_kw) -> Solution:
    """Solve one instance on the GPU; returns host copies of the results.

    With ``escalate`` (default), an FP32/BF16 solve that ends with
    FF_PRECISION is solved again in FP64 on the same device data (the
    returned ``info["escalated"]`` says so).  ``warm``: a Solution of a
    neighbouring problem of the same shape (another date or lambda) to start
    from (ff_options.warm_start; its multipliers are used when present)."""
    dtype = torch.float64 if precision == "f64" else torch.float32
    dp = to_device(prob, dtype=dtype, device=device)
    if warm is not None:
        opt_kw["warm_start"] = 1
        return_duals = return_duals or warm.yD is not None
    opts = options(precision, **opt_kw)
    ws_bytes = L.ff_workspace_size(C.byref(dp.struct), 1, opts)
    if ws_bytes == 0:
        raise ValueError("invalid problem or options")
    res = torch.zeros(L.RESULT_DTYPE.itemsize, dtype=torch.uint8, device=device)
    w = torch.empty(dp.P * dp.n, dtype=dtype, device=device)
    yA = torch.empty(max(dp.P * dp.m, 1), dtype=dtype, device=device) if return_duals else None
    yD = torch.empty(dp.R * dp.n, dtype=dtype, device=device) if return_duals else None
    s = stream if stream is not None else torch.cuda.current_stream(device)
    fn = L.ff_solve_multi if dp.P > 1 or int(prob.T) >= 2 else L.ff_solve_single
    if warm is not None:
        w.copy_(torch.as_tensor(np.asarray(warm.w, dtype=np.float64).reshape(-1), dtype=dtype))
        if yA is not None:
            yA.zero_()
            if warm.yA is not None and dp.m > 0:
                yA[:dp.P * dp.m].copy_(torch.as_tensor(np.asarray(warm.yA).reshape(-1), dtype=dtype))
        if yD is not None:
            yD.zero_()
            if warm.yD is not None:
                yD.copy_(torch.as_tensor(np.asarray(warm.yD).reshape(-1), dtype=dtype))

    def call(o, nbytes):
        ws = torch.empty(nbytes, dtype=torch.uint8, device=device)
        rc = fn(dp.struct, o, ws.data_ptr(), nbytes, res.data_ptr(), w.data_ptr(),
                yA.data_ptr() if yA is not None else 0, yD.data_ptr() if yD is not None else 0, s.cuda_stream)
        if rc != L.FF_OK:
            raise RuntimeError(f"solve failed: {L.ff_status_string(rc)} ({rc}) {L.ff_last_error()}")
        s.synchronize()
        return res.cpu().numpy().view(L.RESULT_DTYPE)[0]

    rec = call(opts, ws_bytes)
    escalated = False
    first_seconds = 0.0
    if escalate and int(rec["status"]) == L.FF_PRECISION and opts.precision != L.FF_PREC_F64:
        first_seconds = float(rec["seconds"])
        o64 = escalation_options(opts)     # starts from the FP32 attempt's point in w, yA, yD
        rec = call(o64, L.ff_workspace_size(C.byref(dp.struct), 1, o64))
        escalated = True
    wn = w.cpu().numpy().astype(np.float64)
    if int(prob.T) >= 2:
        wn = wn.reshape(dp.P, dp.n)
    info = _info(rec)
    info["escalated"] = escalated
    info["first_seconds"] = first_seconds   # device time of the FP32 attempt before an FP64 re-solve
    return Solution(wn, yA.cpu().numpy().astype(np.float64)[:dp.P * dp.m].reshape(dp.P, dp.m) if yA is not None else None,
                    yD.cpu().numpy().astype(np.float64).reshape(dp.R, dp.n) if yD is not None else None,
                    info)


_FIELDS = ("F", "Omega", "D", "alpha", "s", "q", "w0", "wT", "A", "L", "U")
_ALIGN = 64   # elements: every packed array starts on a 256-byte boundary


def _omega_arg(prob):
    """(array, omega_diag): the diagonal of Omega when it has no off-diagonal entries."""
    Om = np.asarray(prob.Omega, dtype=np.float64)
    if Om.ndim == 2 and np.count_nonzero(Om - np.diag(np.diag(Om))) == 0:
        return np.diag(Om), 1
    return Om, 0


def pack(problems: Sequence, np_dtype) -> tuple:
    """Lay the arrays of every instance out in one flat host buffer.

    Returns (flat, layout) where layout[i] maps a field name to (offset, size)
    in elements of ``flat`` and carries ``omega_diag``.  One buffer means one
    host-to-device copy for the whole batch."""
    layout, chunks, off = [], [], 0
    for p in problems:
        ent = {}
        multi = int(p.T) >= 2
        for nm in _FIELDS:
            if nm == "wT" and not multi:
                continue
            if nm == "Omega":
                a, ent["omega_diag"] = _omega_arg(p)
            else:
                a = np.asarray(getattr(p, nm), dtype=np.float64)
            a = a.reshape(-1)
            ent[nm] = (off, a.size)
            chunks.append((off, a))
            off += (a.size + _ALIGN - 1) // _ALIGN * _ALIGN
        layout.append(ent)
    flat = np.zeros(max(off, 1), dtype=np_dtype)
    for o, a in chunks:
        flat[o:o + a.size] = a
    return flat, layout


def _struct(p, ent, base_ptr: int, elem: int, ff_dtype: int) -> L.ff_problem:
    st = L.ff_problem()
    multi = int(p.T) >= 2
    st.n, st.k = int(p.F.shape[0]), int(p.F.shape[1])
    st.m = int(np.asarray(p.A).shape[0])
    st.T = int(p.T) if multi else 0
    st.dtype = ff_dtype
    st.omega_diag = ent["omega_diag"]
    for nm in _FIELDS:
        if nm in ent and ent[nm][1] > 0:
            setattr(st, nm, base_ptr + ent[nm][0] * elem)
        else:
            setattr(st, nm, None)
    st.GMV, st.lambda1, st.lambda2, st.lambda3, st.d = (float(p.GMV), float(p.lam1), float(p.lam2),
                                                         float(p.lam3), float(p.d))
    return st


class BatchRunner:
    """A batch packed into one device buffer; ``run()`` solves every instance
    in one call of ``ff_solve_batch`` (what the throughput benchmark times).

    ``run_from_host()`` is the end-to-end form: one copy of the packed inputs
    from pinned host memory, the solve, and one copy of the portfolios and
    results back to pinned host memory, all on one stream."""

    def __init__(self, problems: Sequence, precision: str = "bf16", device: str = "cuda", duals: bool = False,
                 escalate: bool = True, **opt_kw):
        self.precision = precision
        self.escalate = escalate
        self.escalated: List[int] = []
        self._esc_cache = {}
        self.device = torch.device(device)
        self.dtype = torch.float64 if precision == "f64" else torch.float32
        np_dtype = np.float64 if precision == "f64" else np.float32
        self.problems = list(problems)
        self.count = len(self.problems)
        flat, self.layout = pack(self.problems, np_dtype)
        self.host_in = torch.from_numpy(flat).pin_memory() if torch.cuda.is_available() else torch.from_numpy(flat)
        self.dev_in = self.host_in.to(self.device)
        elem = self.dev_in.element_size()
        ffd = L.FF_F64 if self.dtype == torch.float64 else L.FF_F32
        base = self.dev_in.data_ptr()
        self.structs = (L.ff_problem * self.count)(
            *[_struct(p, e, base, elem, ffd) for p, e in zip(self.problems, self.layout)])
        self.P = [int(p.T) - 1 if int(p.T) >= 2 else 1 for p in self.problems]
        self.n = [int(p.F.shape[0]) for p in self.problems]
        self.w_off = np.concatenate([[0], np.cumsum([(P * n + _ALIGN - 1) // _ALIGN * _ALIGN
                                                     for P, n in zip(self.P, self.n)])]).astype(np.int64)
        self.opts = options(precision, **opt_kw)
        self.ws_bytes = L.ff_workspace_size(self.structs, self.count, self.opts)
        if self.ws_bytes == 0:
            raise ValueError("invalid problem or options")
        self.ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device=self.device)
        self.res = torch.zeros(L.RESULT_DTYPE.itemsize * self.count, dtype=torch.uint8, device=self.device)
        self.w_dev = torch.empty(int(self.w_off[-1]), dtype=self.dtype, device=self.device)
        welem = self.w_dev.element_size()
        self.w_ptrs = [self.w_dev.data_ptr() + int(o) * welem for o in self.w_off[:-1]]
        self.yA_ptrs = self.yD_ptrs = None
        if duals:
            m_ = [int(np.asarray(p.A).shape[0]) for p in self.problems]
            R_ = [int(p.T) if int(p.T) >= 2 else 1 for p in self.problems]
            self.yA_off = np.concatenate([[0], np.cumsum([(P * m + _ALIGN) // _ALIGN * _ALIGN
                                                          for P, m in zip(self.P, m_)])]).astype(np.int64)
            self.yD_off = np.concatenate([[0], np.cumsum([(R * n + _ALIGN - 1) // _ALIGN * _ALIGN
                                                          for R, n in zip(R_, self.n)])]).astype(np.int64)
            self.yA_dev = torch.zeros(int(self.yA_off[-1]), dtype=self.dtype, device=self.device)
            self.yD_dev = torch.zeros(int(self.yD_off[-1]), dtype=self.dtype, device=self.device)
            self.yA_ptrs = [self.yA_dev.data_ptr() + int(o) * welem for o in self.yA_off[:-1]]
            self.yD_ptrs = [self.yD_dev.data_ptr() + int(o) * welem for o in self.yD_off[:-1]]
        pin = torch.cuda.is_available()
        self.w_host = torch.empty(self.w_dev.shape, dtype=self.dtype, pin_memory=pin)
        self.res_host = torch.empty(self.res.shape, dtype=torch.uint8, pin_memory=pin)
        self.graph = None

    def plan(self):
        """(cluster size per instance, solver launches per call)."""
        return L.ff_batch_plan(self.structs, self.count, self.opts)

    def solver_launches(self) -> int:
        return self.plan()[1]

    @property
    def h2d_bytes(self) -> int:
        return self.host_in.numel() * self.host_in.element_size()

    @property
    def d2h_bytes(self) -> int:
        return self.w_dev.numel() * self.w_dev.element_size() + self.res.numel()

    def run(self, stream: Optional[torch.cuda.Stream] = None) -> None:
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        rc = L.ff_solve_batch(self.structs, self.count, self.opts, self.ws.data_ptr(), self.ws_bytes,
                              self.res.data_ptr(), self.w_ptrs, s.cuda_stream, self.yA_ptrs, self.yD_ptrs)
        if rc != L.FF_OK:
            raise RuntimeError(f"batch solve failed: {L.ff_status_string(rc)} ({rc}) {L.ff_last_error()}")

    def capture(self, stream: Optional[torch.cuda.Stream] = None) -> None:
        """Capture one solve of the batch (repack + persistent launches) in a
        CUDA graph; ``replay()`` then re-solves from the current contents of
        the device input buffer with a single graph launch.  The instance
        table is uploaded by an ordinary call first (capture cannot copy from
        pageable host memory); the captured call reuses it (mode 2)."""
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.run(s)
        s.synchronize()
        saved = self.opts.reuse_workspace
        self.opts.reuse_workspace = 2
        try:
            cap = torch.cuda.Stream(self.device)
            cap.wait_stream(s)
            self.graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(self.graph, stream=cap, capture_error_mode="thread_local"):
                self.run(cap)
            s.wait_stream(cap)
        finally:
            self.opts.reuse_workspace = saved

    def replay(self, stream: Optional[torch.cuda.Stream] = None) -> None:
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        with torch.cuda.stream(s):
            self.graph.replay()

    def finish(self, stream: Optional[torch.cuda.Stream] = None) -> int:
        """Wait for the solve on ``stream``; then (``escalate``) solve the
        instances that ended with FF_PRECISION again in FP64, on the same
        device inputs and output slots, and put their results in place.
        Returns the number of instances solved again (``escalated`` lists them)."""
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        s.synchronize()
        self.escalated = []
        if not self.escalate or self.opts.precision == L.FF_PREC_F64:
            return 0
        st = self.res.view(self.count, -1)[:, :4].contiguous().view(torch.int32).cpu().numpy().ravel()
        idx = [int(i) for i in np.nonzero(st == L.FF_PRECISION)[0]]
        if not idx:
            return 0
        key = tuple(idx)
        if key not in self._esc_cache:
            structs = (L.ff_problem * len(idx))(*[self.structs[i] for i in idx])
            o64 = escalation_options(self.opts)
            nb = L.ff_workspace_size(structs, len(idx), o64)
            if nb == 0:
                raise ValueError("invalid problem for the FP64 re-solve")
            ws = torch.empty(nb, dtype=torch.uint8, device=self.device)
            res = torch.zeros(L.RESULT_DTYPE.itemsize * len(idx), dtype=torch.uint8, device=self.device)
            self._esc_cache[key] = (structs, o64, ws, nb, res)
        structs, o64, ws, nb, res = self._esc_cache[key]
        def pick(v):
            return [v[i] for i in idx]
        rc = L.ff_solve_batch(structs, len(idx), o64, ws.data_ptr(), nb, res.data_ptr(), pick(self.w_ptrs),
                              s.cuda_stream, pick(self.yA_ptrs) if self.yA_ptrs is not None else None,
                              pick(self.yD_ptrs) if self.yD_ptrs is not None else None)
        if rc != L.FF_OK:
            raise RuntimeError(f"FP64 re-solve failed: {L.ff_status_string(rc)} ({rc}) {L.ff_last_error()}")
        rows = torch.tensor(idx, device=self.device)
        self.res.view(self.count, -1).index_copy_(0, rows, res.view(len(idx), -1))
        s.synchronize()
        self.escalated = idx
        return len(idx)

    def run_from_host(self, stream: Optional[torch.cuda.Stream] = None) -> None:
        """Copy the packed inputs from pinned host memory, solve (with the
        FP64 re-solve of ``finish``), copy the portfolios and results back."""
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        with torch.cuda.stream(s):
            self.dev_in.copy_(self.host_in, non_blocking=True)
            if getattr(self, "graph", None) is not None:
                self.graph.replay()
            else:
                self.run(s)
        self.finish(s)
        with torch.cuda.stream(s):
            self.w_host.copy_(self.w_dev, non_blocking=True)
            self.res_host.copy_(self.res, non_blocking=True)

    def prepare_backward(self) -> None:
        """Buffers of the batched adjoint (duals on): ``g_dev`` holds the
        upstream gradients in the portfolio layout, ``grad_dev`` the gradients
        of alpha, F, D, s, q, w0 (and w_T for multi-period instances) in the
        packed input layout (``layout``).  Single-period instances go to
        ``ff_backward_batch``, multi-period ones to ``ff_backward_multi_batch``;
        ``bstatus`` holds every instance's adjoint status (instance order)."""
        if self.yD_ptrs is None:
            raise ValueError("BatchRunner(duals=True) is needed for the adjoint")
        self.g_dev = torch.zeros_like(self.w_dev)
        self.grad_dev = torch.zeros_like(self.dev_in)
        elem = self.grad_dev.element_size()
        base = self.grad_dev.data_ptr()
        welem = self.w_dev.element_size()
        self.g_ptrs = [self.g_dev.data_ptr() + int(o) * welem for o in self.w_off[:-1]]
        self.grads = []
        for ent in self.layout:
            gr = L.ff_grads()
            for nm in ("alpha", "F", "D", "s", "q", "w0", "wT"):
                setattr(gr, nm, base + ent[nm][0] * elem if nm in ent else None)
            self.grads.append(gr)
        single = [i for i, p in enumerate(self.problems) if int(p.T) < 2]
        multi = [i for i, p in enumerate(self.problems) if int(p.T) >= 2]
        self._bstatus_sub = torch.zeros(self.count, dtype=torch.int32, device=self.device)
        self._border = single + multi
        self._bsets = []
        pos = 0
        for idx, size_fn, call in ((single, L.ff_backward_batch_workspace_size, L.ff_backward_batch),
                                   (multi, L.ff_backward_multi_workspace_size, L.ff_backward_multi_batch)):
            if not idx:
                continue
            structs = (L.ff_problem * len(idx))(*[self.structs[i] for i in idx])
            nb = size_fn(structs, len(idx))
            if nb == 0:
                raise ValueError("invalid problem for the adjoint")
            ws = torch.empty(nb, dtype=torch.uint8, device=self.device)
            self._bsets.append((idx, structs, ws, nb, call, self._bstatus_sub.data_ptr() + 4 * pos))
            pos += len(idx)

    def backward_launches(self) -> int:
        """Kernels one ``backward()`` enqueues: one for the single-period
        instances and one cooperative launch for the multi-period ones (the
        launch sequence of ff_backward_batch and ff_backward_multi_batch)."""
        return len(self._bsets)

    @property
    def bstatus(self) -> torch.Tensor:
        """Adjoint status of every instance, in instance order."""
        out = torch.empty_like(self._bstatus_sub)
        out[torch.tensor(self._border, device=self.device)] = self._bstatus_sub
        return out

    def backward(self, stream: Optional[torch.cuda.Stream] = None) -> None:
        """Vector-Jacobian products of every instance for the gradients in g_dev."""
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        for idx, structs, ws, nb, call, status in self._bsets:
            pick = lambda v: [v[i] for i in idx]   # noqa: E731
            rc = call(structs, len(idx), pick(self.w_ptrs), pick(self.yA_ptrs), pick(self.yD_ptrs),
                      pick(self.g_ptrs), pick(self.grads), ws.data_ptr(), nb, status, s.cuda_stream)
            if rc != L.FF_OK:
                raise RuntimeError(f"backward failed: {L.ff_status_string(rc)} ({rc}) {L.ff_last_error()}")

    def gradient(self, i: int, name: str) -> np.ndarray:
        off, size = self.layout[i][name]
        a = self.grad_dev[off:off + size].cpu().numpy().astype(np.float64)
        return a.reshape(np.shape(getattr(self.problems[i], name)))

    def results(self) -> List[dict]:
        recs = self.res.cpu().numpy().view(L.RESULT_DTYPE)
        out = [_info(r) for r in recs]
        for i, d in enumerate(out):
            d["escalated"] = i in self.escalated
        return out

    def portfolios(self) -> List[np.ndarray]:
        flat = self.w_dev.cpu().numpy().astype(np.float64)
        out = []
        for i, p in enumerate(self.problems):
            a = flat[self.w_off[i]:self.w_off[i] + self.P[i] * self.n[i]]
            out.append(a.reshape(self.P[i], self.n[i]) if int(p.T) >= 2 else a)
        return out


def solve_batch(problems: Sequence, precision: str = "bf16", device: str = "cuda", **opt_kw):
    """Solve many instances in one persistent launch; returns (portfolios, infos)."""
    br = BatchRunner(problems, precision=precision, device=device, **opt_kw)
    br.run()
    br.finish()
    return br.portfolios(), br.results()


def solve_joint(problems: Sequence, device: str = "cuda", stream: Optional[torch.cuda.Stream] = None,
                **opt_kw) -> List[Solution]:
    """Single-period instances through the joint primal prox variant
    (ff_solve_joint_batch: trading cost and budget set in one primal prox, FP64,
    one CTA per instance); returns host copies of w, y_A, the recovered trade
    multiplier y_D and the result record of every instance."""
    probs = list(problems)
    if any(int(getattr(p, "T", 0)) >= 2 for p in probs):
        raise ValueError("the joint prox variant solves single-period instances only")
    dps = [to_device(p, dtype=torch.float64, device=device) for p in probs]
    count = len(dps)
    structs = (L.ff_problem * count)(*[d.struct for d in dps])
    opts = options("f64", **opt_kw)
    nb = L.ff_joint_workspace_size(structs, count)
    if nb == 0:
        raise ValueError("invalid problem for the joint prox variant")
    ws = torch.empty(nb + 256, dtype=torch.uint8, device=device)
    base = (ws.data_ptr() + 255) // 256 * 256
    res = torch.zeros(count * L.RESULT_DTYPE.itemsize, dtype=torch.uint8, device=device)
    ws_ = [torch.empty(d.n, dtype=torch.float64, device=device) for d in dps]
    ya = [torch.empty(max(d.m, 1), dtype=torch.float64, device=device) for d in dps]
    yd = [torch.empty(d.n, dtype=torch.float64, device=device) for d in dps]
    s = stream if stream is not None else torch.cuda.current_stream(device)
    rc = L.ff_solve_joint_batch(structs, count, opts, base, nb, res.data_ptr(), [t.data_ptr() for t in ws_],
                                s.cuda_stream, [t.data_ptr() for t in ya], [t.data_ptr() for t in yd])
    if rc != L.FF_OK:
        raise RuntimeError(f"ff_solve_joint_batch: {L.ff_status_string(rc)} ({rc}) {L.ff_last_error()}")
    s.synchronize()
    recs = res.cpu().numpy().view(L.RESULT_DTYPE)
    return [Solution(w.cpu().numpy(), a[:d.m].cpu().numpy(), y.cpu().numpy(), _info(r))
            for w, a, y, d, r in zip(ws_, ya, yd, dps, recs)]


@dataclass
class RiskModels:
    """Device results of ``estimate_risk`` for ``count`` windows."""
    beta: torch.Tensor      # (count, n, p) float64
    sigma_f: torch.Tensor   # (count, p, p) float64
    D: torch.Tensor         # (count, n) float64, NaN where not estimated
    nobs: torch.Tensor      # (count, n) int32: days with a return, -1 irregular, -2 singular


def estimate_risk(F, R, min_obs: int = 42, device: str = "cuda",
                  stream: Optional[torch.cuda.Stream] = None) -> RiskModels:
    """Factor model of Sec. 3.2 for a batch of estimation windows through
    ff_risk_estimate.  F: (count, T, p) factor returns, R: (count, T, n) stock
    returns (NaN = no return), as arrays or tensors; stored as float32 on the
    device."""
    Ft = torch.as_tensor(np.asarray(F) if not torch.is_tensor(F) else F).to(device=device, dtype=torch.float32)
    Rt = torch.as_tensor(np.asarray(R) if not torch.is_tensor(R) else R).to(device=device, dtype=torch.float32)
    if Ft.dim() == 2:
        Ft, Rt = Ft[None], Rt[None]
    Ft, Rt = Ft.contiguous(), Rt.contiguous()
    count, T, p = Ft.shape
    n = Rt.shape[2]
    nb = L.ff_risk_workspace_size(count, T, n, p)
    if nb == 0:
        raise ValueError("invalid sizes for the risk-model estimation")
    ws = torch.empty(nb, dtype=torch.uint8, device=device)
    out = RiskModels(torch.empty(count, n, p, dtype=torch.float64, device=device),
                     torch.empty(count, p, p, dtype=torch.float64, device=device),
                     torch.empty(count, n, dtype=torch.float64, device=device),
                     torch.empty(count, n, dtype=torch.int32, device=device))
    s = stream if stream is not None else torch.cuda.current_stream(device)
    rc = L.ff_risk_estimate(count, T, n, p, Ft.data_ptr(), Rt.data_ptr(), min_obs, out.beta.data_ptr(),
                            out.sigma_f.data_ptr(), out.D.data_ptr(), out.nobs.data_ptr(), ws.data_ptr(), nb,
                            s.cuda_stream)
    if rc != L.FF_OK:
        raise RuntimeError(f"risk estimation failed: {L.ff_status_string(rc)} ({rc}) {L.ff_risk_last_error()}")
    out._keep = (Ft, Rt, ws)
    return out
