"""ctypes binding of libflashfolio.so (the C ABI of include/flashfolio.h).

Argument marshalling only: every step of the solve runs in the library's
CUDA kernels.  The names mirror the C entry points.  Loading fails loudly
when the library has not been built.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libflashfolio.so")

FF_OK = 0
FF_ERR_INVALID_ARG = 1
FF_ERR_CUDA = 2
FF_ERR_WORKSPACE = 3
FF_ERR_UNSUPPORTED = 4
FF_ERR_DEVICE = 5

FF_CONVERGED = 0
FF_MAX_ITER = 1
FF_TIME_LIMIT = 2
FF_NUMERICAL = 3
FF_STALLED = 4
FF_PRECISION = 5

FF_F64 = 0
FF_F32 = 1

FF_PREC_F64 = 0
FF_PREC_F32 = 1
FF_PREC_BF16 = 2

FF_STATIC_WORKSPACE_BYTES = 32 * 1024 * 1024

STATUS_NAMES = {FF_CONVERGED: "converged", FF_MAX_ITER: "max_iter", FF_TIME_LIMIT: "time_limit",
                FF_NUMERICAL: "numerical", FF_STALLED: "stalled", FF_PRECISION: "precision_floor"}


class ff_problem(C.Structure):
    _fields_ = [("n", C.c_int32), ("k", C.c_int32), ("m", C.c_int32), ("T", C.c_int32),
                ("dtype", C.c_int32), ("omega_diag", C.c_int32),
                ("F", C.c_void_p), ("Omega", C.c_void_p), ("D", C.c_void_p), ("alpha", C.c_void_p),
                ("s", C.c_void_p), ("q", C.c_void_p), ("w0", C.c_void_p), ("wT", C.c_void_p),
                ("A", C.c_void_p), ("L", C.c_void_p), ("U", C.c_void_p),
                ("GMV", C.c_double), ("lambda1", C.c_double), ("lambda2", C.c_double),
                ("lambda3", C.c_double), ("d", C.c_double)]


class ff_options(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_iter", C.c_int64), ("time_limit", C.c_double),
                ("precision", C.c_int32), ("check_every", C.c_int32), ("reflection", C.c_double),
                ("restart_sufficient", C.c_double), ("restart_necessary", C.c_double),
                ("step_fraction", C.c_double), ("cluster_size", C.c_int32), ("max_teams", C.c_int32),
                ("beta", C.c_double), ("reuse_workspace", C.c_int32), ("cta_work", C.c_double),
                ("restart_artificial", C.c_double), ("stall_checks", C.c_int32), ("round_panels_bf16", C.c_int32),
                ("warm_start", C.c_int32), ("panel_l2_keep", C.c_int32), ("primal_weight", C.c_int32),
                ("test_expire_first_wait", C.c_int32)]


class ff_grads(C.Structure):
    _fields_ = [("alpha", C.c_void_p), ("F", C.c_void_p), ("D", C.c_void_p), ("s", C.c_void_p),
                ("q", C.c_void_p), ("w0", C.c_void_p), ("wT", C.c_void_p)]


class ff_result(C.Structure):
    _fields_ = [("status", C.c_int32), ("restarts", C.c_int32), ("iterations", C.c_int64),
                ("rel_kkt", C.c_double), ("r_primal", C.c_double), ("r_dual", C.c_double),
                ("r_gap", C.c_double), ("primal_obj", C.c_double), ("dual_obj", C.c_double),
                ("paper_obj", C.c_double), ("fixed_point_res", C.c_double), ("seconds", C.c_double),
                ("lipschitz", C.c_double), ("threshold_rounds", C.c_int64),
                ("phase_seconds", C.c_double * 6), ("term_scale", C.c_double)]


RESULT_DTYPE = np.dtype([(name, {C.c_int32: np.int32, C.c_int64: np.int64, C.c_double: np.float64}[ct])
                         if ct in (C.c_int32, C.c_int64, C.c_double) else (name, np.float64, (6,))
                         for name, ct in ff_result._fields_], align=True)
assert RESULT_DTYPE.itemsize == C.sizeof(ff_result)

EXPORTS = ("ff_default_options", "ff_workspace_size", "ff_solve_single", "ff_solve_multi",
           "ff_solve_batch", "ff_status_string", "ff_version", "ff_last_error",
           "ff_solve_single_static", "ff_batch_plan", "ff_backward", "ff_backward_single", "ff_backward_workspace_size",
           "ff_backward_batch", "ff_backward_batch_workspace_size", "ff_backward_multi_batch",
           "ff_backward_multi_workspace_size", "ff_risk_workspace_size", "ff_risk_estimate", "ff_risk_last_error",
           "ff_joint_workspace_size", "ff_solve_joint_batch")

_lib = None


def load(path: str = LIB_PATH) -> C.CDLL:
    """Load the library (once).  Raises if it is missing: there is no fallback."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2604_22625_gb300.build.build()")
    lib = C.CDLL(path)
    lib.ff_default_options.argtypes = [C.POINTER(ff_options)]
    lib.ff_default_options.restype = None
    lib.ff_workspace_size.argtypes = [C.POINTER(ff_problem), C.c_int, C.POINTER(ff_options)]
    lib.ff_workspace_size.restype = C.c_size_t
    sig = [C.POINTER(ff_problem), C.POINTER(ff_options), C.c_void_p, C.c_size_t, C.c_void_p,
           C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    for name in ("ff_solve_single", "ff_solve_multi"):
        getattr(lib, name).argtypes = sig
        getattr(lib, name).restype = C.c_int
    lib.ff_backward_workspace_size.argtypes = [C.POINTER(ff_problem)]
    lib.ff_backward_workspace_size.restype = C.c_size_t
    lib.ff_backward_single.argtypes = [C.POINTER(ff_problem), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                       C.POINTER(ff_grads), C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p]
    lib.ff_backward_single.restype = C.c_int
    lib.ff_backward.argtypes = lib.ff_backward_single.argtypes
    lib.ff_backward.restype = C.c_int
    lib.ff_backward_batch_workspace_size.argtypes = [C.POINTER(ff_problem), C.c_int]
    lib.ff_backward_batch_workspace_size.restype = C.c_size_t
    vp = C.POINTER(C.c_void_p)
    lib.ff_backward_batch.argtypes = [C.POINTER(ff_problem), C.c_int, vp, vp, vp, vp, C.POINTER(ff_grads),
                                      C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p]
    lib.ff_backward_batch.restype = C.c_int
    lib.ff_backward_multi_workspace_size.argtypes = [C.POINTER(ff_problem), C.c_int]
    lib.ff_backward_multi_workspace_size.restype = C.c_size_t
    lib.ff_backward_multi_batch.argtypes = lib.ff_backward_batch.argtypes
    lib.ff_backward_multi_batch.restype = C.c_int
    lib.ff_batch_plan.argtypes = [C.POINTER(ff_problem), C.c_int, C.POINTER(ff_options),
                                  C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
    lib.ff_batch_plan.restype = C.c_int
    lib.ff_solve_single_static.argtypes = [C.POINTER(ff_problem), C.POINTER(ff_options), C.c_void_p,
                                           C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    lib.ff_solve_single_static.restype = C.c_int
    lib.ff_solve_batch.argtypes = [C.POINTER(ff_problem), C.c_int, C.POINTER(ff_options), C.c_void_p,
                                   C.c_size_t, C.c_void_p, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                                   C.POINTER(C.c_void_p), C.c_void_p]
    lib.ff_solve_batch.restype = C.c_int
    lib.ff_joint_workspace_size.argtypes = [C.POINTER(ff_problem), C.c_int]
    lib.ff_joint_workspace_size.restype = C.c_size_t
    lib.ff_solve_joint_batch.argtypes = lib.ff_solve_batch.argtypes
    lib.ff_solve_joint_batch.restype = C.c_int
    lib.ff_status_string.argtypes = [C.c_int]
    lib.ff_status_string.restype = C.c_char_p
    lib.ff_last_error.argtypes = []
    lib.ff_last_error.restype = C.c_char_p
    lib.ff_version.argtypes = []
    lib.ff_version.restype = C.c_int
    lib.ff_risk_workspace_size.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int]
    lib.ff_risk_workspace_size.restype = C.c_size_t
    lib.ff_risk_estimate.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_int,
                                     C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t,
                                     C.c_void_p]
    lib.ff_risk_estimate.restype = C.c_int
    lib.ff_risk_last_error.argtypes = []
    lib.ff_risk_last_error.restype = C.c_char_p
    _lib = lib
    return lib


def default_options(**kw) -> ff_options:
    o = ff_options()
    load().ff_default_options(C.byref(o))
    for key, val in kw.items():
        setattr(o, key, val)
    return o


def ff_workspace_size(probs, count: int, opts: ff_options) -> int:
    return int(load().ff_workspace_size(probs, count, C.byref(opts)))


def ff_solve_single(prob: ff_problem, opts: ff_options, ws: int, ws_bytes: int, res: int, w: int,
                    yA: int = 0, yD: int = 0, stream: int = 0) -> int:
    return int(load().ff_solve_single(C.byref(prob), C.byref(opts), C.c_void_p(ws), ws_bytes, C.c_void_p(res),
                                      C.c_void_p(w), C.c_void_p(yA or None), C.c_void_p(yD or None),
                                      C.c_void_p(stream or None)))


def ff_solve_multi(prob: ff_problem, opts: ff_options, ws: int, ws_bytes: int, res: int, w: int,
                   yA: int = 0, yD: int = 0, stream: int = 0) -> int:
    return int(load().ff_solve_multi(C.byref(prob), C.byref(opts), C.c_void_p(ws), ws_bytes, C.c_void_p(res),
                                     C.c_void_p(w), C.c_void_p(yA or None), C.c_void_p(yD or None),
                                     C.c_void_p(stream or None)))


def ff_solve_single_static(prob: ff_problem, opts: ff_options, res: int, w: int, yA: int = 0, yD: int = 0,
                           stream: int = 0) -> int:
    return int(load().ff_solve_single_static(C.byref(prob), C.byref(opts), C.c_void_p(res), C.c_void_p(w),
                                             C.c_void_p(yA or None), C.c_void_p(yD or None),
                                             C.c_void_p(stream or None)))


def ff_backward_workspace_size(prob: ff_problem) -> int:
    return int(load().ff_backward_workspace_size(C.byref(prob)))


def ff_backward_single(prob: ff_problem, w: int, yA: int, yD: int, grad_w: int, grads: ff_grads, ws: int,
                       ws_bytes: int, status: int = 0, stream: int = 0) -> int:
    return int(load().ff_backward_single(C.byref(prob), C.c_void_p(w), C.c_void_p(yA or None), C.c_void_p(yD),
                                         C.c_void_p(grad_w), C.byref(grads), C.c_void_p(ws), ws_bytes,
                                         C.c_void_p(status or None), C.c_void_p(stream or None)))


def ff_backward(prob: ff_problem, w: int, yA: int, yD: int, grad_w: int, grads: ff_grads, ws: int,
                ws_bytes: int, status: int = 0, stream: int = 0) -> int:
    return int(load().ff_backward(C.byref(prob), C.c_void_p(w), C.c_void_p(yA or None), C.c_void_p(yD),
                                  C.c_void_p(grad_w), C.byref(grads), C.c_void_p(ws), ws_bytes,
                                  C.c_void_p(status or None), C.c_void_p(stream or None)))


def ff_batch_plan(probs, count: int, opts: ff_options):
    """(cluster size per instance, number of solver launches) of ff_solve_batch."""
    cl = (C.c_int32 * count)()
    nl = C.c_int32(0)
    rc = int(load().ff_batch_plan(probs, count, C.byref(opts), cl, C.byref(nl)))
    if rc != FF_OK:
        raise ValueError(f"ff_batch_plan: {ff_status_string(rc)}")
    return list(cl), int(nl.value)


def ff_solve_batch(probs, count: int, opts: ff_options, ws: int, ws_bytes: int, res: int, w_ptrs,
                   stream: int = 0, yA_ptrs=None, yD_ptrs=None) -> int:
    arr = (C.c_void_p * count)(*w_ptrs)
    ya = (C.c_void_p * count)(*yA_ptrs) if yA_ptrs is not None else None
    yd = (C.c_void_p * count)(*yD_ptrs) if yD_ptrs is not None else None
    return int(load().ff_solve_batch(probs, count, C.byref(opts), C.c_void_p(ws), ws_bytes, C.c_void_p(res),
                                     arr, ya, yd, C.c_void_p(stream or None)))


def ff_joint_workspace_size(probs, count: int) -> int:
    return int(load().ff_joint_workspace_size(probs, count))


def ff_solve_joint_batch(probs, count: int, opts: ff_options, ws: int, ws_bytes: int, res: int, w_ptrs,
                         stream: int = 0, yA_ptrs=None, yD_ptrs=None) -> int:
    arr = (C.c_void_p * count)(*w_ptrs)
    ya = (C.c_void_p * count)(*yA_ptrs) if yA_ptrs is not None else None
    yd = (C.c_void_p * count)(*yD_ptrs) if yD_ptrs is not None else None
    return int(load().ff_solve_joint_batch(probs, count, C.byref(opts), C.c_void_p(ws), ws_bytes,
                                           C.c_void_p(res), arr, ya, yd, C.c_void_p(stream or None)))


def ff_backward_batch_workspace_size(probs, count: int) -> int:
    return int(load().ff_backward_batch_workspace_size(probs, count))


def ff_backward_batch(probs, count: int, w_ptrs, yA_ptrs, yD_ptrs, g_ptrs, grads, ws: int, ws_bytes: int,
                      status: int = 0, stream: int = 0) -> int:
    def arr(v):
        return (C.c_void_p * count)(*v) if v is not None else None
    gr = (ff_grads * count)(*grads)
    return int(load().ff_backward_batch(probs, count, arr(w_ptrs), arr(yA_ptrs), arr(yD_ptrs), arr(g_ptrs), gr,
                                        C.c_void_p(ws), ws_bytes, C.c_void_p(status or None),
                                        C.c_void_p(stream or None)))


def ff_backward_multi_workspace_size(probs, count: int) -> int:
    return int(load().ff_backward_multi_workspace_size(probs, count))


def ff_backward_multi_batch(probs, count: int, w_ptrs, yA_ptrs, yD_ptrs, g_ptrs, grads, ws: int, ws_bytes: int,
                            status: int = 0, stream: int = 0) -> int:
    def arr(v):
        return (C.c_void_p * count)(*v) if v is not None else None
    gr = (ff_grads * count)(*grads)
    return int(load().ff_backward_multi_batch(probs, count, arr(w_ptrs), arr(yA_ptrs), arr(yD_ptrs), arr(g_ptrs),
                                              gr, C.c_void_p(ws), ws_bytes, C.c_void_p(status or None),
                                              C.c_void_p(stream or None)))


def ff_status_string(code: int) -> str:
    return load().ff_status_string(code).decode()


def ff_last_error() -> str:
    return load().ff_last_error().decode()


def ff_version() -> int:
    return int(load().ff_version())


def ff_risk_workspace_size(count: int, T: int, n: int, p: int) -> int:
    return int(load().ff_risk_workspace_size(count, T, n, p))


def ff_risk_estimate(count: int, T: int, n: int, p: int, F: int, R: int, min_obs: int, beta: int, sigma_f: int,
                     D: int, nobs: int, ws: int, ws_bytes: int, stream: int = 0) -> int:
    return int(load().ff_risk_estimate(count, T, n, p, C.c_void_p(F), C.c_void_p(R), min_obs, C.c_void_p(beta),
                                       C.c_void_p(sigma_f), C.c_void_p(D), C.c_void_p(nobs or None), C.c_void_p(ws),
                                       ws_bytes, C.c_void_p(stream or None)))


def ff_risk_last_error() -> str:
    return load().ff_risk_last_error().decode()
