"""The C-ABI library builds, loads and exports every entry point of include/flashfolio.h
(no compute call: runs without a GPU)."""
import ctypes as C
import os
import re

import pytest

from paper_2604_22625_gb300 import _lib
from paper_2604_22625_gb300.build import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build()
    return _lib.load()


def _declared():
    src = open(os.path.join(ROOT, "include", "flashfolio.h")).read()
    return sorted(set(re.findall(r"\b(ff_[a-z_]+)\s*\(", src)))


def test_exports(lib):
    names = _declared()
    assert set(names) >= {"ff_solve_single", "ff_solve_multi", "ff_solve_batch", "ff_workspace_size",
                          "ff_status_string", "ff_default_options", "ff_version"}
    for nm in names:
        assert hasattr(lib, nm), nm


def test_struct_sizes_match_header(lib, tmp_path):
    """The ctypes mirrors have the size and field offsets of the header's
    structs, as a C compiler lays them out (gcc on this host)."""
    import shutil
    import subprocess
    assert _lib.RESULT_DTYPE.itemsize == C.sizeof(_lib.ff_result)
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"ff_result": _lib.ff_result, "ff_options": _lib.ff_options, "ff_problem": _lib.ff_problem,
               "ff_grads": _lib.ff_grads}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "flashfolio.h"', "int main(void) {"]
    for nm, cls in structs.items():
        lines.append(f'printf("{nm} %zu\\n", sizeof({nm}));')
        for fname, _ in cls._fields_:
            lines.append(f'printf("{nm}.{fname} %zu\\n", offsetof({nm}, {fname}));')
    lines.append("return 0; }")
    src = tmp_path / "abi.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "abi"
    inc = os.path.join(ROOT, "include")
    subprocess.run([cc, "-I", inc, str(src), "-o", str(exe)], check=True, capture_output=True)
    out = dict(line.rsplit(" ", 1) for line in subprocess.run([str(exe)], check=True, capture_output=True,
                                                               text=True).stdout.splitlines())
    for nm, cls in structs.items():
        assert int(out[nm]) == C.sizeof(cls), nm
        for fname, _ in cls._fields_:
            assert int(out[f"{nm}.{fname}"]) == getattr(cls, fname).offset, (nm, fname)


def test_host_only_calls(lib):
    assert _lib.ff_version() >= 100
    assert _lib.ff_status_string(_lib.FF_ERR_WORKSPACE).startswith("workspace")
    o = _lib.default_options()
    assert o.tol == 1e-6 and o.check_every == 64 and o.precision == _lib.FF_PREC_F32
    assert abs(o.reflection - 1 / 3) < 1e-15 and o.beta == 0.75 and o.step_fraction == 0.4
    # invalid problem -> workspace size 0, solve rejects before touching the GPU
    p = _lib.ff_problem()
    assert _lib.ff_workspace_size(C.byref(p), 1, o) == 0
    rc = _lib.ff_solve_single(p, o, 0, 0, 0, 0)
    assert rc == _lib.FF_ERR_INVALID_ARG


def test_workspace_size_grows_with_n(lib):
    o = _lib.default_options()

    def ws(n, T=0):
        p = _lib.ff_problem()
        p.n, p.k, p.m, p.T, p.dtype, p.omega_diag = n, 10, 10, T, _lib.FF_F32, 1
        for nm in ("F", "Omega", "D", "alpha", "s", "q", "w0", "A", "L", "U", "wT"):
            setattr(p, nm, 1024)    # non-null placeholders: size query only
        p.GMV, p.lambda1, p.lambda2, p.lambda3, p.d = 1e9, 1e-8, 1.0, 1.0, 1.5
        return _lib.ff_workspace_size(C.byref(p), 1, o)

    assert 0 < ws(100) < ws(1000) < ws(1000, T=5)


def test_batch_plan_groups_by_cluster_size(lib):
    """The host-only plan gives small single-period instances one CTA and
    spreads large multi-period ones over clusters (no GPU needed)."""
    import numpy as np
    from paper_2604_22625_gb300 import api, synthetic as S
    probs = [S.make_single(n, 20, i) for i, n in enumerate([600, 3000, 7000] * 40)]
    probs += [S.make_multi(30, 3500, 20, 99)]
    flat, lay = api.pack(probs, np.float32)
    st = (_lib.ff_problem * len(probs))(*[api._struct(p, e, 1 << 20, 4, _lib.FF_F32) for p, e in zip(probs, lay)])
    o = _lib.default_options(precision=_lib.FF_PREC_BF16)
    cl, nl = _lib.ff_batch_plan(st, len(probs), o)
    assert cl[:120] == [1] * 120
    assert cl[-1] == 16 and nl == 2          # 29 * 3500 asset-periods > 8 * 8192
    o.cluster_size = 4
    cl, nl = _lib.ff_batch_plan(st, len(probs), o)
    assert set(cl) == {4} and nl == 2          # one launch per kind: single- and multi-period


def _placeholder_problem(T=0, n=100, k=10, m=10):
    p = _lib.ff_problem()
    p.n, p.k, p.m, p.T, p.dtype, p.omega_diag = n, k, m, T, _lib.FF_F32, 1
    for nm in ("F", "Omega", "D", "alpha", "s", "q", "w0", "A", "L", "U", "wT"):
        setattr(p, nm, 1024)    # non-null placeholders: host-side checks only
    p.GMV, p.lambda1, p.lambda2, p.lambda3, p.d = 1e9, 1e-8, 1.0, 1.0, 1.5
    return p


def test_invalid_options_are_rejected_on_host(lib):
    p = _placeholder_problem()
    ok = _lib.default_options()
    assert _lib.ff_workspace_size(C.byref(p), 1, ok) > 0
    for field, value in (("reflection", 0.9), ("cta_work", 0.5), ("restart_artificial", 1.0),
                         ("reuse_workspace", 3), ("cluster_size", 3), ("tol", 0.0), ("check_every", 0)):
        o = _lib.default_options()
        setattr(o, field, value)
        assert _lib.ff_workspace_size(C.byref(p), 1, o) == 0, field
        assert _lib.ff_solve_single(p, o, 0, 0, 0, 0) == _lib.FF_ERR_INVALID_ARG, field


def test_backward_host_checks(lib):
    single = _placeholder_problem()
    multi = _placeholder_problem(T=5)
    assert _lib.ff_backward_workspace_size(single) > 0
    g = _lib.ff_grads()
    rc = _lib.ff_backward_single(multi, 4096, 4096, 4096, 4096, g, 0, 0)
    assert rc == _lib.FF_ERR_INVALID_ARG
    rc = _lib.ff_backward_single(single, 4096, 4096, 4096, 4096, g, 0, 0)   # no workspace
    assert rc == _lib.FF_ERR_WORKSPACE
    # the general entry point routes by kind; both stop at the missing workspace
    assert _lib.ff_backward(single, 4096, 4096, 4096, 4096, g, 0, 0) == _lib.FF_ERR_WORKSPACE
    assert _lib.ff_backward(multi, 4096, 4096, 4096, 4096, g, 0, 0) == _lib.FF_ERR_WORKSPACE
    bad = _placeholder_problem(T=5)
    bad.wT = None                                  # w_T is required for a multi-period adjoint
    assert _lib.ff_backward(bad, 4096, 4096, 4096, 4096, g, 0, 0) == _lib.FF_ERR_INVALID_ARG


def test_multi_backward_host_checks(lib):
    """Workspace sizes and argument checks of the multi-period adjoint (host only)."""
    assert C.sizeof(_lib.ff_grads) == 7 * C.sizeof(C.c_void_p)
    multi = _placeholder_problem(T=5)
    one = (_lib.ff_problem * 1)(multi)
    ws1 = _lib.ff_backward_multi_workspace_size(one, 1)
    assert ws1 > 0 and _lib.ff_backward_workspace_size(multi) == ws1
    two = (_lib.ff_problem * 2)(multi, _placeholder_problem(T=9, n=300))
    assert _lib.ff_backward_multi_workspace_size(two, 2) > ws1
    mixed = (_lib.ff_problem * 2)(multi, _placeholder_problem())
    assert _lib.ff_backward_multi_workspace_size(mixed, 2) == 0      # single-period instance
    # the documented estimate: about 333 (T-1) n + 16 ((T-1)(m+1))^2 bytes
    big = (_lib.ff_problem * 1)(_placeholder_problem(T=50, n=2000, k=60, m=60))
    est = 333 * 49 * 2000 + 16 * (49 * 61) ** 2
    assert abs(_lib.ff_backward_multi_workspace_size(big, 1) / est - 1) < 0.02
    g = [_lib.ff_grads()]
    ptr = [4096]
    rc = _lib.ff_backward_multi_batch(mixed, 2, ptr * 2, ptr * 2, ptr * 2, ptr * 2, g * 2, 0, 0)
    assert rc == _lib.FF_ERR_INVALID_ARG
    rc = _lib.ff_backward_multi_batch(one, 1, ptr, ptr, ptr, ptr, g, 0, 0)
    assert rc == _lib.FF_ERR_WORKSPACE
    rc = _lib.ff_backward_multi_batch(one, 1, ptr, ptr, ptr, ptr, g, 256 * 17, 1024)   # too small
    assert rc == _lib.FF_ERR_WORKSPACE
    rc = _lib.ff_backward_multi_batch(one, 1, ptr, ptr, None, ptr, g, 256 * 17, ws1)   # no yD
    assert rc == _lib.FF_ERR_INVALID_ARG
    rc = _lib.ff_backward_multi_batch(one, 70000, ptr, ptr, ptr, ptr, g, 256 * 17, ws1)
    assert rc == _lib.FF_ERR_INVALID_ARG


def test_batch_count_limit(lib):
    probs = (_lib.ff_problem * 1)(_placeholder_problem())
    o = _lib.default_options()
    rc = _lib.ff_solve_batch(probs, 70000, o, 0, 0, 4096, [4096] * 70000)
    assert rc == _lib.FF_ERR_UNSUPPORTED


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    """Without the built library the binding raises; there is no CPU fallback
    (the package never routes a solve through the oracle)."""
    monkeypatch.setattr(_lib, "_lib", None)
    with pytest.raises(RuntimeError, match="missing"):
        _lib.load(str(tmp_path / "libflashfolio.so"))


def test_package_does_not_import_the_oracle():
    """Only tests, the smoke check and the bench's CPU legs may use oracle/."""
    pkg = os.path.join(ROOT, "paper_2604_22625_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import oracle|from oracle)", src, re.M), f


def test_joint_host_checks(lib):
    """Workspace size and argument checks of the joint prox variant (host only):
    about 8 n (k + m + 12) bytes per instance; FP64 only; single-period only;
    k, m <= 256; a short workspace is refused before anything is enqueued."""
    single = _placeholder_problem(n=1000, k=10, m=10)
    one = (_lib.ff_problem * 1)(single)
    ws1 = _lib.ff_joint_workspace_size(one, 1)
    est = 8 * 1000 * (10 + 10 + 12)
    assert est <= ws1 <= est + 16 * 256 + 4096
    multi = (_lib.ff_problem * 1)(_placeholder_problem(T=5))
    assert _lib.ff_joint_workspace_size(multi, 1) == 0
    o32 = _lib.default_options(precision=_lib.FF_PREC_F32)
    o64 = _lib.default_options(precision=_lib.FF_PREC_F64)
    assert _lib.ff_solve_joint_batch(one, 1, o32, 4096, ws1, 4096, [4096]) == _lib.FF_ERR_UNSUPPORTED
    assert _lib.ff_solve_joint_batch(multi, 1, o64, 4096, ws1, 4096, [4096]) == _lib.FF_ERR_UNSUPPORTED
    wide = (_lib.ff_problem * 1)(_placeholder_problem(n=1000, k=300, m=10))
    assert _lib.ff_solve_joint_batch(wide, 1, o64, 4096, 1 << 30, 4096, [4096]) == _lib.FF_ERR_UNSUPPORTED
    assert _lib.ff_solve_joint_batch(one, 1, o64, 4096, ws1 - 256, 4096, [4096]) == _lib.FF_ERR_WORKSPACE
    assert _lib.ff_solve_joint_batch(one, 1, o64, 4096 + 8, ws1, 4096, [4096]) == _lib.FF_ERR_WORKSPACE
    assert _lib.ff_solve_joint_batch(one, 1, o64, 4096, ws1, 4096, [None]) == _lib.FF_ERR_INVALID_ARG
    # no options: the defaults in FP64, so only the short workspace is refused
    rc = _lib.load().ff_solve_joint_batch(one, 1, None, C.c_void_p(4096), ws1 - 256, C.c_void_p(4096),
                                          (C.c_void_p * 1)(4096), None, None, None)
    assert rc == _lib.FF_ERR_WORKSPACE
