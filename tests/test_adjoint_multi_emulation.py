"""Serial CPU transcription of the multi-period adjoint kernels
(csrc/ff_adjoint_multi.cu), checked against the oracle's implicit derivative.

Each function below mirrors one phase of the cooperative kernel adjm_kernel
(classify, rows, zcols, cfill, chol, inverse, pcg_init, ez, w, update_res,
rz, pdir, prodF, omega, hp, alpha, step, grad_asset, grad_F) with the same
storage (period-major P x n group-space vectors at each group's first
period, the kNB-column panel of M^-1 E^T, row-major C with leading dimension
rmax), the same index arithmetic and the same phase order; threads become
loops.  Every
workspace buffer starts as NaN and is bounds-checked (a negative or
out-of-range index raises), so a read before a write or an index outside a
buffer fails here, on the CPU.  This checks the GPU algorithm and its
indexing; the GPU kernels themselves are compared with the oracle in
test_gpu_adjoint_multi.py.  Nothing in the package imports this file, and it
shares no code with the oracle.
"""
from dataclasses import replace

import numpy as np
import pytest

import oracle
from oracle import grad as OG
from paper_2604_22625_gb300 import synthetic as S

# the constants of csrc/ff_adjoint_multi.cu
kNB, kMaxPcg, kPcgTol, kDropRel, kZFloor = 32, 600, 1e-11, 1e-12, 1e-14


class Inst:
    """Fields of one instance record (the AdjM struct)."""

def sgn(x): return 1.0 if x > 0 else (-1.0 if x < 0 else 0.0)

def setup(p, w, yA, yD, gw, f64=1):
    I = Inst()
    I.n, I.k = p.F.shape; I.m = p.A.shape[0]; I.P = p.T - 1; I.R = p.T
    I.F = np.asarray(p.F, float).ravel(); I.Om = np.asarray(p.Omega, float)
    I.omega_diag = 0
    I.D = np.asarray(p.D, float).ravel(); I.s = np.asarray(p.s, float).ravel(); I.q = np.asarray(p.q, float).ravel()
    I.w0 = np.asarray(p.w0, float); I.wT = np.asarray(p.wT, float); I.A = np.asarray(p.A, float).ravel()
    I.w = np.asarray(w, float).ravel(); I.yA = np.asarray(yA, float).ravel(); I.yD = np.asarray(yD, float).ravel()
    I.gw = np.asarray(gw, float).ravel()
    I.kappa = p.lam1 * p.GMV; I.lam2 = p.lam2; I.lam3 = p.lam3; I.d = p.d; I.f64 = f64
    PN = I.P * I.n
    I.rmax = I.P * (I.m + 1)
    I.gfirst = np.full(PN, -7, np.int64); I.src = np.full(PN, -9, np.int64); I.xfix = np.full(PN, np.nan)
    I.hz = np.full(I.R * I.n, np.nan); I.ldd = np.full(PN, np.nan); I.ldl = np.full(PN, np.nan)
    for nm in ("u", "res", "zz", "pd", "hp"): setattr(I, nm, np.full(PN, np.nan))
    for nm in ("Uk", "Wk", "Uk2", "Wk2"): setattr(I, nm, np.full(I.P * I.k, np.nan))
    I.rowp = np.full(I.rmax, -5); I.rowj = np.full(I.rmax, -5); I.rowoff = np.full(I.P + 1, -5)
    I.drop = np.zeros(I.rmax, int)
    I.C = np.full(I.rmax * I.rmax, np.nan); I.Ci = np.full(I.rmax * I.rmax, np.nan); I.Cd = np.full(I.rmax, np.nan)
    I.Z = np.full(PN * kNB, np.nan)
    I.ez = np.full(I.rmax, np.nan); I.wv = np.full(I.rmax, np.nan); I.nu = np.full(I.rmax, np.nan)
    I.part = np.full(I.n, np.nan); I.sc = np.zeros(8); I.flags = np.zeros(8, int)
    T = p.T; n = I.n
    I.dalpha = np.full(T * n, np.nan); I.dD = np.full(T * n, np.nan); I.ds = np.full(T * n, np.nan)
    I.dq = np.full(T * n, np.nan); I.dF = np.full(n * I.k, np.nan); I.dw0 = np.full(n, np.nan); I.dwT = np.full(n, np.nan)
    return I

def dead_trade(I, r, i):
    o = r * I.n + i
    return abs(I.yD[o]) < I.lam2 * I.s[o]

def xe(I, p, i):
    if p < 0: return I.w0[i]
    if p >= I.P: return I.wT[i]
    o = p * I.n + i
    return I.w[o] if I.gfirst[o] >= 0 else I.xfix[o]

def gv(I, v, p, i):
    if p < 0 or p >= I.P: return 0.0
    g = I.gfirst[p * I.n + i]
    return v[g * I.n + i] if g >= 0 else 0.0

def erow(I, p, j, i):
    if j < 0: return sgn(I.w[p * I.n + i])
    return I.A[j * I.n + i]

def chain_solve(I, i, b, z, stride, col):
    n, P = I.n, I.P
    yprev = 0.0
    for p in range(P):
        o = p * n + i
        if I.gfirst[o] != p: continue
        y = b[o * stride + col] - I.ldl[o] * yprev
        z[o * stride + col] = y; yprev = y
    znext = lnext = 0.0
    for p in range(P - 1, -1, -1):
        o = p * n + i
        g = I.gfirst[o]
        if g < 0: znext = lnext = 0.0; continue
        if g != p: continue
        zg = z[o * stride + col] / I.ldd[o] - lnext * znext
        z[o * stride + col] = zg; znext = zg; lnext = I.ldl[o]

def classify(I):
    n, P = I.n, I.P
    for i in range(n):
        p = 0
        while p < P:
            q = p
            while q + 1 < P and dead_trade(I, q + 1, i): q += 1
            code, fv = -1, 0.0
            if p == 0 and dead_trade(I, 0, i): code, fv = 1, I.w0[i]
            if code < 0 and q == P - 1 and dead_trade(I, P, i): code, fv = 2, I.wT[i]
            if code < 0:
                for pp in range(p, q + 1):
                    if I.w[pp * n + i] == 0.0: code, fv = 0, 0.0; break
            for pp in range(p, q + 1):
                o = pp * n + i
                I.gfirst[o] = p if code < 0 else -1
                I.src[o] = code; I.xfix[o] = 0.0 if code < 0 else fv
                I.ldd[o] = 0.0; I.ldl[o] = 0.0
            p = q + 1
        for r in range(P + 1):
            h = 0.0
            if not dead_trade(I, r, i):
                c2 = I.lam3 * I.q[r * n + i]
                az = max(abs(xe(I, r, i) - xe(I, r - 1, i)), kZFloor)
                h = c2 * I.d * (I.d - 1) * az ** (I.d - 2) if c2 > 0 else 0.0
            I.hz[r * n + i] = h
        dprev, prev_end, p = 0.0, -2, 0
        while p < P:
            o = p * n + i
            if I.gfirst[o] < 0: p += 1; continue
            q = p
            while q + 1 < P and I.gfirst[(q + 1) * n + i] == p: q += 1
            b = I.hz[o] + I.hz[(q + 1) * n + i]
            for pp in range(p, q + 1): b += 2 * I.kappa * I.D[pp * n + i]
            l = 0.0
            if prev_end == p - 1:
                e = -I.hz[o]; l = e / dprev; b -= l * e
            I.ldd[o] = b; I.ldl[o] = l; dprev = b; prev_end = q; p = q + 1

def rows(I):
    n, P, m = I.n, I.P, I.m
    ym = max([abs(I.yA[e]) for e in range(P * m)], default=0.0)
    btol = 1e-10 if I.f64 else 1e-6   # FP32 outputs carry their rounding into the l1 norm
    r = 0
    for p in range(P):
        l1 = sum(abs(I.w[p * n + i]) for i in range(n))
        I.rowoff[p] = r
        if l1 >= 1.0 - btol: I.rowp[r] = p; I.rowj[r] = -1; r += 1
        for j in range(m):
            if ym > 0 and abs(I.yA[p * m + j]) > 1e-12 * ym: I.rowp[r] = p; I.rowj[r] = j; r += 1
    I.rowoff[P] = r; I.flags[:4] = [r, 0, 0, 0]; I.sc[:4] = 0
    I.nu[:] = 0; I.wv[:] = 0; I.ez[:] = 0; I.drop[:] = 0

def zcols(I, c0):
    r = I.flags[0]; n, P = I.n, I.P
    if c0 >= r: return
    for i in range(n):
        for cc in range(kNB):
            c = c0 + cc
            if c >= r: break
            pc, jc = I.rowp[c], I.rowj[c]
            for p in range(P):
                o = p * n + i
                if I.gfirst[o] == p: I.Z[o * kNB + cc] = 0.0
            g = I.gfirst[pc * n + i]
            if g < 0: continue
            I.Z[(g * n + i) * kNB + cc] = erow(I, pc, jc, i)
            chain_solve(I, i, I.Z, I.Z, kNB, cc)

def cfill(I, c0):
    r = I.flags[0]; n = I.n
    for a in range(r):
        for cc in range(32):
            c = c0 + cc
            if c >= r: continue
            pa, ja = I.rowp[a], I.rowj[a]
            acc = 0.0
            for i in range(n):
                g = I.gfirst[pa * n + i]
                if g < 0: continue
                acc += erow(I, pa, ja, i) * I.Z[(g * n + i) * kNB + cc]
            I.C[a * I.rmax + c] = acc

def chol(I):
    r, ld = I.flags[0], I.rmax; A = I.C
    for j in range(r): I.Cd[j] = A[j * ld + j]
    for j in range(r):
        piv = A[j * ld + j]
        dr = not (piv > kDropRel * I.Cd[j])
        I.drop[j] = int(dr)
        A[j * ld + j] = 1.0 if dr else np.sqrt(piv)
        if dr:
            for i in range(j + 1, r): A[i * ld + j] = 0.0
            for l in range(j): A[j * ld + l] = 0.0
            continue
        ljj = A[j * ld + j]
        for i in range(j + 1, r): A[i * ld + j] /= ljj
        for ii in range(j + 1, r):
            for l in range(j + 1, ii + 1):
                A[ii * ld + l] -= A[ii * ld + j] * A[l * ld + j]

def inverse(I):
    r, ld = I.flags[0], I.rmax; L = I.C; X = I.Ci
    for c in range(r):
        for i in range(r):
            v = 1.0 if i == c else 0.0
            if i > c:
                for l in range(c, i): v -= L[i * ld + l] * X[l * ld + c]
            X[i * ld + c] = 0.0 if i < c else v / L[i * ld + i]
        for i in range(r - 1, -1, -1):
            v = X[i * ld + c]
            for l in range(i + 1, r): v -= L[l * ld + i] * X[l * ld + c]
            X[i * ld + c] = v / L[i * ld + i]
        for i in range(r):
            if I.drop[c] or I.drop[i]: X[i * ld + c] = 0.0

def pcg_init(I):
    n, P = I.n, I.P
    for i in range(n):
        for p in range(P):
            o = p * n + i; g = I.gfirst[o]
            if g < 0: continue
            if g == p: I.res[o] = -I.gw[o]; I.u[o] = 0; I.pd[o] = 0; I.hp[o] = 0
            else: I.res[g * n + i] -= I.gw[o]
        chain_solve(I, i, I.res, I.zz, 1, 0)

def ez(I):
    if I.flags[1]: return
    n = I.n
    for a in range(I.flags[0]):
        pa, ja = I.rowp[a], I.rowj[a]; acc = 0.0
        for i in range(n):
            g = I.gfirst[pa * n + i]
            if g >= 0: acc += erow(I, pa, ja, i) * I.zz[g * n + i]
        I.ez[a] = acc

def wk(I):
    if I.flags[1]: return
    r = I.flags[0]
    for a in range(r):
        acc = sum(I.Ci[a * I.rmax + c] * I.ez[c] for c in range(r))
        I.wv[a] = acc; I.nu[a] -= acc

def update_res(I):
    if I.flags[1]: return
    n, P = I.n, I.P
    for i in range(n):
        for p in range(P):
            o = p * n + i; g = I.gfirst[o]
            if g < 0: continue
            qv = sum(I.wv[a] * erow(I, p, I.rowj[a], i) for a in range(I.rowoff[p], I.rowoff[p + 1]))
            I.res[g * n + i] -= qv
        chain_solve(I, i, I.res, I.zz, 1, 0)
        s = 0.0
        for p in range(P):
            o = p * n + i
            if I.gfirst[o] == p: s += I.res[o] * I.zz[o]
        I.part[i] = s

def rz(I, init):
    if I.flags[1]: return
    s = I.part[:I.n].sum()
    if not np.isfinite(s): I.flags[3] = 4; I.flags[1] = 1; return
    if init:
        I.sc[0] = s; I.sc[1] = s; I.sc[3] = 0.0
        if not s > 0: I.flags[1] = 1
        return
    I.flags[2] += 1
    I.sc[3] = s / I.sc[0]; I.sc[0] = s
    if not s > kPcgTol ** 2 * I.sc[1]: I.flags[1] = 1
    elif I.flags[2] >= kMaxPcg: I.flags[3] = 3; I.flags[1] = 1

def pdir(I):
    if I.flags[1]: return
    beta = I.sc[3]
    for i in range(I.n):
        for p in range(I.P):
            o = p * I.n + i
            if I.gfirst[o] == p: I.pd[o] = -I.zz[o] + beta * I.pd[o]

def prodF(I, which):
    if which == 0 and I.flags[1]: return
    n, k = I.n, I.k
    for e in range(I.P * k):
        p, j = e // k, e % k; acc = 0.0
        if which == 2:
            for i in range(n): acc += (xe(I, p, i) - I.wT[i]) * I.F[i * k + j]
            I.Uk2[e] = acc
        else:
            v = I.pd if which == 0 else I.u
            for i in range(n):
                g = I.gfirst[p * n + i]
                if g >= 0: acc += v[g * n + i] * I.F[i * k + j]
            I.Uk[e] = acc

def omega(I, which, in_pcg):
    if in_pcg and I.flags[1]: return
    k = I.k
    U = I.Uk if which == 0 else I.Uk2; W = I.Wk if which == 0 else I.Wk2
    for e in range(I.P * k):
        p, j = e // k, e % k
        acc = sum(I.Om[j, l] * U[p * k + l] for l in range(k))
        W[e] = 2 * I.kappa * acc

def hp(I):
    if I.flags[1]: return
    n, P, k = I.n, I.P, I.k
    for i in range(n):
        vprev, vcur = 0.0, gv(I, I.pd, 0, i)
        for p in range(P):
            vnext = gv(I, I.pd, p + 1, i)
            o = p * n + i; g = I.gfirst[o]
            if g >= 0:
                y = 2 * I.kappa * I.D[o] * vcur
                for j in range(k): y += I.F[i * k + j] * I.Wk[p * k + j]
                y += I.hz[o] * (vcur - vprev) - I.hz[(p + 1) * n + i] * (vnext - vcur)
                if g == p: I.hp[o] = y
                else: I.hp[g * n + i] += y
            vprev, vcur = vcur, vnext
        s = 0.0
        for p in range(P):
            o = p * n + i
            if I.gfirst[o] == p: s += I.pd[o] * I.hp[o]
        I.part[i] = s

def alpha(I):
    if I.flags[1]: return
    s = I.part[:I.n].sum()
    if not (s > 0) or not np.isfinite(s): I.flags[3] = 4; I.flags[1] = 1; return
    I.sc[2] = I.sc[0] / s

def step(I):
    if I.flags[1]: return
    al = I.sc[2]
    for i in range(I.n):
        for p in range(I.P):
            o = p * I.n + i
            if I.gfirst[o] != p: continue
            I.u[o] += al * I.pd[o]; I.res[o] += al * I.hp[o]
        chain_solve(I, i, I.res, I.zz, 1, 0)

def grad_asset(I):
    n, P, k = I.n, I.P, I.k
    kap, dexp = I.kappa, I.d
    for i in range(n):
        wTi = I.wT[i]; dw0 = dwT = 0.0
        for r in range(P + 1):
            o = r * n + i
            live = not dead_trade(I, r, i)
            z = xe(I, r, i) - xe(I, r - 1, i)
            duz = gv(I, I.u, r, i) - gv(I, I.u, r - 1, i)
            sz = sgn(z)
            I.ds[o] = -I.lam2 * sz * duz if live else 0.0
            I.dq[o] = -I.lam3 * dexp * abs(z) ** (dexp - 1) * sz * duz if live else 0.0
            hd = I.hz[o] * duz
            if r == 0: dw0 += hd
            if r == P: dwT -= hd
        for p in range(P):
            o = p * n + i
            up = gv(I, I.u, p, i); dX = xe(I, p, i) - wTi
            y = 2 * kap * I.D[o] * up
            for j in range(k): y += I.F[i * k + j] * I.Wk[p * k + j]
            I.dalpha[o] = up; I.dD[o] = -2 * kap * dX * up
            dwT += y
            sc = I.src[o]
            if sc == 1 or sc == 2:
                hl = I.hz[o] * (gv(I, I.u, p, i) - gv(I, I.u, p - 1, i))
                hr = I.hz[(p + 1) * n + i] * (gv(I, I.u, p + 1, i) - gv(I, I.u, p, i))
                cf = I.gw[o] - y - (hl - hr)
                sx = sgn(I.xfix[o])
                for a in range(I.rowoff[p], I.rowoff[p + 1]):
                    j = I.rowj[a]
                    cf -= I.nu[a] * (sx if j < 0 else I.A[j * n + i])
                if sc == 1: dw0 += cf
                else: dwT += cf
        I.dalpha[P * n + i] = 0.0; I.dD[P * n + i] = 0.0
        I.dw0[i] = dw0; I.dwT[i] = dwT

def grad_F(I):
    n, k = I.n, I.k
    for e in range(n * k):
        i, j = e // k, e % k
        acc = 0.0
        for p in range(I.P):
            acc += gv(I, I.u, p, i) * I.Wk2[p * k + j] + (xe(I, p, i) - I.wT[i]) * I.Wk[p * k + j]
        I.dF[e] = -acc

def run(I):
    classify(I); rows(I)
    for c0 in range(0, I.rmax, kNB):
        zcols(I, c0); cfill(I, c0)
    chol(I); inverse(I)
    pcg_init(I); ez(I); wk(I); update_res(I); rz(I, 1); pdir(I)
    for it in range(kMaxPcg):
        if I.flags[1]: break
        prodF(I, 0); omega(I, 0, 1); hp(I); alpha(I); step(I); ez(I); wk(I); update_res(I); rz(I, 0); pdir(I)
    prodF(I, 1); omega(I, 0, 0); prodF(I, 2); omega(I, 1, 0); grad_asset(I); grad_F(I)
    return I



class Checked:
    """1-D buffer whose scalar indexing is bounds-checked (slices pass through)."""

    def __init__(self, a, name):
        self.a, self.name = a, name

    def _chk(self, i):
        if not isinstance(i, slice) and not (0 <= i < self.a.size):
            raise IndexError(f"{self.name}[{i}] outside 0..{self.a.size - 1}")

    def __getitem__(self, i):
        self._chk(i)
        return self.a[i]

    def __setitem__(self, i, v):
        self._chk(i)
        self.a[i] = v


def emulate(p, w, yA, yD, gw, f64=1):
    I = setup(p, w, yA, yD, gw, f64)
    for nm, v in list(vars(I).items()):
        if isinstance(v, np.ndarray) and v.ndim == 1 and nm not in ("F", "D", "s", "q", "w0", "wT", "A", "w",
                                                                     "yA", "yD", "gw"):
            setattr(I, nm, Checked(v, nm))
    run(I)
    T, n, k = p.T, I.n, I.k
    grads = {"alpha": I.dalpha.a.reshape(T, n), "D": I.dD.a.reshape(T, n), "s": I.ds.a.reshape(T, n),
             "q": I.dq.a.reshape(T, n), "F": I.dF.a.reshape(n, k), "w0": I.dw0.a, "wT": I.dwT.a}
    return I, grads


def _no_rows(p):
    return replace(p, A=np.zeros((0, p.F.shape[0])), L=np.zeros(0), U=np.zeros(0))


CASES = {
    "ties_w0_wT": lambda: S.make_multi(4, 20, 4, 12, n_onehot=2),
    "zeros_budget": lambda: S.make_multi(6, 200, 12, 1),
    "quadratic_impact": lambda: S.make_multi(5, 60, 6, 3, n_onehot=2, d=2.0),
    "one_free_period": lambda: S.make_multi(2, 30, 4, 5, n_onehot=2),
    "no_exposure_rows": lambda: _no_rows(S.make_multi(3, 30, 4, 6, n_onehot=2)),
}


def _compare(p, sol, g, grads, rng):
    for nm in OG.MULTI_PARAMS:
        assert np.all(np.isfinite(grads[nm])), nm
        delta = rng.standard_normal(np.shape(getattr(p, nm)))
        a = float(np.sum(grads[nm] * delta))
        b = OG.directional_vjp(p, sol, g, nm, delta)
        scale = float(np.linalg.norm(grads[nm]) * np.linalg.norm(delta))
        # 1e-5: the oracle takes its w0 and w_T derivatives by central differences
        # with a step tied to the smallest live trade (about 1e-6 relative error)
        assert abs(a - b) <= 1e-5 * abs(b) + 1e-9 * scale, (nm, a, b)


@pytest.mark.parametrize("case", sorted(CASES))
def test_emulated_kernels_match_oracle(case):
    p = CASES[case]()
    sol = oracle.solve(p)
    assert sol.polished
    rng = np.random.default_rng(1)
    g = rng.standard_normal(sol.x.shape)
    I, grads = emulate(p, sol.x, sol.yA, sol.yD, g)
    assert I.flags[3] == 0 and 0 < I.flags[2] < 50
    _compare(p, sol, g, grads, rng)


def test_emulated_kernels_drop_a_dependent_row():
    """A duplicated active exposure row makes E M^-1 E^T singular: the Cholesky
    drops the copy and the gradients are those of the problem without it."""
    p = S.make_multi(5, 60, 6, 3, n_onehot=2)
    sol = oracle.solve(p)
    j = sorted({jj for (_, jj, _, _) in sol.reduced.box})[0]
    p2 = replace(p, A=np.vstack([p.A, p.A[j:j + 1]]), L=np.append(p.L, p.L[j]), U=np.append(p.U, p.U[j]))
    yA2 = np.hstack([sol.yA, sol.yA[:, j:j + 1]])
    yA2[:, j] *= 0.5
    yA2[:, -1] *= 0.5
    rng = np.random.default_rng(1)
    g = rng.standard_normal(sol.x.shape)
    I, grads = emulate(p2, sol.x, yA2, sol.yD, g)
    r = I.flags[0]
    assert int(np.sum(I.drop.a[:r])) >= 1 and I.flags[3] == 0
    _compare(p, sol, g, grads, rng)


def test_emulated_kernels_on_fp32_outputs():
    """FP32 data and FP32 solver outputs (w, yA, yD rounded): the budget rows
    are found with the FP32 tolerance, zero holdings stay exact zeros, and
    the gradients match the oracle's on the same rounded data."""
    p = S.make_multi(5, 60, 6, 3, n_onehot=2).rounded(np.float32)
    sol = oracle.solve(p)
    assert sol.polished
    f32 = lambda a: np.asarray(a, dtype=np.float32).astype(np.float64)   # noqa: E731
    rng = np.random.default_rng(4)
    g = f32(rng.standard_normal(sol.x.shape))
    I, grads = emulate(p, f32(sol.x), f32(sol.yA), f32(sol.yD), g, f64=0)
    r = I.flags[0]
    assert I.flags[3] == 0
    assert sum(1 for a in range(r) if I.rowj[a] == -1) == int(np.sum(sol.reduced.budget))
    for nm in OG.MULTI_PARAMS:
        delta = rng.standard_normal(np.shape(getattr(p, nm)))
        a = float(np.sum(grads[nm] * delta))
        b = OG.directional_vjp(p, sol, g, nm, delta)
        scale = float(np.linalg.norm(grads[nm]) * np.linalg.norm(delta))
        # FP32-rounded outputs move the point by ~1e-7 relative
        assert abs(a - b) <= 1e-4 * abs(b) + 1e-7 * scale, (nm, a, b)
