"""Serial CPU transcription of the joint prox kernel's prox step
(csrc/ff_joint.cu: joint_coord, impact_root and the safeguarded Newton search
for the budget multiplier), checked against the oracle's definition-based
prox_joint.  The transcription follows the kernel's branches, constants and
order of operations; threads become loops.  This checks the GPU algorithm on
the CPU (every branch of the coordinate solve, the multiplier search with and
without a warm start); the GPU kernel itself is compared with the oracle in
test_gpu_joint.py.  Nothing in the package imports this file, and it shares
no code with the oracle."""
import math

import numpy as np
import pytest

from oracle.prox import prox_joint

kMuRounds = 64


def sgn(x):
    return 1.0 if x > 0 else (-1.0 if x < 0 else 0.0)


def impact_root(t, gc, d, dk):
    if not t > 0.0:
        return 0.0
    if not gc > 0.0:
        return t
    if dk == 1:
        be = 1.5 * gc
        rho = 2.0 * t / (be + math.sqrt(be * be + 4.0 * t))
        return rho * rho
    if dk == 2:
        return t / (1.0 + 2.0 * gc)
    lo, hi, r = 0.0, t, t
    for _ in range(100):
        rp = r ** (d - 1.0)
        h = r + gc * d * rp - t
        if h > 0:
            hi = r
        else:
            lo = r
        dh = 1.0 + gc * d * (d - 1.0) * (rp / r if r > 0 else 0.0)
        rn = r - h / dh
        if not (lo < rn < hi):
            rn = 0.5 * (lo + hi)
        if abs(rn - r) <= 1e-16 * t:
            return rn
        r = rn
    return r


def joint_coord(v, a, mu, g, c1, c2, cp0, d, dk):
    gc1, gc2 = g * c1, g * c2
    lo_b, hi_b = min(0.0, a), max(0.0, a)

    def sides(b):
        if a == 0.0:
            return -v - gc1 - mu, -v + gc1 + mu
        if b == 0.0:
            return -v + cp0 - mu, -v + cp0 + mu
        base = (a - v) + mu * sgn(a)
        return base - gc1, base + gc1

    L1, R1 = sides(lo_b)
    if L1 <= 0.0 <= R1:
        return lo_b, 0.0
    if L1 > 0.0:
        s0, s1 = -1.0, -1.0
    elif a == 0.0:
        s0, s1 = 1.0, 1.0
    else:
        L2, R2 = sides(hi_b)
        if L2 <= 0.0 <= R2:
            return hi_b, 0.0
        if L2 > 0.0:
            s0, s1 = (1.0, -1.0) if a > 0 else (-1.0, 1.0)
        else:
            s0, s1 = 1.0, 1.0
    t = v - a - gc1 * s1 - mu * s0
    r = impact_root(s1 * t, gc2, d, dk)
    w = a + s1 * r
    dw = 0.0
    if r > 0.0 and w != 0.0:
        curv = 0.0
        if gc2 > 0.0:
            curv = gc2 * d * (d - 1.0) * (1.0 if dk == 2 else (1.0 / math.sqrt(r) if dk == 1 else r ** (d - 2.0)))
        dw = -1.0 / (1.0 + curv)
    return w, dw


def joint_prox_kernel(v, a, g, c1, c2, d, mu_prev=0.0):
    """The kernel's prox step: the multiplier search, then x_bar."""
    dk = 1 if d == 1.5 else (2 if d == 2.0 else 0)
    n = len(v)
    cp0 = [g * (sgn(-ai) * (c1[i] + c2[i] * d * abs(ai) ** (d - 1.0))) if ai != 0.0 else 0.0
           for i, ai in enumerate(a)]

    def S_at(mu):
        s, ds = 0.0, 0.0
        for i in range(n):
            w, dw = joint_coord(v[i], a[i], mu, g, c1[i], c2[i], cp0[i], d, dk)
            s += abs(w)
            ds += dw
        return s, ds

    lo, hi, mt = 0.0, math.inf, mu_prev
    search = True
    if mt > 0.0:
        St, dSt = S_at(mt)
        if St <= 1.0 and S_at(0.0)[0] <= 1.0:
            search = False
    else:
        St, dSt = S_at(0.0)
        if St <= 1.0:
            search = False
    mu = 0.0
    if search:
        exact = False
        for _ in range(kMuRounds):
            if abs(St - 1.0) <= 1e-15:
                exact = True
                break
            if St > 1.0:
                lo = mt
            else:
                hi = mt
            if math.isfinite(hi) and hi - lo <= 1e-16 * hi:
                break
            mn = mt + (St - 1.0) / (-dSt) if dSt < 0.0 else -1.0
            if not (lo < mn < hi):
                mn = 0.5 * (lo + hi) if math.isfinite(hi) else (4.0 * lo if lo > 0.0 else (St - 1.0) / n)
            mt = mn
            St, dSt = S_at(mt)
        mu = mt if exact else (hi if math.isfinite(hi) else mt)
    x = np.array([joint_coord(v[i], a[i], mu, g, c1[i], c2[i], cp0[i], d, dk)[0] for i in range(n)])
    return x, mu


@pytest.mark.parametrize("d", [1.5, 2.0, 1.3])
@pytest.mark.parametrize("case", ["binding", "inside", "zeros_in_w0", "no_impact"])
def test_kernel_prox_step_matches_oracle(d, case):
    rng = np.random.default_rng({"binding": 1, "inside": 2, "zeros_in_w0": 3, "no_impact": 4}[case])
    n = 60
    a = rng.normal(0, 0.02, n)
    if case == "zeros_in_w0":
        a[::3] = 0.0
    v = a + rng.normal(0, 0.03 if case != "binding" else 0.2, n)
    if case == "inside":
        v *= 0.2
        a *= 0.2
    g = 0.7
    c1 = rng.uniform(0.0, 5e-3, n)
    c2 = rng.uniform(0.0, 5e-2, n) if case != "no_impact" else np.zeros(n)
    x, mu = joint_prox_kernel(list(v), list(a), g, list(c1), list(c2), d)
    ref, mu_ref = prox_joint(v, a, g, c1, c2, d)
    assert np.max(np.abs(x - ref)) <= 1e-12, (np.max(np.abs(x - ref)), mu, mu_ref)
    assert abs(mu - mu_ref) <= 1e-10 * max(1.0, mu_ref)
    assert np.abs(x).sum() <= 1.0 + 1e-13
    if case == "binding":
        assert mu > 0.0
        # a warm start from a nearby multiplier reaches the same point
        xw, muw = joint_prox_kernel(list(v), list(a), g, list(c1), list(c2), d, mu_prev=1.3 * mu)
        assert np.max(np.abs(xw - ref)) <= 1e-12
    if case == "inside":
        assert mu == 0.0
