"""Seeded synthetic portfolio instances (inputs only, no solver arithmetic).

This module is the single source of problem data for both the CUDA solver and
the FP64 CPU oracle. It draws the arrays of the single-period model (Sec. 2.1,
Eqs. 1-3) and of the multi-period model (Sec. 2.2, Eqs. 4-6) from fixed
distributions; it never evaluates an objective, a gradient or a projection.

The paper builds its instances from market data (Sec. 3: 5-day forward returns
plus noise for alpha, a Fama-French factor regression for the risk model, CRSP
spreads and ADV-based impact). Those data are not available here; the
distributions below stand in for them:

* F (n x k): ``k - n_onehot`` columns of N(0, 1) style loadings followed by
  ``n_onehot`` one-hot columns (industry or sector membership), the factor
  exposure matrix beta of the risk model Sigma = beta Sigma_f beta^T + D (Sec. 3.2).
* Omega (k x k): diagonal factor covariance, entries U[1e-5, 1e-4].
* D: specific variances U[1e-4, 9e-4].
* alpha ~ N(0, (2e-3)^2); multi-period alpha_t follows an AR(1) with
  correlation 0.8 across t and the same stationary variance.
* s ~ U[2e-4, 2e-3] (spread), q ~ U[1e-3, 1e-2] (impact), d = 1.5.
* w0: |w0_i| ~ U(0, 1) with random signs, rescaled to ||w0||_1 = 0.9; the
  terminal target w_T of the multi-period model is drawn the same way.
* GMV = 1e9, lambda1 = 10 / GMV, lambda2 = lambda3 = 1.

All arrays are float64 and C-contiguous. Per-period arrays of the
multi-period model have T rows indexed t = 1..T as in Eq. 4; ``D[T-1]`` and
``alpha[T-1]`` only enter constants of the objective.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
from typing import Optional

import numpy as np

GMV_DEFAULT = 1e9


@dataclass
class Problem:
    """One portfolio instance in the paper's units (Eqs. 1-6).

    Single period (``T == 0``): alpha, D, s, q are (n,); the decision is w.
    Multi-period (``T >= 2``): alpha, D, s, q are (T, n); the decisions are
    w_1..w_{T-1}; w0 and wT are fixed.
    """

    F: np.ndarray            # (n, k) factor exposures
    Omega: np.ndarray        # (k, k) factor covariance (symmetric positive definite)
    D: np.ndarray            # (n,) or (T, n) specific variances (> 0)
    alpha: np.ndarray        # (n,) or (T, n) predicted returns
    s: np.ndarray            # (n,) or (T, n) spread coefficients (>= 0)
    q: np.ndarray            # (n,) or (T, n) impact coefficients (>= 0)
    w0: np.ndarray           # (n,) initial portfolio
    A: np.ndarray            # (m, n) exposure matrix
    L: np.ndarray            # (m,) lower exposure bounds
    U: np.ndarray            # (m,) upper exposure bounds
    GMV: float = GMV_DEFAULT
    lam1: float = 10.0 / GMV_DEFAULT
    lam2: float = 1.0
    lam3: float = 1.0
    d: float = 1.5
    T: int = 0               # 0 = single-period model, else the horizon T
    wT: Optional[np.ndarray] = None   # (n,) terminal portfolio (multi-period)
    tag: str = field(default="")

    @property
    def n(self) -> int:
        return int(self.F.shape[0])

    @property
    def k(self) -> int:
        return int(self.F.shape[1])

    @property
    def m(self) -> int:
        return int(self.A.shape[0])

    @property
    def multi(self) -> bool:
        return self.T >= 2

    @property
    def periods(self) -> int:
        """Number of free portfolios: 1 (single) or T - 1 (multi)."""
        return self.T - 1 if self.multi else 1

    def rounded(self, dtype) -> "Problem":
        """Copy whose arrays are rounded to ``dtype`` and widened back to float64.

        The GPU solves the storage-rounded data; the oracle is given exactly the
        same numbers through this copy.
        """
        def r(a):
            if a is None:
                return None
            return np.ascontiguousarray(np.asarray(a, dtype=dtype).astype(np.float64))
        kw = {}
        for name in ("F", "Omega", "D", "alpha", "s", "q", "w0", "A", "L", "U", "wT"):
            kw[name] = r(getattr(self, name))
        return replace(self, **kw)

    def with_F_rounded_bf16(self) -> "Problem":
        """Copy with F and A rounded to bfloat16 (round to nearest even), as
        stored by the batched solver; every other array is rounded to float32."""
        p = self.rounded(np.float32)
        return replace(p, F=_round_bf16(p.F), A=_round_bf16(p.A))


def _round_bf16(a: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(a, dtype=np.float32)
    u = x.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    u = (u + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _signed_l1(rng: np.random.Generator, n: int, l1: float) -> np.ndarray:
    mag = rng.uniform(0.0, 1.0, n)
    sign = np.where(rng.uniform(0.0, 1.0, n) < 0.5, -1.0, 1.0)
    w = sign * mag
    return w * (l1 / np.abs(w).sum())


def _loadings(rng: np.random.Generator, n: int, k: int, n_onehot: int,
              groups: np.ndarray) -> np.ndarray:
    """k - n_onehot Gaussian columns, then one-hot membership of ``groups``."""
    F = np.zeros((n, k))
    F[:, : k - n_onehot] = rng.standard_normal((n, k - n_onehot))
    F[np.arange(n), k - n_onehot + (groups % n_onehot)] = 1.0
    return F


def make_single(n: int, k: int, seed: int, *, n_onehot: int = 10, n_industries: Optional[int] = None,
                bound: float = 0.05, lam1: float = 10.0 / GMV_DEFAULT, lam2: float = 1.0,
                lam3: float = 1.0, d: float = 1.5, tag: str = "") -> Problem:
    """Single-period instance (Eqs. 1-3).

    ``n_industries is None``: A = F^T (k rows, factor exposure bounds).
    Otherwise the industries (uniform among ``n_industries``) define the
    one-hot sector columns of F (sector = industry mod ``n_onehot``) and
    A = [F^T; H] with H the industry net-exposure rows.
    """
    rng = np.random.default_rng(seed)
    ngroups = n_industries if n_industries is not None else n_onehot
    groups = rng.integers(0, ngroups, n)
    F = _loadings(rng, n, k, n_onehot, groups)
    Omega = np.diag(rng.uniform(1e-5, 1e-4, k))
    D = rng.uniform(1e-4, 9e-4, n)
    alpha = rng.normal(0.0, 2e-3, n)
    s = rng.uniform(2e-4, 2e-3, n)
    q = rng.uniform(1e-3, 1e-2, n)
    w0 = _signed_l1(rng, n, 0.9)
    if n_industries is None:
        A = F.T.copy()
    else:
        H = np.zeros((n_industries, n))
        H[groups, np.arange(n)] = 1.0
        A = np.vstack([F.T, H])
    m = A.shape[0]
    L = np.full(m, -bound)
    U = np.full(m, bound)
    return Problem(F=F, Omega=Omega, D=D, alpha=alpha, s=s, q=q, w0=w0, A=np.ascontiguousarray(A),
                   L=L, U=U, lam1=lam1, lam2=lam2, lam3=lam3, d=d, T=0, tag=tag)


def make_multi(T: int, n: int, k: int, seed: int, *, n_onehot: int = 10, bound: float = 0.05,
               rho: float = 0.8, d_scale: tuple = (0.8, 1.2), lam1: float = 10.0 / GMV_DEFAULT,
               lam2: float = 1.0, lam3: float = 1.0, d: float = 1.5, tag: str = "") -> Problem:
    """Multi-period instance (Eqs. 4-6) with T periods.

    alpha_t: AR(1) with correlation ``rho`` and stationary sd 2e-3;
    D_t = D * u_t, u_t ~ U[d_scale]; s_t, q_t constant over t; A = F^T.
    """
    assert T >= 2
    rng = np.random.default_rng(seed)
    groups = rng.integers(0, n_onehot, n)
    F = _loadings(rng, n, k, n_onehot, groups)
    Omega = np.diag(rng.uniform(1e-5, 1e-4, k))
    D0 = rng.uniform(1e-4, 9e-4, n)
    D = D0[None, :] * rng.uniform(d_scale[0], d_scale[1], (T, n))
    alpha = np.empty((T, n))
    alpha[0] = rng.normal(0.0, 2e-3, n)
    innov = np.sqrt(1.0 - rho * rho)
    for t in range(1, T):
        alpha[t] = rho * alpha[t - 1] + innov * rng.normal(0.0, 2e-3, n)
    s = np.repeat(rng.uniform(2e-4, 2e-3, n)[None, :], T, axis=0)
    q = np.repeat(rng.uniform(1e-3, 1e-2, n)[None, :], T, axis=0)
    w0 = _signed_l1(rng, n, 0.9)
    wT = _signed_l1(rng, n, 0.9)
    A = np.ascontiguousarray(F.T.copy())
    m = A.shape[0]
    return Problem(F=F, Omega=Omega, D=D, alpha=alpha, s=s, q=q, w0=w0, A=A,
                   L=np.full(m, -bound), U=np.full(m, bound), lam1=lam1, lam2=lam2,
                   lam3=lam3, d=d, T=T, wT=wT, tag=tag)


# ---------------------------------------------------------------------------
# The five benchmark workloads (seeded).
# ---------------------------------------------------------------------------

def config_single_small(seed: int = 0) -> Problem:
    """n=500, k=20 (10 Gaussian + 10 one-hot industries), A = F^T, bounds +-0.05."""
    return make_single(500, 20, seed, n_onehot=10, bound=0.05, tag="single n=500 k=20")


def config_single_large(seed: int = 1) -> Problem:
    """n=10000, k=100 (90 Gaussian + 10 one-hot sectors), 60 industries,
    A = [F^T; industry rows] (m=160), bounds +-0.02."""
    return make_single(10000, 100, seed, n_onehot=10, n_industries=60, bound=0.02,
                       tag="single n=10000 k=100 m=160")


def config_multi(seed: int = 2) -> Problem:
    """T=20, n=5000, k=80, A = F^T, bounds +-0.05."""
    return make_multi(20, 5000, 80, seed, tag="multi T=20 n=5000 k=80")


def config_batch(seed: int = 3, n_single: int = 512, n_multi: int = 64) -> list:
    """512 single-period instances (n ~ U{500..8000}, k in {40, 80}) and 64
    multi-period instances (T ~ U{5..40}, n ~ U{1000..4000}, k in {40, 80}).
    Instance i is drawn from seed ``seed * 10**6 + i``."""
    out = []
    for i in range(n_single + n_multi):
        r = np.random.default_rng(seed * 10 ** 6 + i)
        k = int(r.choice([40, 80]))
        if i < n_single:
            n = int(r.integers(500, 8001))
            out.append(make_single(n, k, seed * 10 ** 6 + i + 7 * 10 ** 5,
                                   tag=f"batch single n={n} k={k}"))
        else:
            T = int(r.integers(5, 41))
            n = int(r.integers(1000, 4001))
            out.append(make_multi(T, n, k, seed * 10 ** 6 + i + 7 * 10 ** 5,
                                  tag=f"batch multi T={T} n={n} k={k}"))
    return out


def config_diff(seed: int = 4, n_single: int = 64, n_multi: int = 8) -> list:
    """64 single-period (n=3000, k=60) and 8 multi-period (T=50, n=2000, k=60)."""
    out = []
    for i in range(n_single):
        out.append(make_single(3000, 60, seed * 10 ** 6 + i, tag="diff single n=3000 k=60"))
    for i in range(n_multi):
        out.append(make_multi(50, 2000, 60, seed * 10 ** 6 + n_single + i,
                              tag="diff multi T=50 n=2000 k=60"))
    return out


# ---------------------------------------------------------------------------
# Returns for the risk-model estimation of Sec. 3.2 (seeded).
# ---------------------------------------------------------------------------

@dataclass
class Returns:
    """One estimation window: factor returns F (T x p) and stock returns R
    (T x n, NaN where a stock has no return), both stored in float32 and kept
    here as float64 copies of the float32 values.  ``beta``, ``sigma_f`` and
    ``spec_var`` are the true parameters the data were drawn from."""
    F: np.ndarray
    R: np.ndarray
    beta: np.ndarray
    sigma_f: np.ndarray
    spec_var: np.ndarray


def make_returns(T: int, n: int, seed: int, p: int = 6, late_frac: float = 0.1, irregular_frac: float = 0.0,
                 noise: bool = True) -> Returns:
    """Daily returns from a p-factor model (the paper's market factor and five
    Fama-French factors, p = 6): factor returns f_k ~ N(0, Sigma_f) with daily
    volatilities U[0.4 %, 1.2 %] and random correlations; loadings: market
    N(1, 0.3^2), the others N(0, 0.5^2); specific volatilities U[1 %, 3 %];
    r_k = beta f_k + eps_k.  A share ``late_frac`` of the stocks start on a
    day drawn uniformly from [1, T - 20] (NaN before: a listing inside the
    window), a share ``irregular_frac`` has one NaN after its first return."""
    rng = np.random.default_rng(seed)
    vol = rng.uniform(0.004, 0.012, p)
    Z = rng.standard_normal((p, p))
    C = Z @ Z.T + p * np.eye(p)
    d = np.sqrt(np.diag(C))
    corr = C / np.outer(d, d)
    sigma_f = corr * np.outer(vol, vol)
    F = rng.multivariate_normal(np.zeros(p), sigma_f, size=T)
    beta = np.empty((n, p))
    beta[:, 0] = rng.normal(1.0, 0.3, n)
    beta[:, 1:] = rng.normal(0.0, 0.5, (n, p - 1))
    spec = rng.uniform(0.01, 0.03, n) ** 2
    R = F @ beta.T
    if noise:
        R = R + rng.standard_normal((T, n)) * np.sqrt(spec)[None, :]
    late = rng.uniform(0.0, 1.0, n) < late_frac
    starts = rng.integers(1, max(2, T - 20), n)
    for i in np.nonzero(late)[0]:
        R[: starts[i], i] = np.nan
    irr = np.nonzero(rng.uniform(0.0, 1.0, n) < irregular_frac)[0]
    for i in irr:
        first = int(np.argmax(~np.isnan(R[:, i])))
        if first < T - 2:
            R[rng.integers(first + 1, T), i] = np.nan
    f32 = lambda a: np.ascontiguousarray(np.asarray(a, dtype=np.float32).astype(np.float64))  # noqa: E731
    return Returns(F=f32(F), R=f32(R), beta=beta, sigma_f=sigma_f, spec_var=spec)


# ---------------------------------------------------------------------------
# Paper-shaped instances of the lambda grid (Sec. 4.1; data recipe of Sec. 3)
# ---------------------------------------------------------------------------
PAPER_LAMBDA1 = (1e-8, 1e-7, 1e-6, 1e-5, 1e-4)
PAPER_LAMBDA23 = (1.0, 10.0, 100.0, 1000.0, 10000.0)
PAPER_DATES = 21


def eta_profile(T: int, reading: str = "literal") -> np.ndarray:
    """Intraday scaling of the costs for t = 1..T (Sec. 3.4): eta_t = 0.5 +
    2 (t/T - 0.5)^2, normalised by sum_{k=1}^{T-1} eta_k as printed.  The
    formula makes costs largest at the ends while the text says liquidity is
    greatest there: ``reading="inverted"`` uses 1 / eta_t (normalised the
    same way) for the other reading."""
    t = np.arange(1, T + 1, dtype=np.float64)
    eta = 0.5 + 2.0 * (t / T - 0.5) ** 2
    if reading == "inverted":
        eta = 1.0 / eta
    elif reading != "literal":
        raise ValueError(reading)
    return eta / eta[: T - 1].sum()


def make_paper_date(date: int, n: int = 2000, p: int = 6, seed_base: int = 6 * 10 ** 6) -> dict:
    """The lambda-independent data of one date: a p-factor risk model with a
    full factor covariance (market + five style factors), alpha as the mean of
    the next five daily returns plus half a daily volatility of noise (the
    paper's construction, on simulated returns), spreads, the impact
    coefficient q = sigma (GMV / ADV)^(d - 1) with ADV log-uniform in
    [1e7, 1e9], w0 and a terminal target w_T (random signs, l1 norm 0.9)."""
    rng = np.random.default_rng(seed_base + date)
    vol = rng.uniform(0.004, 0.012, p)
    Z = rng.standard_normal((p, p))
    C = Z @ Z.T + p * np.eye(p)
    dd = np.sqrt(np.diag(C))
    sigma_f = (C / np.outer(dd, dd)) * np.outer(vol, vol)
    beta = np.empty((n, p))
    beta[:, 0] = rng.normal(1.0, 0.3, n)
    beta[:, 1:] = rng.normal(0.0, 0.5, (n, p - 1))
    D = rng.uniform(1e-4, 9e-4, n)
    sig_tot = np.sqrt(np.einsum("ij,jk,ik->i", beta, sigma_f, beta) + D)
    f5 = rng.multivariate_normal(np.zeros(p), sigma_f, size=5)
    r5 = f5 @ beta.T + rng.standard_normal((5, n)) * np.sqrt(D)[None, :]
    alpha = r5.mean(axis=0) + 0.5 * sig_tot * rng.standard_normal(n)
    s = rng.uniform(2e-4, 2e-3, n)
    adv = np.exp(rng.uniform(np.log(1e7), np.log(1e9), n))
    w0 = _signed_l1(rng, n, 0.9)
    wT = _signed_l1(rng, n, 0.9)
    return dict(beta=beta, sigma_f=sigma_f, D=D, alpha=alpha, s=s, adv=adv, sig_tot=sig_tot, w0=w0, wT=wT)


def make_paper_instance(date: int, lam1: float, lam23: float, kind: str = "single", n: int = 2000, T: int = 10,
                        d: float = 1.5, eta_reading: str = "literal", bound: float = 0.05,
                        GMV: float = GMV_DEFAULT) -> Problem:
    """One instance of the paper's grid: date ``date`` (0..20), lambda1, lambda2 =
    lambda3, single-period or multi-period (T = 10, alpha_t = alpha and Sigma
    fixed over the horizon, s_t and q_t scaled by the eta profile).  A = beta^T
    (factor exposure rows, bounds +-bound)."""
    b = make_paper_date(date, n)
    q = b["sig_tot"] * (GMV / b["adv"]) ** (d - 1.0)
    A = np.ascontiguousarray(b["beta"].T.copy())
    m = A.shape[0]
    tag = f"paper {kind} date={date} lam1={lam1:g} lam23={lam23:g}"
    if kind == "single":
        return Problem(F=b["beta"], Omega=b["sigma_f"], D=b["D"], alpha=b["alpha"], s=b["s"], q=q, w0=b["w0"],
                       A=A, L=np.full(m, -bound), U=np.full(m, bound), GMV=GMV, lam1=lam1, lam2=lam23,
                       lam3=lam23, d=d, T=0, tag=tag)
    eta = eta_profile(T, eta_reading)
    return Problem(F=b["beta"], Omega=b["sigma_f"], D=np.repeat(b["D"][None, :], T, axis=0),
                   alpha=np.repeat(b["alpha"][None, :], T, axis=0), s=eta[:, None] * b["s"][None, :],
                   q=eta[:, None] * q[None, :], w0=b["w0"], A=A, L=np.full(m, -bound), U=np.full(m, bound),
                   GMV=GMV, lam1=lam1, lam2=lam23, lam3=lam23, d=d, T=T, wT=b["wT"], tag=tag + f" eta={eta_reading}")
