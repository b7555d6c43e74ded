"""Risk-model estimation of Sec. 3.2 in FP64 (test infrastructure).

ORACLE: test infrastructure only; shares no code with the CUDA estimator.

For one estimation window of T days (the paper uses the previous T = 504
business days of every date) with factor returns F (T x p, row k = f_k) and
stock returns R (T x n, column i = r_i):

* the factor covariance is the sample covariance of the factor returns,
      Sigma_f = (F - 1 1^T F / T)^T (F - 1 1^T F / T) / (T - 1);
* the loadings of stock i are the least-squares coefficients of the
  regression r_i ~ F beta_i (no intercept, as the regression is stated),
  over the days on which the stock has a return;
* the residuals theta_{k,i} = r_{k,i} - beta_i^T f_k give the specific
  variance D_ii as their sample variance over those days (mean removed,
  divisor count - 1).

A stock is estimated only with at least ``min_obs`` days of history (the
paper: two months).  Reading of "history": a stock has returns from its first
day in the window on (missing days are NaN and come first); a NaN after the
first return makes the stock irregular and it is not estimated either.
Unestimated stocks get beta = 0, D = NaN and valid = False.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class RiskModel:
    beta: np.ndarray      # (n, p)
    sigma_f: np.ndarray   # (p, p)
    D: np.ndarray         # (n,)
    valid: np.ndarray     # (n,) bool
    count: np.ndarray     # (n,) days with a return


def factor_covariance(F: np.ndarray) -> np.ndarray:
    """Sample covariance of the rows of F, written out as in Sec. 3.2."""
    F = np.asarray(F, dtype=np.float64)
    T = F.shape[0]
    C = F - np.ones((T, 1)) @ (np.ones((1, T)) @ F) / T
    return C.T @ C / (T - 1)


def history(r: np.ndarray):
    """(first day with a return, number of days, regular) of one return column."""
    ok = ~np.isnan(r)
    if not ok.any():
        return len(r), 0, True
    first = int(np.argmax(ok))
    regular = bool(ok[first:].all())
    return first, int(ok.sum()), regular


def estimate(F, R, min_obs: int = 42) -> RiskModel:
    """Loadings, factor covariance and specific variances of one window."""
    F = np.asarray(F, dtype=np.float64)
    R = np.asarray(R, dtype=np.float64)
    T, p = F.shape
    n = R.shape[1]
    beta = np.zeros((n, p))
    D = np.full(n, np.nan)
    valid = np.zeros(n, dtype=bool)
    count = np.zeros(n, dtype=np.int64)
    for i in range(n):
        first, cnt, regular = history(R[:, i])
        count[i] = cnt
        if not regular or cnt < min_obs:
            continue
        Fi = F[first:]
        ri = R[first:, i]
        b, *_ = np.linalg.lstsq(Fi, ri, rcond=None)
        theta = ri - Fi @ b
        beta[i] = b
        D[i] = float(np.sum((theta - theta.mean()) ** 2) / (cnt - 1))
        valid[i] = True
    return RiskModel(beta, factor_covariance(F), D, valid, count)
