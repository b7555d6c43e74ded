"""Pins of the risk-model oracle (oracle/risk.py, Sec. 3.2): the factor
covariance against numpy's covariance routine, exact recovery of noise-free
loadings, the one-factor closed form, the normal equations of the residuals,
the history rules, and statistical consistency on a long window."""
import numpy as np

from oracle import risk
from paper_2604_22625_gb300 import synthetic as S


def test_factor_covariance_is_the_sample_covariance():
    ret = S.make_returns(504, 10, 1)
    assert np.allclose(risk.factor_covariance(ret.F), np.cov(ret.F, rowvar=False), rtol=1e-13, atol=0)


def test_noise_free_loadings_are_recovered():
    ret = S.make_returns(300, 40, 2, late_frac=0.3, noise=False)
    # the float32 rounding of R breaks exactness slightly: regress the float64 model values
    R = ret.F @ ret.beta.T
    R[np.isnan(ret.R)] = np.nan
    m = risk.estimate(ret.F, R, min_obs=42)
    ok = m.valid
    assert ok.sum() > 20
    assert np.max(np.abs(m.beta[ok] - ret.beta[ok])) <= 1e-10
    assert np.max(m.D[ok]) <= 1e-24


def test_one_factor_closed_form():
    rng = np.random.default_rng(3)
    f = rng.normal(0, 0.01, (200, 1))
    r = 0.7 * f[:, 0] + rng.normal(0, 0.02, 200)
    m = risk.estimate(f, r[:, None], min_obs=10)
    b = float(np.sum(f[:, 0] * r) / np.sum(f[:, 0] ** 2))
    theta = r - b * f[:, 0]
    var = float(np.sum((theta - theta.mean()) ** 2) / 199)
    assert abs(m.beta[0, 0] - b) <= 1e-14 * abs(b)
    assert abs(m.D[0] - var) <= 1e-13 * var


def test_residuals_satisfy_the_normal_equations():
    ret = S.make_returns(504, 30, 4, late_frac=0.3)
    m = risk.estimate(ret.F, ret.R)
    for i in np.nonzero(m.valid)[0]:
        first, cnt, _ = risk.history(ret.R[:, i])
        Fi = ret.F[first:]
        theta = ret.R[first:, i] - Fi @ m.beta[i]
        assert np.max(np.abs(Fi.T @ theta)) <= 1e-12 * np.linalg.norm(Fi) * np.linalg.norm(ret.R[first:, i])


def test_history_rules():
    ret = S.make_returns(504, 400, 5, late_frac=0.5, irregular_frac=0.05)
    m = risk.estimate(ret.F, ret.R, min_obs=42)
    for i in range(400):
        first, cnt, regular = risk.history(ret.R[:, i])
        assert m.count[i] == cnt
        assert m.valid[i] == (regular and cnt >= 42)
        if not m.valid[i]:
            assert np.all(m.beta[i] == 0) and np.isnan(m.D[i])
    assert 0 < (~m.valid).sum() < 400
    # a late starter is the full-history regression of its own days
    i = next(i for i in range(400) if m.valid[i] and np.isnan(ret.R[0, i]))
    first = risk.history(ret.R[:, i])[0]
    sub = risk.estimate(ret.F[first:], ret.R[first:, i:i + 1], min_obs=42)
    assert np.allclose(sub.beta[0], m.beta[i], rtol=0, atol=1e-15) and abs(sub.D[0] - m.D[i]) <= 1e-18


def test_consistency_on_a_long_window():
    ret = S.make_returns(20000, 25, 6, late_frac=0.0)
    m = risk.estimate(ret.F, ret.R)
    # standard errors: sigma_eps / (sqrt(T) * factor vol) ~ 0.02 / (141 * 0.004) ~ 0.035
    assert np.max(np.abs(m.beta - ret.beta)) <= 0.25
    assert np.max(np.abs(m.D / ret.spec_var - 1.0)) <= 0.06
    assert np.max(np.abs(m.sigma_f - ret.sigma_f)) <= 0.05 * np.max(np.abs(ret.sigma_f))
