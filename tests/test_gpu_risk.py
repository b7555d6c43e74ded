"""GPU risk-model estimation (ff_risk_estimate, Sec. 3.2) against the FP64
oracle (oracle/risk.py) on the same float32 returns, element by element.

Tolerances from the arithmetic: the factor covariance and the Gram matrices
are sums of exact products of FP32 inputs (FP64 for Sigma_f, 1e-12 relative;
double-float pairs of about 48 bits for the Gram tables); b = F^T r, sum r
and sum r^2 are FP32 sums over chunks of 16 days folded into double-float
accumulators, so each carries at most 16 u32 = 9.5e-7 of the sum of its
terms' magnitudes: beta to 1e-5 absolute (loadings are O(1)) and D to 1e-5
relative.  History counts and the estimated / not-estimated decision are
exact."""
import numpy as np
import pytest

from oracle import risk
from paper_2604_22625_gb300 import synthetic as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2604_22625_gb300 import api as _api
    from paper_2604_22625_gb300.build import build
    build()
    return _api


def _compare(api, windows, min_obs=42):
    F = np.stack([w.F for w in windows])
    R = np.stack([w.R for w in windows])
    out = api.estimate_risk(F, R, min_obs=min_obs)
    beta = out.beta.cpu().numpy()
    sig = out.sigma_f.cpu().numpy()
    D = out.D.cpu().numpy()
    nobs = out.nobs.cpu().numpy()
    for d, w in enumerate(windows):
        ref = risk.estimate(w.F, w.R, min_obs=min_obs)
        assert np.allclose(sig[d], ref.sigma_f, rtol=1e-12, atol=0)
        hist = [risk.history(w.R[:, i]) for i in range(w.R.shape[1])]
        exp_nobs = np.array([c if reg else -1 for _, c, reg in hist])
        assert np.array_equal(nobs[d], exp_nobs)
        ok = ref.valid
        assert np.array_equal(~np.isnan(D[d]), ok)
        assert np.max(np.abs(beta[d][ok] - ref.beta[ok]), initial=0.0) <= 1e-5
        assert np.all(beta[d][~ok] == 0.0)
        if ok.any():
            assert np.max(np.abs(D[d][ok] / ref.D[ok] - 1.0)) <= 1e-5


def test_windows_with_listings_and_gaps(api):
    _compare(api, [S.make_returns(504, 3000, 10 + s, late_frac=0.2, irregular_frac=0.02) for s in range(3)])


@pytest.mark.parametrize("n", [1, 255, 257, 1000])
def test_ragged_stock_counts(api, n):
    _compare(api, [S.make_returns(504, n, 20 + n, late_frac=0.3)])


@pytest.mark.parametrize("p,T", [(1, 60), (3, 131), (8, 504)])
def test_factor_counts_and_window_lengths(api, p, T):
    _compare(api, [S.make_returns(T, 700, 30 + p, p=p, late_frac=0.2)], min_obs=min(42, T // 2))
