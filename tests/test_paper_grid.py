"""The paper-shaped instances of the lambda grid (Sec. 4.1 with the data
recipe of Sec. 3) and the SGM1 statistic, on the CPU."""
import numpy as np

import bench
from paper_2604_22625_gb300 import synthetic as S


def test_eta_profile_hand_values():
    # T = 10: eta_t = 0.5 + 2 (t/10 - 0.5)^2 = 0.82, 0.68, 0.58, 0.52, 0.50, 0.52, 0.58, 0.68, 0.82, 1.00;
    # the first nine sum to 5.70
    e = S.eta_profile(10)
    raw = np.array([0.82, 0.68, 0.58, 0.52, 0.50, 0.52, 0.58, 0.68, 0.82, 1.00])
    assert np.allclose(e, raw / 5.70, rtol=1e-14, atol=0)
    inv = S.eta_profile(10, "inverted")
    assert np.allclose(inv, (1 / raw) / np.sum(1 / raw[:9]), rtol=1e-14, atol=0)
    assert inv[4] > inv[0]       # inverted: costs smallest at the ends (most liquid), largest mid-horizon


def test_instances_follow_the_recipe():
    single = S.make_paper_instance(3, 1e-6, 100.0, "single", n=300)
    multi = S.make_paper_instance(3, 1e-6, 100.0, "multi", n=300)
    assert single.F.shape == (300, 6) and single.A.shape == (6, 300)
    assert np.all(np.linalg.eigvalsh(single.Omega) > 0) and np.count_nonzero(single.Omega - np.diag(np.diag(single.Omega)))
    assert single.lam2 == single.lam3 == 100.0 and single.lam1 == 1e-6
    assert multi.T == 10 and np.all(multi.alpha == multi.alpha[0]) and np.all(multi.D == single.D)
    eta = S.eta_profile(10)
    assert np.allclose(multi.s, eta[:, None] * single.s[None, :]) and np.allclose(multi.q, eta[:, None] * single.q[None, :])
    b = S.make_paper_date(3, 300)
    assert np.allclose(single.q, b["sig_tot"] * np.sqrt(single.GMV / b["adv"]))      # d = 1.5
    assert abs(np.abs(single.w0).sum() - 0.9) < 1e-12 and abs(np.abs(multi.wT).sum() - 0.9) < 1e-12


def test_sgm1():
    assert abs(bench.sgm1([0.0, 3.0]) - 1.0) < 1e-15          # sqrt(1 * 4) - 1
    assert abs(bench.sgm1([1.0, 1.0, 1.0]) - 1.0) < 1e-15
