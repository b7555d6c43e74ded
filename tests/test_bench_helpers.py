"""Host logic of bench.py: the stratified samples shared by the oracle check,
the plain per-instance form and both CPU baselines, and the oracle check of a
GPU output (run here on the oracle's own solution and on a perturbed copy)."""
import numpy as np

import bench
import oracle
from paper_2604_22625_gb300 import synthetic as S


def _batch():
    return S.config_batch(n_single=40, n_multi=12)


def test_strata_pick_centres_of_equal_count_strata():
    probs = _batch()
    for kind, cnt in (("single", 4), ("multi", 4), ("multi", 30)):
        pick = bench.strata(probs, kind, cnt)
        assert len(pick) == min(cnt, 40 if kind == "single" else 12)
        assert len(set(pick)) == len(pick)
        assert all((int(probs[i].T) >= 2) == (kind == "multi") for i in pick)
        assert pick == bench.strata(probs, kind, cnt)          # deterministic
    size = lambda i: probs[i].F.shape[0] * max(1, int(probs[i].T) - 1) * (probs[i].F.shape[1] + probs[i].A.shape[0])  # noqa: E731
    pick = bench.strata(probs, "single", 4)
    assert [size(i) for i in pick] == sorted(size(i) for i in pick)


def test_extremes_include_both_ends():
    probs = _batch()
    pick = bench.extremes(probs, "multi", 3)
    multis = [i for i, p in enumerate(probs) if int(p.T) >= 2]
    size = lambda i: (probs[i].F.shape[0] * (int(probs[i].T) - 1), i)  # noqa: E731
    assert pick[0] == min(multis, key=size) and pick[-1] == max(multis, key=size)
    assert len(pick) == 3


def test_cpu_rate_weights_the_strata():
    probs = _batch()
    r = bench.cpu_rate(probs, [1.0, 3.0], [10.0])
    assert abs(r - len(probs) / (40 * 2.0 + 12 * 10.0)) < 1e-12


def test_oracle_check_of_a_point():
    prob = S.make_single(80, 6, 5, n_onehot=2)
    ref = oracle.solve(prob)
    row = bench._oracle_check_one(("t", prob, "f64", ref.x, ref.yA, ref.yD))
    assert row["err_inf"] == 0.0 and row["obj_gap"] == 0.0 and row["oracle_certified"]
    assert row["rel_kkt"] <= 1e-10
    bad = ref.x + 2e-5
    row2 = bench._oracle_check_one(("t", prob, "f64", bad, ref.yA, ref.yD))
    assert abs(row2["err_inf"] - 2e-5) < 1e-12
    summ = bench.summarize_check([row, row2])
    assert summ["n"] == 2 and not summ["within_bars"] and summ["max_err_inf"] == row2["err_inf"]
