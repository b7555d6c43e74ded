"""Regression against tests/golden/oracle_tiny.json (written by
tests/golden/make_golden.py from the oracle only)."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2604_22625_gb300 import synthetic as S

HERE = os.path.dirname(os.path.abspath(__file__))
with open(os.path.join(HERE, "golden", "oracle_tiny.json")) as f:
    GOLDEN = json.load(f)


def _make(spec):
    if spec["kind"] == "single":
        return S.make_single(spec["n"], spec["k"], spec["seed"], n_onehot=spec["n_onehot"])
    return S.make_multi(spec["T"], spec["n"], spec["k"], spec["seed"], n_onehot=spec["n_onehot"])


@pytest.mark.parametrize("name", sorted(GOLDEN))
def test_oracle_reproduces_record(name):
    rec = GOLDEN[name]
    sol = oracle.solve(_make(rec["spec"]))
    assert np.max(np.abs(sol.x - np.array(rec["x"]))) <= 1e-10
    assert abs(sol.obj - rec["obj"]) <= 1e-12 * max(1.0, abs(rec["obj"]))


@pytest.mark.gpu
@pytest.mark.parametrize("name", sorted(GOLDEN))
def test_cuda_matches_record(name):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2604_22625_gb300 import api
    from paper_2604_22625_gb300.build import build
    build()
    rec = GOLDEN[name]
    sol = api.solve(_make(rec["spec"]), precision="f64", tol=2e-7)
    assert sol.info["status_name"] == "converged"
    assert np.max(np.abs(sol.x - np.array(rec["x"]))) <= 1e-5
