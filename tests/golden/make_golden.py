"""Write tests/golden/oracle_tiny.json: the oracle's solution of two tiny
seeded instances (one single-period, one multi-period).

The paper prints no worked example (its only table reports solve times), so
no stored value here comes from the paper.  This fixture is a regression
record written by the oracle alone (the oracle's correctness rests on the
pins in tests/test_oracle_*.py); the CUDA path is compared with it in
tests/test_golden.py.  Run from the repository root:

    python tests/golden/make_golden.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2604_22625_gb300 import synthetic as S  # noqa: E402

CASES = {
    "single_n12_k3": dict(kind="single", n=12, k=3, seed=77, n_onehot=1),
    "multi_T3_n8_k2": dict(kind="multi", T=3, n=8, k=2, seed=78, n_onehot=1),
}


def make(spec):
    if spec["kind"] == "single":
        return S.make_single(spec["n"], spec["k"], spec["seed"], n_onehot=spec["n_onehot"])
    return S.make_multi(spec["T"], spec["n"], spec["k"], spec["seed"], n_onehot=spec["n_onehot"])


def main():
    out = {}
    for name, spec in CASES.items():
        sol = oracle.solve(make(spec))
        out[name] = {"spec": spec, "x": sol.x.tolist(), "obj": sol.obj, "paper_obj": sol.paper_obj,
                     "rel_kkt": sol.kkt.rel_kkt}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_tiny.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(path)


if __name__ == "__main__":
    main()
