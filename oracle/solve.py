"""Oracle entry point: interior point, then active-set polish, then certificate.

ORACLE: test infrastructure only; shares no code with the CUDA solver.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import active, ipm
from .kkt import KKT, evaluate
from .model import Scaled


@dataclass
class OracleSolution:
    x: np.ndarray        # (P, n) minimiser
    yA: np.ndarray       # (P, m)
    yD: np.ndarray       # (R, n)
    obj: float           # scaled minimisation objective
    paper_obj: float     # Eq. 1 / Eq. 4 value in paper units
    kkt: KKT             # relative KKT residuals of (x, yA, yD)
    polished: bool
    ipm_iters: int
    reduced: object = None

    @property
    def w(self):
        return self.x[0] if self.x.shape[0] == 1 else self.x


def solve(prob, polish: bool = True, polish_max_vars: int = 120000,
          polish_seconds: float = 60.0) -> OracleSolution:
    """FP64 minimiser of the scaled model of ``prob`` (single or multi-period).
    The active-set polish gets ``polish_seconds`` of wall clock; when it does
    not certify a point in that time the interior-point point is returned
    (``polished`` False), with its own KKT evaluation."""
    sc = Scaled(prob)
    sol = ipm.solve(prob)
    if polish and sc.P * sc.n <= polish_max_vars:
        ref = active.refine(prob, sol, seconds=polish_seconds)
        if ref is not None:
            x, yA, yD, res, red = ref
            return OracleSolution(x, yA, yD, sc.objective(x), sc.paper_objective(x), res, True,
                                  sol.iters, red)
    res = evaluate(sc, sol.x, sol.yA, sol.yD)
    return OracleSolution(sol.x, sol.yA, sol.yD, sol.obj, sol.paper_obj, res, False, sol.iters)
