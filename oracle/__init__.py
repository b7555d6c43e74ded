"""FP64 CPU oracle for the portfolio models (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. It shares no code with the CUDA solver
and never calls it.
"""
from .model import Scaled  # noqa: F401
from . import ipm, kkt, prox  # noqa: F401
from . import active  # noqa: F401
from .solve import OracleSolution, solve  # noqa: F401
