"""FP64 CPU oracle of the Zeus method (PSO -> many BFGS runs -> argmin).

TEST INFRASTRUCTURE ONLY.  This package is the independent reference the
CUDA path is checked against.  Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it; the library under
``paper_2603_28770_gb300`` never does.  It shares no code with the CUDA
library: the arithmetic lives in ``zeus_oracle.c`` (plain C, FP64, compiled
without FMA contraction), this module only marshals numpy arrays.

Every function cites the part of the paper (Zeus, arXiv 2603.28770) it
follows.  Parity pins live in ``tests/test_oracle_*.py``.
"""
from .oracle import (  # noqa: F401
    OBJECTIVES, Problem, build, lib, philox4x64_10, uniform, f, grad_forward,
    dual_op, sincos2pi, exp, argmin, pso, line_search, bfgs_update, bfgs, bfgs_many, solve,
    bfgs_quadratic_exact, max_threads, lbfgs_direction, cluster, CLUSTER_METHODS, dot_split,
    dot_plain, direction, ORDER_LIB, ORDER_PLAIN,
)
