"""Plain CPU FP64 oracle for robust value iteration on IMDPs (arXiv 2401.04068).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers.  The CUDA library never
imports this package and shares no code with it.

``imdp_oracle.c`` holds the arithmetic (value iteration, Eq. 2; O-maximization,
Sec. 4, sequential procedure).  This module compiles it with gcc and wraps it
with ctypes.  The exact-rational checker that pins it lives with the tests
(``tests/exact_lp.py``).
"""
from .oracle import (  # noqa: F401
    OracleIMDP,
    OracleSpec,
    build_oracle,
    omax_column,
    validate,
    value_iteration,
    has_openmp,
    REACH,
    REACH_AVOID,
    REWARD,
    STATUS,
)
