"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module only *builds problems*: planted linear programs whose optimum is
known in closed form, storage rounding of the constraint matrix, and a
strictly feasible start for planted problems.  It contains none of the
interior-point method's arithmetic (no normal equations, no sketch, no
step lengths), so that the CPU oracle and the CUDA path can both consume it
without sharing any of the method.

Problem form (the paper's primal, Section 1, eq. primal):
    min c^T x  s.t.  A x = b,  x >= 0,
with dual  max b^T y  s.t.  A^T y + s = c,  s >= 0  (eq. dual).

A planted instance draws (x*, y*, s*) with x* o s* = 0 and sets b = A x*,
c = A^T y* + s*, so (x*, y*, s*) is primal-dual optimal by construction.
When A is stored in a reduced precision, b and c are formed in FP64 from the
*rounded* A, so the planted optimum stays exact for the stored problem.
"""

from .planted import (  # noqa: F401
    PlantedLP,
    planted_dense,
    planted_dense_blocked,
    make,
    planted_sparse,
    round_bf16,
    bf16_bits,
    feasible_start,
    config_small,
    CONFIGS,
    batch_family,
)
from .random_lp import RandomLP, random_lp  # noqa: F401
