"""Phase-1 LP for a primal feasible start (test infrastructure; see package
docstring).

Appendix "Feasible starting point": with every b_i >= 0 (rows with b_i < 0
are negated, which changes neither the feasible set nor x), (x, z) = (x, 0)
solves
    min 1^T z   s.t.   A x + I z = b,   x, z >= 0
exactly when A x = b, x >= 0 is feasible (the printed objective "min z" is
read as 1^T z).  The phase-1 LP always has the feasible point (0, b), so the
IPM applies to it from the usual infeasible start.  Its interior solution has
x > 0 and a small z; the start is made exactly primal feasible by the
minimum-norm correction x0 = x + A^T (A A^T)^{-1} (b - A x).
"""

from __future__ import annotations

import dataclasses

import numpy as np

from . import ipm


@dataclasses.dataclass
class Phase1:
    feasible: bool
    x0: np.ndarray        # primal start (valid when feasible)
    z_sum: float          # 1^T z at the phase-1 solution
    iterations: int


def phase1_lp(A: np.ndarray, b: np.ndarray):
    """The phase-1 data (A1, b1, c1) after making b nonnegative."""
    m, n = A.shape
    sign = np.where(b < 0, -1.0, 1.0)
    A1 = np.hstack([A * sign[:, None], np.eye(m)])
    b1 = b * sign
    c1 = np.concatenate([np.zeros(n), np.ones(m)])
    return A1, b1, c1


def phase1_start(A: np.ndarray, b: np.ndarray, tol: float = 1e-9,
                 feas_tol: float = 1e-6) -> Phase1:
    m, n = A.shape
    A1, b1, c1 = phase1_lp(A, b)
    res = ipm.solve(A1, b1, c1, ipm.Options(solver="exact", mode="infeasible", tol=tol))
    x, z = res.x[:n], res.x[n:]
    z_sum = float(z.sum())
    feasible = z_sum <= feas_tol * (1.0 + np.linalg.norm(b))
    r = b - A @ x
    x0 = x + A.T @ np.linalg.solve(A @ A.T, r)
    return Phase1(feasible=bool(feasible and (x0 > 0).all()), x0=x0, z_sum=z_sum,
                  iterations=res.iterations)
