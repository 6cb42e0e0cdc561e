"""Brute-force vertex enumeration for tiny standard-form LPs (oracle).

Test infrastructure only.  For min c^T x s.t. A x = b, x >= 0 with A of full
row rank m, an optimum (if one exists) is attained at a basic feasible
solution: a set B of m columns with A_B nonsingular and x_B = A_B^{-1} b >= 0,
x_N = 0.  Enumerating all C(n, m) bases therefore finds the optimal value of
the primal of eq. (primal) exactly (up to the linear solves' rounding).
"""

from __future__ import annotations

import itertools

import numpy as np


def enumerate_vertices(A: np.ndarray, b: np.ndarray, c: np.ndarray,
                       feas_tol: float = 1e-10):
    """Returns (best objective, best x, number of feasible bases)."""
    m, n = A.shape
    best = np.inf
    best_x = None
    count = 0
    for B in itertools.combinations(range(n), m):
        AB = A[:, B]
        if abs(np.linalg.det(AB)) < 1e-12:
            continue
        xB = np.linalg.solve(AB, b)
        if (xB < -feas_tol).any():
            continue
        count += 1
        x = np.zeros(n)
        x[list(B)] = xB
        obj = c @ x
        if obj < best:
            best, best_x = obj, x
    return best, best_x, count
