"""The correction vector v (oracle; test infrastructure only).

Section 4, eq. (compv):
    v = (X S)^{1/2} W (A D W)^+ (A D^2 A^T dy_hat - p),
which satisfies the invariant of eq. (addl), A S^{-1} v = A D^2 A^T dy_hat - p,
whenever A D W has full row rank (Lemma 4.1), and has
||v|| <= sqrt(3 n mu) ||f^(t)|| (Lemma 4.2).

The exact minimum-norm alternative v = (A S^{-1})^+ (A D^2 A^T dy_hat - p)
(Section 4, "Construction of v") is provided for small cross-checks only.
"""

from __future__ import annotations

import numpy as np


def correction_v(x: np.ndarray, s: np.ndarray, W, ADW: np.ndarray,
                 r_v: np.ndarray) -> np.ndarray:
    """eq. (compv); ``W`` dense or scipy.sparse (n x w), ``r_v`` = M dy_hat - p."""
    g = np.linalg.pinv(ADW) @ r_v          # (ADW)^+ r_v, a w-vector
    Wg = W @ g
    return np.sqrt(x * s) * np.asarray(Wg).reshape(-1)


def correction_v_minnorm(A: np.ndarray, s: np.ndarray, r_v: np.ndarray) -> np.ndarray:
    """v = (A S^{-1})^+ r_v (the O(m^2 n) choice the paper rejects)."""
    return np.linalg.pinv(A / s) @ r_v
