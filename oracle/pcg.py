"""Algorithm 1: the sketched preconditioner and the inner solvers (oracle).

Test infrastructure only (see the package docstring).

Notation follows Section 3: M = A D^2 A^T (eq. normal), the preconditioner
Q = A D W W^T D A^T (eq. pdprecond), and the symmetric preconditioned system
of eq. (precond_alt):

    B z = Q^{-1/2} p,   B = Q^{-1/2} A D^2 A^T Q^{-1/2},   dy = Q^{-1/2} z.

The residual of iterate z^j is f^(j) = B z^j - Q^{-1/2} p (Section 3.1).
"""

from __future__ import annotations

import dataclasses
from typing import Callable, List, Optional

import numpy as np


@dataclasses.dataclass
class Preconditioner:
    U: np.ndarray        # U_Q, left singular vectors of A D W  (m x m)
    sv: np.ndarray       # Sigma_Q^{1/2}: singular values of A D W
    Vt: np.ndarray       # right singular vectors (m x w), for (ADW)^+
    Q_mhalf: np.ndarray  # Q^{-1/2} = U_Q Sigma_Q^{-1/2} U_Q^T

    @property
    def Q_inv(self) -> np.ndarray:
        return self.Q_mhalf @ self.Q_mhalf


def preconditioner(ADW: np.ndarray) -> Preconditioner:
    """Algorithm 1, steps 1-2: thin SVD of A D W and Q^{-1/2}.

    Step 1 takes U_Q (left singular vectors) and Sigma_Q^{1/2} (singular
    values) of ADW; step 2 forms Q^{-1/2} = U_Q Sigma_Q^{-1/2} U_Q^T, i.e.
    U_Q diag(1/singular value) U_Q^T (eq. pdprecond and the text below it).
    """
    U, sv, Vt = np.linalg.svd(ADW, full_matrices=False)
    Q_mhalf = (U / sv) @ U.T
    return Preconditioner(U=U, sv=sv, Vt=Vt, Q_mhalf=Q_mhalf)


@dataclasses.dataclass
class SolveTrace:
    z: np.ndarray
    res_norms: List[float]        # ||f^(j)||_2 for j = 0..t
    iterations: int


def cg(Bmv: Callable[[np.ndarray], np.ndarray], rhs: np.ndarray, t_max: int,
       tol: float = 0.0, z0: Optional[np.ndarray] = None) -> SolveTrace:
    """Standard conjugate gradient on B z = rhs (Algorithm 1, step 3).

    Starts from z^0 = 0 (or ``z0``) and stops after t_max iterations or when
    ||f^(j)|| = ||B z^j - rhs|| <= tol.  The residual is the recursively
    updated CG residual (Hestenes-Stiefel form).
    """
    z = np.zeros_like(rhs) if z0 is None else z0.copy()
    r = rhs - Bmv(z)                   # r = -f
    d = r.copy()
    rr = r @ r
    norms = [np.sqrt(rr)]
    j = 0
    while j < t_max and norms[-1] > tol:
        Bd = Bmv(d)
        a = rr / (d @ Bd)
        z = z + a * d
        r = r - a * Bd
        rr_new = r @ r
        d = r + (rr_new / rr) * d
        rr = rr_new
        j += 1
        norms.append(np.sqrt(rr))
    return SolveTrace(z=z, res_norms=norms, iterations=j)


def chebyshev(Bmv: Callable[[np.ndarray], np.ndarray], rhs: np.ndarray,
              lam_min: float, lam_max: float, t_max: int, tol: float = 0.0,
              true_residual_every: int = 0) -> SolveTrace:
    """Chebyshev iteration on B z = rhs for spec(B) in [lam_min, lam_max].

    Section 3.2 uses Chebyshev iteration in place of CG; it needs only the
    spectral interval, no inner products.  This is the classical three-term
    form: with theta = (lam_max+lam_min)/2, delta = (lam_max-lam_min)/2 and
    s1 = theta/delta, the residual after j steps is
        r^j = T_j((theta - B)/delta) r^0 / T_j(s1),
    computed by  rho_0 = 1/s1, d^0 = r^0/theta,
                 z^{j+1} = z^j + d^j,  r^{j+1} = r^j - B d^j,
                 rho_{j+1} = 1/(2 s1 - rho_j),
                 d^{j+1} = rho_{j+1} rho_j d^j + (2 rho_{j+1}/delta) r^{j+1}.
    The residual norm is only *observed* for stopping (every step here).
    """
    theta = 0.5 * (lam_max + lam_min)
    delta = 0.5 * (lam_max - lam_min)
    s1 = theta / delta
    z = np.zeros_like(rhs)
    r = rhs.copy()
    rho = 1.0 / s1
    d = r / theta
    norms = [np.linalg.norm(r)]
    j = 0
    while j < t_max and norms[-1] > tol:
        z = z + d
        r = r - Bmv(d)
        rho_new = 1.0 / (2.0 * s1 - rho)
        d = rho_new * rho * d + (2.0 * rho_new / delta) * r
        rho = rho_new
        j += 1
        norms.append(np.linalg.norm(r))
    return SolveTrace(z=z, res_norms=norms, iterations=j)


def chebyshev_bound(U: float, t: int) -> float:
    """Right side of eq. (cs): 2 / (((sqrt U+1)/(sqrt U-1))^t + ((sqrt U-1)/(sqrt U+1))^t)."""
    q = (np.sqrt(U) + 1.0) / (np.sqrt(U) - 1.0)
    return 2.0 / (q ** t + q ** (-t))


def cg_contraction(zeta: float) -> float:
    """Per-step residual contraction of eq. (rec): zeta / (2 - zeta)."""
    return zeta / (2.0 - zeta)


def theory_inner_tol(mu: float, n: int, gamma: float, sigma: float) -> float:
    """||f^(t)|| target that makes Lemma 4.2's bound give ||v|| <= gamma sigma mu / 4.

    Lemma 4.2: ||v|| <= sqrt(3 n mu) ||f^(t)||; Lemma 4.4 needs
    ||v|| <= gamma sigma mu / 4, hence ||f^(t)|| <= gamma sigma sqrt(mu) / (4 sqrt(3 n)).
    """
    return gamma * sigma * np.sqrt(mu) / (4.0 * np.sqrt(3.0 * n))


def inner_iteration_count(n: int, gamma: float, sigma: float, zeta: float = 0.5) -> int:
    """Lemma 4.4: t >= log(n psi) / log(1/zeta), psi = 4 sqrt6 (1 + sigma/sqrt(1-gamma)) / (gamma sigma)."""
    psi = 4.0 * np.sqrt(6.0) * (1.0 + sigma / np.sqrt(1.0 - gamma)) / (gamma * sigma)
    return int(np.ceil(np.log(n * psi) / np.log(1.0 / zeta)))
