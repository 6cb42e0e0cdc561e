"""Algorithms 2 (feasible) and 3 (infeasible) IPM, CPU oracle in FP64.

Test infrastructure only (see the package docstring).

Two normal-equation modes:
  * ``solver="exact"``: A D^2 A^T dy = p solved by Cholesky, v = 0 -- the
    "standard analysis" case of Section 4.1; this is the oracle of record for
    the LP optimum.
  * ``solver="sketch"``: the paper's method -- sketch W (step 2), Algorithm 1
    (SVD of ADW, Q^{-1/2}, CG or Chebyshev on eq. precond_alt), the
    correction v of eq. (compv), then the directions of eqs. (delxhat),
    (delshat) / (delxhat_i), (delshat_i).

Readings of points the paper leaves open:
  * alpha_max (Alg. 2 step 5, Alg. 3 step 6) is the first exit from N(gamma)
    along the direction: the largest alpha in [0,1] with the whole segment
    [0, alpha] inside N(gamma); positivity of (x, s) is enforced explicitly.
  * alpha_bar minimises the quadratic gap (x+a dx)^T (s+a ds) on [0, alpha_max]
    in closed form; ties go to the largest step.
  * stopping: relative gap |c^T x - b^T y|/(1+|c^T x|), ||r_p||/(1+||b||),
    ||r_d||/(1+||c||) all <= tol, or k_max iterations.
  * inner stopping: ||f^(t)|| <= gamma sigma sqrt(mu)/(4 sqrt(3n))
    (the level at which Lemma 4.2 gives Lemma 4.4's ||v|| <= gamma sigma mu/4),
    or the relative rule ||f^(t)|| <= tol_cg ||f^(0)|| used in Section 7.
"""

from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sps

from . import correction, pcg, sketch


@dataclasses.dataclass
class Options:
    sigma: float = 0.5          # centering parameter, sigma in (0, 4/5)
    gamma: float = 0.999        # neighbourhood width, gamma in (0, 1)
    tol: float = 1e-8
    k_max: int = 200
    mode: str = "infeasible"    # "feasible" (Alg. 2) or "infeasible" (Alg. 3)
    solver: str = "exact"       # "exact" (Cholesky, v = 0), "sketch", or "cg" (unpreconditioned)
    sketch: str = "countsketch"  # or "gaussian"
    w: Optional[int] = None     # sketch width (default 4m)
    s: int = 2                  # nonzeros per row of a CountSketch
    seed: int = 0
    inner: str = "cg"           # "cg" or "chebyshev"
    inner_rule: str = "theory"  # "theory" or "relative"
    tol_cg: float = 1e-5
    t_max: int = 500
    v_correction: bool = True
    cheb_lanczos: int = 10      # CG steps used to estimate the Chebyshev interval
    keep_vectors: bool = False
    sigma_rule: str = "fixed"   # "fixed" (the paper) or "adaptive" (two right-hand sides)
    sigma_range: tuple = (0.1, 0.75)


@dataclasses.dataclass
class IterRecord:
    k: int
    mu: float
    gap: float
    rp_norm: float
    rd_norm: float
    inner_its: int = 0
    f_norm: float = 0.0
    f0_norm: float = 0.0
    v_norm: float = 0.0
    alpha_max: float = 0.0
    alpha_bar: float = 0.0
    vectors: Optional[dict] = None
    sigma_used: float = 0.0



@dataclasses.dataclass
class Result:
    x: np.ndarray
    y: np.ndarray
    s: np.ndarray
    status: str
    iterations: int
    history: List[IterRecord]


# ---------------------------------------------------------------------------
# building blocks
# ---------------------------------------------------------------------------

def residuals(A, b, c, x, y, s):
    """eq. (primalres), (dualres): r_p = A x - b (m), r_d = A^T y + s - c (n)."""
    return A @ x - b, A.T @ y + s - c


def rhs(A, x, s, r_p, r_d, sigma, mu, feasible: bool):
    """Right-hand side p of the normal equations.

    feasible  (eq. pdef):  p = -sigma mu A S^{-1} 1 + A x
    infeasible (Sec. 5):   p = -r_p - sigma mu A S^{-1} 1 + A x - A D^2 r_d
    """
    p = -sigma * mu * (A @ (1.0 / s)) + A @ x
    if not feasible:
        d2 = x / s
        p = p - r_p - A @ (d2 * r_d)
    return p


def normal_matrix(A, d2):
    """M = A D^2 A^T (eq. normal), formed densely (oracle only).  A sparse A
    (scipy.sparse) gives the same matrix through a sparse product."""
    if sps.issparse(A):
        return (A @ sps.diags(d2) @ A.T).toarray()
    return (A * d2) @ A.T


def directions(A, x, s, r_d, dy, v, sigma, mu, feasible: bool):
    """Directions given dy_hat and v.

    ds_hat = -A^T dy_hat            (eq. delshat, feasible)
    ds_hat = -r_d - A^T dy_hat      (eq. delshat_i, infeasible)
    dx_hat = -x + sigma mu S^{-1} 1 - D^2 ds_hat - S^{-1} v   (eq. delxhat)
    """
    ds = -(A.T @ dy)
    if not feasible:
        ds = ds - r_d
    dx = -x + sigma * mu / s - (x / s) * ds - v / s
    return dx, ds


def _first_exit(a, b, c):
    """Per element, the first alpha > 0 where g = a t^2 + b t + c crosses
    from >= 0 to < 0 (a downward crossing); +inf where there is none.

    A root at or below 0 is not an exit: the element is then either inside
    its feasible interval already or (c slightly < 0 from rounding) moving
    back into it.  Elements whose g is negative on all of (0, inf) exit at 0.
    """
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    c = np.asarray(c, float)
    out = np.full(a.shape, np.inf)
    lin = a == 0.0
    # linear: b t + c, decreasing when b < 0, crossing zero at -c/b
    lb = lin & (b < 0)
    out[lb] = np.maximum(-c[lb] / b[lb], 0.0)
    q = ~lin
    disc = b * b - 4.0 * a * c
    neg_disc = q & (disc < 0)
    out[neg_disc & (a < 0)] = 0.0          # g < 0 everywhere
    real = q & (disc >= 0)
    sq = np.sqrt(np.where(real, disc, 0.0))
    # stable roots (Numerical Recipes, quadratic equations)
    qq = -0.5 * (b + np.where(b >= 0, sq, -sq))
    with np.errstate(divide="ignore", invalid="ignore"):
        r1 = np.where(qq != 0, qq / np.where(a != 0, a, 1.0), 0.0)
        r2 = np.where(qq != 0, c / np.where(qq != 0, qq, 1.0), 0.0)
    lo = np.minimum(r1, r2)
    hi = np.maximum(r1, r2)
    up = real & (a > 0)         # negative between the roots: exit at lo
    sel = up & (lo > 0)
    out[sel] = lo[sel]
    dn = real & (a < 0)         # negative outside the roots: exit at hi
    sel = dn & (hi > 0)
    out[sel] = hi[sel]
    sel = dn & (hi <= 0)
    out[sel] = 0.0
    return out


def step_lengths(x, s, dx, ds, gamma, feasible: bool, res_ratio: float = 0.0,
                 mu0: float = 1.0):
    """alpha_max and alpha_bar of Alg. 2 steps 5-6 / Alg. 3 steps 6-7.

    N(gamma) (eq. neigh): x_i s_i >= (1-gamma) mu, (x, s) > 0; infeasible
    adds ||r||/||r^0|| <= mu/mu_0 (Section 5) where, with v satisfying the
    invariant, r(alpha) = (1-alpha) r (Appendix A.2, eqs. iip_3_1, iip_3_2),
    so ||r(alpha)||/||r^0|| = (1-alpha) res_ratio.

    mu(alpha) = mu + alpha c1 + alpha^2 c2 with c1 = (x^T ds + s^T dx)/n,
    c2 = dx^T ds / n, so every condition is a quadratic in alpha.
    """
    n = x.size
    mu = x @ s / n
    c1 = (x @ ds + s @ dx) / n
    c2 = (dx @ ds) / n
    g = 1.0 - gamma
    # x_i(a) s_i(a) - (1-gamma) mu(a) >= 0
    exits = _first_exit(dx * ds - g * c2, x * ds + s * dx - g * c1, x * s - g * mu)
    alpha = min(1.0, float(np.min(exits)))
    # mu(alpha) > 0
    alpha = min(alpha, float(_first_exit(np.array([c2]), np.array([c1]), np.array([mu]))[0]))
    if not feasible:
        # mu(a)/mu0 - (1-a) res_ratio >= 0
        e = _first_exit(np.array([c2 / mu0]), np.array([c1 / mu0 + res_ratio]),
                        np.array([mu / mu0 - res_ratio]))[0]
        alpha = min(alpha, float(e))
    # strict positivity of x and s
    with np.errstate(divide="ignore"):
        px = np.where(dx < 0, -x / dx, np.inf)
        ps = np.where(ds < 0, -s / ds, np.inf)
    apos = float(min(np.min(px), np.min(ps)))
    if apos <= alpha:
        alpha = apos * (1.0 - 1e-12)
    alpha_max = max(alpha, 0.0)
    # alpha_bar = argmin over [0, alpha_max] of n mu(alpha)
    if c2 > 0:
        alpha_bar = min(max(-c1 / (2.0 * c2), 0.0), alpha_max)
    else:
        alpha_bar = alpha_max
    return alpha_max, alpha_bar


def in_neighbourhood(x, s, gamma, feasible=True, res_ratio=0.0, mu0=1.0,
                     rel_slack=0.0) -> bool:
    """Membership test of N(gamma) on (x, s) (eq. neigh / Section 5)."""
    n = x.size
    mu = x @ s / n
    if not ((x > 0).all() and (s > 0).all()):
        return False
    if np.min(x * s) < (1.0 - gamma) * mu * (1.0 - rel_slack):
        return False
    if not feasible and res_ratio > (mu / mu0) * (1.0 + rel_slack):
        return False
    return True


def sketch_matrix(opt: Options, n: int, w: int, k: int, retry: int):
    if opt.sketch == "countsketch":
        return sketch.countsketch_matrix(opt.seed, k, retry, n, w, opt.s)
    return sketch.gaussian_matrix(opt.seed, k, retry, n, w)


@dataclasses.dataclass
class NormalSolve:
    dy: np.ndarray
    v: np.ndarray
    z: np.ndarray
    trace: pcg.SolveTrace
    f_norm: float             # ||f^(t)|| = ||Q^{-1/2}(M dy - p)||
    f0_norm: float            # ||Q^{-1/2} p||
    precond: pcg.Preconditioner
    ADW: np.ndarray
    retry: int
    lam: tuple = (0.0, 0.0)


def lanczos_interval(alphas, betas):
    """Extreme Ritz values from CG coefficients (the Lanczos tridiagonal)."""
    k = len(alphas)
    T = np.zeros((k, k))
    for j in range(k):
        T[j, j] = 1.0 / alphas[j] + (betas[j - 1] / alphas[j - 1] if j > 0 else 0.0)
        if j + 1 < k:
            T[j, j + 1] = T[j + 1, j] = np.sqrt(betas[j]) / alphas[j]
    ev = np.linalg.eigvalsh(T)
    return ev[0], ev[-1]


def normal_solve(A, x, s, p, opt: Options, k: int, inner_tol: float,
                 W=None, retry_start: int = 0) -> NormalSolve:
    """Algorithm 1 plus eq. (compv) for one outer iteration.

    D = X^{1/2} S^{-1/2} (eq. normal).  A sketch whose ADW is numerically
    rank deficient (probability delta, Lemma 4.1) is redrawn.
    """
    m, n = A.shape
    w = opt.w or 4 * m
    d = np.sqrt(x / s)
    d2 = x / s
    AD = A * d
    for retry in range(retry_start, sketch.MAX_RETRY):
        Wk = W if W is not None else sketch_matrix(opt, n, w, k, retry)
        ADW = np.asarray(AD @ Wk) if not hasattr(Wk, "tocsc") else np.asarray((Wk.T @ AD.T).T)
        # Lemma 4.1 needs rank(ADW) = m: m singular values, none negligible
        pre = pcg.preconditioner(ADW) if ADW.shape[1] >= m else None
        if pre is not None and pre.sv[-1] > 1e-13 * pre.sv[0]:
            break
        if W is not None:
            raise np.linalg.LinAlgError("sketch rank deficient")
    else:
        raise np.linalg.LinAlgError("sketch rank deficient after retries")
    Qmh = pre.Q_mhalf

    def Bmv(z):
        u = Qmh @ z
        return Qmh @ (A @ (d2 * (A.T @ u)))

    rhs_ = Qmh @ p
    f0 = float(np.linalg.norm(rhs_))
    tol = inner_tol if opt.inner_rule == "theory" else opt.tol_cg * f0
    lam = (0.0, 0.0)
    if opt.inner == "cg":
        tr = pcg.cg(Bmv, rhs_, opt.t_max, tol)
    else:
        # Chebyshev interval from a few CG (Lanczos) steps on the same system:
        # [0.5 theta_min, 1.05 theta_max]  (an implementation choice; the paper
        # assumes the band of Lemma 3.1 is known)
        alphas, betas = _cg_coeffs(Bmv, rhs_, opt.cheb_lanczos)
        tmin, tmax = lanczos_interval(alphas, betas)
        lam = (0.5 * tmin, 1.05 * tmax)
        tr = pcg.chebyshev(Bmv, rhs_, lam[0], lam[1], opt.t_max, tol)
    z = tr.z
    dy = Qmh @ z
    r_v = A @ (d2 * (A.T @ dy)) - p        # A D^2 A^T dy_hat - p
    f_norm = float(np.linalg.norm(Qmh @ r_v))
    if opt.v_correction:
        v = correction.correction_v(x, s, Wk, ADW, r_v)
    else:
        v = np.zeros(n)
    return NormalSolve(dy=dy, v=v, z=z, trace=tr, f_norm=f_norm, f0_norm=f0,
                       precond=pre, ADW=ADW, retry=retry, lam=lam)


def _adaptive_sigma_solve(A, x, s, r_p, r_d, mu, feasible, opt: Options, k: int, rec):
    """Two right-hand sides on one normal matrix (and, for the sketched solver,
    one sketch and Q): the RHS is affine in sigma, p(sigma) = p_aff + sigma p_c
    with p_aff = p(0) and p_c = -mu A S^{-1} 1, so dy and v are affine in sigma
    too.  sigma comes from the affine direction's largest positivity-keeping
    step: sigma = clip((mu_aff / mu)^3, sigma_range) (Mehrotra's centering
    heuristic), inside the paper's sigma range (0, 4/5).  Returns (dy, v, sigma)."""
    m, n = A.shape
    p_aff = rhs(A, x, s, r_p, r_d, 0.0, mu, feasible)
    p_c = rhs(A, x, s, r_p, r_d, 1.0, mu, feasible) - p_aff
    lo, hi = opt.sigma_range
    if opt.solver == "exact":
        cf = sla.cho_factor(normal_matrix(A, x / s))
        dy_a, dy_c = sla.cho_solve(cf, p_aff), sla.cho_solve(cf, p_c)
        v_a = v_c = np.zeros(n)
    else:
        tol_f = pcg.theory_inner_tol(mu, n, opt.gamma, lo)
        solve = normal_solve if opt.solver == "sketch" else (
            lambda A_, x_, s_, p_, o_, k_, t_: normal_solve_unpreconditioned(A_, x_, s_, p_, o_, t_))
        na = solve(A, x, s, p_aff, opt, k, tol_f)
        nc = solve(A, x, s, p_c, opt, k, tol_f)
        dy_a, dy_c, v_a, v_c = na.dy, nc.dy, na.v, nc.v
        rec.inner_its = na.trace.iterations + nc.trace.iterations
    dx_a, ds_a = directions(A, x, s, r_d, dy_a, v_a, 0.0, mu, feasible)
    a_aff = 1.0
    neg = dx_a < 0
    if neg.any():
        a_aff = min(a_aff, float(np.min(-x[neg] / dx_a[neg])))
    neg = ds_a < 0
    if neg.any():
        a_aff = min(a_aff, float(np.min(-s[neg] / ds_a[neg])))
    mu_aff = float((x + a_aff * dx_a) @ (s + a_aff * ds_a)) / n
    sigma = float(np.clip((mu_aff / mu) ** 3, lo, hi))
    return dy_a + sigma * dy_c, v_a + sigma * v_c, sigma


def normal_solve_unpreconditioned(A, x, s, p, opt: Options, inner_tol: float) -> NormalSolve:
    """The standard IPM's inner solve (the comparison system of Section 7):
    CG on eq. (normal) itself, i.e. Q = I in eq. (precond), and no correction
    (v = 0, there is no sketch).  ||f|| = ||p - A D^2 A^T dy||."""
    m, n = A.shape
    d2 = x / s

    def Mmv(z):
        return A @ (d2 * (A.T @ z))

    f0 = float(np.linalg.norm(p))
    tol = inner_tol if opt.inner_rule == "theory" else opt.tol_cg * f0
    tr = pcg.cg(Mmv, p, opt.t_max, tol)
    dy = tr.z
    f_norm = float(np.linalg.norm(Mmv(dy) - p))
    return NormalSolve(dy=dy, v=np.zeros(n), z=dy, trace=tr, f_norm=f_norm, f0_norm=f0,
                       precond=None, ADW=None, retry=0, lam=(0.0, 0.0))


def _cg_coeffs(Bmv, rhs_, steps):
    r = rhs_.copy()
    d = r.copy()
    rr = r @ r
    alphas, betas = [], []
    for _ in range(steps):
        Bd = Bmv(d)
        a = rr / (d @ Bd)
        r = r - a * Bd
        rr_new = r @ r
        beta = rr_new / rr
        alphas.append(a)
        betas.append(beta)
        d = r + beta * d
        rr = rr_new
        if rr == 0:
            break
    return alphas, betas


# ---------------------------------------------------------------------------
# outer loop
# ---------------------------------------------------------------------------

def converged(A, b, c, x, y, r_p, r_d, tol):
    cx = c @ x
    gap = abs(cx - b @ y) / (1.0 + abs(cx))
    rp = np.linalg.norm(r_p) / (1.0 + np.linalg.norm(b))
    rd = np.linalg.norm(r_d) / (1.0 + np.linalg.norm(c))
    return gap <= tol and rp <= tol and rd <= tol, gap


def solve(A, b, c, opt: Options, x0=None, y0=None, s0=None) -> Result:
    """Algorithm 2 (``opt.mode == "feasible"``) or 3 (``"infeasible"``).

    Default start (infeasible): x0 = s0 = 1, y0 = 0.  The feasible mode needs
    a strictly feasible start in N(gamma) from the caller.  A may be a
    scipy.sparse matrix with the exact solver (fixed sigma): every step then
    uses A only in products with vectors and in eq. normal's A D^2 A^T.
    """
    if sps.issparse(A):
        if opt.solver != "exact" or opt.sigma_rule == "adaptive":
            raise ValueError("a sparse A is taken by the exact solver with fixed sigma only")
        A = sps.csr_matrix(A, dtype=np.float64)
    else:
        A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    feasible = opt.mode == "feasible"
    x = np.ones(n) if x0 is None else np.array(x0, dtype=float)
    y = np.zeros(m) if y0 is None else np.array(y0, dtype=float)
    s = np.ones(n) if s0 is None else np.array(s0, dtype=float)
    r_p, r_d = residuals(A, b, c, x, y, s)
    r0_norm = np.sqrt(r_p @ r_p + r_d @ r_d)
    mu0 = x @ s / n
    if feasible and not in_neighbourhood(x, s, opt.gamma):
        raise ValueError("feasible mode needs a start in N(gamma)")
    history: List[IterRecord] = []
    status = "max_iter"
    for k in range(opt.k_max + 1):
        mu = x @ s / n
        r_p, r_d = residuals(A, b, c, x, y, s)
        done, gap = converged(A, b, c, x, y, r_p, r_d, opt.tol)
        rec = IterRecord(k=k, mu=mu, gap=gap, rp_norm=float(np.linalg.norm(r_p)),
                         rd_norm=float(np.linalg.norm(r_d)))
        history.append(rec)
        if done:
            status = "optimal"
            break
        if k == opt.k_max:
            break
        if feasible:
            r_d_used = np.zeros(n)
            p = rhs(A, x, s, r_p, r_d_used, opt.sigma, mu, True)
        else:
            r_d_used = r_d
            p = rhs(A, x, s, r_p, r_d, opt.sigma, mu, False)
        d2 = x / s
        if opt.sigma_rule == "adaptive":
            dy, v, sigma_k = _adaptive_sigma_solve(A, x, s, r_p, r_d_used, mu, feasible, opt, k, rec)
            dx, ds = directions(A, x, s, r_d_used, dy, v, sigma_k, mu, feasible)
            rec.sigma_used = sigma_k
        elif opt.solver == "exact":
            M = normal_matrix(A, d2)
            cf = sla.cho_factor(M)
            dy = sla.cho_solve(cf, p)
            v = np.zeros(n)
        elif opt.solver == "cg":
            tol_f = pcg.theory_inner_tol(mu, n, opt.gamma, opt.sigma)
            ns = normal_solve_unpreconditioned(A, x, s, p, opt, tol_f)
            dy, v = ns.dy, ns.v
            rec.inner_its = ns.trace.iterations
            rec.f_norm = ns.f_norm
            rec.f0_norm = ns.f0_norm
        else:
            tol_f = pcg.theory_inner_tol(mu, n, opt.gamma, opt.sigma)
            ns = normal_solve(A, x, s, p, opt, k, tol_f)
            dy, v = ns.dy, ns.v
            rec.inner_its = ns.trace.iterations
            rec.f_norm = ns.f_norm
            rec.f0_norm = ns.f0_norm
            rec.v_norm = float(np.linalg.norm(v))
        if opt.sigma_rule != "adaptive":
            dx, ds = directions(A, x, s, r_d_used, dy, v, opt.sigma, mu, feasible)
            rec.sigma_used = opt.sigma
        res_ratio = 0.0 if feasible else np.sqrt(r_p @ r_p + r_d @ r_d) / r0_norm
        a_max, a_bar = step_lengths(x, s, dx, ds, opt.gamma, feasible, res_ratio, mu0)
        rec.alpha_max, rec.alpha_bar = a_max, a_bar
        if opt.keep_vectors:
            rec.vectors = dict(x=x.copy(), y=y.copy(), s=s.copy(), p=p, dy=dy, v=v,
                               dx=dx, ds=ds, r_p=r_p, r_d=r_d)
        if a_bar <= 0.0:
            status = "stalled"
            break
        x = x + a_bar * dx
        y = y + a_bar * dy
        s = s + a_bar * ds
    return Result(x=x, y=y, s=s, status=status, iterations=len(history) - 1,
                  history=history)
