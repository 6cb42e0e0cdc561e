"""Pins for oracle.ipm / oracle.correction (Algorithms 2-3, Sections 4-5).

Every check here comes from something other than the oracle itself: the
planted closed-form optimum, brute-force vertex enumeration, a library LP
solver (HiGHS via scipy), the paper's identities (Lemma 4.5, Appendix eqs.
iip_3) and inequalities (Lemmas 4.2, 4.6, Lemma 3.6 of the cited work), and
a brute-force grid for the step lengths.
"""

import numpy as np
import pytest

import lpgen
from oracle import correction, ipm, pcg, sketch, vertex


def _tiny_planted(m, n, seed):
    return lpgen.planted_dense(m, n, seed=seed)


# ---------------------------------------------------------------------------
# end-to-end optimum
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("solver", ["exact", "sketch"])
@pytest.mark.parametrize("seed", [0, 1])
def test_planted_optimum_reached(solver, seed):
    lp = lpgen.planted_dense(16, 600, seed=seed, col_scale_log10=(-1, 1))
    opt = ipm.Options(mode="infeasible", solver=solver, s=2, w=64)
    res = ipm.solve(lp.A, lp.b, lp.c, opt)
    assert res.status == "optimal"
    obj = lp.c @ res.x
    assert abs(obj - lp.objective) <= 1e-7 * (1 + abs(lp.objective))
    assert abs(obj - lp.b @ res.y) <= 1e-8 * (1 + abs(obj))


def test_feasible_mode_planted():
    lp = lpgen.planted_dense(12, 400, seed=3)
    x0, y0, s0 = lpgen.feasible_start(lp, gamma=0.999)
    for solver in ["exact", "sketch"]:
        opt = ipm.Options(mode="feasible", solver=solver, s=2, w=48)
        res = ipm.solve(lp.A, lp.b, lp.c, opt, x0, y0, s0)
        assert res.status == "optimal"
        assert abs(lp.c @ res.x - lp.objective) <= 1e-7 * (1 + abs(lp.objective))


@pytest.mark.parametrize("seed", range(4))
def test_vertex_enumeration_and_highs_agree_with_oracle(seed):
    rng = np.random.default_rng(100 + seed)
    m, n = 3, 9
    A = rng.standard_normal((m, n))
    # a bounded feasible LP: x0 > 0 feasible, c = A^T y + s with s > 0
    x_feas = rng.uniform(0.5, 1.5, n)
    b = A @ x_feas
    c = A.T @ rng.standard_normal(m) + rng.uniform(0.1, 1.0, n)
    best, _, count = vertex.enumerate_vertices(A, b, c)
    assert count > 0
    res = ipm.solve(A, b, c, ipm.Options(mode="infeasible", solver="exact"))
    assert res.status == "optimal"
    assert abs(c @ res.x - best) <= 1e-7 * (1 + abs(best))
    from scipy.optimize import linprog
    hi = linprog(c, A_eq=A, b_eq=b, bounds=[(0, None)] * n, method="highs")
    assert abs(hi.fun - best) <= 1e-7 * (1 + abs(best))
    # sketched method on the same tiny LP (w >= m, s = 1)
    res2 = ipm.solve(A, b, c, ipm.Options(mode="infeasible", solver="sketch", w=8, s=1))
    assert abs(c @ res2.x - best) <= 1e-7 * (1 + abs(best))


def test_planted_tiny_matches_vertex_enumeration():
    lp = _tiny_planted(3, 10, seed=5)
    best, xb, _ = vertex.enumerate_vertices(lp.A, lp.b, lp.c)
    assert best == pytest.approx(lp.objective, rel=1e-10, abs=1e-10)
    assert np.allclose(xb, lp.x_star, atol=1e-9)


# ---------------------------------------------------------------------------
# sparse A: the exact solver takes a scipy.sparse matrix (eq. normal's
# A D^2 A^T by a sparse product)
# ---------------------------------------------------------------------------

def _csc(lp):
    import scipy.sparse as sps
    return sps.csc_matrix((lp.val, lp.row_idx, lp.col_ptr), shape=(lp.m, lp.n))


@pytest.mark.parametrize("seed", [0, 1])
def test_sparse_input_reaches_the_planted_optimum(seed):
    # the planted (x*, y*, s*) of a sparse LP fixes its optimal value in
    # closed form; the solve from the infeasible start must reach it
    lp = lpgen.planted_sparse(24, 900, nnz_per_col=4, seed=seed)
    A = _csc(lp)
    res = ipm.solve(A, lp.b, lp.c, ipm.Options(mode="infeasible", solver="exact"))
    assert res.status == "optimal"
    obj = lp.c @ res.x
    assert abs(obj - lp.objective) <= 1e-7 * (1 + abs(lp.objective))
    assert abs(obj - lp.b @ res.y) <= 1e-8 * (1 + abs(obj))
    assert np.linalg.norm(A @ res.x - lp.b) <= 1e-8 * (1 + np.linalg.norm(lp.b))
    assert np.all(res.x > 0) and np.all(res.s > 0)


@pytest.mark.parametrize("seed", range(3))
def test_sparse_input_matches_vertex_enumeration(seed):
    # brute force over every basis of a tiny sparse LP: the optimal value
    # the oracle reaches from the sparse matrix is the best vertex
    lp = lpgen.planted_sparse(3, 12, nnz_per_col=2, seed=seed)
    best, _, count = vertex.enumerate_vertices(lp.dense(), lp.b, lp.c)
    assert count > 0 and best == pytest.approx(lp.objective, rel=1e-9, abs=1e-9)
    res = ipm.solve(_csc(lp), lp.b, lp.c, ipm.Options(mode="infeasible", solver="exact"))
    assert res.status == "optimal"
    assert abs(lp.c @ res.x - best) <= 1e-7 * (1 + abs(best))


def test_sparse_input_is_refused_by_the_sketched_solver():
    lp = lpgen.planted_sparse(8, 100, nnz_per_col=3, seed=0)
    with pytest.raises(ValueError):
        ipm.solve(_csc(lp), lp.b, lp.c, ipm.Options(mode="infeasible", solver="sketch"))


# ---------------------------------------------------------------------------
# per-step identities and invariants
# ---------------------------------------------------------------------------

def _trajectory(mode, solver="sketch", m=10, n=300, seed=7, k_max=40, v_corr=True, sigma=0.5):
    lp = lpgen.planted_dense(m, n, seed=seed)
    opt = ipm.Options(mode=mode, solver=solver, s=2, w=4 * m, keep_vectors=True,
                      k_max=k_max, v_correction=v_corr, sigma=sigma)
    if mode == "feasible":
        x0, y0, s0 = lpgen.feasible_start(lp, opt.gamma)
        res = ipm.solve(lp.A, lp.b, lp.c, opt, x0, y0, s0)
    else:
        res = ipm.solve(lp.A, lp.b, lp.c, opt)
    return lp, opt, res


@pytest.mark.parametrize("mode", ["feasible", "infeasible"])
def test_lemma_4_5_identities(mode):
    # (a) x(a) o s(a) = (1-a) x o s + a sigma mu 1 - a v + a^2 dx o ds
    # (b) mu(a) = [1 - a(1-sigma)] mu - a v^T 1/n  (+ a^2 dx^T ds / n, which
    #     is zero in the feasible case)
    lp, opt, res = _trajectory(mode)
    for rec in res.history[:-1]:
        V = rec.vectors
        x, s, dx, ds, v = V["x"], V["s"], V["dx"], V["ds"], V["v"]
        mu = x @ s / x.size
        for a in (0.3, 0.77, 1.0):
            xa, sa = x + a * dx, s + a * ds
            lhs = xa * sa
            rhs = (1 - a) * x * s + a * opt.sigma * mu - a * v + a * a * dx * ds
            assert np.allclose(lhs, rhs, rtol=1e-9, atol=1e-12 * mu)
            mua = xa @ sa / x.size
            pred = (1 - a * (1 - opt.sigma)) * mu - a * v.sum() / x.size + a * a * (dx @ ds) / x.size
            assert mua == pytest.approx(pred, rel=1e-9, abs=1e-14)
        if mode == "feasible":
            # dx^T ds = 0 (proof of Lemma 4.5)
            assert abs(dx @ ds) <= 1e-8 * np.linalg.norm(dx) * np.linalg.norm(ds)


def test_feasible_iterates_stay_feasible_and_in_neighbourhood():
    lp, opt, res = _trajectory("feasible")
    for rec in res.history[:-1]:
        V = rec.vectors
        x, y, s = V["x"], V["y"], V["s"]
        assert np.linalg.norm(lp.A @ x - lp.b) <= 1e-9 * (1 + np.linalg.norm(lp.b))
        assert np.linalg.norm(lp.A.T @ y + s - lp.c) <= 1e-9 * (1 + np.linalg.norm(lp.c))
        assert ipm.in_neighbourhood(x, s, opt.gamma, rel_slack=1e-9)


def test_infeasible_residual_shrinks_linearly():
    # eqs. iip_3_1, iip_3_2: r(alpha) = (1 - alpha) r
    lp, opt, res = _trajectory("infeasible")
    H = res.history
    for k in range(len(H) - 2):
        V = H[k].vectors
        a = H[k].alpha_bar
        rp1 = lp.A @ (V["x"] + a * V["dx"]) - lp.b
        rd1 = lp.A.T @ (V["y"] + a * V["dy"]) + V["s"] + a * V["ds"] - lp.c
        scale = 1e-9 * (1 + np.linalg.norm(V["r_p"]) + np.linalg.norm(V["r_d"]))
        assert np.linalg.norm(rp1 - (1 - a) * V["r_p"]) <= scale + 1e-12 * np.linalg.norm(lp.b)
        assert np.linalg.norm(rd1 - (1 - a) * V["r_d"]) <= scale + 1e-12 * np.linalg.norm(lp.c)


def test_correction_invariant_and_norm_bound():
    # eq. (addl): A S^{-1} v = A D^2 A^T dy_hat - p ; Lemma 4.2: ||v|| <= sqrt(3 n mu) ||f||
    rng = np.random.default_rng(21)
    m, n = 8, 2000
    A = rng.standard_normal((m, n))
    x = rng.uniform(0.1, 2, n)
    s = rng.uniform(0.1, 2, n)
    p = rng.standard_normal(m)
    opt = ipm.Options(solver="sketch", sketch="gaussian", w=800, t_max=3, inner_rule="relative",
                      tol_cg=0.0)
    ns = ipm.normal_solve(A, x, s, p, opt, k=0, inner_tol=0.0)
    d2 = x / s
    r_v = A @ (d2 * (A.T @ ns.dy)) - p
    assert np.allclose(A @ (ns.v / s), r_v, rtol=1e-9, atol=1e-12 * np.linalg.norm(p))
    mu = x @ s / n
    assert np.linalg.norm(ns.v) <= np.sqrt(3 * n * mu) * ns.f_norm
    # ||f|| is ||Q^{-1/2} (M dy - p)|| with the inexact dy (3 iterations)
    assert ns.f_norm > 0


def test_correction_with_identity_sketch_and_minnorm_alternative():
    rng = np.random.default_rng(22)
    m, n = 4, 30
    A = rng.standard_normal((m, n))
    x = rng.uniform(0.1, 2, n)
    s = rng.uniform(0.1, 2, n)
    r_v = rng.standard_normal(m)
    W = np.eye(n)
    ADW = A * np.sqrt(x / s)
    v = correction.correction_v(x, s, W, ADW, r_v)
    vmin = correction.correction_v_minnorm(A, s, r_v)
    assert np.allclose(A @ (v / s), r_v, atol=1e-10)
    assert np.allclose(A @ (vmin / s), r_v, atol=1e-10)
    assert np.linalg.norm(vmin) <= np.linalg.norm(v) * (1 + 1e-12)


def test_mu_decrease_lemma_3_6():
    # mu(alpha_bar) <= [1 - alpha_bar/2 (1 - 5 sigma/4)] mu  (read as an inequality)
    lp, opt, res = _trajectory("feasible")
    H = res.history
    for k in range(len(H) - 1):
        a = H[k].alpha_bar
        assert H[k + 1].mu <= (1 - a / 2 * (1 - 1.25 * opt.sigma)) * H[k].mu * (1 + 1e-9)


def test_outer_iteration_bound_lemma_4_7():
    # k <= (n / beta) log(1/eps) with beta of eq. pdbeta1 and
    # lambda = max{1/gamma, 1/(1-gamma), 1/sigma, 1/(1 - 5 sigma/4)}
    lp, opt, res = _trajectory("feasible")
    g, sg = opt.gamma, opt.sigma
    lam = max(1 / g, 1 / (1 - g), 1 / sg, 1 / (1 - 1.25 * sg))
    beta = 1.0 / (8 * lam ** 3 * (1 + lam * sg ** 2 + lam * g ** 2 * sg ** 2 / 16 + g * sg ** 2 / 2))
    mu0 = res.history[0].mu
    eps = res.history[-1].mu / mu0
    assert res.iterations <= lp.n / beta * np.log(1 / eps)


def test_without_v_correction_still_converges():
    # Table 2: the method still converges without v (the counts there are on
    # other data; here only convergence and a modest change are asserted)
    lp = lpgen.planted_dense(12, 500, seed=8)
    out = []
    for vc in (True, False):
        opt = ipm.Options(mode="infeasible", solver="sketch", s=2, w=48, v_correction=vc)
        res = ipm.solve(lp.A, lp.b, lp.c, opt)
        assert res.status == "optimal"
        out.append(res.iterations)
    assert out[1] <= 1.5 * out[0]


def test_sketched_cg_needs_far_fewer_inner_iterations_than_plain_cg():
    # Table 1 / Figure 1 qualitatively: near a degenerate vertex A D^2 A^T is
    # ill-conditioned (m/2 large entries of D^2); the sketched preconditioner
    # keeps the inner count small while plain CG needs many more iterations
    rng = np.random.default_rng(30)
    m, n = 80, 3000
    A = rng.standard_normal((m, n))
    d2 = 10.0 ** rng.uniform(-6, -2, n)
    big = rng.choice(n, m // 2, replace=False)
    d2[big] = 10.0 ** rng.uniform(2, 6, m // 2)
    x, s = np.sqrt(d2), 1.0 / np.sqrt(d2)
    p = rng.standard_normal(m)
    M = (A * d2) @ A.T
    assert np.linalg.cond(M) > 1e6
    plain = pcg.cg(lambda z: M @ z, p, 20000, 1e-6 * np.linalg.norm(p))
    opt = ipm.Options(solver="sketch", w=4 * m, s=2, inner_rule="relative", tol_cg=1e-6)
    ns = ipm.normal_solve(A, x, s, p, opt, k=0, inner_tol=0.0)
    assert plain.iterations >= 10 * ns.trace.iterations


def test_unpreconditioned_normal_solve_is_cg_on_eq_normal():
    # the comparison system: Q = I, so at a tight tolerance dy is the Cholesky
    # solution, and there is no correction vector
    rng = np.random.default_rng(31)
    m, n = 20, 400
    A = rng.standard_normal((m, n))
    x, s = np.exp(rng.uniform(-1, 1, n)), np.exp(rng.uniform(-1, 1, n))
    p = rng.standard_normal(m)
    M = (A * (x / s)) @ A.T
    exact = np.linalg.solve(M, p)
    opt = ipm.Options(solver="cg", inner_rule="relative", tol_cg=1e-13, t_max=500)
    ns = ipm.normal_solve_unpreconditioned(A, x, s, p, opt, inner_tol=0.0)
    assert np.linalg.norm(ns.dy - exact) <= 1e-9 * np.linalg.norm(exact)
    assert not ns.v.any()
    assert ns.f_norm <= 1e-12 * np.linalg.norm(p)


def test_standard_ipm_with_plain_cg_vs_sketched_inner_counts():
    # Section 7 / Tables 1-2 qualitatively, at the IPM level: with the
    # experiments' relative inner rule the sketched method converges, and over
    # the same outer iterations the standard IPM's plain CG needs >= 10x more
    # inner steps on a column-scaled LP
    m, n = 64, 3000
    lp = lpgen.planted_dense(m, n, seed=32, storage="f64", col_scale_log10=(-2, 2))
    common = dict(mode="infeasible", inner_rule="relative", tol_cg=1e-5, t_max=20000)
    sk = ipm.solve(lp.A, lp.b, lp.c, ipm.Options(solver="sketch", w=4 * m, s=2, k_max=60, **common))
    assert sk.status == "optimal"
    plain = ipm.solve(lp.A, lp.b, lp.c, ipm.Options(solver="cg", k_max=sk.iterations, **common))
    n_plain = sum(r.inner_its for r in plain.history)
    n_sk = sum(r.inner_its for r in sk.history)
    assert n_plain >= 10 * n_sk, (n_plain, n_sk)


def test_w_sweep_inner_iterations_fall_with_w():
    # Figures 2-3 qualitatively: a wider sketch embeds better (Lemma 3.1), so
    # the mean inner iteration count falls as w grows
    m, n = 64, 3000
    lp = lpgen.planted_dense(m, n, seed=33, storage="f64", col_scale_log10=(-2, 2))
    means = []
    for wf in (2, 4, 16):
        r = ipm.solve(lp.A, lp.b, lp.c, ipm.Options(solver="sketch", w=wf * m, s=2))
        assert r.status == "optimal"
        its = [h.inner_its for h in r.history if h.inner_its]
        means.append(sum(its) / len(its))
    assert means[0] > means[1] > means[2], means


# ---------------------------------------------------------------------------
# step lengths
# ---------------------------------------------------------------------------

def test_first_exit_hand_built_quadratics():
    # g = a t^2 + b t + c with known downward crossings
    a = np.array([1.0, -1.0, 0.0, 0.0, 1.0, -1.0, 2.0, -1.0])
    b = np.array([-3.0, 0.0, -2.0, 1.0, 1.0, 0.5, -1.0, -1.0])
    c = np.array([2.0, 4.0, 1.0, 1.0, 1.0, 0.0, 1.0, -1.0])
    # 1) (t-1)(t-2): exits at 1     2) 4 - t^2: exits at 2     3) 1-2t: exits at 0.5
    # 4) 1+t: never                 5) t^2+t+1 > 0: never       6) -t^2+0.5t: exits at 0.5
    # 7) 2t^2 - t + 1 > 0: never    8) -t^2 - t - 1 < 0 everywhere: exits at 0
    expect = np.array([1.0, 2.0, 0.5, np.inf, np.inf, 0.5, np.inf, 0.0])
    got = ipm._first_exit(a, b, c)
    assert np.allclose(got, expect)


@pytest.mark.parametrize("mode,sigma", [("feasible", 0.5), ("infeasible", 0.5), ("infeasible", 0.3)])
def test_step_length_against_grid(mode, sigma):
    # at sigma = 0.5 the residual condition of the infeasible neighbourhood
    # never binds on this LP; at sigma = 0.3 it stops some steps
    lp, opt, res = _trajectory(mode, k_max=12 if sigma == 0.5 else 6, sigma=sigma)
    feasible = mode == "feasible"
    r0 = np.sqrt(res.history[0].vectors["r_p"] @ res.history[0].vectors["r_p"]
                 + res.history[0].vectors["r_d"] @ res.history[0].vectors["r_d"])
    mu0 = res.history[0].mu
    grid = np.linspace(0, 1, 20001)
    tight = 0
    for rec in res.history[:-1]:
        V = rec.vectors
        x, s, dx, ds = V["x"], V["s"], V["dx"], V["ds"]
        rr = 0.0 if feasible else np.sqrt(V["r_p"] @ V["r_p"] + V["r_d"] @ V["r_d"]) / r0
        amax = rec.alpha_max
        ok = [ipm.in_neighbourhood(x + a * dx, s + a * ds, opt.gamma, feasible,
                                   (1 - a) * rr, mu0, rel_slack=1e-9)
              for a in grid]
        ok = np.array(ok)
        inside = grid <= amax
        assert ok[inside].all()
        if amax < 1.0:
            beyond = grid > amax * (1 + 1e-6) + 1e-9
            assert not ok[beyond][:5].all()
        # alpha_bar minimises the gap on [0, alpha_max]
        gaps = [(x + a * dx) @ (s + a * ds) for a in grid[inside]]
        ab = rec.alpha_bar
        gap_ab = (x + ab * dx) @ (s + ab * ds)
        assert gap_ab <= min(gaps) * (1 + 1e-9) + 1e-15
        if not feasible:
            mu_a = (x + amax * dx) @ (s + amax * ds) / x.size
            tight += abs(mu_a / mu0 - (1 - amax) * rr) <= 1e-7 * mu_a / mu0
    if sigma < 0.5:
        assert tight >= 1


def _grid_membership(x, s, dx, ds, grid, gamma, feasible, rr, mu0, slack=1e-9):
    """Brute force: is (x + a dx, s + a ds) in N(gamma) for every a of the
    grid?  eq. neigh: x, s > 0 and x_i s_i >= (1 - gamma) mu; infeasible
    (Section 5) adds ||r(a)||/||r0|| = (1 - a) rr <= mu(a)/mu0.  Also
    returns the duality gap at every grid point."""
    X = x[None, :] + grid[:, None] * dx[None, :]
    S = s[None, :] + grid[:, None] * ds[None, :]
    gap = (X * S).sum(axis=1)
    mu = gap / x.size
    ok = (X > 0).all(axis=1) & (S > 0).all(axis=1)
    ok &= (X * S).min(axis=1) >= (1 - gamma) * mu * (1 - slack)
    if not feasible:
        ok &= (1 - grid) * rr <= mu / mu0 * (1 + slack)
    return ok, gap


@pytest.mark.parametrize("feasible", [True, False])
def test_step_lengths_on_random_states_against_grid(feasible):
    # Trajectories rarely make every condition bind (with gamma = 0.999 the
    # neighbourhood hardly ever does, and the gap is usually smallest at
    # alpha_max), so random states in N(gamma) with directions built to make
    # each condition bind are checked too: alpha_max is the first exit from
    # N(gamma) on a grid of 20001 steps, alpha_bar minimises the gap on
    # [0, alpha_max].  Half the directions shrink one group of coordinates and
    # grow the rest, which puts the gap's minimiser inside the interval.
    rng = np.random.default_rng(50 + feasible)
    grid = np.linspace(0, 1, 20001)
    n = 40
    interior = tight = 0
    for trial in range(36):
        gamma = (0.3, 0.6, 0.9)[trial % 3]
        x = np.exp(rng.uniform(-1, 1, n))
        s = (1 + 0.8 * gamma * rng.uniform(-1, 1, n)) / x
        shrink = rng.uniform(0.2, 1.0) if feasible else rng.uniform(0.5, 1.0)
        if trial % 4 < 2:
            dx = x * (-shrink + rng.uniform(0.2, 1.2) * rng.standard_normal(n))
            ds = s * (-shrink + rng.uniform(0.2, 1.2) * rng.standard_normal(n))
        else:
            grow = rng.random(n) < rng.uniform(0.15, 0.4)
            u = np.where(grow, 1.0, -rng.uniform(0.6, 1.0)) * (1 + 0.1 * rng.standard_normal(n))
            dx = x * u
            ds = s * (u + 0.1 * rng.standard_normal(n))
        mu = x @ s / n
        mu0 = mu * rng.uniform(1, 3)
        rr = 0.0 if feasible else mu / mu0 * rng.uniform(0.9, 1.0)
        amax, abar = ipm.step_lengths(x, s, dx, ds, gamma, feasible, rr, mu0)
        ok, gap = _grid_membership(x, s, dx, ds, grid, gamma, feasible, rr, mu0)
        assert ok[0]
        inside = grid <= amax
        assert ok[inside].all(), trial
        if amax < 1.0:
            beyond = grid > amax * (1 + 1e-6) + 1e-9
            assert not ok[beyond][:5].all(), trial
        assert 0.0 <= abar <= amax
        gap_ab = (x + abar * dx) @ (s + abar * ds)
        assert gap_ab <= gap[inside].min() * (1 + 1e-9) + 1e-15, trial
        interior += 1e-3 < abar < amax * (1 - 1e-3)
        if not feasible:
            mu_a = (x + amax * dx) @ (s + amax * ds) / n
            tight += abs(mu_a / mu0 - (1 - amax) * rr) <= 1e-7 * mu_a / mu0
    # the cases above really exercised the interior minimiser and, for the
    # infeasible neighbourhood, the residual condition
    assert interior >= 3
    assert feasible or tight >= 3


def test_feasible_start_is_strictly_feasible_and_central_enough():
    lp = lpgen.planted_dense(10, 200, seed=4)
    x0, y0, s0 = lpgen.feasible_start(lp, gamma=0.9)
    assert (x0 > 0).all() and (s0 > 0).all()
    assert np.allclose(lp.A @ x0, lp.b, atol=1e-10 * np.linalg.norm(lp.b))
    assert np.allclose(lp.A.T @ y0 + s0, lp.c, atol=1e-10 * np.linalg.norm(lp.c))
    assert ipm.in_neighbourhood(x0, s0, 0.9)


def test_normal_solve_matches_cholesky_at_tight_tolerance():
    rng = np.random.default_rng(40)
    m, n = 12, 1500
    A = rng.standard_normal((m, n))
    x = np.exp(rng.uniform(-5, 2, n))
    s = np.exp(rng.uniform(-5, 2, n))
    p = rng.standard_normal(m)
    for inner in ("cg", "chebyshev"):
        opt = ipm.Options(solver="sketch", w=4 * m, s=2, inner=inner, t_max=400)
        ns = ipm.normal_solve(A, x, s, p, opt, k=0, inner_tol=1e-11 * np.linalg.norm(p))
        exact = np.linalg.solve((A * (x / s)) @ A.T, p)
        assert np.allclose(ns.dy, exact, rtol=1e-7, atol=1e-9 * np.linalg.norm(exact))


def test_sketch_redraw_on_rank_failure():
    # a CountSketch narrower than m is rank deficient every draw -> error
    rng = np.random.default_rng(41)
    m, n = 6, 100
    A = rng.standard_normal((m, n))
    x = np.ones(n)
    s = np.ones(n)
    opt = ipm.Options(solver="sketch", w=4, s=1)
    with pytest.raises(np.linalg.LinAlgError):
        ipm.normal_solve(A, x, s, rng.standard_normal(m), opt, k=0, inner_tol=1e-8)


# ---------------------------------------------------------------------------
# two right-hand sides per outer iteration (adaptive sigma)
# ---------------------------------------------------------------------------
def test_two_rhs_combination_is_the_solve_with_p_sigma():
    # p is affine in sigma, so dy_aff + sigma dy_c must equal the direct solve
    # with p(sigma) (exact solver: v = 0)
    lp = lpgen.planted_dense(24, 600, seed=40)
    rng = np.random.default_rng(41)
    x, s = np.exp(rng.uniform(-1, 1, lp.n)), np.exp(rng.uniform(-1, 1, lp.n))
    y = rng.standard_normal(lp.m)
    r_p, r_d = ipm.residuals(lp.A, lp.b, lp.c, x, y, s)
    mu = x @ s / lp.n
    opt = ipm.Options(solver="exact", sigma_rule="adaptive")
    rec = ipm.IterRecord(k=0, mu=mu, gap=0.0, rp_norm=0.0, rd_norm=0.0)
    dy, v, sigma = ipm._adaptive_sigma_solve(lp.A, x, s, r_p, r_d, mu, False, opt, 0, rec)
    assert 0.1 <= sigma <= 0.75
    M = ipm.normal_matrix(lp.A, x / s)
    direct = np.linalg.solve(M, ipm.rhs(lp.A, x, s, r_p, r_d, sigma, mu, False))
    assert np.linalg.norm(dy - direct) <= 1e-9 * np.linalg.norm(direct)
    assert not v.any()


@pytest.mark.parametrize("col_scale", [None, (-2, 2)])
def test_two_rhs_adaptive_sigma_needs_fewer_outer_iterations(col_scale):
    lp = lpgen.planted_dense(48, 3000, seed=42, storage="f64", col_scale_log10=col_scale)
    out = {}
    for rule in ("fixed", "adaptive"):
        r = ipm.solve(lp.A, lp.b, lp.c, ipm.Options(solver="sketch", sigma_rule=rule, w=4 * 48, s=2))
        assert r.status == "optimal"
        assert abs(lp.c @ r.x - lp.objective) <= 1e-7 * (1 + abs(lp.objective))
        out[rule] = r
    assert out["adaptive"].iterations <= 0.7 * out["fixed"].iterations
    sig = [h.sigma_used for h in out["adaptive"].history if h.sigma_used > 0]
    assert min(sig) >= 0.1 and max(sig) <= 0.75


@pytest.mark.parametrize("col_scale", [None, (-2, 2)])
def test_gamma_sensitivity(col_scale):
    # gamma is never given numerically; the default 0.999 is a reading.  On
    # the planted family every gamma in {0.9, 0.99, 0.999} reaches the
    # optimum, in outer iteration counts within 25 % of one another
    lp = lpgen.planted_dense(64, 4096, seed=0, col_scale_log10=col_scale)
    outer = []
    for g in (0.9, 0.99, 0.999):
        r = ipm.solve(lp.A, lp.b, lp.c, ipm.Options(mode="infeasible", solver="sketch", gamma=g, s=2, w=256))
        assert r.status == "optimal"
        assert abs(lp.c @ r.x - lp.objective) <= 1e-7 * (1 + abs(lp.objective))
        outer.append(r.iterations)
    assert max(outer) <= 1.25 * min(outer), outer


def test_orthonormal_rows_and_unit_scaling_give_the_identity_normal_matrix():
    # A with orthonormal rows and D = I (x = s) make M = A A^T = I, so the
    # inexact solve must return dy = p
    rng = np.random.default_rng(60)
    m, n = 10, 400
    Qn, _ = np.linalg.qr(rng.standard_normal((n, m)))
    A = Qn.T
    x = s = np.exp(rng.uniform(-1, 1, n))
    p = rng.standard_normal(m)
    opt = ipm.Options(solver="sketch", w=4 * m, s=2, t_max=100)
    ns = ipm.normal_solve(A, x, s, p, opt, k=0, inner_tol=1e-12 * np.linalg.norm(p))
    assert np.allclose(ns.dy, p, rtol=0, atol=1e-10 * np.linalg.norm(p))


def test_identity_sketch_correction_is_the_min_norm_solution_of_ad():
    # W = I: v = (XS)^{1/2} (AD)^+ r, and (AD)^+ r is the minimum-norm solution
    # of (AD) z = r, here from a least-squares solver
    rng = np.random.default_rng(61)
    m, n = 6, 40
    A = rng.standard_normal((m, n))
    x, s = rng.uniform(0.1, 2, n), rng.uniform(0.1, 2, n)
    r = rng.standard_normal(m)
    AD = A * np.sqrt(x / s)
    v = correction.correction_v(x, s, np.eye(n), AD, r)
    z, *_ = np.linalg.lstsq(AD, r, rcond=None)
    assert np.allclose(v, np.sqrt(x * s) * z, rtol=1e-10, atol=1e-12 * np.linalg.norm(v))


def test_inner_solves_stop_at_the_theory_bound():
    # with the default (theory) rule every inner solve ends at
    # ||f|| <= gamma sigma sqrt(mu) / (4 sqrt(3 n)), the level Lemma 4.4 needs
    lp, opt, res = _trajectory("infeasible", k_max=25)
    n = lp.n
    for rec in res.history[:-1]:
        assert rec.inner_its < opt.t_max
        assert rec.f_norm <= pcg.theory_inner_tol(rec.mu, n, opt.gamma, opt.sigma) * (1 + 1e-9)
        # and so, by Lemma 4.2, the correction meets Lemma 4.4's ||v|| <= gamma sigma mu / 4
        assert rec.v_norm <= opt.gamma * opt.sigma * rec.mu / 4 * (1 + 1e-9)
