"""Parity of each CUDA hot-path step with the CPU oracle, through the C ABI.

Rows of the hot path (paper references in brackets):
  a1+a2  residuals and right-hand side      [Alg. 3 step 3, eq. pdef]
  a3     CountSketch A D W                   [Section 2, eq. pdprec]
  a4     preconditioner Q^{-1}               [Alg. 1 steps 1-2]
  a5     the product A D^2 A^T v and the inexact solve  [eq. normal, Alg. 1 step 3]
  a6     correction v                        [eq. compv]
  a7     directions                          [eqs. delshat(_i), delxhat]
  a8     step lengths                        [Alg. 2 steps 5-6, Alg. 3 steps 6-7]

Tolerances: FP64 arithmetic is held to c * (length) * 2^-53 times the
absolute-value bound of the same expression; the FP32 product to
4 (m + L + 64) 2^-24 times |A| D^2 |A|^T |v| (forward error of a dot product of
length m followed by FP32 sums of L columns per warp; the per-CTA partials
are summed in double-float, ~2^-48).
"""

import numpy as np
import pytest

import lpgen
from oracle import correction, ipm, pcg, sketch
from tests.gpu_helpers import EPS32, EPS64, adat_bound, dev, fp32_lane_columns, host, solver_for, torch_cuda

pytestmark = pytest.mark.gpu

SHAPES = [
    # (m, n, storage): several tiles and a ragged last tile; m not a multiple of the vector width
    (64, 4099, "f64"),
    (37, 3001, "f64"),
    (512, 20011, "f32"),
    (45, 7777, "f32"),
    (128, 513, "f32"),
    (256, 9000, "bf16"),
    (19, 1000, "bf16"),
    (2048, 3000, "bf16"),
    # tall columns: the row-split kernels (several column groups, one group,
    # and two slabs per warp), with ragged row vectors and a ragged last tile
    (600, 5003, "f32"),
    (1500, 7001, "f32"),
    (2048, 3001, "f32"),
    (1100, 4003, "bf16"),
    (4096, 6007, "bf16"),
    (5000, 6001, "bf16"),
]


def _lp(m, n, storage, seed=0):
    return lpgen.planted_dense(m, n, seed=seed, storage=storage,
                               col_scale_log10=(-1, 1) if storage != "f64" else None)


@pytest.mark.parametrize("m,n,storage", SHAPES)
@pytest.mark.parametrize("precision", [0, 1])
def test_adat_matches_fp64_product(m, n, storage, precision):
    torch = torch_cuda()
    lp = _lp(m, n, storage)
    rng = np.random.default_rng(1)
    d2 = np.exp(rng.uniform(-6, 6, n))
    v = rng.standard_normal(m)
    ref = lp.A @ (d2 * (lp.A.T @ v))
    with solver_for(lp) as S:
        u = host(S.adat(dev(torch, d2), dev(torch, v), precision))
    bound = adat_bound(lp.A, d2, v)
    if storage == "f64" or precision == 1:
        tol = 8 * (m + n) * EPS64 * bound
    else:
        L = fp32_lane_columns(m, n, storage)
        tol = 4 * (m + L + 64) * EPS32 * bound
    assert np.all(np.abs(u - ref) <= tol + 1e-300), np.max(np.abs(u - ref) / bound)


@pytest.mark.parametrize("mode", ["infeasible", "feasible"])
@pytest.mark.parametrize("m,n,storage", [(64, 4099, "f64"), (512, 20011, "f32"), (37, 2000, "bf16"),
                                         (700, 4001, "f32"), (2048, 3001, "bf16"), (5000, 6001, "bf16")])
def test_residual_rhs(mode, m, n, storage):
    torch = torch_cuda()
    lp = _lp(m, n, storage, seed=2)
    rng = np.random.default_rng(3)
    x = np.exp(rng.uniform(-3, 3, n))
    s = np.exp(rng.uniform(-3, 3, n))
    y = rng.standard_normal(m)
    A = lp.A
    rp_ref, rd_ref = ipm.residuals(A, lp.b, lp.c, x, y, s)
    mu = x @ s / n
    p_ref = ipm.rhs(A, x, s, rp_ref, np.zeros(n) if mode == "feasible" else rd_ref, 0.5, mu,
                    mode == "feasible")
    with solver_for(lp) as S:
        rp, rd, p, sc = S.residual_rhs(dev(torch, x), dev(torch, y), dev(torch, s), mode)
        rp, rd, p = host(rp), host(rd), host(p)
    ax = np.abs(A)
    tol_rp = 8 * n * EPS64 * (ax @ x + np.abs(lp.b))
    tol_rd = 8 * m * EPS64 * (ax.T @ np.abs(y) + s + np.abs(lp.c))
    assert np.all(np.abs(rp - rp_ref) <= tol_rp)
    assert np.all(np.abs(rd - rd_ref) <= tol_rd)
    d2 = x / s
    t_abs = x + 0.5 * mu / s + (0 if mode == "feasible" else d2 * np.abs(rd_ref))
    tol_p = 16 * n * EPS64 * (ax @ t_abs + ax @ x + np.abs(lp.b))
    assert np.all(np.abs(p - p_ref) <= tol_p)
    assert sc["mu"] == pytest.approx(mu, rel=1e-12)
    assert sc["cx"] == pytest.approx(lp.c @ x, rel=1e-10)
    assert sc["by"] == pytest.approx(lp.b @ y, rel=1e-10, abs=1e-12)
    assert sc["rp_norm"] == pytest.approx(np.linalg.norm(rp_ref), rel=1e-9)
    assert sc["rd_norm"] == pytest.approx(np.linalg.norm(rd_ref), rel=1e-9)


# FP32/BF16 storage sums in double-float arithmetic: products exact up to the
# 2^-48 split of d_j / sqrt(s); the pair sums (renormalised every 8 steps) add
# at most ~16 2^-48 of the bound per step, over at most twice the mean bucket
# size n s / w of steps
DF_U = 2.0 ** -48


@pytest.mark.parametrize("m,n,storage,s_blocks,w", [
    (64, 4099, "f64", 2, 0), (512, 20011, "f32", 4, 0), (30, 1500, "bf16", 3, 0), (8, 100, "f32", 1, 0),
    (600, 5003, "f32", 2, 0), (520, 3001, "bf16", 2, 0), (130, 2000, "f64", 2, 0),
    # several rows per thread of the bucket kernel (4 BF16, 8 FP32, 4 FP64), and
    # columns above its 4096 rows (the slab kernel)
    (2048, 9001, "bf16", 4, 0), (2100, 4001, "f32", 2, 0), (1100, 3001, "f64", 2, 0),
    (4500, 5003, "bf16", 2, 0),
    # more buckets than columns: most buckets of the bucket kernel are empty,
    # the others hold an odd or even number of columns
    (600, 701, "f32", 1, 0), (1030, 1100, "bf16", 1, 0),
    # buckets of ~10^4 columns: above the in-CTA sort capacity
    (4, 40000, "f32", 1, 4), (6, 30000, "f64", 2, 6)])
def test_countsketch_matches_oracle(m, n, storage, s_blocks, w):
    torch = torch_cuda()
    lp = _lp(m, n, storage, seed=4)
    rng = np.random.default_rng(5)
    D = np.exp(rng.uniform(-3, 3, n))
    seed, k, retry = 12345, 7, 1
    with solver_for(lp, s=s_blocks, w=w) as S:
        w = S.sketch_width
        adw = host(S.sketch(dev(torch, D), seed, k, retry))
    W = sketch.countsketch_matrix(seed, k, retry, n, w, s_blocks)
    ref = np.asarray((W.T @ (lp.A * D).T).T)
    bound = np.asarray((abs(W).T @ np.abs(lp.A * D).T).T)
    assert adw.shape == (m, w)
    eps = 8 * n * EPS64 if storage == "f64" else max(8 * n * EPS64, (32 * n * s_blocks / w + 64) * DF_U)
    assert np.all(np.abs(adw - ref) <= eps * bound + 1e-300)


@pytest.mark.parametrize("storage", ["f32", "bf16", "f64"])
def test_countsketch_is_bitwise_reproducible(storage):
    # the summation order depends only on the hashes, not on scheduling
    torch = torch_cuda()
    lp = _lp(300, 30011, storage, seed=13)
    D = dev(torch, np.exp(np.random.default_rng(14).uniform(-4, 4, lp.n)))
    with solver_for(lp, s=3) as S:
        a = host(S.sketch(D, 99, 2, 0))
        b = host(S.sketch(D, 99, 2, 0))
        c = host(S.sketch(D, 99, 2, 1))
    assert np.array_equal(a.view(np.uint64), b.view(np.uint64))
    assert not np.array_equal(a, c)


def test_precond_apply_is_q_inverse():
    torch = torch_cuda()
    lp = _lp(40, 3000, "f32", seed=6)
    rng = np.random.default_rng(7)
    D = np.exp(rng.uniform(-1, 1, lp.n))
    with solver_for(lp) as S:
        adw = S.sketch(dev(torch, D), 0, 0)
        r = rng.standard_normal(lp.m)
        z = host(S.precond_apply(adw, dev(torch, r)))
        adw_h = host(adw)
    pre = pcg.preconditioner(adw_h)
    ref = pre.Q_inv @ r
    cond = (pre.sv[0] / pre.sv[-1]) ** 2
    assert np.linalg.norm(z - ref) <= 1e3 * cond * EPS64 * np.linalg.norm(ref)


def test_precond_rank_failure_is_reported():
    torch = torch_cuda()
    from paper_2209_08722_gb300.solver import LPError
    lp = _lp(16, 500, "f32", seed=8)
    with solver_for(lp) as S:
        adw = torch.zeros(lp.m, S.sketch_width, dtype=torch.float64, device="cuda")
        adw[:, :3] = 1.0
        with pytest.raises(LPError) as ei:
            S.precond_apply(adw.contiguous(), torch.ones(lp.m, dtype=torch.float64, device="cuda"))
        assert "SKETCH_RANK" in str(ei.value)


@pytest.mark.parametrize("storage", ["f64", "f32", "bf16"])
def test_normal_solve_fixed_iterations_matches_oracle_cg(storage):
    # t CG iterations on eq. (precond) with Q^{-1} = R^{-1}R^{-T} give the same
    # iterates as CG on eq. (precond_alt) with the SVD-based Q^{-1/2}
    m, n = 48, 6000
    lp = _lp(m, n, storage, seed=9)
    rng = np.random.default_rng(10)
    x = np.exp(rng.uniform(-4, 2, n))
    s = np.exp(rng.uniform(-4, 2, n))
    D = np.sqrt(x / s)
    p = rng.standard_normal(m)
    t = 6
    opt = ipm.Options(solver="sketch", w=4 * m, s=2, t_max=t, seed=0)
    ref = ipm.normal_solve(lp.A, x, s, p, opt, k=3, inner_tol=0.0)
    assert ref.trace.iterations == t
    with solver_for(lp, s=2, t_max=t, seed=0) as S:
        dy, v, info = S.normal_solve(D, p, xs=x * s, k=3, tol_f=1e-300)
    assert info["inner_iterations"] == t
    rel = 1e-4 if storage != "f64" else 1e-9
    assert np.linalg.norm(dy - ref.dy) <= rel * np.linalg.norm(ref.dy)
    # v for the GPU's own dy (eq. compv, same W) and its invariant (eq. addl)
    d2 = x / s
    r_v = lp.A @ (d2 * (lp.A.T @ dy)) - p
    W = sketch.countsketch_matrix(0, 3, 0, n, 4 * m, 2)
    v_ref = correction.correction_v(x, s, W, ref.ADW, r_v)
    assert np.linalg.norm(v - v_ref) <= 1e-7 * np.linalg.norm(v_ref)
    inv = lp.A @ (v / s)
    assert np.linalg.norm(inv - r_v) <= 1e-8 * np.linalg.norm(r_v)
    mu = x @ s / n
    assert np.linalg.norm(v) <= np.sqrt(3 * n * mu) * info["f_norm"] * (1 + 1e-6)


@pytest.mark.parametrize("storage,m,n", [("f64", 96, 12000), ("f32", 96, 12000), ("bf16", 96, 12000),
                                         ("f32", 700, 30000), ("bf16", 1100, 40000)])
@pytest.mark.parametrize("inner", [0, 1])
def test_normal_solve_converges_to_cholesky(storage, m, n, inner):
    lp = _lp(m, n, storage, seed=11)
    rng = np.random.default_rng(12)
    D = np.exp(rng.uniform(-3, 3, n))
    p = rng.standard_normal(m)
    M = (lp.A * D * D) @ lp.A.T
    exact = np.linalg.solve(M, p)
    with solver_for(lp, s=2, inner=inner) as S:
        tol_f = 1e-11 * np.linalg.norm(p) / np.sqrt(np.linalg.eigvalsh(M)[-1])
        dy, _, info = S.normal_solve(D, p, k=0, tol_f=tol_f)
    assert info["f_norm"] <= tol_f
    assert np.linalg.norm(dy - exact) <= 1e-7 * np.linalg.norm(exact)


@pytest.mark.parametrize("mode", ["infeasible", "feasible"])
@pytest.mark.parametrize("m,n,storage", [(64, 4099, "f64"), (512, 20011, "f32"), (33, 3000, "bf16"),
                                         (700, 4001, "f32"), (2048, 3001, "bf16"), (5000, 6001, "bf16")])
def test_directions(mode, m, n, storage):
    torch = torch_cuda()
    lp = _lp(m, n, storage, seed=13)
    rng = np.random.default_rng(14)
    x = np.exp(rng.uniform(-3, 3, n))
    s = np.exp(rng.uniform(-3, 3, n))
    rd = rng.standard_normal(n)
    dy = rng.standard_normal(m)
    v = 1e-3 * rng.standard_normal(n)
    mu = x @ s / n
    feas = mode == "feasible"
    dx_ref, ds_ref = ipm.directions(lp.A, x, s, np.zeros(n) if feas else rd, dy, v, 0.5, mu, feas)
    with solver_for(lp) as S:
        dx, ds = S.directions(dev(torch, x), dev(torch, s), dev(torch, rd), dev(torch, dy),
                              dev(torch, v), mu, mode)
        dx, ds = host(dx), host(ds)
    ds_bound = np.abs(lp.A).T @ np.abs(dy) + (0 if feas else np.abs(rd))
    assert np.all(np.abs(ds - ds_ref) <= 8 * m * EPS64 * ds_bound)
    dx_bound = x + 0.5 * mu / s + (x / s) * ds_bound + np.abs(v) / s
    assert np.all(np.abs(dx - dx_ref) <= 16 * m * EPS64 * dx_bound)


@pytest.mark.parametrize("mode", ["feasible", "infeasible"])
def test_step_lengths_match_oracle_on_a_trajectory(mode):
    torch = torch_cuda()
    lp = lpgen.planted_dense(10, 3000, seed=15)
    opt = ipm.Options(mode=mode, solver="sketch", s=2, w=40, keep_vectors=True, k_max=25)
    if mode == "feasible":
        x0, y0, s0 = lpgen.feasible_start(lp, opt.gamma)
        res = ipm.solve(lp.A, lp.b, lp.c, opt, x0, y0, s0)
    else:
        res = ipm.solve(lp.A, lp.b, lp.c, opt)
    V0 = res.history[0].vectors
    r0 = np.sqrt(V0["r_p"] @ V0["r_p"] + V0["r_d"] @ V0["r_d"])
    mu0 = res.history[0].mu
    with solver_for(lp) as S:
        for rec in res.history[:-1]:
            V = rec.vectors
            rr = 0.0 if mode == "feasible" else np.sqrt(V["r_p"] @ V["r_p"] + V["r_d"] @ V["r_d"]) / r0
            am, ab = S.step_lengths(dev(torch, V["x"]), dev(torch, V["s"]), dev(torch, V["dx"]),
                                    dev(torch, V["ds"]), mode, rr, mu0)
            assert am == pytest.approx(rec.alpha_max, rel=1e-9, abs=1e-12)
            assert ab == pytest.approx(rec.alpha_bar, rel=1e-9, abs=1e-12)


def test_step_lengths_hand_built():
    # two elements: element 0 exits N(gamma) at alpha = 1/2 by construction
    torch = torch_cuda()
    lp = lpgen.planted_dense(2, 64, seed=16)
    n = lp.n
    x = np.ones(n)
    s = np.ones(n)
    dx = np.zeros(n)
    ds = np.zeros(n)
    dx[0] = -1.0   # x_0 s_0 = 1 - a; mu(a) = (n - a)/n; exit where 1 - a = (1-g)(n-a)/n
    g = 0.999
    with solver_for(lp, gamma=g) as S:
        am, ab = S.step_lengths(dev(torch, x), dev(torch, s), dev(torch, dx), dev(torch, ds),
                                "feasible", 0.0, 1.0)
    expect = (1 - (1 - g)) / (1 - (1 - g) / n)
    assert am == pytest.approx(min(1.0, expect), rel=1e-12)
    assert ab == pytest.approx(am)
