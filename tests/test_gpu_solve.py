"""End-to-end parity of lp_solve (Algorithms 2 and 3 on the GPU) with the CPU
oracle and the planted closed-form optimum.

Bar: relative duality gap <= 1e-8 and FP64 objective agreement <= 1e-7 with
the oracle and with c^T x*.
"""

import numpy as np
import pytest

import lpgen
from oracle import ipm
from tests.gpu_helpers import dev, host, solver_for, torch_cuda

pytestmark = pytest.mark.gpu


def _check(lp, x, y, s, info, ref=None):
    assert info["status"] == 0, info
    assert info["rel_gap"] <= 1e-8
    obj = float(lp.c @ x)
    assert abs(obj - lp.objective) <= 1e-7 * (1 + abs(lp.objective)), (obj, lp.objective)
    assert abs(obj - float(lp.b @ y)) <= 1e-8 * (1 + abs(obj)) * 1.01
    assert (x > 0).all() and (s > 0).all()
    A = lp.dense()
    assert np.linalg.norm(A @ x - lp.b) <= 1e-8 * (1 + np.linalg.norm(lp.b)) * 1.01
    assert np.linalg.norm(A.T @ y + s - lp.c) <= 1e-8 * (1 + np.linalg.norm(lp.c)) * 1.01
    if ref is not None:
        assert abs(obj - float(lp.c @ ref.x)) <= 1e-7 * (1 + abs(obj))


@pytest.mark.parametrize("name,div", [("c2", 8), ("c2", 32), ("c4", 16), ("c1", 1)])
def test_infeasible_solve_small_configs(name, div):
    lp = lpgen.config_small(name, div)
    cfg = lpgen.CONFIGS[name]
    ref = ipm.solve(lp.dense(), lp.b, lp.c, ipm.Options(mode="infeasible"))
    with solver_for(lp, s=cfg["s"], w_factor=cfg["w_factor"]) as S:
        x, y, s, info = S.solve(tol=1e-8, mode="infeasible")
    _check(lp, x, y, s, info, ref)
    # outer iterations close to the exact-solve oracle (inexact solve + v)
    assert abs(info["outer_iterations"] - ref.iterations) <= max(3, 0.2 * ref.iterations)


def test_feasible_solve_c1_fp64():
    lp = lpgen.planted_dense(64, 4096, seed=0, storage="f64")
    x0, y0, s0 = lpgen.feasible_start(lp, gamma=0.999)
    ref = ipm.solve(lp.A, lp.b, lp.c, ipm.Options(mode="feasible"), x0, y0, s0)
    with solver_for(lp, s=2) as S:
        x, y, s, info = S.solve(tol=1e-8, mode="feasible", x0=x0, y0=y0, s0=s0)
    _check(lp, x, y, s, info, ref)


def test_solve_with_device_buffers_and_chebyshev():
    torch = torch_cuda()
    lp = lpgen.planted_dense(96, 12000, seed=3, storage="f32", col_scale_log10=(-1, 1))
    with solver_for(lp, s=2, inner=1) as S:
        x, y, s, info = S.solve(tol=1e-8, x0=dev(torch, np.ones(lp.n)),
                                y0=dev(torch, np.zeros(lp.m)), s0=dev(torch, np.ones(lp.n)))
    _check(lp, host(x), host(y), host(s), info)


def test_solve_without_v_correction_table2():
    # Table 2 ablation: without v the iteration still drives mu and the duality
    # gap down by many orders; the primal residual is then no longer corrected
    # and settles at the inexact-solve level (the CPU oracle shows the same), so
    # the 1e-8 residual test is not asserted here.
    lp = lpgen.planted_dense(64, 8000, seed=5, storage="f32")
    with solver_for(lp, s=2, v_correction=0, k_max=60) as S:
        x, y, s, info = S.solve(tol=1e-8)
        hist = S.history()
    assert info["status"] in (0, 1, 3)
    assert min(h["mu"] for h in hist) <= 1e-8 * hist[0]["mu"]
    assert min(h["rel_gap"] for h in hist) <= 1e-3


def test_solve_is_deterministic():
    lp = lpgen.planted_dense(128, 10000, seed=6, storage="f32", col_scale_log10=(-1, 1))
    with solver_for(lp, s=2) as S:
        x1, y1, _, i1 = S.solve(tol=1e-8)
        x2, y2, _, i2 = S.solve(tol=1e-8)
    assert np.array_equal(x1, x2) and np.array_equal(y1, y2)
    assert i1["inner_total"] == i2["inner_total"]


def test_feasible_mode_rejects_infeasible_start():
    from paper_2209_08722_gb300.solver import LPError
    lp = lpgen.planted_dense(16, 500, seed=7, storage="f64")
    with solver_for(lp) as S:
        with pytest.raises(LPError) as ei:
            S.solve(mode="feasible", x0=np.ones(lp.n), y0=np.zeros(lp.m), s0=np.ones(lp.n))
        assert "NOT_FEASIBLE" in str(ei.value)


def test_create_rejects_bad_arguments():
    from paper_2209_08722_gb300 import LPSolver
    from paper_2209_08722_gb300.solver import LPError
    lp = lpgen.planted_dense(16, 500, seed=8, storage="f32")
    with pytest.raises(LPError) as ei:   # sketch narrower than m
        LPSolver(lp.storage_array(), lp.b, lp.c, lp.m, lp.n, dtype="f32", w=8)
    assert "LP_ERR_ARG" in str(ei.value)
    b = lp.b.copy()
    b[0] = np.nan
    with pytest.raises(LPError):
        LPSolver(lp.storage_array(), b, lp.c, lp.m, lp.n, dtype="f32")
    with pytest.raises(LPError):          # m > n
        LPSolver(np.ones((4, 8), dtype=np.float32), np.ones(8), np.ones(4), 8, 4, dtype="f32")


def test_tiny_lp_matches_vertex_enumeration():
    from oracle import vertex
    lp = lpgen.planted_dense(3, 10, seed=5, storage="f64")
    best, _, _ = vertex.enumerate_vertices(lp.A, lp.b, lp.c)
    with solver_for(lp, s=1) as S:
        x, y, s, info = S.solve(tol=1e-9)
    assert info["status"] == 0
    assert abs(lp.c @ x - best) <= 1e-7 * (1 + abs(best))


def test_standard_ipm_plain_cg_needs_10x_more_inner_steps():
    # Section 7 / Tables 1-2: precondition = 0 is the standard IPM with
    # unpreconditioned CG (Q = I, v = 0); with the experiments' relative inner
    # rule, over the outer iterations the sketched method needs, plain CG
    # takes >= 10x the inner steps on a column-scaled LP
    lp = lpgen.planted_dense(64, 8000, seed=37, storage="f32", col_scale_log10=(-2, 2))
    common = dict(s=2, inner_rule=1, tol_cg=1e-5, t_max=20000)
    with solver_for(lp, k_max=60, **common) as S:
        _, _, _, sk = S.solve(tol=1e-8)
    assert sk["status"] == 0, sk
    with solver_for(lp, precondition=0, k_max=sk["outer_iterations"], **common) as S:
        _, _, _, plain = S.solve(tol=1e-8)
    assert plain["inner_total"] >= 10 * sk["inner_total"], (plain["inner_total"], sk["inner_total"])


def test_w_sweep_inner_iterations_fall_with_w():
    # Figures 2-3 qualitatively: a wider sketch is a better embedding, so the
    # mean inner iteration count falls as w grows (same LP, same outer path)
    lp = lpgen.planted_dense(64, 8000, seed=38, storage="f32", col_scale_log10=(-2, 2))
    means = []
    for wf in (2.0, 4.0, 16.0):
        with solver_for(lp, s=2, w_factor=wf) as S:
            _, _, _, info = S.solve(tol=1e-8)
        assert info["status"] == 0, info
        means.append(info["inner_total"] / info["outer_iterations"])
    assert means[0] > means[1] > means[2], means


def test_autotuned_handles_of_one_shape_take_the_same_kernel():
    # the tuned choice is cached per (dtype, leading dimension, n): a second
    # handle of the same shape computes the same products bit for bit, and the
    # tuned product agrees with the default one to FP32 rounding
    torch = torch_cuda()
    lp = lpgen.planted_dense(300, 40000, seed=23, storage="f32", col_scale_log10=(-1, 1))
    rng = np.random.default_rng(24)
    d2 = dev(torch, np.exp(rng.uniform(-4, 4, lp.n)))
    v = dev(torch, rng.standard_normal(lp.m))
    with solver_for(lp, s=2, autotune=1) as S1, solver_for(lp, s=2, autotune=1) as S2, \
            solver_for(lp, s=2) as S0:
        u1, u2, u0 = host(S1.adat(d2, v, 0)), host(S2.adat(d2, v, 0)), host(S0.adat(d2, v, 0))
    assert np.array_equal(u1, u2)
    assert np.allclose(u1, u0, rtol=1e-4, atol=1e-6 * np.abs(u0).max())


def test_batched_solve_matches_sequential_solves():
    # the batched-LP family (uneven m, n): lp_solve_batch runs the LPs
    # concurrently on their own streams; every LP reaches its planted optimum
    # and the results equal the one-at-a-time solves bit for bit
    # (with the graph path on: blocks of inner steps replayed from CUDA graphs,
    # and the product's tile shape from the autotuner)
    from paper_2209_08722_gb300 import solve_batch
    lps = lpgen.batch_family(6, seed=3, m_range=(32, 160), k_range=(64, 128))
    solvers = [solver_for(lp, s=2, autotune=1) for lp in lps]
    try:
        seq = [S.solve(tol=1e-8) for S in solvers]
        for S in solvers:
            S.reset_kernel_stats()
        bat = solve_batch(solvers, tol=1e-8, max_threads=0)
        replays = [S.kernel_stats()["graph_replays"] for S in solvers]
    finally:
        for S in solvers:
            S.close()
    assert all(r > 0 for r in replays), replays
    for lp, (x1, y1, _, i1), (x2, y2, _, i2) in zip(lps, seq, bat):
        assert i2["status"] == 0, i2
        assert abs(lp.c @ x2 - lp.objective) <= 1e-7 * (1 + abs(lp.objective))
        assert np.array_equal(x1, x2) and np.array_equal(y1, y2)
        assert i1["inner_total"] == i2["inner_total"]


@pytest.mark.parametrize("storage,m,n,inner", [("f32", 128, 20000, 0), ("bf16", 1100, 30000, 0),
                                               ("f32", 96, 12000, 1)])
def test_graph_replayed_blocks_equal_plain_launches(storage, m, n, inner):
    # the same kernels with the same arguments: the solve with every block of
    # inner steps replayed from a CUDA graph equals the one with plain
    # launches bit for bit (warp-per-column and row-split products, CG and
    # Chebyshev)
    lp = lpgen.planted_dense(m, n, seed=17, storage=storage, col_scale_log10=(-1, 1))
    out = {}
    for graphs in (0, 1):
        with solver_for(lp, s=2, graphs=graphs, inner=inner) as S:
            S.reset_kernel_stats()
            out[graphs] = S.solve(tol=1e-8)
            out[graphs] += (S.kernel_stats()["graph_replays"],)
    (x0, y0, s0, i0, r0), (x1, y1, s1, i1, r1) = out[0], out[1]
    assert r0 == 0 and r1 > 0
    assert i1["status"] == 0 and abs(lp.c @ x1 - lp.objective) <= 1e-7 * (1 + abs(lp.objective))
    assert np.array_equal(x0, x1) and np.array_equal(y0, y1) and np.array_equal(s0, s1)
    assert i0["inner_total"] == i1["inner_total"]


@pytest.mark.parametrize("col_scale", [None, (-2, 2)])
def test_two_rhs_adaptive_sigma_matches_oracle_and_cuts_iterations(col_scale):
    # sigma_rule = 1: two right-hand sides on one sketch and Q per outer
    # iteration; the oracle implements the same variant
    from oracle import ipm
    m, n = 48, 3000
    lp = lpgen.planted_dense(m, n, seed=42, storage="f64", col_scale_log10=col_scale)
    ref = ipm.solve(lp.A, lp.b, lp.c, ipm.Options(solver="sketch", sigma_rule="adaptive", w=4 * m, s=2))
    with solver_for(lp, s=2) as S:
        _, _, _, fixed = S.solve(tol=1e-8)
    with solver_for(lp, s=2, sigma_rule=1) as S:
        x, y, s, info = S.solve(tol=1e-8)
        hist = S.history()
    assert info["status"] == 0, info
    assert abs(lp.c @ x - lp.objective) <= 1e-7 * (1 + abs(lp.objective))
    assert info["outer_iterations"] <= 0.7 * fixed["outer_iterations"]
    assert abs(info["outer_iterations"] - ref.iterations) <= 2
    sig = [h["sigma"] for h in hist[:-1]]
    assert min(sig) >= 0.1 - 1e-12 and max(sig) <= 0.75 + 1e-12
    ref_sig = [h.sigma_used for h in ref.history[:-1]]
    k = min(5, len(sig), len(ref_sig))
    assert np.allclose(sig[:k], ref_sig[:k], rtol=1e-3, atol=1e-6)


@pytest.mark.gpu
def test_failed_sketch_draws_are_redrawn_and_inner_solves_stay_short():
    """With s = 2, draws of W whose rows for the basic columns are dependent
    leave PCG with a Ritz spread ~1e6 near the optimum (this LP once needed
    2 x t_max = 1000 steps in one outer iteration); the solver redraws them, so
    every outer iteration ends within a few dozen steps."""
    torch_cuda()
    lp = lpgen.planted_dense(64, 8192, seed=1000, storage="bf16")
    with solver_for(lp, s=2) as S:
        x, y, s, info = S.solve(tol=1e-8)
        assert info["status"] == 0, info
        assert abs(lp.c @ x - lp.objective) <= 1e-7 * (1 + abs(lp.objective))
        assert info["inner_max"] <= 100, info
        assert info["sketch_retries"] >= 1, info


@pytest.mark.gpu
def test_lp_whose_sketches_collapsed_near_the_optimum_is_solved():
    """LP 23 of the batched family (284 x 53,392, s = 2): near mu ~ 1e-10 every
    draw it tried had a singular W_B, kappa(ADW) ~ 1e9 against kappa(AD) ~ 600,
    and the stored Q^{-1} turned indefinite; it stalled at gap 4.3e-8 before
    the redraw and refactor rules."""
    torch_cuda()
    rng = np.random.default_rng(0)
    for _ in range(24):  # the family's sizes, as lpgen.batch_family draws them
        m = int(rng.integers(32, 513))
        k = int(rng.integers(64, 257))
    lp = lpgen.planted_dense(m, m * k, seed=23, storage="f32")
    with solver_for(lp, s=2) as S:
        x, y, s, info = S.solve(tol=1e-8)
        assert info["status"] == 0, info
        assert info["rel_gap"] <= 1e-8
        assert abs(lp.c @ x - lp.objective) <= 1e-7 * (1 + abs(lp.objective))
        assert info["inner_max"] <= 200, info


def test_handles_reuse_cached_device_memory():
    # a destroyed handle's device blocks go to the library's cache and the next
    # handle of the same shape takes them (zeroed again): the solves agree bit
    # for bit, a guarded handle (other block sizes) keeps intact guards, and
    # releasing the cache leaves the library usable
    torch_cuda()
    from paper_2209_08722_gb300 import release_cached_memory
    lp = lpgen.planted_dense(96, 6001, seed=31, storage="f32")
    with solver_for(lp, s=2, guard=0) as S:
        x1, y1, _, i1 = S.solve(tol=1e-8)
    with solver_for(lp, s=2, guard=0) as S:
        x2, y2, _, i2 = S.solve(tol=1e-8)
    assert i1["status"] == i2["status"] == 0
    assert np.array_equal(x1, x2) and np.array_equal(y1, y2)
    with solver_for(lp, s=2, guard=1) as S:
        x3, _, _, _ = S.solve(tol=1e-8)
        assert S.check_guards()[1] == 0
    assert np.array_equal(x1, x3)
    release_cached_memory()
    with solver_for(lp, s=2, guard=0) as S:
        x4, _, _, _ = S.solve(tol=1e-8)
    assert np.array_equal(x1, x4)
