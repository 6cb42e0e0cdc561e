"""Parity of the CSC (sparse A) path with the CPU oracle, through the C ABI.

Same rows as tests/test_gpu_kernels.py for a CSC A with a fixed number of
nonzeros per column and heavy-tailed row counts (20% Zipf(1.2) rows).  The
tolerances are the forward-error bounds of the sums in any order; the sums
themselves run in a fixed order (two-pass product, sketch summed per bucket),
so repeated calls and CSR/CSC input agree bit for bit.
"""

import numpy as np
import pytest

import lpgen
from oracle import ipm, sketch
from tests.gpu_helpers import EPS32, EPS64, dev, host, solver_for, torch_cuda

pytestmark = pytest.mark.gpu

SHAPES = [(64, 5000, 8), (300, 20011, 8), (37, 3001, 5)]


def _lp(m, n, k, seed=0):
    return lpgen.planted_sparse(m, n, nnz_per_col=k, seed=seed, storage="f32")


@pytest.mark.parametrize("m,n,k", SHAPES)
@pytest.mark.parametrize("precision", [0, 1])
def test_sparse_adat(m, n, k, precision):
    torch = torch_cuda()
    lp = _lp(m, n, k)
    A = lp.scipy_csc()
    rng = np.random.default_rng(1)
    d2 = np.exp(rng.uniform(-5, 5, n))
    v = rng.standard_normal(m)
    ref = A @ (d2 * (A.T @ v))
    absA = abs(A)
    bound = absA @ (d2 * (absA.T @ np.abs(v)))
    with solver_for(lp) as S:
        u = host(S.adat(dev(torch, d2), dev(torch, v), precision))
    eps = EPS64 if precision else EPS32
    # dot of k terms, then a sum over the columns of one CTA and the CTA tree
    per_cta = n // 304 + 1
    tol = 4 * (k + per_cta + 64) * eps * bound
    assert np.all(np.abs(u - ref) <= tol + 1e-300)


@pytest.mark.parametrize("mode", ["infeasible", "feasible"])
def test_sparse_residual_rhs_and_directions(mode):
    torch = torch_cuda()
    m, n, k = 64, 5000, 8
    lp = _lp(m, n, k, seed=2)
    A = lp.dense()
    rng = np.random.default_rng(3)
    x = np.exp(rng.uniform(-3, 3, n))
    s = np.exp(rng.uniform(-3, 3, n))
    y = rng.standard_normal(m)
    feas = mode == "feasible"
    rp_ref, rd_ref = ipm.residuals(A, lp.b, lp.c, x, y, s)
    mu = x @ s / n
    p_ref = ipm.rhs(A, x, s, rp_ref, np.zeros(n) if feas else rd_ref, 0.5, mu, feas)
    with solver_for(lp) as S:
        rp, rd, p, sc = S.residual_rhs(dev(torch, x), dev(torch, y), dev(torch, s), mode)
        rp, rd, p = host(rp), host(rd), host(p)
        dy = rng.standard_normal(m)
        v = 1e-3 * rng.standard_normal(n)
        dx, ds = S.directions(dev(torch, x), dev(torch, s), dev(torch, rd_ref), dev(torch, dy),
                              dev(torch, v), mu, mode)
        dx, ds = host(dx), host(ds)
    ax = np.abs(A)
    assert np.all(np.abs(rp - rp_ref) <= 64 * n * EPS64 * (ax @ x + np.abs(lp.b)))
    assert np.all(np.abs(rd - rd_ref) <= 16 * k * EPS64 * (ax.T @ np.abs(y) + s + np.abs(lp.c)))
    t_abs = x + 0.5 * mu / s + (0 if feas else (x / s) * np.abs(rd_ref))
    assert np.all(np.abs(p - p_ref) <= 64 * n * EPS64 * (ax @ t_abs + ax @ x + np.abs(lp.b)))
    dx_ref, ds_ref = ipm.directions(A, x, s, np.zeros(n) if feas else rd_ref, dy, v, 0.5, mu, feas)
    ds_bound = ax.T @ np.abs(dy) + (0 if feas else np.abs(rd_ref))
    assert np.all(np.abs(ds - ds_ref) <= 16 * k * EPS64 * ds_bound)
    assert np.all(np.abs(dx - dx_ref) <= 32 * k * EPS64 * (x + 0.5 * mu / s + (x / s) * ds_bound + np.abs(v) / s))


@pytest.mark.parametrize("m,n,k,s_blocks,w_factor", [
    (64, 5000, 8, 2, 4.0), (300, 20011, 8, 3, 4.0),
    # buckets of ~10^4 entries: above the per-bucket sort capacity (FP64 atomics)
    (16, 20000, 8, 1, 1.0)])
def test_sparse_countsketch(m, n, k, s_blocks, w_factor):
    torch = torch_cuda()
    lp = _lp(m, n, k, seed=4)
    rng = np.random.default_rng(5)
    D = np.exp(rng.uniform(-3, 3, n))
    with solver_for(lp, s=s_blocks, w_factor=w_factor) as S:
        w = S.sketch_width
        adw = host(S.sketch(dev(torch, D), 99, 3, 0))
        again = host(S.sketch(dev(torch, D), 99, 3, 0))
    W = sketch.countsketch_matrix(99, 3, 0, n, w, s_blocks)
    AD = lp.scipy_csc().multiply(D[None, :]).tocsc()
    ref = (AD @ W).toarray()
    bound = (abs(AD) @ abs(W)).toarray()
    assert np.all(np.abs(adw - ref) <= 16 * n * EPS64 * bound + 1e-300)
    if w_factor > 1.0:
        # buckets within the sort capacity are summed in a fixed order
        assert np.array_equal(adw.view(np.uint64), again.view(np.uint64))


def test_sparse_solve_from_csr_equals_csc_bit_for_bit():
    # the CSR input is sorted into the CSC the generator built, and every
    # sparse kernel (products, passes, sketch) sums in a fixed order
    torch_cuda()
    import scipy.sparse as sp
    from paper_2209_08722_gb300 import LPSolver
    lp = _lp(128, 30011, 8, seed=9)
    vals = lp.val.astype(np.float32)
    csr = sp.csc_matrix((vals, lp.row_idx, lp.col_ptr), shape=(lp.m, lp.n)).tocsr()
    rp, ci = csr.indptr.astype(np.int64), csr.indices.astype(np.int32)
    with LPSolver(None, lp.b, lp.c, lp.m, lp.n, dtype="f32", csr=(rp, ci, csr.data), s=2) as S:
        x1, y1, _, i1 = S.solve(tol=1e-8)
    with solver_for(lp, s=2) as S:
        x2, y2, _, i2 = S.solve(tol=1e-8)
    assert i1["status"] == i2["status"] == 0
    assert i1["inner_total"] == i2["inner_total"]
    assert np.array_equal(x1, x2) and np.array_equal(y1, y2)


def test_sparse_normal_solve_matches_cholesky():
    m, n, k = 96, 12000, 8
    lp = _lp(m, n, k, seed=6)
    A = lp.dense()
    rng = np.random.default_rng(7)
    D = np.exp(rng.uniform(-2, 2, n))
    p = rng.standard_normal(m)
    M = (A * D * D) @ A.T
    exact = np.linalg.solve(M, p)
    with solver_for(lp, s=2) as S:
        tol_f = 1e-11 * np.linalg.norm(p) / np.sqrt(np.linalg.eigvalsh(M)[-1])
        dy, _, info = S.normal_solve(D, p, k=0, tol_f=tol_f)
    assert np.linalg.norm(dy - exact) <= 1e-7 * np.linalg.norm(exact)


@pytest.mark.parametrize("m,n", [(128, 62500), (256, 20000)])
def test_sparse_solve_planted(m, n):
    # A_B may be singular for a sparse planted LP: compare objectives (the
    # optimal value is unique even where the optimal x is not)
    lp = lpgen.planted_sparse(m, n, nnz_per_col=8, seed=8, storage="f32")
    with solver_for(lp, s=2, w_factor=3.0) as S:
        x, y, s, info = S.solve(tol=1e-8)
    assert info["status"] == 0, info
    obj = float(lp.c @ x)
    assert abs(obj - lp.objective) <= 1e-7 * (1 + abs(lp.objective))
    A = lp.scipy_csc()
    assert np.linalg.norm(A @ x - lp.b) <= 1.01e-8 * (1 + np.linalg.norm(lp.b))
    assert np.linalg.norm(A.T @ y + s - lp.c) <= 1.01e-8 * (1 + np.linalg.norm(lp.c))
