"""Parity at the full sizes of the workloads: the 512 x 131072 FP32 planted LP
with columns scaled by 10^U(-2, 2) (seed 0) with its solver options
(CountSketch w = 4m, s = 4); the 2048 x 524288 BF16 LP (CountSketch w = 4m,
s = 4), which the bench times; the 4096 x 2,000,000 sparse LP (w = 3m, s = 2).  The oracle checks every output of the
product (one FP64 matrix product), sampled columns of the sketch (one bucket
at a time, from the oracle's own hash), and the solve against the planted
closed-form optimum.

Tolerances as in test_gpu_kernels: the FP32 product to 4 (m + L + 64) 2^-24
times |A| D^2 |A|^T |v| (L = n / 1216 + 64 columns summed in FP32 per warp),
the double-float product to 8 (m + n) 2^-53 times the same bound, the
double-float sketch to (32 n s / w + 64) 2^-48 times |A D| |W|.
"""

import json
import os

import numpy as np
import pytest

import lpgen
from oracle import sketch
from tests.gpu_helpers import EPS32, EPS64, adat_bound, dev, fp32_lane_columns, host, solver_for, torch_cuda

pytestmark = pytest.mark.gpu

M, N, S_BLOCKS, W_FACTOR = 512, 131072, 4, 4.0
DF_U = 2.0 ** -48


def _oracle_objective(name, lp):
    """The objective of the CPU oracle's own whole solve of this very LP,
    written by tests/golden/make_oracle_records.py (which calls only the
    oracle)."""
    rec = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "oracle_solves.json")))[name]
    assert (rec["m"], rec["n"], rec["seed"]) == (lp.m, lp.n, 0)
    assert abs(rec["planted_objective"] - lp.objective) <= 1e-9 * (1 + abs(lp.objective))
    return rec["objective"]


@pytest.fixture(scope="module")
def bench_lp():
    return lpgen.planted_dense(M, N, seed=0, storage="f32", col_scale_log10=(-2.0, 2.0))


@pytest.mark.parametrize("precision", [0, 1])
def test_full_size_product_matches_fp64(bench_lp, precision):
    torch = torch_cuda()
    lp = bench_lp
    rng = np.random.default_rng(11)
    d2 = np.exp(rng.uniform(-6, 6, N))
    v = rng.standard_normal(M)
    ref = lp.A @ (d2 * (lp.A.T @ v))
    with solver_for(lp, s=S_BLOCKS, w_factor=W_FACTOR) as S:
        u = host(S.adat(dev(torch, d2), dev(torch, v), precision))
    bound = adat_bound(lp.A, d2, v)
    if precision == 1:
        tol = 8 * (M + N) * EPS64 * bound
    else:
        tol = 4 * (M + N // 1216 + 64 + 64) * EPS32 * bound
    assert np.all(np.abs(u - ref) <= tol), np.max(np.abs(u - ref) / bound)


def test_full_size_countsketch_sampled_columns(bench_lp):
    torch = torch_cuda()
    lp = bench_lp
    rng = np.random.default_rng(12)
    D = np.exp(rng.uniform(-3, 3, N))
    seed, k, retry = 0, 5, 0
    with solver_for(lp, s=S_BLOCKS, w_factor=W_FACTOR) as S:
        w = S.sketch_width
        adw = host(S.sketch(dev(torch, D), seed, k, retry))
    assert adw.shape == (M, w)
    cols, signs = sketch.countsketch_hash(seed, k, retry, N, w, S_BLOCKS)
    eps = max(8 * N * EPS64, (32 * N * S_BLOCKS / w + 64) * DF_U)
    for bucket in rng.choice(w, 24, replace=False):
        b = bucket // (w // S_BLOCKS)  # the block this sketch column belongs to
        members = np.nonzero(cols[b] == bucket)[0]
        scale = signs[b, members] * D[members] / np.sqrt(S_BLOCKS)
        ref = lp.A[:, members] @ scale
        bound = np.abs(lp.A[:, members]) @ np.abs(scale)
        assert np.all(np.abs(adw[:, bucket] - ref) <= eps * bound + 1e-300), bucket


def test_full_size_solve_reaches_the_planted_optimum(bench_lp):
    torch_cuda()
    lp = bench_lp
    with solver_for(lp, s=S_BLOCKS, w_factor=W_FACTOR) as S:
        x, y, s, info = S.solve(tol=1e-8)
    assert info["status"] == 0, info
    assert info["rel_gap"] <= 1e-8 and info["rp_rel"] <= 1e-8 and info["rd_rel"] <= 1e-8
    assert abs(float(lp.c @ x) - lp.objective) <= 1e-7 * (1 + abs(lp.objective))
    o = _oracle_objective("c2", lp)
    assert abs(float(lp.c @ x) - o) <= 1e-7 * (1 + abs(o))
    assert np.all(x > 0) and np.all(s > 0)
    # the planted support is identified: the m largest x_j are the basic columns
    basis = np.nonzero(lp.x_star > 0)[0]
    assert set(np.argsort(-x)[:M]) == set(basis)


# ---- the sparse configuration at its full size --------------------------------

def test_c3_full_size_sparse_product_matches_fp64():
    torch = torch_cuda()
    # c3: CSC 4096 x 2,000,000, 8 nonzeros per column, 20 % Zipf rows, w = 3m, s = 2
    lp = lpgen.config_small("c3", 1)
    A = lp.scipy_csc()
    rng = np.random.default_rng(14)
    d2 = np.exp(rng.uniform(-5, 5, lp.n))
    v = rng.standard_normal(lp.m)
    ref = A @ (d2 * (A.T @ v))
    absA = abs(A)
    bound = absA @ (d2 * (absA.T @ np.abs(v)))
    with solver_for(lp, s=2, w_factor=3.0) as S:
        u = host(S.adat(dev(torch, d2), dev(torch, v), 0))
    per_cta = lp.n // 304 + 1
    tol = 4 * (8 + per_cta + 64) * EPS32 * bound
    assert np.all(np.abs(u - ref) <= tol + 1e-300)


# ---- the other full-size workloads ----------------------------------------------

def _blocked_product(lp, d2, v, block=32768):
    """A (d2 o (A^T v)) and |A| (d2 o (|A|^T |v|)) in FP64 from the stored
    values, one column block at a time (the FP64 copy of a 10^9-entry A would
    take 8.6 GB)."""
    u = np.zeros(lp.m)
    bound = np.zeros(lp.m)
    cols = lp.storage_array()
    for j0 in range(0, lp.n, block):
        blk = cols[j0:j0 + block]
        if lp.storage == "bf16":
            blk = (blk.astype(np.uint32) << np.uint32(16)).view(np.float32)
        blk = blk.astype(np.float64)                     # (cols, m) = A[:, j0:j1]^T
        u += blk.T @ (d2[j0:j0 + block] * (blk @ v))
        ab = np.abs(blk)
        bound += ab.T @ (d2[j0:j0 + block] * (ab @ np.abs(v)))
    return u, bound


@pytest.fixture(scope="module")
def c4_lp():
    return lpgen.make(lpgen.CONFIGS["c4"])


@pytest.mark.parametrize("precision", [0, 1])
def test_c4_full_size_product_matches_fp64(c4_lp, precision):
    # 2048 x 524288 BF16 (2.1 GB): the row-split kernels, every output
    torch = torch_cuda()
    lp = c4_lp
    rng = np.random.default_rng(15)
    d2 = np.exp(rng.uniform(-6, 6, lp.n))
    v = rng.standard_normal(lp.m)
    ref, bound = _blocked_product(lp, d2, v)
    cfg = lpgen.CONFIGS["c4"]
    with solver_for(lp, s=cfg["s"], w_factor=cfg["w_factor"]) as S:
        u = host(S.adat(dev(torch, d2), dev(torch, v), precision))
    if precision == 1:
        tol = 8 * (lp.m + lp.n) * EPS64 * bound
    else:
        tol = 4 * (lp.m + fp32_lane_columns(lp.m, lp.n, "bf16") + 64) * EPS32 * bound
    assert np.all(np.abs(u - ref) <= tol), np.max(np.abs(u - ref) / bound)


def test_c4_full_size_solve_reaches_the_planted_optimum(c4_lp):
    # BF16 storage, FP32 products, FP64-class refinement; CountSketch w = 4m, s = 4
    torch_cuda()
    lp = c4_lp
    cfg = lpgen.CONFIGS["c4"]
    with solver_for(lp, s=cfg["s"], w_factor=cfg["w_factor"]) as S:
        x, y, s, info = S.solve(tol=1e-8)
    assert info["status"] == 0, info
    assert info["rel_gap"] <= 1e-8 and info["rp_rel"] <= 1e-8 and info["rd_rel"] <= 1e-8
    assert abs(float(lp.c @ x) - lp.objective) <= 1e-7 * (1 + abs(lp.objective))
    assert abs(float(lp.b @ y) - lp.objective) <= 1e-7 * (1 + abs(lp.objective))
    o = _oracle_objective("c4", lp)
    assert abs(float(lp.c @ x) - o) <= 1e-7 * (1 + abs(o))
    assert np.all(x > 0) and np.all(s > 0)
    basis = np.nonzero(lp.x_star > 0)[0]
    assert set(np.argsort(-x)[:lp.m]) == set(basis)


def test_c3_full_size_sparse_countsketch_sampled_columns():
    # the reproducible sparse sketch (entries of each bucket gathered in column
    # order, sorted by row, summed per row) at 4096 x 2,000,000, w = 3m, s = 2:
    # sampled buckets against the oracle's hash, and two calls bit for bit
    torch = torch_cuda()
    lp = lpgen.config_small("c3", 1)
    A = lp.scipy_csc()
    rng = np.random.default_rng(16)
    D = np.exp(rng.uniform(-3, 3, lp.n))
    seed, k, retry, s_blocks = 3, 4, 0, 2
    with solver_for(lp, s=s_blocks, w_factor=3.0) as S:
        w = S.sketch_width
        adw = host(S.sketch(dev(torch, D), seed, k, retry))
        again = host(S.sketch(dev(torch, D), seed, k, retry))
    assert np.array_equal(adw.view(np.uint64), again.view(np.uint64))
    cols, signs = sketch.countsketch_hash(seed, k, retry, lp.n, w, s_blocks)
    for bucket in rng.choice(w, 16, replace=False):
        b = bucket // (w // s_blocks)
        members = np.nonzero(cols[b] == bucket)[0]
        scale = signs[b, members] * D[members] / np.sqrt(s_blocks)
        sub = A[:, members]
        ref = sub @ scale
        bound = abs(sub) @ np.abs(scale)
        nnz_col = int(np.diff(A.indptr)[members].max()) if len(members) else 1
        eps = 4 * (len(members) * nnz_col + 8) * EPS64
        assert np.all(np.abs(adw[:, bucket] - ref) <= eps * bound + 1e-300), bucket


def test_c4_full_size_countsketch_sampled_columns(c4_lp):
    # the bucket kernel (whole 2048-row BF16 columns by bulk copy, double-float
    # sums) at 2048 x 524288, w = 4m, s = 4: sampled buckets against the
    # oracle's hash; two calls bit for bit
    torch = torch_cuda()
    lp = c4_lp
    cfg = lpgen.CONFIGS["c4"]
    rng = np.random.default_rng(17)
    D = np.exp(rng.uniform(-3, 3, lp.n))
    seed, k, retry = 0, 6, 0
    with solver_for(lp, s=cfg["s"], w_factor=cfg["w_factor"]) as S:
        w = S.sketch_width
        adw = host(S.sketch(dev(torch, D), seed, k, retry))
        again = host(S.sketch(dev(torch, D), seed, k, retry))
    assert adw.shape == (lp.m, w)
    assert np.array_equal(adw.view(np.uint64), again.view(np.uint64))
    cols, signs = sketch.countsketch_hash(seed, k, retry, lp.n, w, cfg["s"])
    store = lp.storage_array()
    eps = max(8 * lp.n * EPS64, (32 * lp.n * cfg["s"] / w + 64) * DF_U)
    for bucket in rng.choice(w, 12, replace=False):
        b = bucket // (w // cfg["s"])
        members = np.nonzero(cols[b] == bucket)[0]
        blk = (store[members].astype(np.uint32) << np.uint32(16)).view(np.float32).astype(np.float64)  # (cols, m)
        scale = signs[b, members] * D[members] / np.sqrt(cfg["s"])
        ref = blk.T @ scale
        bound = np.abs(blk).T @ np.abs(scale)
        assert np.all(np.abs(adw[:, bucket] - ref) <= eps * bound + 1e-300), bucket


def test_c3_full_size_solve_from_csr_reaches_the_planted_objective():
    # 4096 x 2,000,000 with 16 M nonzeros, given as CSR (the configured format):
    # lp_create sorts it into exactly the CSC the generator built (checked on
    # the host with the same sort), and the solve reaches the planted
    # objective; A_B may be singular (empty rows), so only the objective and
    # the residuals are compared (several optimal x may exist).  Every sparse
    # kernel sums in a fixed order, so the CSR and CSC solves agree bit for bit.
    torch_cuda()
    import scipy.sparse as sp
    from paper_2209_08722_gb300 import LPSolver, csr_to_csc
    lp = lpgen.config_small("c3", 1)
    vals = lp.val.astype(np.float32)
    csr = sp.csc_matrix((vals, lp.row_idx, lp.col_ptr), shape=(lp.m, lp.n)).tocsr()
    rp, ci = csr.indptr.astype(np.int64), csr.indices.astype(np.int32)
    cp, ri, vo = csr_to_csc(rp, ci, csr.data, lp.m, lp.n, "f32")
    assert np.array_equal(cp, lp.col_ptr) and np.array_equal(ri, lp.row_idx) and np.array_equal(vo, vals)
    opts = dict(s=2, w_factor=3.0)
    with LPSolver(None, lp.b, lp.c, lp.m, lp.n, dtype="f32", csr=(rp, ci, csr.data), **opts) as S:
        x, y, s, info = S.solve(tol=1e-8)
    assert info["status"] == 0, info
    assert info["rel_gap"] <= 1e-8 and info["rp_rel"] <= 1e-8 and info["rd_rel"] <= 1e-8
    assert abs(float(lp.c @ x) - lp.objective) <= 1e-7 * (1 + abs(lp.objective))
    assert abs(float(lp.b @ y) - lp.objective) <= 1e-7 * (1 + abs(lp.objective))
    o = _oracle_objective("c3", lp)
    assert abs(float(lp.c @ x) - o) <= 1e-7 * (1 + abs(o))
    assert np.all(x > 0) and np.all(s > 0)
    with solver_for(lp, **opts) as S:
        x2, y2, _, info2 = S.solve(tol=1e-8)
    assert info2["status"] == 0
    assert np.array_equal(x2, x) and np.array_equal(y2, y)
