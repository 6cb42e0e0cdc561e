"""Gaussian-sketch variant (Section 6): parity with the oracle's W_G.

The CUDA path draws W_G on the fly with the same counter-based generator and
the same FP32-exact uniforms as oracle.sketch.gaussian_matrix; it differs only
in the rounding of log/cos (FP32 on the GPU) and in folding D into W in FP32,
so the entries agree to a few FP32 ulps.  The product runs either as an FP32
SIMT GEMM or on the tensor cores (tcgen05, TF32 with both operands split in a
high and a low TF32 part); both must keep FP32 accuracy.
"""

import numpy as np
import pytest

import lpgen
from oracle import correction, ipm, pcg, sketch
from tests.gpu_helpers import EPS32, dev, host, solver_for, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("m,n,storage,tensor", [
    (64, 4099, "f32", 0), (200, 9000, "f32", 0), (37, 3001, "bf16", 0), (48, 2000, "f64", 0),
    (64, 4099, "f32", 1), (200, 9000, "f32", 1), (37, 3001, "bf16", 1), (300, 5003, "f32", 1),
    (512, 6007, "f32", 1), (130, 2500, "bf16", 1), (600, 3000, "f32", 1)])
def test_gaussian_sketch_matches_oracle(m, n, storage, tensor):
    torch = torch_cuda()
    lp = lpgen.planted_dense(m, n, seed=31, storage=storage, col_scale_log10=(-1, 1))
    rng = np.random.default_rng(32)
    D = np.exp(rng.uniform(-3, 3, n))
    with solver_for(lp, sketch=1, tensor_sketch=tensor) as S:
        w = S.sketch_width
        adw = host(S.sketch(dev(torch, D), 77, 4, 1))
    W = sketch.gaussian_matrix(77, 4, 1, n, w)
    AD = lp.A * D
    ref = AD @ W
    bound = np.abs(AD) @ np.abs(W)
    if tensor and storage != "f64":
        # split operands: 3 * 2^-22 per product; tensor-core FP32 accumulation
        # (rounding mode unspecified): 2^-23 per step over at most n steps
        tol = (16 * EPS32 + 2 * (n + 8) * EPS32 + 64 * EPS32) * bound
    else:
        kper = max(1, n // 64) if n > 4096 * 64 else 4096
        tol = (64 * EPS32 + (min(n, kper) + 64) * EPS32) * bound
    assert np.all(np.abs(adw - ref) <= tol)
    # in norm the error must be at FP32 level: dropping the low TF32 part of
    # either operand leaves ~2^-12 / sqrt(n) of the bound, above this threshold
    assert np.linalg.norm(adw - ref) <= 8 * EPS32 * np.linalg.norm(bound)


def test_gaussian_tensor_and_simt_wide_range():
    # columns scaled by 10^U(-2, 2) and D by e^U(-2, 2): the sums cancel, so the
    # error is measured against the magnitude of the terms, |A D| |W|
    torch = torch_cuda()
    m, n = 256, 20000
    lp = lpgen.planted_dense(m, n, seed=36, storage="f32", col_scale_log10=(-2, 2))
    D = np.exp(np.random.default_rng(37).uniform(-2, 2, n))
    out = []
    for tensor in (0, 1):
        with solver_for(lp, sketch=1, tensor_sketch=tensor) as S:
            w = S.sketch_width
            out.append(host(S.sketch(dev(torch, D), 5, 1, 0)))
    W = sketch.gaussian_matrix(5, 1, 0, n, w)
    AD = lp.A * D
    ref = AD @ W
    scale = np.linalg.norm(np.abs(AD) @ np.abs(W))
    errs = [np.linalg.norm(o - ref) / scale for o in out]
    assert max(errs) <= 8 * EPS32, errs


def test_gaussian_normal_solve_and_correction():
    m, n = 48, 6000
    lp = lpgen.planted_dense(m, n, seed=33, storage="f32")
    rng = np.random.default_rng(34)
    x = np.exp(rng.uniform(-2, 2, n))
    s = np.exp(rng.uniform(-2, 2, n))
    D = np.sqrt(x / s)
    p = rng.standard_normal(m)
    M = (lp.A * D * D) @ lp.A.T
    exact = np.linalg.solve(M, p)
    with solver_for(lp, sketch=1, t_max=4) as S:
        dy, v, info = S.normal_solve(D, p, xs=x * s, k=2, tol_f=1e-300)
    assert info["inner_iterations"] == 4
    # t = 4 CG steps: the same iterate as the oracle's CG on eq. (precond_alt)
    opt = ipm.Options(solver="sketch", sketch="gaussian", w=4 * m, t_max=4)
    ref = ipm.normal_solve(lp.A, x, s, p, opt, k=2, inner_tol=0.0)
    assert np.linalg.norm(dy - ref.dy) <= 1e-4 * np.linalg.norm(ref.dy)
    # v and the invariant of eq. (addl), A S^{-1} v = A D^2 A^T dy - p
    r_v = lp.A @ ((x / s) * (lp.A.T @ dy)) - p
    assert np.linalg.norm(lp.A @ (v / s) - r_v) <= 1e-5 * np.linalg.norm(r_v)
    v_ref = correction.correction_v(x, s, sketch.gaussian_matrix(0, 2, 0, n, 4 * m), ref.ADW, r_v)
    assert np.linalg.norm(v - v_ref) <= 1e-5 * np.linalg.norm(v_ref)
    del exact


def test_gaussian_lp_solve():
    lp = lpgen.planted_dense(64, 8000, seed=35, storage="f32", col_scale_log10=(-1, 1))
    with solver_for(lp, sketch=1) as S:
        x, y, s, info = S.solve(tol=1e-8)
    assert info["status"] == 0, info
    assert abs(lp.c @ x - lp.objective) <= 1e-7 * (1 + abs(lp.objective))
    assert np.linalg.norm(lp.A @ x - lp.b) <= 1.01e-8 * (1 + np.linalg.norm(lp.b))
