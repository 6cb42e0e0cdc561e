"""lp_adat_noalloc: the product A diag(d2) A^T v for callers that cannot allocate.

Some callers own all device memory themselves (a fixed arena, a serving loop
with a hard memory budget, code that must not call the CUDA allocator
after start-up) and so cannot create a solver handle, which allocates its
workspaces.  lp_adat_noalloc takes the caller's A, d2, v and u and keeps its
scratch in a fixed-size device array inside the library.  This test calls it
through the C ABI twice in a row and compares each result, element by
element, with the product in FP64 on the CPU (the plain definition
A (d2 o (A^T v))) at the FP32 rounding bound the other product tests use,
and with lp_adat, the handle-based entry point computing the same product.
Padding rows between m and the leading dimension hold NaN in one case: they
must not reach the result.
"""

import ctypes

import numpy as np
import pytest

import lpgen
from tests.gpu_helpers import EPS32, adat_bound, dev, fp32_lane_columns, host, solver_for, torch_cuda

pytestmark = pytest.mark.gpu


def _caller_matrix(torch, lp, storage, ld=None, fill=0.0):
    """Column-major A with a leading dimension that is a multiple of 16 bytes;
    rows m .. ld-1 of every column hold ``fill``."""
    vec = 4 if storage == "f32" else 8
    ld = ld or (lp.m + vec - 1) // vec * vec
    st = lp.storage_array()                      # (n, m): row j = column a_j
    if storage == "bf16":
        pad = np.full((lp.n, ld), lpgen.bf16_bits(np.array([fill]))[0], dtype=np.uint16)
    else:
        pad = np.full((lp.n, ld), fill, dtype=st.dtype)
    pad[:, :lp.m] = st
    if storage == "bf16":
        pad = pad.view(np.int16)
    return torch.from_numpy(pad).cuda(), ld


def _noalloc(lib, nat, A_d, dtype, m, n, ld, d2_d, v_d, u):
    return lib.lp_adat_noalloc(ctypes.c_void_p(A_d.data_ptr()), dtype, m, n, ld,
                               ctypes.c_void_p(d2_d.data_ptr()), ctypes.c_void_p(v_d.data_ptr()),
                               ctypes.c_void_p(u.data_ptr()), None)


@pytest.mark.parametrize("m,n,storage,ld,fill", [
    (512, 20011, "f32", None, 0.0), (256, 9000, "bf16", None, 0.0), (45, 7777, "f32", None, 0.0),
    (45, 7777, "f32", 48, float("nan")), (250, 5000, "bf16", 264, float("inf")),
    (2048, 3001, "f32", None, 0.0)])
def test_noalloc_matches_fp64_and_lp_adat_on_two_calls(m, n, storage, ld, fill):
    torch = torch_cuda()
    from paper_2209_08722_gb300 import _native as nat
    lib = nat.load()
    lp = lpgen.planted_dense(m, n, seed=21, storage=storage, col_scale_log10=(-1, 1))
    rng = np.random.default_rng(22)
    d2 = np.exp(rng.uniform(-5, 5, n))
    v = rng.standard_normal(m)
    exact = lp.A @ (d2 * (lp.A.T @ v))             # FP64 on the CPU
    d2_d, v_d = dev(torch, d2), dev(torch, v)
    with solver_for(lp) as S:
        handle = host(S.adat(d2_d, v_d, 0))
    A_d, ld = _caller_matrix(torch, lp, storage, ld, fill)
    dtype = nat.LP_F32 if storage == "f32" else nat.LP_BF16
    # FP32 products, FP32 per-lane sums over at most n / 1216 + 64 columns, FP64 beyond
    bound = adat_bound(lp.A, d2, v)
    tol = 4 * (m + n // 1216 + 64) * EPS32 * bound
    tol_handle = 4 * (m + fp32_lane_columns(m, n, storage) + 64) * EPS32 * bound
    u = torch.empty(m, dtype=torch.float64, device="cuda")
    for _ in range(2):
        u.fill_(float("nan"))
        torch.cuda.synchronize()
        assert _noalloc(lib, nat, A_d, dtype, m, n, ld, d2_d, v_d, u) == nat.LP_OK
        got = host(u)
        assert np.all(np.isfinite(got))
        assert np.all(np.abs(got - exact) <= tol + 1e-300)
        assert np.all(np.abs(got - handle) <= tol + tol_handle + 1e-300)


def test_noalloc_rejects_sizes_beyond_its_scratch_and_bad_layouts():
    torch = torch_cuda()
    from paper_2209_08722_gb300 import _native as nat
    lib = nat.load()
    buf = torch.zeros(16, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(buf.data_ptr())
    # a leading dimension beyond the kernel's register tile (FP32: 2048, BF16: 4096)
    assert lib.lp_adat_noalloc(p, nat.LP_F32, 4096, 8, 4096, p, p, p, None) == nat.LP_ERR_ARG
    assert lib.lp_adat_noalloc(p, nat.LP_F32, 2000, 8, 2052, p, p, p, None) == nat.LP_ERR_ARG
    assert lib.lp_adat_noalloc(p, nat.LP_BF16, 4100, 8, 4104, p, p, p, None) == nat.LP_ERR_ARG
    # leading dimension not a multiple of 16 bytes
    assert lib.lp_adat_noalloc(p, nat.LP_F32, 5, 8, 5, p, p, p, None) == nat.LP_ERR_ARG
    # FP64 storage is not served by this entry point
    assert lib.lp_adat_noalloc(p, nat.LP_F64, 4, 8, 4, p, p, p, None) == nat.LP_ERR_ARG
