"""lp_adat_noalloc: the product A diag(d2) A^T v for callers that cannot allocate.

Some callers own all device memory themselves (a fixed arena, a serving loop
with a hard memory budget, code that must not call the CUDA allocator
after start-up) and so cannot create a solver handle, which allocates its
workspaces.  lp_adat_noalloc takes the caller's A, d2, v and u and keeps its
scratch in a fixed-size device array inside the library.  This test calls it
through the C ABI twice in a row and compares each result with lp_adat, the
handle-based entry point computing the same product.
"""

import ctypes

import numpy as np
import pytest

import lpgen
from tests.gpu_helpers import EPS32, adat_bound, dev, host, solver_for, torch_cuda

pytestmark = pytest.mark.gpu


def _caller_matrix(torch, lp, storage):
    """Column-major A with a leading dimension that is a multiple of 16 bytes."""
    vec = 4 if storage == "f32" else 8
    ld = (lp.m + vec - 1) // vec * vec
    st = lp.storage_array()                      # (n, m): row j = column a_j
    pad = np.zeros((lp.n, ld), dtype=st.dtype)
    pad[:, :lp.m] = st
    if storage == "bf16":
        pad = pad.view(np.int16)
    return torch.from_numpy(pad).cuda(), ld


@pytest.mark.parametrize("m,n,storage", [(512, 20011, "f32"), (256, 9000, "bf16"), (45, 7777, "f32")])
def test_noalloc_matches_lp_adat_on_two_calls(m, n, storage):
    torch = torch_cuda()
    from paper_2209_08722_gb300 import _native as nat
    lib = nat.load()
    lp = lpgen.planted_dense(m, n, seed=21, storage=storage, col_scale_log10=(-1, 1))
    rng = np.random.default_rng(22)
    d2 = np.exp(rng.uniform(-5, 5, n))
    v = rng.standard_normal(m)
    d2_d, v_d = dev(torch, d2), dev(torch, v)
    with solver_for(lp) as S:
        ref = host(S.adat(d2_d, v_d, 0))
    A_d, ld = _caller_matrix(torch, lp, storage)
    dtype = nat.LP_F32 if storage == "f32" else nat.LP_BF16
    tol = 4 * (m + n // 1216 + 64) * EPS32 * adat_bound(lp.A, d2, v)
    u = torch.empty(m, dtype=torch.float64, device="cuda")
    for _ in range(2):
        u.fill_(float("nan"))
        torch.cuda.synchronize()
        rc = lib.lp_adat_noalloc(ctypes.c_void_p(A_d.data_ptr()), dtype, m, n, ld,
                                 ctypes.c_void_p(d2_d.data_ptr()), ctypes.c_void_p(v_d.data_ptr()),
                                 ctypes.c_void_p(u.data_ptr()), None)
        assert rc == nat.LP_OK
        got = host(u)
        assert np.all(np.isfinite(got))
        assert np.all(np.abs(got - ref) <= 2 * tol + 1e-300)


def test_noalloc_rejects_sizes_beyond_its_scratch_and_bad_layouts():
    torch = torch_cuda()
    from paper_2209_08722_gb300 import _native as nat
    lib = nat.load()
    buf = torch.zeros(16, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(buf.data_ptr())
    # m beyond the largest register tile of the kernel (FP32: 2048 rows)
    assert lib.lp_adat_noalloc(p, nat.LP_F32, 4096, 8, 4096, p, p, p, None) == nat.LP_ERR_ARG
    # leading dimension not a multiple of 16 bytes
    assert lib.lp_adat_noalloc(p, nat.LP_F32, 5, 8, 5, p, p, p, None) == nat.LP_ERR_ARG
    # FP64 storage is not served by this entry point
    assert lib.lp_adat_noalloc(p, nat.LP_F64, 4, 8, 4, p, p, p, None) == nat.LP_ERR_ARG
