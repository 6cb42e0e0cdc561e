"""CPU checks of the C ABI's argument errors.

Every case here is rejected before the library makes any CUDA call (the
header promises that for errors in the arguments themselves), so these run
without a GPU: each call returns the documented code, leaves the output
handle NULL and says why in lp_create_error().
"""

import ctypes
import math

import numpy as np
import pytest

from paper_2209_08722_gb300 import _native as nat


@pytest.fixture(scope="module")
def lib():
    from paper_2209_08722_gb300 import build_native
    import os
    if not os.path.exists(build_native.lib_path()):
        build_native.build()
    return nat.load()


M, N = 8, 32
_A = np.ones((N, M), dtype=np.float32)      # column-major m x n: column j = row j here
_B = np.ones(M)
_C = np.ones(N)


def _dense(m=M, n=N, fmt=nat.LP_DENSE_COLMAJOR, dtype=nat.LP_F32, ld=M, val=_A):
    A = nat.LpMatrix()
    A.m, A.n, A.fmt, A.dtype, A.ld, A.on_device = m, n, fmt, dtype, ld, 0
    A.val = val.ctypes.data if val is not None else None
    return A


def _csc(ptr, idx, val, m=M, n=N, dtype=nat.LP_F32):
    A = nat.LpMatrix()
    A.m, A.n, A.fmt, A.dtype, A.on_device = m, n, nat.LP_CSC, dtype, 0
    A.ptr, A.idx, A.val = ptr.ctypes.data, idx.ctypes.data, val.ctypes.data
    A.nnz = int(ptr[-1]) if len(ptr) else 0
    return A


def _csr(ptr, idx, val, m=M, n=N, dtype=nat.LP_F32):
    A = nat.LpMatrix()
    A.m, A.n, A.fmt, A.dtype, A.on_device = m, n, nat.LP_CSR, dtype, 0
    A.ptr, A.idx, A.val = ptr.ctypes.data, idx.ctypes.data, val.ctypes.data
    A.nnz = int(ptr[-1]) if len(ptr) else 0
    return A


def _opts(lib, **kw):
    o = nat.LpOptions()
    lib.lp_options_default(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _create(lib, A, b=_B, c=_C, opt=None):
    h = ctypes.c_void_p(12345)           # must come back NULL
    rc = lib.lp_create(ctypes.byref(h), ctypes.byref(A) if A is not None else None,
                       b.ctypes.data if b is not None else None,
                       c.ctypes.data if c is not None else None, 0,
                       ctypes.byref(opt) if opt is not None else None)
    assert h.value is None, "the handle must be NULL after a failed lp_create"
    return rc, lib.lp_create_error().decode()


def test_options_default_are_the_documented_defaults(lib):
    o = _opts(lib)
    assert (o.sigma, o.gamma, o.tol_cg) == (0.5, 0.999, 1e-5)
    assert (o.inner_rule, o.sketch, o.s, o.inner) == (nat.LP_RULE_THEORY, nat.LP_SKETCH_COUNT, 2, nat.LP_INNER_CG)
    assert (o.refine_every, o.k_max, o.t_max, o.v_correction, o.cheb_lanczos) == (8, 200, 500, 1, 10)
    assert (o.profile, o.w_factor, o.w, o.seed, o.stream) == (0, 4.0, 0, 0, None)
    assert (o.tensor_sketch, o.precondition, o.sigma_rule, o.graphs, o.autotune) == (1, 1, 0, 1, 0)


def test_null_and_shape_errors(lib):
    assert lib.lp_create(None, ctypes.byref(_dense()), _B.ctypes.data, _C.ctypes.data, 0, None) == nat.LP_ERR_ARG
    rc, why = _create(lib, None)
    assert rc == nat.LP_ERR_ARG and "required" in why
    rc, why = _create(lib, _dense(), b=None)
    assert rc == nat.LP_ERR_ARG and "required" in why
    rc, why = _create(lib, _dense(m=N, n=M, ld=N))           # m > n
    assert rc == nat.LP_ERR_ARG and "m <= n" in why
    rc, why = _create(lib, _dense(m=0))
    assert rc == nat.LP_ERR_ARG and "m <= n" in why
    rc, why = _create(lib, _dense(fmt=7))
    assert rc == nat.LP_ERR_ARG and "format" in why
    rc, why = _create(lib, _dense(dtype=3))
    assert rc == nat.LP_ERR_ARG and "dtype" in why
    rc, why = _create(lib, _dense(ld=M - 1))
    assert rc == nat.LP_ERR_ARG and "ld >= m" in why
    rc, why = _create(lib, _dense(val=None))
    assert rc == nat.LP_ERR_ARG and "ld >= m" in why


def test_host_csc_structure_is_checked(lib):
    ptr = np.arange(N + 1, dtype=np.int64)                  # one entry per column
    idx = (np.arange(N) % M).astype(np.int32)
    val = np.ones(N, dtype=np.float32)
    bad_ptr = ptr.copy()
    bad_ptr[5], bad_ptr[6] = 7, 6                           # not monotone
    rc, why = _create(lib, _csc(bad_ptr, idx, val))
    assert rc == nat.LP_ERR_ARG and "monotone" in why
    bad_idx = idx.copy()
    bad_idx[3] = M                                          # row index out of range
    rc, why = _create(lib, _csc(ptr, bad_idx, val))
    assert rc == nat.LP_ERR_ARG and "out of range" in why
    A = _csc(ptr, idx, val)
    A.nnz = N - 1                                           # ptr[n] != nnz
    rc, why = _create(lib, A)
    assert rc == nat.LP_ERR_ARG and "ptr[n]" in why
    rc, why = _create(lib, _csc(ptr, idx, val.astype(np.float32), dtype=nat.LP_BF16))
    assert rc == nat.LP_ERR_UNSUPPORTED and "FP32 or FP64" in why
    rc, why = _create(lib, _csc(ptr, idx, val), opt=_opts(lib, sketch=nat.LP_SKETCH_GAUSS))
    assert rc == nat.LP_ERR_UNSUPPORTED and "dense A only" in why


def test_host_csr_structure_is_checked(lib):
    ptr = np.arange(0, 4 * M + 1, 4, dtype=np.int64)        # four entries per row
    idx = (np.arange(4 * M) * 3 % N).astype(np.int32)
    val = np.ones(4 * M, dtype=np.float32)
    bad_ptr = ptr.copy()
    bad_ptr[2], bad_ptr[3] = 13, 11                         # not monotone
    rc, why = _create(lib, _csr(bad_ptr, idx, val))
    assert rc == nat.LP_ERR_ARG and "monotone" in why
    bad_idx = idx.copy()
    bad_idx[5] = N                                          # column index out of range
    rc, why = _create(lib, _csr(ptr, bad_idx, val))
    assert rc == nat.LP_ERR_ARG and "out of range" in why
    bad_idx[5] = -1
    rc, why = _create(lib, _csr(ptr, bad_idx, val))
    assert rc == nat.LP_ERR_ARG and "out of range" in why
    A = _csr(ptr, idx, val)
    A.nnz = 4 * M - 1                                       # ptr[m] != nnz
    rc, why = _create(lib, A)
    assert rc == nat.LP_ERR_ARG and "ptr[m]" in why
    A = _csr(ptr, idx, val)
    A.ptr = None
    rc, why = _create(lib, A)
    assert rc == nat.LP_ERR_ARG and "CSR A needs" in why
    rc, why = _create(lib, _csr(ptr, idx, val, dtype=nat.LP_BF16))
    assert rc == nat.LP_ERR_UNSUPPORTED and "FP32 or FP64" in why
    rc, why = _create(lib, _csr(ptr, idx, val), opt=_opts(lib, sketch=nat.LP_SKETCH_GAUSS))
    assert rc == nat.LP_ERR_UNSUPPORTED and "dense A only" in why


@pytest.mark.parametrize("field,value,message", [
    ("sigma", 0.0, "sigma"), ("sigma", 1.0, "sigma"), ("sigma", math.nan, "sigma"),
    ("gamma", 0.0, "gamma"), ("gamma", 1.0, "gamma"),
    ("s", 0, "s must be"), ("s", 17, "s must be"), ("graphs", 2, "graphs"), ("autotune", 3, "autotune"),
    ("sketch", 2, "sketch"), ("precondition", 2, "precondition"), ("sigma_rule", 2, "sigma_rule"),
    ("inner", 2, "inner must be"), ("t_max", 0, "t_max"), ("k_max", -1, "k_max"),
    ("inner_rule", 2, "inner_rule"), ("tol_cg", -1e-3, "tol_cg"), ("tol_cg", math.inf, "tol_cg"),
    ("w", -4, "w must be"), ("w_factor", 0.0, "w_factor"), ("w_factor", math.nan, "w_factor"),
])
def test_bad_options_are_rejected(lib, field, value, message):
    rc, why = _create(lib, _dense(), opt=_opts(lib, **{field: value}))
    assert rc == nat.LP_ERR_ARG and message in why, why


@pytest.mark.parametrize("opts", [dict(w=4), dict(w_factor=0.5), dict(w=2**31)])
def test_sketch_width_is_checked_before_any_device_work(lib, opts):
    rc, why = _create(lib, _dense(), opt=_opts(lib, **opts))
    assert rc == nat.LP_ERR_ARG and "sketch width" in why, why


def test_null_handles_are_argument_errors(lib):
    d = np.ones(N)
    p = d.ctypes.data
    assert lib.lp_destroy(None) == nat.LP_OK
    assert lib.lp_release_cached_memory() == nat.LP_OK  # an empty cache: nothing to free
    assert lib.lp_last_error(None) == b""
    assert lib.lp_adat(None, p, p, p, 0) == nat.LP_ERR_ARG
    assert lib.lp_residual_rhs(None, p, p, p, 1, None, None, None, None) == nat.LP_ERR_ARG
    assert lib.lp_sketch(None, p, 0, 0, 0, p, None) == nat.LP_ERR_ARG
    assert lib.lp_precond_apply(None, p, p, p) == nat.LP_ERR_ARG
    assert lib.lp_directions(None, p, p, p, p, p, 1.0, 1, p, p) == nat.LP_ERR_ARG
    assert lib.lp_step_lengths(None, p, p, p, p, 1, 0.0, 1.0, p) == nat.LP_ERR_ARG
    assert lib.lp_normal_solve(None, p, p, p, 0, 0.0, 0, p, p, None) == nat.LP_ERR_ARG
    assert lib.lp_solve(None, 1e-8, 1, None, None, None, 0, None, None, None, None) == nat.LP_ERR_ARG
    assert lib.lp_get_history(None, None, 0) == nat.LP_ERR_ARG
    assert lib.lp_get_kernel_stats(None, None) == nat.LP_ERR_ARG
    assert lib.lp_reset_kernel_stats(None) == nat.LP_ERR_ARG
    assert lib.lp_set_warm_start(None, 0, None, None, None, 0) == nat.LP_ERR_ARG
    assert lib.lp_get_warm_start_stats(None, None, None, None) == nat.LP_ERR_ARG
    st = nat.LpState(3, 1, 0, 0, 1.0, 1.0, 0.0, 0, 1.0)
    assert lib.lp_get_state(None, ctypes.byref(st), p, p, p, None, 0) == nat.LP_ERR_ARG
    assert lib.lp_set_state(None, ctypes.byref(st), p, p, p, None, 0) == nat.LP_ERR_ARG
    hs = (ctypes.c_void_p * 1)(None)
    assert lib.lp_solve_batch(hs, 1, 1e-8, 1, 0, None, None, None, 1, None) == nat.LP_ERR_ARG
    assert lib.lp_solve_batch(None, 1, 1e-8, 1, 0, None, None, None, 1, None) == nat.LP_ERR_ARG


def test_mlp_and_standalone_entry_points_check_their_arguments(lib):
    out = ctypes.c_void_p(None)
    assert lib.lp_mlp_create(None, 4, 8, 4, 0, None) == nat.LP_ERR_ARG
    for dims in ((0, 8, 4), (4, 0, 4), (4, 8, 0)):
        assert lib.lp_mlp_create(ctypes.byref(out), *dims, 0, None) == nat.LP_ERR_ARG
    assert lib.lp_mlp_destroy(None) == nat.LP_OK
    assert lib.lp_mlp_num_params(None) == -1
    buf = np.ones(16, dtype=np.float32)
    assert lib.lp_mlp_get_params(None, buf.ctypes.data) == nat.LP_ERR_ARG
    assert lib.lp_mlp_forward(None, buf.ctypes.data, 1, buf.ctypes.data) == nat.LP_ERR_ARG
    # the allocation-free product: null pointers, FP64 storage, an ld that is
    # not a 16-byte multiple, a misaligned A
    d = np.ones(N)
    A = np.ones(16 * N + 8, dtype=np.float32)
    base = A.ctypes.data + (-A.ctypes.data) % 16            # a 16-byte-aligned start inside A
    p = d.ctypes.data
    assert lib.lp_adat_noalloc(None, nat.LP_F32, M, N, M, p, p, p, None) == nat.LP_ERR_ARG
    assert lib.lp_adat_noalloc(base, nat.LP_F64, M, N, M, p, p, p, None) == nat.LP_ERR_ARG
    assert lib.lp_adat_noalloc(base, nat.LP_F32, 6, N, 6, p, p, p, None) == nat.LP_ERR_ARG
    assert lib.lp_adat_noalloc(base + 4, nat.LP_F32, M, N, M, p, p, p, None) == nat.LP_ERR_ARG
    assert lib.lp_adat_noalloc(base, nat.LP_F32, M, N, M - 4, p, p, p, None) == nat.LP_ERR_ARG
    # phase 1 wants a host matrix and tol > 0
    x0 = np.zeros(N)
    dense = _dense()
    assert lib.lp_phase1_start(ctypes.byref(dense), _B.ctypes.data, None, 0.0, x0.ctypes.data, None) == nat.LP_ERR_ARG
    dense.on_device = 1
    assert lib.lp_phase1_start(ctypes.byref(dense), _B.ctypes.data, None, 1e-7, x0.ctypes.data, None) == nat.LP_ERR_ARG


def test_create_error_message_is_per_thread(lib):
    # two threads fail lp_create with different argument errors at the same
    # time; each reads back its own message
    import threading
    results = {}

    def worker(tag, opt):
        seen = set()
        for _ in range(300):
            rc, why = _create(lib, _dense(), opt=opt)
            assert rc == nat.LP_ERR_ARG
            seen.add(why)
        results[tag] = seen

    t1 = threading.Thread(target=worker, args=("sigma", _opts(lib, sigma=2.0)))
    t2 = threading.Thread(target=worker, args=("t_max", _opts(lib, t_max=0)))
    t1.start(); t2.start(); t1.join(); t2.join()
    assert len(results["sigma"]) == 1 and "sigma" in next(iter(results["sigma"]))
    assert len(results["t_max"]) == 1 and "t_max" in next(iter(results["t_max"]))


def test_phase1_checks_a_host_matrix_before_reading_it(lib):
    x0 = np.zeros(N)
    b = _B.ctypes.data

    def call(A):
        return lib.lp_phase1_start(ctypes.byref(A), b, None, 1e-7, x0.ctypes.data, None)

    assert call(_dense(val=None)) == nat.LP_ERR_ARG          # no values
    ptr = np.arange(N + 1, dtype=np.int64)
    idx = (np.arange(N) % M).astype(np.int32)
    val = np.ones(N, dtype=np.float32)
    A = _csc(ptr, idx, val)
    A.ptr = None
    assert call(A) == nat.LP_ERR_ARG                           # no column pointers
    A = _csc(ptr, idx, val)
    A.idx = None
    assert call(A) == nat.LP_ERR_ARG                           # no row indices
    back = ptr.copy()
    back[-1] = 0                                               # ptr[n] < ptr[0]: negative nnz
    assert call(_csc(back, idx, val)) == nat.LP_ERR_ARG
    neg = ptr - 1                                              # ptr[0] < 0
    assert call(_csc(neg, idx, val)) == nat.LP_ERR_ARG
    csr_ptr = np.arange(0, 4 * M + 1, 4, dtype=np.int64)
    csr_idx = (np.arange(4 * M) * 3 % N).astype(np.int32)
    csr_val = np.ones(4 * M, dtype=np.float32)
    bad = csr_idx.copy()
    bad[0] = N                                                 # CSR column index out of range
    assert call(_csr(csr_ptr, bad, csr_val)) == nat.LP_ERR_ARG
    A = _csr(csr_ptr, csr_idx, csr_val)
    A.idx = None
    assert call(A) == nat.LP_ERR_ARG                           # no column indices


def test_wait_probe_rejects_a_null_handle(lib):
    assert lib.lp_wait_probe(None, 1000, 0) == nat.LP_ERR_ARG


def test_csr_to_csc_is_a_stable_column_sort(lib):
    # the conversion lp_create applies to CSR input, on the host (no CUDA call):
    # identical to SciPy's CSR -> CSC (column-major, rows ascending in each
    # column), for a matrix with unsorted and duplicate column indices in rows
    sp = pytest.importorskip("scipy.sparse")
    from paper_2209_08722_gb300.solver import LPError, csr_to_csc
    rng = np.random.default_rng(3)
    m, n = 37, 500
    counts = rng.integers(0, 30, size=m)
    rp = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    ci = rng.integers(0, n, size=int(rp[-1])).astype(np.int32)
    val = rng.standard_normal(int(rp[-1]))
    for dtype, vals in (("f64", val), ("f32", val.astype(np.float32))):
        cp, ri, vo = csr_to_csc(rp, ci, vals, m, n, dtype)
        ref = sp.csr_matrix((vals, ci, rp), shape=(m, n)).tocsc()
        assert np.array_equal(cp, ref.indptr) and np.array_equal(ri, ref.indices)
        assert np.array_equal(vo, ref.data)
    # each column's rows ascend, and the entries are the CSR's
    cp, ri, vo = csr_to_csc(rp, ci, val, m, n, "f64")
    for j in range(n):
        assert np.all(np.diff(ri[cp[j]:cp[j + 1]]) >= 0)
    assert sorted(zip(ri.tolist(), np.repeat(np.arange(n), np.diff(cp)).tolist(), vo.tolist())) == \
        sorted(zip(np.repeat(np.arange(m), counts).tolist(), ci.tolist(), val.tolist()))
    bad = ci.copy()
    bad[0] = n
    with pytest.raises(LPError):
        csr_to_csc(rp, bad, val, m, n, "f64")
    assert lib.lp_csr_to_csc(m, n, 0, None, None, None, nat.LP_F64, None, None, None) == nat.LP_ERR_ARG


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
def test_csr_to_csc_in_parts_equals_scipy_bit_for_bit(lib, dtype):
    # above a million entries the sort runs in parts on host threads; the
    # result must still be the stable sort, bit for bit: empty rows, rows
    # of very different lengths, duplicate column indices, and the reverse
    # direction (CSC -> CSR, as lp_create builds the row copy) too
    sp = pytest.importorskip("scipy.sparse")
    from paper_2209_08722_gb300.solver import csr_to_csc
    rng = np.random.default_rng(11)
    m, n = 3001, 40000
    counts = rng.integers(0, 800, size=m)
    counts[rng.choice(m, 50, replace=False)] = 0
    counts[rng.choice(m, 5, replace=False)] = 20000
    rp = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    nnz = int(rp[-1])
    assert nnz >= 1 << 20
    ci = rng.integers(0, n, size=nnz).astype(np.int32)
    bits = rng.integers(0, 1 << 16, size=nnz, dtype=np.uint16)
    vals = {"f64": rng.standard_normal(nnz), "f32": rng.standard_normal(nnz).astype(np.float32),
            "bf16": bits}[dtype]
    keys = np.arange(nnz, dtype=np.int64)  # SciPy carries the entry's position through its own sort
    ref = sp.csr_matrix((keys + 1, ci, rp), shape=(m, n)).tocsc()
    cp, ri, vo = csr_to_csc(rp, ci, vals, m, n, dtype)
    assert np.array_equal(cp, ref.indptr) and np.array_equal(ri, ref.indices)
    assert np.array_equal(vo.view(np.uint8), vals[ref.data - 1].view(np.uint8))
    # the reverse direction: the CSC read as the CSR of the transpose
    rp2, ci2, vo2 = csr_to_csc(cp, ri, vo, n, m, dtype)
    assert np.array_equal(rp2, rp)
    back = sp.csc_matrix((np.arange(nnz) + 1, ri, cp), shape=(m, n)).tocsr()
    assert np.array_equal(ci2, back.indices)
    assert np.array_equal(vo2.view(np.uint8), vo[back.data - 1].view(np.uint8))
