"""Checks of the seeded problem generators (planted optimality, storage rounding)."""

import numpy as np
import pytest

import lpgen


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    a = np.random.default_rng(0).standard_normal(10000) * 10.0 ** np.random.default_rng(1).uniform(-3, 3, 10000)
    ours = lpgen.round_bf16(a)
    ref = torch.tensor(a.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(ours, ref)


@pytest.mark.parametrize("storage", ["f64", "f32", "bf16"])
def test_planted_dense_is_optimal(storage):
    lp = lpgen.planted_dense(8, 200, seed=2, storage=storage, col_scale_log10=(-2, 2))
    A = lp.A
    if storage == "f32":
        assert np.array_equal(A, A.astype(np.float32).astype(np.float64))
    assert np.allclose(A @ lp.x_star, lp.b)
    s = lp.c - A.T @ lp.y_star
    assert np.allclose(s, lp.s_star)
    assert (lp.x_star >= 0).all() and (lp.s_star >= 0).all()
    assert np.all(lp.x_star * lp.s_star == 0)
    assert lp.objective == pytest.approx(lp.b @ lp.y_star, rel=1e-12)


def test_planted_sparse_structure():
    lp = lpgen.planted_sparse(64, 5000, nnz_per_col=8, seed=3)
    k = 8
    rows = lp.row_idx.reshape(-1, k)
    assert (np.diff(rows, axis=1) > 0).all()          # distinct, sorted rows
    counts = np.bincount(lp.row_idx, minlength=64)
    assert counts.max() > 3 * counts.mean()            # heavy-tailed row counts
    A = lp.dense()
    assert np.allclose(A @ lp.x_star, lp.b)
    assert np.allclose(lp.c - A.T @ lp.y_star, lp.s_star)


def test_storage_array_layout():
    lp = lpgen.planted_dense(5, 7, seed=1, storage="f32")
    st = lp.storage_array()
    assert st.shape == (7, 5) and st.dtype == np.float32
    assert np.array_equal(st.T.astype(np.float64), lp.A)
    lpb = lpgen.planted_dense(5, 7, seed=1, storage="bf16")
    bits = lpb.storage_array()
    assert bits.dtype == np.uint16
    vals = (bits.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    assert np.array_equal(vals.T, lpb.A)


def test_bf16_rounding_ties_go_to_even():
    # FP32 values exactly halfway between two bfloat16 neighbours (low 16 bits
    # 0x8000) round to the neighbour with an even last bit, in both signs
    hi = np.array([0x3F80, 0x3F81, 0x4049, 0x404A, 0xBF80, 0xBF81, 0x0001, 0x7F00], dtype=np.uint32)
    f = ((hi << np.uint32(16)) | np.uint32(0x8000)).view(np.float32)
    got = lpgen.bf16_bits(f).astype(np.uint32)
    expect = np.where(hi % 2 == 0, hi, hi + 1)
    assert np.array_equal(got, expect)
    # just below and just above the halfway point
    below = ((hi << np.uint32(16)) | np.uint32(0x7FFF)).view(np.float32)
    above = ((hi << np.uint32(16)) | np.uint32(0x8001)).view(np.float32)
    assert np.array_equal(lpgen.bf16_bits(below).astype(np.uint32), hi)
    assert np.array_equal(lpgen.bf16_bits(above).astype(np.uint32), hi + 1)


def test_column_scaling_is_log_uniform():
    # col_scale_log10 = (-2, 2): column j is scaled by 10^U(-2, 2)
    m, n = 16, 4000
    plain = lpgen.planted_dense(m, n, seed=5)
    scaled = lpgen.planted_dense(m, n, seed=5, col_scale_log10=(-2.0, 2.0))
    lg = np.log10(np.linalg.norm(scaled.A, axis=0) / np.sqrt(m))
    assert lg.min() < -1.8 and lg.max() > 1.8 and abs(lg.mean()) < 0.2
    assert np.allclose(scaled.A @ scaled.x_star, scaled.b)
    assert plain.A.shape == scaled.A.shape


def test_batch_family_sizes_and_planted_optima():
    lps = lpgen.batch_family(12, seed=4, m_range=(8, 24), k_range=(4, 9))
    for lp in lps:
        assert 8 <= lp.m <= 24 and lp.n % lp.m == 0 and 4 <= lp.n // lp.m <= 9
        assert lp.storage == "f32"
        assert np.allclose(lp.A @ lp.x_star, lp.b)
        assert np.allclose(lp.c - lp.A.T @ lp.y_star, lp.s_star)
        assert np.all(lp.x_star * lp.s_star == 0)
    again = lpgen.batch_family(12, seed=4, m_range=(8, 24), k_range=(4, 9))
    assert all(np.array_equal(a.A, b.A) and np.array_equal(a.b, b.b) for a, b in zip(lps, again))
    assert len({(lp.m, lp.n) for lp in lps}) > 1           # the sizes vary across the family


def test_named_workloads_and_the_bench_agree():
    C = lpgen.CONFIGS
    assert (C["c1"]["m"], C["c1"]["n"], C["c1"]["storage"], C["c1"]["mode"]) == (64, 4096, "f64", "feasible")
    assert (C["c2"]["m"], C["c2"]["n"], C["c2"]["storage"], C["c2"]["col_scale"]) == (512, 131072, "f32", (-2.0, 2.0))
    assert (C["c3"]["kind"], C["c3"]["m"], C["c3"]["n"], C["c3"]["nnz_per_col"]) == ("sparse", 4096, 2_000_000, 8)
    assert (C["c4"]["m"], C["c4"]["n"], C["c4"]["storage"]) == (2048, 524288, "bf16")
    import bench
    for name in ("c2", "c4"):
        b = bench.BENCH[name]
        assert (b["m"], b["n"], b["s"], b["w_factor"], b["dtype"]) == (
            C[name]["m"], C[name]["n"], C[name]["s"], C[name]["w_factor"], C[name]["storage"])
    small = lpgen.config_small("c2", 64)
    assert (small.m, small.n, small.storage) == (8, 2048, "f32")


@pytest.mark.parametrize("storage,scale", [("bf16", None), ("f32", (-2.0, 2.0)), ("f64", None)])
def test_blocked_dense_generator_is_planted_and_thread_independent(storage, scale):
    # the column-block generator of the 10^9-entry workload: every block has its
    # own seeded stream, so the matrix does not depend on the worker count
    m, n = 12, 1000
    one = lpgen.planted_dense_blocked(m, n, seed=7, storage=storage, col_scale_log10=scale,
                                      block=96, threads=1)
    many = lpgen.planted_dense_blocked(m, n, seed=7, storage=storage, col_scale_log10=scale,
                                       block=96, threads=5)
    assert np.array_equal(one.storage_array(), many.storage_array())
    assert np.array_equal(one.b, many.b) and np.array_equal(one.c, many.c)
    st = one.storage_array()
    assert st.shape == (n, m)
    A = one.dense()
    assert A.shape == (m, n) and A.dtype == np.float64
    if storage == "bf16":
        assert st.dtype == np.uint16
        assert np.array_equal(A, lpgen.round_bf16(A))        # values are bf16-representable
    if storage == "f32":
        assert np.array_equal(A, A.astype(np.float32).astype(np.float64))
        lg = np.log10(np.linalg.norm(A, axis=0) / np.sqrt(m))
        assert lg.min() < -1.5 and lg.max() > 1.5
    # the planted optimum is exact for the stored values
    assert np.allclose(A @ one.x_star, one.b, rtol=1e-13, atol=1e-12)
    assert np.allclose(one.c - A.T @ one.y_star, one.s_star, rtol=1e-13, atol=1e-12)
    assert np.all(one.x_star * one.s_star == 0) and np.count_nonzero(one.x_star) == m
    # the entries look like N(0, 1) draws and differ across seeds and blocks
    if scale is None:
        assert abs(A.mean()) < 0.05 and abs(A.std() - 1) < 0.05
    other = lpgen.planted_dense_blocked(m, n, seed=8, storage=storage, block=96)
    assert not np.array_equal(other.storage_array(), st)
    assert not np.array_equal(st[:96], st[96:192])


def test_c4_workload_uses_the_blocked_generator():
    small = lpgen.config_small("c4", 64)
    assert small.cols is not None and small.storage == "bf16"
    assert (small.m, small.n) == (32, 8192)
