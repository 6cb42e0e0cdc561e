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
