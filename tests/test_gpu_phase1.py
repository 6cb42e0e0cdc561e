"""lp_phase1_start on the GPU (Appendix "Feasible starting point"): a strictly
positive x0 with A x0 = b, or LP_ERR_NOT_FEASIBLE with the phase-1 optimum
matching HiGHS's; dense and CSC inputs."""

import numpy as np
import pytest

import lpgen
from oracle import phase1

pytestmark = pytest.mark.gpu
scipy_opt = pytest.importorskip("scipy.optimize")


def _highs_phase1(A, b):
    A1, b1, c1 = phase1.phase1_lp(A, b)
    r = scipy_opt.linprog(c1, A_eq=A1, b_eq=b1, bounds=(0, None), method="highs")
    assert r.status == 0
    return r.fun


def _start(A, b, **kw):
    from paper_2209_08722_gb300 import phase1_start
    m, n = A.shape
    return phase1_start(np.ascontiguousarray(A.T), b, m, n, dtype="f64", **kw)


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_planted_dense_start(storage):
    from paper_2209_08722_gb300 import phase1_start
    lp = lpgen.planted_dense(64, 4000, seed=11, storage=storage, col_scale_log10=(-1, 1))
    flip = np.where(np.arange(lp.m) % 3 == 0, -1.0, 1.0)   # some negative b_i
    A = lp.A * flip[:, None]
    b = lp.b * flip
    store = np.ascontiguousarray(A.T.astype(np.float32 if storage == "f32" else np.float64))
    x0, info = phase1_start(store, b, lp.m, lp.n, dtype=storage, s=2)
    assert (x0 > 0).all() and info["x0_min"] > 0
    scale = (1 + np.linalg.norm(b)) * (1 + np.abs(x0).max())
    assert np.linalg.norm(A @ x0 - b) <= 1e-9 * scale
    assert info["z_sum"] <= 1e-6 * (1 + np.linalg.norm(b))


def test_planted_sparse_start():
    from paper_2209_08722_gb300 import phase1_start
    lp = lpgen.planted_sparse(128, 6000, nnz_per_col=6, seed=12, storage="f64")
    x0, info = phase1_start(None, lp.b, lp.m, lp.n, dtype="f64",
                            csc=(lp.col_ptr, lp.row_idx, lp.val), s=2)
    A = lp.dense()
    assert (x0 > 0).all()
    assert np.linalg.norm(A @ x0 - lp.b) <= 1e-9 * (1 + np.linalg.norm(lp.b)) * (1 + np.abs(x0).max())


def test_random_lp_infeasible_matches_highs():
    from paper_2209_08722_gb300.solver import LPError
    rl = lpgen.random_lp(20, 200, density=0.2, seed=3)
    ref = _highs_phase1(rl.A, rl.b)
    assert ref > 1e-3
    with pytest.raises(LPError) as ei:
        _start(rl.A, rl.b, s=2)
    assert "NOT_FEASIBLE" in str(ei.value)
    assert abs(ei.value.info["z_sum"] - ref) <= 1e-6 * (1 + ref)


def test_random_lp_feasible_right_hand_side():
    rl = lpgen.random_lp(20, 200, density=0.2, seed=4)
    b = rl.A @ np.abs(np.random.default_rng(5).standard_normal(rl.n))
    x0, info = _start(rl.A, b, s=2)
    assert (x0 > 0).all()
    assert np.linalg.norm(rl.A @ x0 - b) <= 1e-9 * (1 + np.linalg.norm(b)) * (1 + np.abs(x0).max())
