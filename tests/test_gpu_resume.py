"""Checkpoint and resume (lp_get_state / lp_set_state): a solve stopped at
k_max and resumed on a fresh handle from the saved state draws the same
sketch sequence (seeded by the outer iteration k) and takes the same
iterates as the uninterrupted solve, bit for bit."""

import numpy as np
import pytest

import lpgen
from tests.gpu_helpers import solver_for, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("warm", ["none", "previous"])
def test_resumed_solve_equals_uninterrupted_solve(warm):
    torch_cuda()
    lp = lpgen.planted_dense(128, 10000, seed=6, storage="f32", col_scale_log10=(-1, 1))
    with solver_for(lp, s=2, seed=11) as S:
        S.set_warm_start(warm)
        x_ref, y_ref, s_ref, i_ref = S.solve(tol=1e-8)
        hist_ref = S.history()
    assert i_ref["status"] == 0 and i_ref["outer_iterations"] > 12
    stop = i_ref["outer_iterations"] // 2
    with solver_for(lp, s=2, seed=11, k_max=stop) as S1:
        S1.set_warm_start(warm)
        _, _, _, i1 = S1.solve(tol=1e-8)
        assert i1["status"] == 1 and i1["outer_iterations"] == stop  # LP_STATUS_MAX_ITER
        state = S1.get_state()
    assert state["k"] == stop and state["mode"] == 1 and state["seed"] == 11
    assert state["has_dy_prev"] == (1 if warm == "previous" else 0)
    # a fresh handle with another seed: the state's seed replaces it
    with solver_for(lp, s=2, seed=999) as S2:
        S2.set_warm_start(warm)
        S2.set_state(state)
        x, y, s, i2 = S2.solve(tol=1e-8)
        hist = S2.history()
    assert i2["status"] == 0
    assert i2["outer_iterations"] == i_ref["outer_iterations"]
    assert i1["inner_total"] + i2["inner_total"] == i_ref["inner_total"]
    assert [h["inner_iterations"] for h in hist] == [h["inner_iterations"] for h in hist_ref[stop:]]
    assert np.array_equal(x, x_ref) and np.array_equal(y, y_ref) and np.array_equal(s, s_ref)


def test_state_misuse_is_rejected():
    torch = torch_cuda()
    from paper_2209_08722_gb300.solver import LPError
    lp = lpgen.planted_dense(32, 2000, seed=3, storage="f64")
    with solver_for(lp, k_max=3) as S:
        with pytest.raises(LPError):  # no solve yet
            S.get_state()
        S.solve(tol=1e-8)
        st = S.get_state()
        S.residual_rhs(*(torch.from_numpy(st[k]).cuda() for k in ("x", "y", "s")))
        with pytest.raises(LPError):  # the iterate was overwritten
            S.get_state()
        S.set_state(st)
        with pytest.raises(LPError):  # the state is from an infeasible-mode solve
            S.solve(tol=1e-8, mode="feasible")
        S.set_state(st)
        with pytest.raises(LPError):  # a resumed solve takes no start point
            S.solve(tol=1e-8, x0=st["x"], y0=st["y"], s0=st["s"])
        for key, bad in (("k", -1), ("mu0", 0.0), ("mu", -1.0), ("r0", float("nan")), ("mode", 7)):
            with pytest.raises(LPError):
                S.set_state(dict(st, **{key: bad}))
        S.set_state(dict(st, k=3))
        _, _, _, info = S.solve(tol=1e-8)
        assert info["status"] == 1 and info["outer_iterations"] == 3
