"""Pins for oracle.phase1 (Appendix "Feasible starting point") and the
paper's random LP generator (Appendix "Random data")."""

import numpy as np
import pytest

import lpgen
from oracle import phase1

scipy_opt = pytest.importorskip("scipy.optimize")


def _highs_phase1(A, b):
    A1, b1, c1 = phase1.phase1_lp(A, b)
    r = scipy_opt.linprog(c1, A_eq=A1, b_eq=b1, bounds=(0, None), method="highs")
    assert r.status == 0
    return r.fun


def _check_start(A, b, res):
    assert res.feasible
    assert (res.x0 > 0).all()
    assert np.linalg.norm(A @ res.x0 - b) <= 1e-9 * (1 + np.linalg.norm(b)) * (1 + np.abs(res.x0).max())


def test_planted_lp_gets_a_strictly_feasible_start():
    lp = lpgen.planted_dense(20, 200, seed=1)
    res = phase1.phase1_start(lp.A, lp.b)
    _check_start(lp.A, lp.b, res)
    assert res.z_sum <= 1e-7 * (1 + np.linalg.norm(lp.b))


def test_negative_right_hand_sides_are_handled():
    # negating rows of (A, b) changes neither the feasible set nor x
    lp = lpgen.planted_dense(16, 160, seed=2)
    flip = np.where(np.arange(16) % 2 == 0, -1.0, 1.0)
    A, b = lp.A * flip[:, None], lp.b * flip
    assert (b < 0).any()
    _check_start(A, b, phase1.phase1_start(A, b))
    # the phase-1 data themselves: b1 >= 0, (0, b1) is feasible, and every
    # feasible x of A x = b (here the planted optimum) gives the feasible
    # point (x, 0) with objective 1^T z = 0
    A1, b1, c1 = phase1.phase1_lp(A, b)
    assert (b1 >= 0).all()
    assert np.allclose(A1 @ np.concatenate([np.zeros(lp.n), b1]), b1)
    xz = np.concatenate([lp.x_star, np.zeros(16)])
    assert np.allclose(A1 @ xz, b1, atol=1e-10 * np.linalg.norm(b))
    assert c1 @ xz == 0.0 and c1 @ np.concatenate([np.zeros(lp.n), b1]) == pytest.approx(b1.sum())


def test_start_is_projected_onto_a_x_equals_b():
    # with a loose phase-1 tolerance the IPM's x misses A x = b by far more
    # than rounding; the minimum-norm correction must still land on it
    lp = lpgen.planted_dense(20, 200, seed=8)
    res = phase1.phase1_start(lp.A, lp.b, tol=1e-3)
    assert np.linalg.norm(lp.A @ res.x0 - lp.b) <= 1e-11 * (1 + np.linalg.norm(lp.b)) * (1 + np.abs(res.x0).max())


def test_random_lp_family_matches_highs_phase1_optimum():
    # the paper's generator usually gives infeasible Ax = b, x >= 0 (x ~ N(0,1));
    # the phase-1 optimum 1^T z is then positive and equals HiGHS's
    rl = lpgen.random_lp(20, 200, density=0.2, seed=3)
    res = phase1.phase1_start(rl.A, rl.b)
    ref = _highs_phase1(rl.A, rl.b)
    assert ref > 1e-3 and not res.feasible
    assert abs(res.z_sum - ref) <= 1e-6 * (1 + ref)


def test_random_lp_family_with_a_feasible_right_hand_side():
    rl = lpgen.random_lp(20, 200, density=0.2, seed=4)
    b = rl.A @ np.abs(np.random.default_rng(5).standard_normal(rl.n))
    res = phase1.phase1_start(rl.A, b)
    assert abs(_highs_phase1(rl.A, b)) <= 1e-7
    _check_start(rl.A, b, res)


def test_constructed_infeasible_lp_is_detected():
    # A >= 0 and x >= 0 give A x >= 0, so a negative b_i cannot be reached
    rl = lpgen.random_lp(12, 80, density=0.3, seed=6)
    b = -np.abs(rl.b) - 0.5
    res = phase1.phase1_start(rl.A, b)
    assert not res.feasible
    ref = _highs_phase1(rl.A, b)
    assert abs(res.z_sum - ref) <= 1e-6 * (1 + ref)
    assert abs(ref - np.abs(b).sum()) <= 1e-6 * np.abs(b).sum()   # z = |b| is optimal


def test_random_lp_generator_structure():
    rl = lpgen.random_lp(30, 100, density=0.1, seed=7)
    assert (rl.A >= 0).all() and (rl.A <= 2).all()
    assert (np.count_nonzero(rl.A, axis=1) >= 1).all()      # the diagonal draw
    assert abs(np.count_nonzero(rl.A) / rl.A.size - 0.1) < 0.05
