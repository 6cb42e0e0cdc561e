"""The solver's host-side numerical helpers (csrc/host_math.h) against the
oracle, on the CPU: the extreme Ritz values that set the Chebyshev interval
(Section 3.2) and drive the check of a sketch draw, from the coefficients of
the oracle's own CG.  The header is plain C++, compiled here with g++ into a
throw-away shim."""

import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import ipm, pcg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2209_08722_gb300", "csrc")
SHIM = os.path.join(ROOT, "tests", "host_math_shim.cpp")


def _build_shim(out_dir, include_dir):
    """Compile the shim against the host_math.h found in include_dir."""
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    out = os.path.join(str(out_dir), "libhostmath.so")
    subprocess.run([gxx, "-O2", "-std=c++17", "-shared", "-fPIC", "-I", str(include_dir), SHIM, "-o", out],
                   check=True)
    lib = ctypes.CDLL(out)
    dp = ctypes.POINTER(ctypes.c_double)
    lib.shim_lanczos_extremes.argtypes = [dp, ctypes.c_int, dp, dp]
    lib.shim_lanczos_extremes.restype = ctypes.c_int
    lib.shim_tridiag_extremes.argtypes = [dp, dp, ctypes.c_int, dp, dp]
    lib.shim_tridiag_extremes.restype = None
    lib.shim_theory_inner_tol.argtypes = [ctypes.c_double, ctypes.c_longlong, ctypes.c_double, ctypes.c_double]
    lib.shim_theory_inner_tol.restype = ctypes.c_double
    lib.shim_stop.argtypes = [ctypes.c_double] * 7 + [dp]
    lib.shim_stop.restype = ctypes.c_int
    return lib


@pytest.fixture(scope="module")
def shim(tmp_path_factory):
    return _build_shim(tmp_path_factory.mktemp("shim"), CSRC)


def _ptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _spd(m, cond, seed):
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((m, m)))
    return (U * np.geomspace(1.0, cond, m)) @ U.T


@pytest.mark.parametrize("m,cond,steps", [(12, 30.0, 5), (40, 1e3, 12), (64, 10.0, 8), (8, 5.0, 8)])
def test_lanczos_extremes_match_the_oracle(shim, m, cond, steps):
    B = _spd(m, cond, seed=m)
    rhs = np.random.default_rng(m + 1).standard_normal(m)
    alphas, betas = ipm._cg_coeffs(lambda z: B @ z, rhs, steps)
    lo_ref, hi_ref = ipm.lanczos_interval(alphas, betas)
    coef = np.empty(2 * len(alphas))
    coef[0::2], coef[1::2] = alphas, betas
    lo, hi = ctypes.c_double(), ctypes.c_double()
    assert shim.shim_lanczos_extremes(_ptr(coef), len(alphas), ctypes.byref(lo), ctypes.byref(hi)) == 1
    assert lo.value == pytest.approx(lo_ref, rel=1e-12)
    assert hi.value == pytest.approx(hi_ref, rel=1e-12)


def test_tridiagonal_extremes_match_a_dense_eigensolver(shim):
    rng = np.random.default_rng(5)
    for k in (1, 2, 7, 50):
        dg = rng.standard_normal(k) * 3
        off = rng.standard_normal(max(k - 1, 0))
        T = np.diag(dg) + np.diag(off, 1) + np.diag(off, -1)
        ev = np.linalg.eigvalsh(T)
        lo, hi = ctypes.c_double(), ctypes.c_double()
        shim.shim_tridiag_extremes(_ptr(dg), _ptr(off if k > 1 else np.zeros(1)), k,
                                   ctypes.byref(lo), ctypes.byref(hi))
        scale = np.abs(ev).max()
        assert abs(lo.value - ev[0]) <= 1e-13 * scale
        assert abs(hi.value - ev[-1]) <= 1e-13 * scale


def test_broken_recurrence_is_reported(shim):
    lo, hi = ctypes.c_double(-7.0), ctypes.c_double(-7.0)
    for coef in (np.array([0.5, 0.1, -1.0, 0.2]),       # alpha_1 <= 0
                 np.array([0.5, -0.1, 1.0, 0.2]),       # beta_0 < 0
                 np.array([np.nan, 0.1])):
        assert shim.shim_lanczos_extremes(_ptr(coef), len(coef) // 2, ctypes.byref(lo), ctypes.byref(hi)) == 0
        assert lo.value == -7.0 and hi.value == -7.0    # left alone


def test_theory_inner_target_matches_the_oracle(shim):
    rng = np.random.default_rng(7)
    for _ in range(50):
        mu, n = 10.0 ** rng.uniform(-12, 2), int(rng.integers(1, 10 ** 7))
        gamma, sigma = rng.uniform(0.01, 0.999), rng.uniform(0.05, 0.8)
        ref = pcg.theory_inner_tol(mu, n, gamma, sigma)
        assert shim.shim_theory_inner_tol(mu, n, gamma, sigma) == pytest.approx(ref, rel=1e-15)


def test_stopping_measures_match_the_oracle(shim):
    # the oracle's test on random iterates, and at a planted optimum moved so
    # that exactly one of the three measures sits at 0.5 or 2 times tol
    import lpgen
    rng = np.random.default_rng(8)
    tol = 1e-8
    lp = lpgen.planted_dense(6, 40, seed=8)
    A, b, c, n = lp.A, lp.b, lp.c, lp.n
    x0, y0, s0 = lp.x_star, lp.y_star, lp.s_star
    cases = [(rng.uniform(0, 2, n), rng.standard_normal(lp.m), rng.uniform(0, 2, n)) for _ in range(10)]
    cases.append((x0, y0, s0))
    null = np.eye(n) - np.linalg.pinv(A) @ A                    # A (null u) = 0
    for scale in (0.5, 2.0):
        u = rng.standard_normal(n)
        u -= (u @ c) / (c @ c) * c                              # keeps c^T x: only r_p moves
        t = scale * tol * (1 + np.linalg.norm(b)) / np.linalg.norm(A @ u)
        cases.append((x0 + t * u, y0, s0))
        e = np.eye(n)[0]                                        # only r_d moves
        cases.append((x0, y0, s0 + scale * tol * (1 + np.linalg.norm(c)) * e))
        g = null @ rng.standard_normal(n)                       # only the gap moves
        t = scale * tol * (1 + abs(c @ x0)) / abs(c @ g)
        cases.append((x0 + t * g, y0, s0))
    out = np.empty(3)
    outcomes = set()
    for x, y, s in cases:
        r_p, r_d = ipm.residuals(A, b, c, x, y, s)
        done_ref, gap_ref = ipm.converged(A, b, c, x, y, r_p, r_d, tol)
        done = shim.shim_stop(c @ x, b @ y, r_p @ r_p, r_d @ r_d, np.linalg.norm(b), np.linalg.norm(c), tol,
                              _ptr(out))
        assert out[0] == pytest.approx(gap_ref, rel=1e-12, abs=1e-15)
        assert out[1] == pytest.approx(np.linalg.norm(r_p) / (1 + np.linalg.norm(b)), rel=1e-12, abs=1e-300)
        assert out[2] == pytest.approx(np.linalg.norm(r_d) / (1 + np.linalg.norm(c)), rel=1e-12, abs=1e-300)
        assert bool(done) == bool(done_ref)
        outcomes.add(bool(done))
    assert outcomes == {True, False}


# One mistake at a time planted in a copy of host_math.h; the tests above,
# run against a shim built from that copy, must catch each of them.
HEADER_MUTANTS = [
    ("diagonal_index", "be_prev / al_prev", "be_prev / al", "lanczos"),
    ("offdiagonal_sqrt_dropped", "std::sqrt(std::max(coef[2 * j + 1], 0.0)) / al",
     "std::max(coef[2 * j + 1], 0.0) / al", "lanczos"),
    ("breakdown_test_strict", "!(be_prev >= 0.0)", "!(be_prev > 0.0)", "lanczos"),
    ("sturm_pivot_sign", "q = dg[i] - x - (i > 0 ? o2 / q : 0.0);", "q = dg[i] - x + (i > 0 ? o2 / q : 0.0);",
     "tridiag"),
    ("gershgorin_radius_dropped", "gl = std::min(gl, dg[i] - r);", "gl = std::min(gl, dg[i]);", "tridiag"),
    ("theory_factor_3_dropped", "std::sqrt(3.0 * (double)n)", "std::sqrt((double)n)", "theory"),
    ("gap_normalised_by_dual", "(1.0 + std::fabs(cx))", "(1.0 + std::fabs(by))", "stop"),
    ("primal_residual_by_c", "std::sqrt(rp2) / (1.0 + bnorm)", "std::sqrt(rp2) / (1.0 + cnorm)", "stop"),
    ("dual_residual_test_dropped", "s.rd_rel <= tol", "s.rp_rel <= tol", "stop"),
]


def _run_checks(lib, which):
    if which == "lanczos":
        for m, cond, steps in ((12, 30.0, 5), (40, 1e3, 12)):
            test_lanczos_extremes_match_the_oracle(lib, m, cond, steps)
    elif which == "tridiag":
        test_tridiagonal_extremes_match_a_dense_eigensolver(lib)
    elif which == "theory":
        test_theory_inner_target_matches_the_oracle(lib)
    else:
        test_stopping_measures_match_the_oracle(lib)


@pytest.mark.parametrize("mid,old,new,which", HEADER_MUTANTS, ids=[m[0] for m in HEADER_MUTANTS])
def test_planted_mistake_in_host_math_is_caught(tmp_path, mid, old, new, which):
    src = open(os.path.join(CSRC, "host_math.h")).read()
    assert src.count(old) == 1, (mid, src.count(old))
    inc = tmp_path / "inc"
    inc.mkdir()
    (inc / "host_math.h").write_text(src.replace(old, new))
    lib = _build_shim(tmp_path, inc)
    with pytest.raises(AssertionError):
        _run_checks(lib, which)
