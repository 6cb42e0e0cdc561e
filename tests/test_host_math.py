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

from oracle import ipm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2209_08722_gb300", "csrc")
SHIM = os.path.join(ROOT, "tests", "host_math_shim.cpp")


@pytest.fixture(scope="module")
def shim(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    out = str(tmp_path_factory.mktemp("shim") / "libhostmath.so")
    subprocess.run([gxx, "-O2", "-std=c++17", "-shared", "-fPIC", "-I", CSRC, SHIM, "-o", out], check=True)
    lib = ctypes.CDLL(out)
    dp = ctypes.POINTER(ctypes.c_double)
    lib.shim_lanczos_extremes.argtypes = [dp, ctypes.c_int, dp, dp]
    lib.shim_lanczos_extremes.restype = ctypes.c_int
    lib.shim_tridiag_extremes.argtypes = [dp, dp, ctypes.c_int, dp, dp]
    lib.shim_tridiag_extremes.restype = None
    return lib


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
