"""CPU checks of the Python binding's argument marshalling.

The library reads exactly as many elements as the sizes say, and takes one
host/device flag per call, so the binding checks buffer lengths, dtypes,
modes and that a call's vectors all live on one side before any pointer
reaches the library.  Calls that pass those checks are sent to the library
with a NULL handle here, where the C side answers LP_ERR_ARG without any
CUDA call.
"""

import ctypes

import numpy as np
import pytest

from paper_2209_08722_gb300 import _native as nat

torch = pytest.importorskip("torch")

M, N = 8, 32


def _bare_solver(m=M, n=N):
    """An LPSolver with a NULL handle: every library call it makes returns
    LP_ERR_ARG before touching CUDA."""
    from paper_2209_08722_gb300.solver import LPSolver
    S = object.__new__(LPSolver)
    S._lib = nat.load()
    S._h = ctypes.c_void_p()
    S.m, S.n, S.dtype = m, n, "f32"
    S.options = nat.LpOptions()
    S._lib.lp_options_default(ctypes.byref(S.options))
    return S


def _reaches_library(call):
    from paper_2209_08722_gb300.solver import LPError
    with pytest.raises(LPError) as ei:
        call()
    assert ei.value.code == nat.LP_ERR_ARG


def test_constructor_checks_sizes_and_dtypes():
    from paper_2209_08722_gb300 import LPSolver
    from paper_2209_08722_gb300.solver import LPError
    A = np.ones((N, M), dtype=np.float32)
    b, c = np.ones(M), np.ones(N)
    with pytest.raises(ValueError, match="b must have 8"):
        LPSolver(A, np.ones(M - 1), c, M, N)
    with pytest.raises(ValueError, match="c must have 32"):
        LPSolver(A, b, np.ones(N + 1), M, N)
    with pytest.raises(ValueError, match="shape"):
        LPSolver(A.T.copy(), b, c, M, N)
    with pytest.raises(ValueError, match="dtype must be"):
        LPSolver(A, b, c, M, N, dtype="f16")
    with pytest.raises(TypeError, match="16-bit patterns"):
        LPSolver(A, b, c, M, N, dtype="bf16")            # values, not bf16 bit patterns
    with pytest.raises(TypeError, match="takes"):
        LPSolver(torch.ones(N, M, dtype=torch.float64), b, c, M, N, dtype="f32")
    with pytest.raises(TypeError, match="unknown option"):
        LPSolver(A, b, c, M, N, no_such_option=1)
    with pytest.raises(ValueError, match="col_ptr"):
        LPSolver(None, b, c, M, N, csc=(np.zeros(N, np.int64), np.zeros(0, np.int32), np.zeros(0)))
    # right sizes but not a valid LP shape (m > n): refused by the library itself
    with pytest.raises(LPError) as ei:
        LPSolver(np.ones((4, 8), dtype=np.float32), np.ones(8), np.ones(4), 8, 4)
    assert ei.value.code == nat.LP_ERR_ARG


def test_solve_checks_mode_lengths_and_outputs():
    S = _bare_solver()
    with pytest.raises(ValueError, match="mode"):
        S.solve(mode="feasable")
    with pytest.raises(ValueError, match="x0 must have 32"):
        S.solve(x0=np.ones(N - 1))
    with pytest.raises(ValueError, match="y0 must have 8"):
        S.solve(x0=np.ones(N), y0=np.ones(N), s0=np.ones(N))
    with pytest.raises(TypeError, match="output x"):
        S.solve(out=(np.ones(N, dtype=np.float32), np.ones(M), np.ones(N)))
    with pytest.raises(ValueError, match="y must have 8"):
        S.solve(out=(np.ones(N), np.ones(N), np.ones(N)))
    # what the end-to-end bench passes: host tensors for the outputs
    outs = tuple(torch.empty(k, dtype=torch.float64) for k in (N, M, N))
    _reaches_library(lambda: S.solve(out=outs))
    _reaches_library(lambda: S.solve(mode="feasible", x0=np.ones(N), y0=np.zeros(M), s0=np.ones(N)))


def test_normal_solve_checks_lengths():
    S = _bare_solver()
    with pytest.raises(ValueError, match="D must have 32"):
        S.normal_solve(np.ones(N - 2), np.ones(M))
    with pytest.raises(ValueError, match="p must have 8"):
        S.normal_solve(np.ones(N), np.ones(M + 1))
    with pytest.raises(ValueError, match="xs must have 32"):
        S.normal_solve(np.ones(N), np.ones(M), xs=np.ones(M))
    _reaches_library(lambda: S.normal_solve(np.ones(N), np.ones(M), xs=np.ones(N)))


def test_kernel_level_calls_take_cuda_float64_tensors():
    S = _bare_solver()
    cpu = torch.ones(N, dtype=torch.float64)
    for call in (lambda: S.adat(cpu, cpu[:M]), lambda: S.sketch(cpu, 0, 0),
                 lambda: S.step_lengths(cpu, cpu, cpu, cpu),
                 lambda: S.directions(cpu, cpu, cpu, cpu[:M], cpu, 1.0)):
        with pytest.raises(TypeError, match="CUDA"):
            call()


def test_size_helper_counts_elements_of_arrays_and_tensors():
    from paper_2209_08722_gb300.solver import _mode, _need
    _need(np.ones((3, 4)), 12, "a")
    _need(torch.ones(3, 4), 12, "t")
    _need(None, 5, "absent")
    with pytest.raises(ValueError, match="t must have 11 elements, got 12"):
        _need(torch.ones(3, 4), 11, "t")
    assert _mode("feasible") == nat.LP_FEASIBLE and _mode("infeasible") == nat.LP_INFEASIBLE
    with pytest.raises(ValueError):
        _mode("Infeasible")


def test_warm_start_arguments():
    S = _bare_solver()
    with pytest.raises(ValueError, match="mode must be"):
        S.set_warm_start("learned")
    with pytest.raises(ValueError, match="needs a model"):
        S.set_warm_start("model")
    with pytest.raises(ValueError, match="both rec_X and rec_T"):
        S.set_warm_start("none", None, torch.zeros(4, 3 * M), None)
    with pytest.raises(TypeError, match="rec_X must be"):
        S.set_warm_start("none", None, torch.zeros(4, 3 * M), torch.zeros(4, M))   # CPU tensors
    _reaches_library(lambda: S.set_warm_start("previous"))


def test_phase1_and_batch_arguments():
    from paper_2209_08722_gb300 import phase1_start, solve_batch
    A = np.ones((N, M))
    with pytest.raises(ValueError, match="b must have 8"):
        phase1_start(A, np.ones(M + 1), M, N)
    with pytest.raises(TypeError, match="16-bit patterns"):
        phase1_start(A, np.ones(M), M, N, dtype="bf16")
    with pytest.raises(ValueError, match="col_ptr"):
        phase1_start(None, np.ones(M), M, N, csc=(np.zeros(3, np.int64), np.zeros(0, np.int32), np.zeros(0)))
    _reaches_library(lambda: phase1_start(A, np.ones(M), M, N, tol=0.0))   # tol must be > 0
    with pytest.raises(ValueError, match="mode"):
        solve_batch([], mode="both")


def test_state_arguments():
    # a checkpoint's vectors must have the LP's sizes before any pointer
    # reaches lp_set_state, which copies exactly n / m values from each
    S = _bare_solver()
    good = {"k": 3, "mode": 1, "has_dy_prev": 0, "mu0": 1.0, "r0": 1.0, "ratio_ref": 0.0, "seed": 0,
            "mu": 0.5, "x": np.ones(N), "y": np.zeros(M), "s": np.ones(N), "dy_prev": np.zeros(M)}
    for key, bad in (("x", np.ones(N - 1)), ("y", np.zeros(M + 1)), ("s", np.ones(M)),
                     ("dy_prev", np.zeros(N))):
        with pytest.raises(ValueError, match=f"{key} must have"):
            S.set_state(dict(good, **{key: bad}))
    with pytest.raises(KeyError):
        S.set_state({k: v for k, v in good.items() if k != "mu"})
    _reaches_library(lambda: S.set_state(good))
    _reaches_library(lambda: S.get_state())
    _reaches_library(lambda: S.check_guards())
