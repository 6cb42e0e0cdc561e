"""ctypes declarations of the C ABI in include/lp_sketch_ipm.h.

Loading fails loudly when the in-tree library has not been built: there is no
fallback of any kind.
"""

from __future__ import annotations

import ctypes
import os
from ctypes import c_float, POINTER, c_char_p, c_double, c_int32, c_int64, c_uint64, c_void_p

from .build_native import lib_path

LP_OK = 0
LP_ERR_ARG = -1
LP_ERR_CUDA = -2
LP_ERR_OOM = -3
LP_ERR_SKETCH_RANK = -4
LP_ERR_NOT_FEASIBLE = -5
LP_ERR_NUMERICAL = -6
LP_ERR_DEVICE_TIMEOUT = -7
LP_ERR_UNSUPPORTED = -8
LP_STATUS_MAX_ITER = 1
LP_WARN_INNER_MAXIT = 2
LP_STATUS_STALLED = 3

LP_DENSE_COLMAJOR, LP_CSC, LP_CSR = 0, 1, 2
LP_F64, LP_F32, LP_BF16 = 0, 1, 2
LP_SKETCH_COUNT, LP_SKETCH_GAUSS = 0, 1
LP_INNER_CG, LP_INNER_CHEBYSHEV = 0, 1
LP_RULE_THEORY, LP_RULE_RELATIVE = 0, 1
LP_FEASIBLE, LP_INFEASIBLE = 0, 1

STATUS_NAMES = {
    0: "LP_OK", -1: "LP_ERR_ARG", -2: "LP_ERR_CUDA", -3: "LP_ERR_OOM",
    -4: "LP_ERR_SKETCH_RANK", -5: "LP_ERR_NOT_FEASIBLE", -6: "LP_ERR_NUMERICAL",
    -7: "LP_ERR_DEVICE_TIMEOUT", -8: "LP_ERR_UNSUPPORTED", 1: "LP_STATUS_MAX_ITER",
    2: "LP_WARN_INNER_MAXIT", 3: "LP_STATUS_STALLED",
}


class LpMatrix(ctypes.Structure):
    _fields_ = [("m", c_int32), ("n", c_int64), ("fmt", c_int32), ("dtype", c_int32),
                ("val", c_void_p), ("ld", c_int64), ("ptr", c_void_p), ("idx", c_void_p),
                ("nnz", c_int64), ("on_device", c_int32)]


class LpOptions(ctypes.Structure):
    _fields_ = [("sigma", c_double), ("gamma", c_double), ("tol_cg", c_double),
                ("inner_rule", c_int32), ("sketch", c_int32), ("s", c_int32),
                ("inner", c_int32), ("refine_every", c_int32), ("k_max", c_int32),
                ("t_max", c_int32), ("v_correction", c_int32), ("cheb_lanczos", c_int32),
                ("profile", c_int32), ("w_factor", c_double), ("w", c_int64),
                ("seed", c_uint64), ("stream", c_void_p), ("tensor_sketch", c_int32),
                ("precondition", c_int32), ("sigma_rule", c_int32), ("graphs", c_int32),
                ("autotune", c_int32), ("guard", c_int32)]


class LpResult(ctypes.Structure):
    _fields_ = [("status", c_int32), ("outer_iterations", c_int32), ("inner_total", c_int64),
                ("inner_max", c_int32), ("sketch_retries", c_int32), ("primal_obj", c_double),
                ("dual_obj", c_double), ("rel_gap", c_double), ("rp_rel", c_double),
                ("rd_rel", c_double), ("mu", c_double), ("ms_total", c_double),
                ("ms_residual", c_double), ("ms_sketch", c_double), ("ms_factor", c_double),
                ("ms_inner", c_double), ("ms_correction", c_double), ("ms_step", c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class LpNsolveInfo(ctypes.Structure):
    _fields_ = [("inner_iterations", c_int32), ("retries", c_int32), ("f_norm", c_double),
                ("f0_norm", c_double), ("v_norm", c_double), ("lam_min", c_double),
                ("lam_max", c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class LpIterRecord(ctypes.Structure):
    _fields_ = [("k", c_int32), ("inner_iterations", c_int32), ("retries", c_int32),
                ("inner_status", c_int32), ("mu", c_double), ("rel_gap", c_double),
                ("rp_rel", c_double), ("rd_rel", c_double), ("f_norm", c_double),
                ("f0_norm", c_double), ("tol_f", c_double), ("alpha_max", c_double),
                ("alpha_bar", c_double), ("sigma", c_double), ("r_ratio", c_double),
                ("factor_kind", c_int32), ("reserved", c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class LpPhase1Info(ctypes.Structure):
    _fields_ = [("z_sum", c_double), ("residual", c_double), ("x0_min", c_double),
                ("outer_iterations", c_int32), ("inner_total", c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class LpState(ctypes.Structure):
    _fields_ = [("k", c_int32), ("mode", c_int32), ("has_dy_prev", c_int32), ("reserved", c_int32),
                ("mu0", c_double), ("r0", c_double), ("ratio_ref", c_double), ("seed", c_uint64),
                ("mu", c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class LpKernelStats(ctypes.Structure):
    _fields_ = [("launches", c_int64), ("ms", c_double), ("bytes_per_launch", c_int64),
                ("all_launches", c_int64), ("graph_replays", c_int64)]


# name -> (restype, argtypes); every symbol of include/lp_sketch_ipm.h
P = c_void_p
SIGNATURES = {
    "lp_options_default": (None, [POINTER(LpOptions)]),
    "lp_create": (c_int32, [POINTER(P), POINTER(LpMatrix), P, P, c_int32, POINTER(LpOptions)]),
    "lp_destroy": (c_int32, [P]),
    "lp_last_error": (c_char_p, [P]),
    "lp_create_error": (c_char_p, []),
    "lp_solve": (c_int32, [P, c_double, c_int32, P, P, P, c_int32, P, P, P, POINTER(LpResult)]),
    "lp_normal_solve": (c_int32, [P, P, P, P, c_int64, c_double, c_int32, P, P,
                                  POINTER(LpNsolveInfo)]),
    "lp_adat": (c_int32, [P, P, P, P, c_int32]),
    "lp_residual_rhs": (c_int32, [P, P, P, P, c_int32, P, P, P, P]),
    "lp_sketch": (c_int32, [P, P, c_uint64, c_int64, c_int32, P, POINTER(c_int64)]),
    "lp_precond_apply": (c_int32, [P, P, P, P]),
    "lp_directions": (c_int32, [P, P, P, P, P, P, c_double, c_int32, P, P]),
    "lp_step_lengths": (c_int32, [P, P, P, P, P, c_int32, c_double, c_double, P]),
    "lp_get_history": (c_int32, [P, POINTER(LpIterRecord), c_int32]),
    "lp_get_state": (c_int32, [P, POINTER(LpState), P, P, P, P, c_int32]),
    "lp_set_state": (c_int32, [P, POINTER(LpState), P, P, P, P, c_int32]),
    "lp_adat_noalloc": (c_int32, [P, c_int32, c_int32, c_int64, c_int64, P, P, P, P]),
    "lp_wait_probe": (c_int32, [P, c_int64, c_int32]),
    "lp_csr_to_csc": (c_int32, [c_int32, c_int64, c_int64, P, P, P, c_int32, P, P, P]),
    "lp_phase1_start": (c_int32, [POINTER(LpMatrix), P, POINTER(LpOptions), c_double, P,
                                  POINTER(LpPhase1Info)]),
    "lp_solve_batch": (c_int32, [POINTER(P), c_int32, c_double, c_int32, c_int32, POINTER(P),
                                 POINTER(P), POINTER(P), c_int32, POINTER(LpResult)]),
    "lp_mlp_create": (c_int32, [POINTER(P), c_int32, c_int32, c_int32, c_uint64, P]),
    "lp_mlp_destroy": (c_int32, [P]),
    "lp_mlp_num_params": (c_int64, [P]),
    "lp_mlp_get_params": (c_int32, [P, P]),
    "lp_mlp_set_params": (c_int32, [P, P]),
    "lp_mlp_get_grads": (c_int32, [P, P]),
    "lp_mlp_forward": (c_int32, [P, P, c_int32, P]),
    "lp_mlp_loss_grad": (c_int32, [P, P, P, c_int32, POINTER(c_double)]),
    "lp_mlp_train_step": (c_int32, [P, P, P, c_int32, c_float, POINTER(c_double)]),
    "lp_set_warm_start": (c_int32, [P, c_int32, P, P, P, c_int32]),
    "lp_get_warm_start_stats": (c_int32, [P, POINTER(c_int64), POINTER(c_int64), POINTER(c_int64)]),
    "lp_get_kernel_stats": (c_int32, [P, POINTER(LpKernelStats)]),
    "lp_check_guards": (c_int32, [P, POINTER(c_int64), POINTER(c_int64)]),
    "lp_release_cached_memory": (c_int32, []),
    "lp_reset_kernel_stats": (c_int32, [P]),
}

_LIB = None


def load(path: str | None = None):
    """The loaded library (ctypes.CDLL) with every prototype declared."""
    global _LIB
    if _LIB is not None and path is None:
        return _LIB
    p = path or lib_path()
    if not os.path.exists(p):
        raise ImportError(
            f"CUDA library {p} is missing: build it with "
            "`python -c 'import __graft_entry__ as g; g.build()'` "
            "(or paper_2209_08722_gb300.build_native.build())")
    lib = ctypes.CDLL(p)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _LIB = lib
    return lib
