"""Thin Python front-end of the CUDA library (argument marshalling only).

Every computation runs in the library's CUDA kernels; this module only turns
NumPy arrays / torch CUDA tensors into pointers and sizes and reports errors.

Entry points mirror the C ABI names (include/lp_sketch_ipm.h):
  LPSolver(...)            -> lp_create / lp_destroy
  .solve(...)              -> lp_solve           (Algorithm 2 or 3)
  .normal_solve(...)       -> lp_normal_solve    (Algorithm 1 + eq. compv)
  .adat / .residual_rhs / .sketch / .precond_apply / .directions / .step_lengths
                           -> the kernel-level entry points (device tensors)
"""

from __future__ import annotations

import ctypes
from typing import Optional

import numpy as np

from . import _native as nat

_DTYPES = {"f64": nat.LP_F64, "f32": nat.LP_F32, "bf16": nat.LP_BF16}
_NP_DT = {"f64": np.float64, "f32": np.float32, "bf16": np.uint16}
# torch dtypes accepted for each storage dtype (bf16 also as raw 16-bit patterns)
_TORCH_DT = {"f64": ("torch.float64",), "f32": ("torch.float32",),
             "bf16": ("torch.bfloat16", "torch.int16", "torch.uint16")}
_MODES = {"feasible": nat.LP_FEASIBLE, "infeasible": nat.LP_INFEASIBLE}


class LPError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{nat.STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _ptr(x) -> Optional[int]:
    if x is None:
        return None
    if _is_torch(x):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        if not x.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    raise TypeError(f"unsupported buffer type {type(x)}")


def _on_device(x) -> bool:
    return _is_torch(x) and x.is_cuda


def _numel(x) -> int:
    return int(x.numel()) if _is_torch(x) else int(np.asarray(x).size)


def _need(x, count: int, name: str):
    """The library reads exactly ``count`` elements of every buffer it is
    given: a shorter one would be read past its end, so sizes are checked here."""
    if x is not None and _numel(x) != count:
        raise ValueError(f"{name} must have {count} elements, got {_numel(x)}")


def _mode(mode: str) -> int:
    if mode not in _MODES:
        raise ValueError(f"mode must be 'feasible' or 'infeasible', got {mode!r}")
    return _MODES[mode]


def _check_dev_f64(*xs):
    for x in xs:
        if x is None:
            continue
        if not (_is_torch(x) and x.is_cuda and str(x.dtype) == "torch.float64" and x.is_contiguous()):
            raise TypeError("kernel-level calls take contiguous float64 CUDA tensors")


def _host_f64(x) -> bool:
    """A writable host buffer of float64: a C-contiguous NumPy array, or a
    contiguous CPU tensor (pinned or not)."""
    if isinstance(x, np.ndarray):
        return x.dtype == np.float64 and x.flags.c_contiguous and x.flags.writeable
    return _is_torch(x) and not x.is_cuda and str(x.dtype) == "torch.float64" and x.is_contiguous()


def _check_dev_f32(x, shape, name: str):
    if not (_is_torch(x) and x.is_cuda and str(x.dtype) == "torch.float32" and x.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous float32 CUDA tensor")
    if tuple(x.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(x.shape)}")


def _same_side(named):
    """Host or device for a whole call: the library takes one flag for all of
    a call's vectors, so a mix would hand it host pointers as device pointers
    (or the reverse).  Device vectors must be contiguous float64 tensors.
    Returns True when they are on the device."""
    given = [(k, v) for k, v in named if v is not None]
    dev = [_on_device(v) for _, v in given]
    if any(dev) and not all(dev):
        raise ValueError("pass all of " + ", ".join(k for k, _ in given)
                         + " as CUDA tensors or all as host arrays")
    if any(dev):
        _check_dev_f64(*[v for _, v in given])
    return any(dev)


class LPSolver:
    """An LP  min c^T x, A x = b, x >= 0  resident on the GPU.

    ``A`` is column-major: an (n, m) C-contiguous array whose row j is column
    a_j (NumPy on the host, or a torch CUDA tensor), in the storage dtype
    ``dtype`` ("f64", "f32" or "bf16"; bf16 given as uint16 bit patterns or a
    torch.bfloat16 tensor).  A sparse A is given instead as
    ``csc=(col_ptr, row_idx, values)`` or ``csr=(row_ptr, col_idx, values)``
    (int64 pointers, int32 indices, "f32" or "f64" values; host arrays or
    CUDA tensors), with ``A=None``; the library sorts CSR into CSC.
    """

    def __init__(self, A, b, c, m: int, n: int, dtype: str = "f32", stream=None, csc=None,
                 csr=None, **options):
        self._lib = nat.load()
        self._h = ctypes.c_void_p()
        if dtype not in _DTYPES:
            raise ValueError(f"dtype must be one of {sorted(_DTYPES)}, got {dtype!r}")
        self.m, self.n, self.dtype = int(m), int(n), dtype
        opt = nat.LpOptions()
        self._lib.lp_options_default(ctypes.byref(opt))
        for k, v in options.items():
            if not hasattr(opt, k):
                raise TypeError(f"unknown option {k}")
            setattr(opt, k, v)
        if stream is not None:
            opt.stream = stream
        self.options = opt
        if csc is not None and csr is not None:
            raise ValueError("give A as csc or as csr, not both")
        sparse = csc if csc is not None else csr
        if sparse is not None:
            # sparse A: CSC (col_ptr int64 [n+1], row_idx int32 [nnz], values [nnz])
            # or CSR (row_ptr int64 [m+1], col_idx int32 [nnz], values [nnz])
            cp, ri, vals = sparse
            if not _is_torch(cp):
                cp = np.ascontiguousarray(cp, dtype=np.int64)
                ri = np.ascontiguousarray(ri, dtype=np.int32)
                vals = np.ascontiguousarray(vals, dtype=_NP_DT[dtype])
            nnz = int(vals.shape[0])
            if csc is not None:
                _need(cp, self.n + 1, "col_ptr")
                _need(ri, nnz, "row_idx")
            else:
                _need(cp, self.m + 1, "row_ptr")
                _need(ri, nnz, "col_idx")
            mat = nat.LpMatrix(m=self.m, n=self.n, fmt=nat.LP_CSC if csc is not None else nat.LP_CSR,
                               dtype=_DTYPES[dtype], val=_ptr(vals), ld=0, ptr=_ptr(cp), idx=_ptr(ri),
                               nnz=nnz, on_device=1 if _on_device(vals) else 0)
            A = (cp, ri, vals)
        elif _is_torch(A):
            if tuple(A.shape) != (self.n, self.m):
                raise ValueError("A must have shape (n, m) (column-major)")
            if str(A.dtype) not in _TORCH_DT[dtype]:
                raise TypeError(f"A is {A.dtype}, storage dtype {dtype!r} takes {_TORCH_DT[dtype]}")
        else:
            if dtype == "bf16" and np.asarray(A).dtype not in (np.uint16, np.int16):
                raise TypeError("bf16 storage takes A as 16-bit patterns (uint16), not as values")
            A = np.ascontiguousarray(A, dtype=_NP_DT[dtype])
            if A.shape != (self.n, self.m):
                raise ValueError("A must have shape (n, m) (column-major)")
        if sparse is None:
            mat = nat.LpMatrix(m=self.m, n=self.n, fmt=nat.LP_DENSE_COLMAJOR, dtype=_DTYPES[dtype],
                               val=_ptr(A), ld=self.m, ptr=None, idx=None, nnz=0,
                               on_device=1 if _on_device(A) else 0)
        bc_dev = _same_side([("b", b), ("c", c)])
        if not bc_dev:
            b = np.ascontiguousarray(b, dtype=np.float64)
            c = np.ascontiguousarray(c, dtype=np.float64)
        _need(b, self.m, "b")
        _need(c, self.n, "c")
        self._keep = (A, b, c)
        rc = self._lib.lp_create(ctypes.byref(self._h), ctypes.byref(mat), _ptr(b), _ptr(c),
                                 1 if bc_dev else 0, ctypes.byref(opt))
        self._keep = None
        if rc != nat.LP_OK:
            raise LPError(rc, self._lib.lp_create_error().decode())

    # -- lifecycle -----------------------------------------------------------
    def close(self):
        if self._h:
            self._lib.lp_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _check(self, rc: int):
        if rc < 0:
            raise LPError(rc, self._lib.lp_last_error(self._h).decode())
        return rc

    # -- solver ------------------------------------------------------------
    def solve(self, tol: float = 1e-8, mode: str = "infeasible", x0=None, y0=None, s0=None,
              out=None):
        """lp_solve.  Host (NumPy) or device (torch CUDA) start/outputs."""
        m, n = self.m, self.n
        mode_c = _mode(mode)
        outs = [None, None, None] if out is None else list(out)
        dev = _same_side([("x0", x0), ("y0", y0), ("s0", s0), ("x", outs[0]), ("y", outs[1]),
                          ("s", outs[2])])
        if out is None:
            if dev:
                import torch
                out = (torch.empty(n, dtype=torch.float64, device="cuda"),
                       torch.empty(m, dtype=torch.float64, device="cuda"),
                       torch.empty(n, dtype=torch.float64, device="cuda"))
            else:
                out = (np.empty(n), np.empty(m), np.empty(n))
        if not dev:
            x0, y0, s0 = [None if v is None else np.ascontiguousarray(v, dtype=np.float64)
                          for v in (x0, y0, s0)]
            for name, o in zip(("x", "y", "s"), out):
                if not _host_f64(o):
                    raise TypeError(f"output {name} must be a contiguous float64 host array or tensor")
        for name, v, k in (("x0", x0, n), ("y0", y0, m), ("s0", s0, n),
                           ("x", out[0], n), ("y", out[1], m), ("s", out[2], n)):
            _need(v, k, name)
        res = nat.LpResult()
        rc = self._lib.lp_solve(self._h, float(tol), mode_c, _ptr(x0), _ptr(y0), _ptr(s0),
                                1 if dev else 0, _ptr(out[0]), _ptr(out[1]), _ptr(out[2]),
                                ctypes.byref(res))
        if rc < 0:
            raise LPError(rc, self._lib.lp_last_error(self._h).decode())
        info = res.as_dict()
        info["status_name"] = nat.STATUS_NAMES.get(rc, str(rc))
        return out[0], out[1], out[2], info

    def normal_solve(self, D, p, xs=None, k: int = 0, tol_f: float = 0.0, want_v: bool = True):
        """lp_normal_solve: returns (dy, v or None, info dict)."""
        dev = _same_side([("D", D), ("p", p), ("xs", xs)])
        if dev:
            import torch
            dy = torch.empty(self.m, dtype=torch.float64, device="cuda")
            v = torch.empty(self.n, dtype=torch.float64, device="cuda") if (want_v and xs is not None) else None
        else:
            D = np.ascontiguousarray(D, dtype=np.float64)
            p = np.ascontiguousarray(p, dtype=np.float64)
            xs = None if xs is None else np.ascontiguousarray(xs, dtype=np.float64)
            dy = np.empty(self.m)
            v = np.empty(self.n) if (want_v and xs is not None) else None
        _need(D, self.n, "D")
        _need(p, self.m, "p")
        _need(xs, self.n, "xs")
        info = nat.LpNsolveInfo()
        rc = self._lib.lp_normal_solve(self._h, _ptr(D), _ptr(p), _ptr(xs), int(k), float(tol_f),
                                       1 if dev else 0, _ptr(dy), _ptr(v), ctypes.byref(info))
        if rc < 0:
            raise LPError(rc, self._lib.lp_last_error(self._h).decode())
        d = info.as_dict()
        d["status"] = rc
        return dy, v, d

    # -- kernel-level (device tensors) ---------------------------------------
    def adat(self, d2, v, precision: int = 0):
        import torch
        _check_dev_f64(d2, v)
        _need(d2, self.n, "d2")
        _need(v, self.m, "v")
        u = torch.empty(self.m, dtype=torch.float64, device="cuda")
        self._check(self._lib.lp_adat(self._h, _ptr(d2), _ptr(v), _ptr(u), int(precision)))
        return u

    def wait_probe(self, spin_cycles: int, complete: bool) -> int:
        """lp_wait_probe: runs the pipelines' bounded device wait once on this
        handle's stream; returns the library's status code (LP_OK when the
        barrier was completed, LP_ERR_DEVICE_TIMEOUT when the wait gave up)."""
        return int(self._lib.lp_wait_probe(self._h, int(spin_cycles), 1 if complete else 0))

    def residual_rhs(self, x, y, s, mode: str = "infeasible"):
        import torch
        _check_dev_f64(x, y, s)
        for name, t, k in (("x", x, self.n), ("y", y, self.m), ("s", s, self.n)):
            _need(t, k, name)
        rp = torch.empty(self.m, dtype=torch.float64, device="cuda")
        rd = torch.empty(self.n, dtype=torch.float64, device="cuda")
        p = torch.empty(self.m, dtype=torch.float64, device="cuda")
        out5 = (ctypes.c_double * 5)()
        mode_c = _mode(mode)
        self._check(self._lib.lp_residual_rhs(self._h, _ptr(x), _ptr(y), _ptr(s), mode_c,
                                              _ptr(rp), _ptr(rd), _ptr(p), out5))
        keys = ("mu", "cx", "by", "rp_norm", "rd_norm")
        return rp, rd, p, dict(zip(keys, list(out5)))

    def sketch(self, D, seed: int, k: int, retry: int = 0):
        import torch
        _check_dev_f64(D)
        _need(D, self.n, "D")
        w = self.sketch_width
        adw = torch.empty(self.m * w, dtype=torch.float64, device="cuda")
        wout = ctypes.c_int64()
        self._check(self._lib.lp_sketch(self._h, _ptr(D), int(seed), int(k), int(retry), _ptr(adw),
                                        ctypes.byref(wout)))
        return adw.view(self.m, w)

    @property
    def sketch_width(self) -> int:
        s = self.options.s
        w = self.options.w if self.options.w > 0 else int(round(self.options.w_factor * self.m))
        w = max(w, s)
        return (w + s - 1) // s * s

    def precond_apply(self, adw, r):
        import torch
        _check_dev_f64(adw, r)
        _need(adw, self.m * self.sketch_width, "adw")
        _need(r, self.m, "r")
        z = torch.empty(self.m, dtype=torch.float64, device="cuda")
        self._check(self._lib.lp_precond_apply(self._h, _ptr(adw), _ptr(r), _ptr(z)))
        return z

    def directions(self, x, s, rd, dy, v, mu: float, mode: str = "infeasible"):
        import torch
        _check_dev_f64(x, s, rd, dy, v)
        mode_c = _mode(mode)
        if rd is None and mode_c == nat.LP_INFEASIBLE:
            raise ValueError("the infeasible directions need rd")
        for name, t, k in (("x", x, self.n), ("s", s, self.n), ("rd", rd, self.n), ("dy", dy, self.m),
                           ("v", v, self.n)):
            _need(t, k, name)
        dx = torch.empty(self.n, dtype=torch.float64, device="cuda")
        ds = torch.empty(self.n, dtype=torch.float64, device="cuda")
        self._check(self._lib.lp_directions(self._h, _ptr(x), _ptr(s), _ptr(rd), _ptr(dy), _ptr(v),
                                            float(mu), mode_c, _ptr(dx), _ptr(ds)))
        return dx, ds

    def step_lengths(self, x, s, dx, ds, mode: str = "infeasible", res_ratio: float = 0.0,
                     mu0: float = 1.0):
        _check_dev_f64(x, s, dx, ds)
        for name, t in (("x", x), ("s", s), ("dx", dx), ("ds", ds)):
            _need(t, self.n, name)
        out2 = (ctypes.c_double * 2)()
        mode_c = _mode(mode)
        self._check(self._lib.lp_step_lengths(self._h, _ptr(x), _ptr(s), _ptr(dx), _ptr(ds), mode_c,
                                              float(res_ratio), float(mu0), out2))
        return out2[0], out2[1]

    def history(self) -> list:
        """lp_get_history: per-outer-iteration records of the last solve."""
        cnt = self._lib.lp_get_history(self._h, None, 0)
        if cnt < 0:
            raise LPError(cnt, "lp_get_history failed")
        recs = (nat.LpIterRecord * max(cnt, 1))()
        self._lib.lp_get_history(self._h, recs, cnt)
        return [recs[i].as_dict() for i in range(cnt)]

    def get_state(self) -> dict:
        """lp_get_state: the state of the last solve as host arrays and scalars
        (a checkpoint: pass it to set_state on this or a fresh solver of the
        same LP to resume the outer iteration where it stopped)."""
        st = nat.LpState()
        x, y, s, dy = np.empty(self.n), np.empty(self.m), np.empty(self.n), np.empty(self.m)
        self._check(self._lib.lp_get_state(self._h, ctypes.byref(st), _ptr(x), _ptr(y), _ptr(s), _ptr(dy), 0))
        out = st.as_dict()
        out.update(x=x, y=y, s=s, dy_prev=dy)
        return out

    def set_state(self, state: dict):
        """lp_set_state: the next solve() (with no start point) resumes from
        `state` (a dict as returned by get_state)."""
        st = nat.LpState(int(state["k"]), int(state["mode"]), int(state["has_dy_prev"]), 0,
                         float(state["mu0"]), float(state["r0"]), float(state["ratio_ref"]), int(state["seed"]),
                         float(state["mu"]))
        arrs = {}
        for name, count in (("x", self.n), ("y", self.m), ("s", self.n), ("dy_prev", self.m)):
            v = np.ascontiguousarray(state[name], dtype=np.float64)
            _need(v, count, name)
            arrs[name] = v
        self._check(self._lib.lp_set_state(self._h, ctypes.byref(st), _ptr(arrs["x"]), _ptr(arrs["y"]),
                                           _ptr(arrs["s"]), _ptr(arrs["dy_prev"]), 0))

    def check_guards(self):
        """lp_check_guards: (regions checked, regions damaged, message) for a
        solver created with guard=1."""
        checked, damaged = ctypes.c_int64(), ctypes.c_int64()
        self._check(self._lib.lp_check_guards(self._h, ctypes.byref(checked), ctypes.byref(damaged)))
        msg = self._lib.lp_last_error(self._h).decode() if damaged.value else ""
        return checked.value, damaged.value, msg

    def kernel_stats(self) -> dict:
        st = nat.LpKernelStats()
        self._check(self._lib.lp_get_kernel_stats(self._h, ctypes.byref(st)))
        return {"launches": st.launches, "ms": st.ms, "bytes_per_launch": st.bytes_per_launch,
                "all_launches": st.all_launches, "graph_replays": st.graph_replays}

    def reset_kernel_stats(self):
        self._check(self._lib.lp_reset_kernel_stats(self._h))


def release_cached_memory():
    """lp_release_cached_memory: return the device blocks the library keeps
    from destroyed solvers to the driver."""
    nat.load().lp_release_cached_memory()


def from_planted(lp, device: bool = False, **options) -> LPSolver:
    """An LPSolver for an ``lpgen.PlantedLP`` (dense or CSC)."""
    if lp.sparse:
        vals = lp.val.astype(np.float32 if lp.storage == "f32" else np.float64)
        return LPSolver(None, lp.b, lp.c, lp.m, lp.n, dtype=lp.storage,
                        csc=(lp.col_ptr, lp.row_idx, vals), **options)
    A = lp.storage_array()
    b, c = lp.b, lp.c
    if device:
        import torch
        A = torch.from_numpy(A).cuda()
        b = torch.from_numpy(np.ascontiguousarray(b)).cuda()
        c = torch.from_numpy(np.ascontiguousarray(c)).cuda()
    return LPSolver(A, b, c, lp.m, lp.n, dtype=lp.storage, **options)


def csr_to_csc(row_ptr, col_idx, values, m: int, n: int, dtype: str = "f32"):
    """lp_csr_to_csc: the CSR -> CSC sort lp_create applies to CSR input, on
    host arrays.  Returns (col_ptr int64 [n+1], row_idx int32 [nnz], values)."""
    lib = nat.load()
    if dtype not in _DTYPES:
        raise ValueError(f"dtype must be one of {sorted(_DTYPES)}, got {dtype!r}")
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    vals = np.ascontiguousarray(values, dtype=_NP_DT[dtype])
    nnz = int(vals.shape[0])
    _need(rp, m + 1, "row_ptr")
    _need(ci, nnz, "col_idx")
    cp = np.empty(n + 1, dtype=np.int64)
    ri = np.empty(nnz, dtype=np.int32)
    vo = np.empty(nnz, dtype=_NP_DT[dtype])
    rc = lib.lp_csr_to_csc(m, n, nnz, _ptr(rp), _ptr(ci), _ptr(vals), _DTYPES[dtype], _ptr(cp), _ptr(ri),
                           _ptr(vo))
    if rc != nat.LP_OK:
        raise LPError(rc, "invalid CSR structure or sizes")
    return cp, ri, vo


def phase1_start(A, b, m: int, n: int, dtype: str = "f64", csc=None, tol: float = 1e-7, **options):
    """lp_phase1_start: a strictly positive x0 with A x0 = b (Appendix
    "Feasible starting point"), from host arrays.  tol is the phase-1 IPM's
    tolerance: the start only needs z small next to x before the exact
    correction, and the phase-1 optimal face is usually unbounded.  A is the (n, m) C-contiguous
    column-major buffer (or csc=(col_ptr, row_idx, values)).  Returns
    (x0, info); raises LPError with code LP_ERR_NOT_FEASIBLE when the phase-1
    optimum shows A x = b, x >= 0 infeasible."""
    lib = nat.load()
    if dtype not in _DTYPES:
        raise ValueError(f"dtype must be one of {sorted(_DTYPES)}, got {dtype!r}")
    opt = nat.LpOptions()
    lib.lp_options_default(ctypes.byref(opt))
    for k, v in options.items():
        if not hasattr(opt, k):
            raise TypeError(f"unknown option {k}")
        setattr(opt, k, v)
    if csc is not None:
        cp = np.ascontiguousarray(csc[0], dtype=np.int64)
        ri = np.ascontiguousarray(csc[1], dtype=np.int32)
        vals = np.ascontiguousarray(csc[2], dtype=_NP_DT[dtype])
        _need(cp, n + 1, "col_ptr")
        _need(ri, int(vals.shape[0]), "row_idx")
        keep = (cp, ri, vals)
        mat = nat.LpMatrix(m=m, n=n, fmt=nat.LP_CSC, dtype=_DTYPES[dtype], val=_ptr(vals), ld=0,
                           ptr=_ptr(cp), idx=_ptr(ri), nnz=int(vals.shape[0]), on_device=0)
    else:
        if dtype == "bf16" and np.asarray(A).dtype not in (np.uint16, np.int16):
            raise TypeError("bf16 storage takes A as 16-bit patterns (uint16), not as values")
        A = np.ascontiguousarray(A, dtype=_NP_DT[dtype])
        if A.shape != (n, m):
            raise ValueError("A must have shape (n, m) (column-major)")
        keep = (A,)
        mat = nat.LpMatrix(m=m, n=n, fmt=nat.LP_DENSE_COLMAJOR, dtype=_DTYPES[dtype], val=_ptr(A),
                           ld=m, ptr=None, idx=None, nnz=0, on_device=0)
    b = np.ascontiguousarray(b, dtype=np.float64)
    _need(b, m, "b")
    x0 = np.empty(n, dtype=np.float64)
    info = nat.LpPhase1Info()
    rc = lib.lp_phase1_start(ctypes.byref(mat), _ptr(b), ctypes.byref(opt), float(tol), _ptr(x0),
                             ctypes.byref(info))
    del keep
    if rc < 0:
        err = LPError(rc, "phase-1 start failed")
        err.info = info.as_dict()
        raise err
    return x0, info.as_dict()


def solve_batch(solvers, tol: float = 1e-8, mode: str = "infeasible", max_threads: int = 0):
    """lp_solve_batch: solve independent LPs (one LPSolver each) concurrently
    from the default start; returns [(x, y, s, info), ...] with host arrays."""
    lib = nat.load()
    count = len(solvers)
    hs = (ctypes.c_void_p * count)(*[S._h.value for S in solvers])
    outs = [(np.empty(S.n), np.empty(S.m), np.empty(S.n)) for S in solvers]
    xs = (ctypes.c_void_p * count)(*[o[0].ctypes.data for o in outs])
    ys = (ctypes.c_void_p * count)(*[o[1].ctypes.data for o in outs])
    ss = (ctypes.c_void_p * count)(*[o[2].ctypes.data for o in outs])
    res = (nat.LpResult * count)()
    m = _mode(mode)
    rc = lib.lp_solve_batch(hs, count, float(tol), m, 0, xs, ys, ss, int(max_threads), res)
    if rc < 0:
        raise LPError(rc, "batched solve failed")
    return [(o[0], o[1], o[2], res[i].as_dict()) for i, o in enumerate(outs)]


class Mlp:
    """lp_mlp: the warm-start model (features 3m -> hidden -> hidden -> m, GELU).
    Batches are torch CUDA float32 tensors of shape (batch, features)."""

    def __init__(self, in_dim: int, hidden: int, out_dim: int, seed: int = 0, stream=None):
        self._lib = nat.load()
        self._h = ctypes.c_void_p()
        rc = self._lib.lp_mlp_create(ctypes.byref(self._h), int(in_dim), int(hidden), int(out_dim),
                                     int(seed), stream)
        if rc != nat.LP_OK:
            raise LPError(rc, "lp_mlp_create failed")
        self.in_dim, self.hidden, self.out_dim = int(in_dim), int(hidden), int(out_dim)

    def close(self):
        if self._h:
            self._lib.lp_mlp_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def num_params(self) -> int:
        return int(self._lib.lp_mlp_num_params(self._h))

    def params(self) -> np.ndarray:
        out = np.empty(self.num_params, dtype=np.float32)
        self._check(self._lib.lp_mlp_get_params(self._h, out.ctypes.data))
        return out

    def set_params(self, flat):
        flat = np.ascontiguousarray(flat, dtype=np.float32)
        _need(flat, self.num_params, "params")
        self._check(self._lib.lp_mlp_set_params(self._h, flat.ctypes.data))

    def grads(self) -> np.ndarray:
        out = np.empty(self.num_params, dtype=np.float32)
        self._check(self._lib.lp_mlp_get_grads(self._h, out.ctypes.data))
        return out

    def forward(self, X):
        import torch
        _check_dev_f32(X, (X.shape[0], self.in_dim) if X.dim() == 2 else (-1,), "X")
        Y = torch.empty(X.shape[0], self.out_dim, dtype=torch.float32, device="cuda")
        self._check(self._lib.lp_mlp_forward(self._h, _ptr(X), int(X.shape[0]), _ptr(Y)))
        return Y

    def _check_batch(self, X, T):
        batch = int(X.shape[0]) if X.dim() == 2 else -1
        _check_dev_f32(X, (batch, self.in_dim), "X")
        _check_dev_f32(T, (batch, self.out_dim), "T")

    def loss_grad(self, X, T) -> float:
        self._check_batch(X, T)
        loss = ctypes.c_double()
        self._check(self._lib.lp_mlp_loss_grad(self._h, _ptr(X), _ptr(T), int(X.shape[0]), ctypes.byref(loss)))
        return loss.value

    def train_step(self, X, T, lr: float) -> float:
        self._check_batch(X, T)
        loss = ctypes.c_double()
        self._check(self._lib.lp_mlp_train_step(self._h, _ptr(X), _ptr(T), int(X.shape[0]), float(lr),
                                                ctypes.byref(loss)))
        return loss.value

    def _check(self, rc):
        if rc != nat.LP_OK:
            raise LPError(rc, "lp_mlp call failed")


def _set_warm_start(self, mode: str = "none", model: Mlp = None, rec_X=None, rec_T=None):
    """lp_set_warm_start: mode "none" | "previous" | "model"; rec_X (cap, 3m) and
    rec_T (cap, m) float32 CUDA tensors receive (features, target) per outer
    iteration when given."""
    modes = {"none": 0, "previous": 1, "model": 2}
    if mode not in modes:
        raise ValueError(f"mode must be one of {sorted(modes)}, got {mode!r}")
    if mode == "model" and model is None:
        raise ValueError("mode 'model' needs a model")
    if model is not None and (model.in_dim, model.out_dim) != (3 * self.m, self.m):
        raise ValueError(f"the model must map 3m = {3 * self.m} features to m = {self.m} outputs")
    if (rec_X is None) != (rec_T is None):
        raise ValueError("give both rec_X and rec_T, or neither")
    cap = 0 if rec_X is None else int(rec_X.shape[0])
    if rec_X is not None:
        _check_dev_f32(rec_X, (cap, 3 * self.m), "rec_X")
        _check_dev_f32(rec_T, (cap, self.m), "rec_T")
    self._warm_keep = (model, rec_X, rec_T)
    self._check(self._lib.lp_set_warm_start(self._h, modes[mode], model._h if model else None, _ptr(rec_X),
                                            _ptr(rec_T), cap))


def _warm_start_stats(self) -> dict:
    a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    self._check(self._lib.lp_get_warm_start_stats(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return {"recorded": a.value, "proposals": b.value, "accepted": c.value}


LPSolver.set_warm_start = _set_warm_start
LPSolver.warm_start_stats = _warm_start_stats
