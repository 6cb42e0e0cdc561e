"""Planted-optimum LP generators (seeded, synthetic).

Every instance is drawn from ``numpy.random.default_rng(seed)`` in a fixed
order, so a (generator, sizes, seed) triple names one problem exactly.

The shapes follow the tall/wide regime the paper targets (m << n, Section 1)
and stand in for its l1-SVM data sets, which are not available here.
"""

from __future__ import annotations

import dataclasses
import os
from typing import Optional

import numpy as np


# ---------------------------------------------------------------------------
# storage rounding
# ---------------------------------------------------------------------------

def bf16_bits(a: np.ndarray) -> np.ndarray:
    """Round FP64/FP32 values to bfloat16 (round to nearest even); uint16 bits."""
    f = np.ascontiguousarray(a, dtype=np.float32)
    u = f.view(np.uint32)
    # NaN is not produced by the generators; plain RNE on the upper 16 bits.
    # For finite values u + 0x8000 stays below 2^32, so 32-bit arithmetic holds.
    rounding = np.uint32(0x7FFF) + ((u >> np.uint32(16)) & np.uint32(1))
    return ((u + rounding) >> np.uint32(16)).astype(np.uint16)


def round_bf16(a: np.ndarray) -> np.ndarray:
    """Values of ``a`` after bfloat16 storage, as FP64."""
    bits = bf16_bits(a).astype(np.uint32) << 16
    return bits.view(np.float32).astype(np.float64)


def _round_storage(a: np.ndarray, storage: str) -> np.ndarray:
    if storage == "f64":
        return np.asarray(a, dtype=np.float64)
    if storage == "f32":
        return np.asarray(a, dtype=np.float32).astype(np.float64)
    if storage == "bf16":
        return round_bf16(a)
    raise ValueError(f"unknown storage {storage!r}")


# ---------------------------------------------------------------------------
# planted problems
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class PlantedLP:
    """A planted LP.  ``A`` holds the stored (rounded) values in FP64.

    Dense problems keep ``A`` as an (m, n) array; sparse problems keep CSC
    arrays (``col_ptr``, ``row_idx``, ``val``) and ``A`` is None unless
    requested with ``dense()``.
    """

    m: int
    n: int
    b: np.ndarray
    c: np.ndarray
    x_star: np.ndarray
    y_star: np.ndarray
    s_star: np.ndarray
    basis: np.ndarray
    storage: str = "f64"
    A: Optional[np.ndarray] = None
    col_ptr: Optional[np.ndarray] = None
    row_idx: Optional[np.ndarray] = None
    val: Optional[np.ndarray] = None
    cols: Optional[np.ndarray] = None   # blocked dense problems: (n, m) storage array

    @property
    def sparse(self) -> bool:
        return self.col_ptr is not None

    @property
    def objective(self) -> float:
        """c^T x* (= b^T y*): the planted optimal value."""
        return float(self.c @ self.x_star)

    def dense(self) -> np.ndarray:
        if self.A is not None:
            return self.A
        if self.cols is not None:
            # FP64 values of the stored (already rounded) entries, (m, n)
            if self.storage == "bf16":
                vals = (self.cols.astype(np.uint32) << np.uint32(16)).view(np.float32)
            else:
                vals = self.cols
            self.A = np.ascontiguousarray(vals.T, dtype=np.float64)
            return self.A
        A = np.zeros((self.m, self.n))
        for j in range(self.n):
            lo, hi = self.col_ptr[j], self.col_ptr[j + 1]
            A[self.row_idx[lo:hi], j] = self.val[lo:hi]
        return A

    def scipy_csc(self):
        import scipy.sparse as sp
        return sp.csc_matrix((self.val, self.row_idx, self.col_ptr), shape=(self.m, self.n))

    def storage_array(self) -> np.ndarray:
        """Column-major storage of dense A in its storage dtype.

        Returned as an (n, m) C-contiguous array (row j = column a_j), i.e. the
        column-major layout with leading dimension m; bf16 is returned as its
        uint16 bit pattern.
        """
        if self.cols is not None:
            return self.cols
        assert self.A is not None
        if self.storage == "f64":
            return np.ascontiguousarray(self.A.T)
        if self.storage == "f32":
            return np.ascontiguousarray(self.A.astype(np.float32).T)
        return np.ascontiguousarray(bf16_bits(self.A).T)


def _plant(rng: np.random.Generator, m: int, n: int):
    basis = np.sort(rng.choice(n, size=m, replace=False))
    x_star = np.zeros(n)
    x_star[basis] = rng.uniform(1.0, 2.0, size=m)
    s_star = rng.uniform(1.0, 2.0, size=n)
    s_star[basis] = 0.0
    y_star = rng.standard_normal(m)
    return basis, x_star, y_star, s_star


def planted_dense(m: int, n: int, seed: int = 0, storage: str = "f64",
                  col_scale_log10: Optional[tuple] = None) -> PlantedLP:
    """Dense planted LP with iid N(0,1) entries.

    ``col_scale_log10=(lo, hi)`` multiplies column j by 10**U(lo, hi)
    (log-uniform column scaling).  A is rounded to ``storage`` first, then
    b = A x*, c = A^T y* + s* are formed in FP64 from the rounded A.
    """
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, n))
    if col_scale_log10 is not None:
        lo, hi = col_scale_log10
        A *= 10.0 ** rng.uniform(lo, hi, size=n)
    A = _round_storage(A, storage)
    basis, x_star, y_star, s_star = _plant(rng, m, n)
    b = A @ x_star
    c = A.T @ y_star + s_star
    return PlantedLP(m=m, n=n, b=b, c=c, x_star=x_star, y_star=y_star,
                     s_star=s_star, basis=basis, storage=storage, A=A)


def _storage_cols(block: np.ndarray, storage: str) -> np.ndarray:
    """(cols, m) float32 draws -> the storage dtype (bf16 as uint16 bits)."""
    if storage == "bf16":
        return bf16_bits(block)
    if storage == "f32":
        return block
    return block.astype(np.float64)


def _cols_values(cols: np.ndarray, storage: str) -> np.ndarray:
    """Stored entries of a column block as FP64 values."""
    if storage == "bf16":
        return (cols.astype(np.uint32) << np.uint32(16)).view(np.float32).astype(np.float64)
    return cols.astype(np.float64)


def planted_dense_blocked(m: int, n: int, seed: int = 0, storage: str = "bf16",
                          col_scale_log10: Optional[tuple] = None, block: int = 8192,
                          threads: Optional[int] = None) -> PlantedLP:
    """Dense planted LP with iid N(0,1) entries, drawn column block by column
    block so that 10^9-entry instances are generated in seconds.

    Block q (columns q*block ... q*block+block-1) is drawn from its own
    generator ``default_rng([seed, 1, q])`` as float32 normals, one row per
    column (the column-major storage order), then multiplied by its columns'
    10**U(lo, hi) scales (drawn after the normals from the same generator)
    and rounded to ``storage``.  The planted optimum comes from
    ``default_rng([seed, 2])``.  b = A x* (only the m basic columns enter) and
    c = A^T y* + s* are formed in FP64 from the stored values.  The blocks are
    independent, so the result does not depend on ``threads``.

    The stored matrix is kept only in its storage dtype (``cols``, an (n, m)
    array = column-major with leading dimension m); ``dense()`` expands it to
    FP64 on request.
    """
    import concurrent.futures as cf
    if storage not in ("f64", "f32", "bf16"):
        raise ValueError(f"unknown storage {storage!r}")
    sdt = {"bf16": np.uint16, "f32": np.float32, "f64": np.float64}[storage]
    cols = np.empty((n, m), dtype=sdt)
    basis, x_star, y_star, s_star = _plant(np.random.default_rng([seed, 2]), m, n)
    c = np.empty(n)
    nblocks = (n + block - 1) // block

    def fill(q):
        j0, j1 = q * block, min(n, (q + 1) * block)
        rng = np.random.default_rng([seed, 1, q])
        blk = rng.standard_normal((j1 - j0, m), dtype=np.float32)
        if col_scale_log10 is not None:
            lo, hi = col_scale_log10
            blk *= (10.0 ** rng.uniform(lo, hi, size=j1 - j0)).astype(np.float32)[:, None]
        cols[j0:j1] = _storage_cols(blk, storage)
        c[j0:j1] = _cols_values(cols[j0:j1], storage) @ y_star + s_star[j0:j1]

    workers = threads or min(32, os.cpu_count() or 1)
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        list(ex.map(fill, range(nblocks)))
    b = _cols_values(cols[basis], storage).T @ x_star[basis]
    return PlantedLP(m=m, n=n, b=b, c=c, x_star=x_star, y_star=y_star,
                     s_star=s_star, basis=basis, storage=storage, cols=cols)


def planted_sparse(m: int, n: int, nnz_per_col: int = 8, seed: int = 0,
                   zipf_frac: float = 0.2, zipf_a: float = 1.2,
                   storage: str = "f32") -> PlantedLP:
    """Sparse planted LP in CSC form.

    Each column has ``nnz_per_col`` distinct rows: a fraction ``1-zipf_frac``
    uniform over rows, the rest drawn from a Zipf(zipf_a) rank distribution
    mapped through a random row permutation (heavy-tailed row counts).
    Values are N(0,1), rounded to ``storage``.
    """
    rng = np.random.default_rng(seed)
    k = nnz_per_col
    if k > m:
        raise ValueError("nnz_per_col > m")
    perm = rng.permutation(m)
    rows = rng.integers(0, m, size=(n, k))
    zipf_mask = rng.random((n, k)) < zipf_frac

    def zipf_rows(cnt):
        out = np.empty(cnt, dtype=np.int64)
        filled = 0
        while filled < cnt:
            z = rng.zipf(zipf_a, size=2 * (cnt - filled) + 16)
            z = z[z <= m]
            take = min(len(z), cnt - filled)
            out[filled:filled + take] = perm[z[:take] - 1]
            filled += take
        return out

    rows[zipf_mask] = zipf_rows(int(zipf_mask.sum()))
    # resample repeated rows within a column (uniformly) until all distinct
    while True:
        srt = np.sort(rows, axis=1)
        dup_cols = np.nonzero((srt[:, 1:] == srt[:, :-1]).any(axis=1))[0]
        if dup_cols.size == 0:
            break
        sub = rows[dup_cols]
        for t in range(1, k):
            clash = (sub[:, t:t + 1] == sub[:, :t]).any(axis=1)
            sub[clash, t] = rng.integers(0, m, size=int(clash.sum()))
        rows[dup_cols] = sub
    rows.sort(axis=1)
    vals = rng.standard_normal((n, k))
    vals = _round_storage(vals, storage)
    col_ptr = np.arange(0, n * k + 1, k, dtype=np.int64)
    row_idx = rows.reshape(-1).astype(np.int32)
    val = vals.reshape(-1)
    basis, x_star, y_star, s_star = _plant(rng, m, n)
    # b = A x*, c = A^T y* + s* in FP64 from the stored values
    b = np.zeros(m)
    np.add.at(b, row_idx, val * np.repeat(x_star, k))
    c = (val * y_star[row_idx]).reshape(n, k).sum(axis=1) + s_star
    return PlantedLP(m=m, n=n, b=b, c=c, x_star=x_star, y_star=y_star,
                     s_star=s_star, basis=basis, storage=storage,
                     col_ptr=col_ptr, row_idx=row_idx, val=val)


# ---------------------------------------------------------------------------
# strictly feasible start for planted problems
# ---------------------------------------------------------------------------

def feasible_start(lp: PlantedLP, gamma: float, shrink: float = 0.5):
    """A strictly feasible (x0, y0, s0) with x0 o s0 >= (1-gamma) mu0.

    With B the planted support (|B| = m, A_B nonsingular):
      primal: delta_N = 1, A_B delta_B = -A_N 1, x0 = x* + t delta  (A x0 = b)
      dual:   A_B^T u = 1, y0 = y* - t u, s0 = c - A^T y0 = s* + t A^T u
              (so s0_B = t).
    t starts at ``shrink`` times the largest value keeping (x0, s0) > 0 and
    is halved until the neighbourhood condition holds.
    """
    A = lp.dense()
    B = lp.basis
    N = np.setdiff1d(np.arange(lp.n), B)
    AB = A[:, B]
    delta = np.ones(lp.n)
    delta[B] = np.linalg.solve(AB, -A[:, N].sum(axis=1))
    u = np.linalg.solve(AB.T, np.ones(lp.m))
    g = A.T @ u
    # largest t with x* + t delta > 0 and s* + t g > 0
    tmax = np.inf
    neg = delta < 0
    if neg.any():
        tmax = min(tmax, np.min(lp.x_star[neg] / -delta[neg]))
    neg = g < 0
    if neg.any():
        tmax = min(tmax, np.min(lp.s_star[neg] / -g[neg]))
    t = shrink * (tmax if np.isfinite(tmax) else 1.0)
    for _ in range(200):
        x0 = lp.x_star + t * delta
        y0 = lp.y_star - t * u
        s0 = lp.c - A.T @ y0
        if (x0 > 0).all() and (s0 > 0).all():
            mu0 = x0 @ s0 / lp.n
            if np.min(x0 * s0) >= (1.0 - gamma) * mu0:
                return x0, y0, s0
        t *= 0.5
    raise RuntimeError("no strictly feasible start found")


# ---------------------------------------------------------------------------
# the five workload shapes
# ---------------------------------------------------------------------------

CONFIGS = {
    # feasible-start IPM, FP64, dense 64 x 4096, CountSketch w=4m, s=2
    "c1": dict(kind="dense", m=64, n=4096, storage="f64", col_scale=None,
               mode="feasible", w_factor=4.0, s=2, seed=0),
    # infeasible-start IPM, FP32 storage, dense 512 x 131072,
    # columns scaled by 10**U(-2, 2), CountSketch w=4m, s=4
    "c2": dict(kind="dense", m=512, n=131072, storage="f32", col_scale=(-2.0, 2.0),
               mode="infeasible", w_factor=4.0, s=4, seed=0),
    # infeasible-start IPM, sparse CSC 4096 x 2,000,000, 8 nnz per column,
    # 20% Zipf(1.2) rows, CountSketch w=3m, s=2
    "c3": dict(kind="sparse", m=4096, n=2_000_000, storage="f32", nnz_per_col=8,
               mode="infeasible", w_factor=3.0, s=2, seed=0),
    # BF16 storage, dense 2048 x 524288, CountSketch w=4m, s=4 (s is not
    # given for this workload; 4 as for the 512 x 131072 one, whose sketches
    # stay well conditioned near the optimum); drawn column block by column
    # block (10^9 entries)
    "c4": dict(kind="dense_blocked", m=2048, n=524288, storage="bf16", col_scale=None,
               mode="infeasible", w_factor=4.0, s=4, seed=0),
}


def make(cfg: dict, m: Optional[int] = None, n: Optional[int] = None,
         seed: Optional[int] = None) -> PlantedLP:
    m = cfg["m"] if m is None else m
    n = cfg["n"] if n is None else n
    seed = cfg["seed"] if seed is None else seed
    if cfg["kind"] == "dense":
        return planted_dense(m, n, seed=seed, storage=cfg["storage"],
                             col_scale_log10=cfg.get("col_scale"))
    if cfg["kind"] == "dense_blocked":
        return planted_dense_blocked(m, n, seed=seed, storage=cfg["storage"],
                                     col_scale_log10=cfg.get("col_scale"))
    return planted_sparse(m, n, nnz_per_col=cfg.get("nnz_per_col", 8), seed=seed,
                          storage=cfg["storage"])


def config_small(name: str, div: int = 8, seed: Optional[int] = None) -> PlantedLP:
    """The named workload with m and n divided by ``div`` (CI-sized)."""
    cfg = CONFIGS[name]
    return make(cfg, m=max(4, cfg["m"] // div), n=max(16, cfg["n"] // div), seed=seed)


def batch_family(count: int, seed: int = 0, m_range=(32, 512), k_range=(64, 256),
                 storage: str = "f32"):
    """The batched-LP family: LP i has m_i ~ U{m_range}, n_i = m_i k_i with
    k_i ~ U{k_range}, N(0,1) entries, planted optimum, seed (seed, i)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        m = int(rng.integers(m_range[0], m_range[1] + 1))
        k = int(rng.integers(k_range[0], k_range[1] + 1))
        out.append(planted_dense(m, m * k, seed=int(seed * 100003 + i), storage=storage))
    return out
