"""The paper's random synthetic LP family (Appendix, "Random data").

A (m x n): each entry i.i.d. U(0,1) with probability p, else 0; then
min(m, n) further U(0,1) draws are added to the main diagonal, so every row
has a nonzero.  b = A x + 0.1 z with x, z ~ N(0,1); c ~ N(0,1).

Nothing guarantees that such an LP is feasible or bounded (x has negative
entries), so its optimum is not known in closed form; it serves as a smoke
workload and as input to the phase-1 start.
"""

from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class RandomLP:
    A: np.ndarray   # FP64 dense
    b: np.ndarray
    c: np.ndarray
    m: int
    n: int
    density: float

    def storage_array(self, storage: str = "f64") -> np.ndarray:
        """A as the (n, m) C-contiguous buffer = column-major m x n."""
        dt = {"f64": np.float64, "f32": np.float32}[storage]
        return np.ascontiguousarray(self.A.T.astype(dt))


def random_lp(m: int, n: int, density: float = 0.1, seed: int = 0) -> RandomLP:
    rng = np.random.default_rng(seed)
    mask = rng.random((m, n)) < density
    A = np.where(mask, rng.random((m, n)), 0.0)
    k = min(m, n)
    A[np.arange(k), np.arange(k)] += rng.random(k)
    x = rng.standard_normal(n)
    z = rng.standard_normal(m)
    b = A @ x + 0.1 * z
    c = rng.standard_normal(n)
    return RandomLP(A=A, b=b, c=c, m=m, n=n, density=density)
