"""Sketching matrices W (test infrastructure; see package docstring).

Section 2 (eq. pdprec) uses a sparse embedding W in R^{n x w} with
O(log(r/delta)) nonzeros per row; Section 6 (Extensions) names the Gaussian
alternative W_G with N(0,1) entries.  The paper does not fix how the nonzeros
of a row are placed, nor the scaling; the readings used here are:

* CountSketch with s nonzeros per row: the w columns are split into s blocks
  of width w/s; row i has one nonzero in each block b, at column
  b*(w/s) + h_b(i), with value sign_b(i)/sqrt(s)  (so E[W W^T] = I).
* Gaussian: iid N(0, 1/w) entries (CG and v are invariant to scaling W;
  only the spectral-band checks depend on it).
* W is redrawn at every outer iteration k (Algorithms 2 and 3, step 2) and
  the same W serves the preconditioner and v (Section 4, after Lemma 4.1).

Random numbers come from SplitMix64 (Steele, Lea, Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), used as a counter-based
generator: output t (t = 1, 2, ...) of the stream seeded with S is
mix64(S + t * GAMMA) mod 2^64.
"""

from __future__ import annotations

import numpy as np

MASK64 = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15
MAX_RETRY = 16   # redraws per outer iteration (rank failure, Lemma 4.1)
MAX_BLOCKS = 16  # s <= 16

_U64 = np.uint64


def mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function (variant 13 of Stafford's mixers)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> _U64(30))) * _U64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> _U64(27))) * _U64(0x94D049BB133111EB)
        z = z ^ (z >> _U64(31))
    return z


def splitmix64_stream(seed: int, count: int) -> np.ndarray:
    """The first ``count`` outputs of SplitMix64 seeded with ``seed``."""
    t = np.arange(1, count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return mix64(_U64(seed & MASK64) + t * _U64(GAMMA))


def draw(seed: int, ctr: np.ndarray) -> np.ndarray:
    """Counter-based draw: output (ctr + 1) of the stream seeded with ``seed``."""
    ctr = np.asarray(ctr, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return mix64(_U64(seed & MASK64) + (ctr + _U64(1)) * _U64(GAMMA))


def countsketch_counter(k: int, retry: int, block: int, i: np.ndarray) -> np.ndarray:
    """Counter of row i, block b, outer iteration k, redraw ``retry``."""
    hi = ((k * MAX_RETRY + retry) * MAX_BLOCKS + block) << 40
    return _U64(hi & MASK64) + np.asarray(i, dtype=np.uint64)


def countsketch_hash(seed: int, k: int, retry: int, n: int, w: int, s: int):
    """Bucket and sign of every row of W for each of the s blocks.

    Returns (cols, signs): int64 arrays of shape (s, n) with the W column
    index b*(w/s) + h_b(i) and the sign +-1.
    """
    if w % s != 0:
        raise ValueError("w must be a multiple of s")
    wb = w // s
    i = np.arange(n, dtype=np.uint64)
    cols = np.empty((s, n), dtype=np.int64)
    signs = np.empty((s, n), dtype=np.float64)
    for b in range(s):
        val = draw(seed, countsketch_counter(k, retry, b, i))
        with np.errstate(over="ignore"):
            h = ((val >> _U64(32)) * _U64(wb)) >> _U64(32)   # multiply-shift range map
        cols[b] = b * wb + h.astype(np.int64)
        signs[b] = np.where((val & _U64(1)) == 0, 1.0, -1.0)
    return cols, signs


def countsketch_matrix(seed: int, k: int, retry: int, n: int, w: int, s: int):
    """W as a scipy.sparse CSR matrix (n x w), entries sign/sqrt(s)."""
    import scipy.sparse as sp
    cols, signs = countsketch_hash(seed, k, retry, n, w, s)
    rows = np.tile(np.arange(n), s)
    data = (signs / np.sqrt(s)).reshape(-1)
    return sp.csr_matrix((data, (rows, cols.reshape(-1))), shape=(n, w))


def gaussian_matrix(seed: int, k: int, retry: int, n: int, w: int) -> np.ndarray:
    """Dense W_G (n x w) with N(0, 1/w) entries via Box-Muller, both outputs.

    The draw for (k, retry) uses its own stream, seeded with
    S_kr = draw(draw(seed, 0), k*MAX_RETRY + retry).  Entry (i, j) has the flat
    index f = i*w + j and uses the draw at counter floor(f / 2) of that
    stream: its 64 bits give two uniforms that are exact in FP32,
    u1 = (bits 41..63 + 1) / 2^23 in (0, 1] and u2 = (bits 18..40) / 2^23 in
    [0, 1), and the entry is z = sqrt(-2 ln u1) cos(2 pi u2) for even f and
    z = sqrt(-2 ln u1) sin(2 pi u2) for odd f (the two independent normals of
    one Box-Muller draw).
    """
    u1, u2 = gaussian_uniforms(seed, k, retry, n, w)
    f = np.arange(n * w)
    r = np.sqrt(-2.0 * np.log(u1))[f // 2]
    ang = 2.0 * np.pi * u2[f // 2]
    z = np.where(f % 2 == 0, r * np.cos(ang), r * np.sin(ang))
    return (z / np.sqrt(w)).reshape(n, w)


def gaussian_uniforms(seed: int, k: int, retry: int, n: int, w: int):
    """The two uniforms of every draw of W_G: draws 0 .. ceil(n w / 2) - 1."""
    s_g = int(draw(seed, np.array([0], dtype=np.uint64))[0])
    s_kr = int(draw(s_g, np.array([k * MAX_RETRY + retry], dtype=np.uint64))[0])
    idx = np.arange((n * w + 1) // 2, dtype=np.uint64)
    with np.errstate(over="ignore"):
        val = draw(s_kr, idx)
    u1 = ((val >> _U64(41)).astype(np.float64) + 1.0) / 8388608.0
    u2 = ((val >> _U64(18)) & _U64(0x7FFFFF)).astype(np.float64) / 8388608.0
    return u1, u2
