"""Shared helpers for the GPU tests (imported by tests only)."""

import numpy as np
import pytest

EPS32 = 2.0 ** -24
EPS64 = 2.0 ** -53


def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def solver_for(lp, **opts):
    """A solver for a planted LP, created with guard regions around its device
    buffers (unless guard=0 is asked for); closing it fails the test when a
    kernel wrote past the end of a buffer."""
    from paper_2209_08722_gb300 import from_planted
    opts.setdefault("guard", 1)
    S = from_planted(lp, **opts)
    if opts["guard"]:
        close = S.close

        def close_checked():
            if S._h:
                checked, damaged, msg = S.check_guards()
                close()
                assert checked > 0 and damaged == 0, msg
            close()

        S.close = close_checked
    return S


def adat_bound(A, d2, v):
    """|A| diag(d2) |A|^T |v|: the scale of the rounding error of A diag(d2) A^T v."""
    return np.abs(A) @ (d2 * (np.abs(A).T @ np.abs(v)))


def fp32_lane_columns(m, n, storage):
    """Bound on the columns one lane sums in FP32 in the inner-loop product:
    the warp-per-column kernel (columns of at most 7 16-byte vectors per lane,
    m <= 512 in FP32, m <= 1024 in BF16) spreads a CTA's columns over 16 warps
    (n / 1216 + 64); the row-split kernel for taller columns gives each lane
    4 columns of every tile of its CTA (n / 152 + 64)."""
    vec = 4 if storage == "f32" else 8
    vpl = -(-((m + vec - 1) // vec) // 32)
    return n // 1216 + 64 if vpl < 8 else n // 152 + 64
