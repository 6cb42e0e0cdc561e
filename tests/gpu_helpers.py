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
    from paper_2209_08722_gb300 import from_planted
    return from_planted(lp, **opts)


def adat_bound(A, d2, v):
    """|A| diag(d2) |A|^T |v|: the scale of the rounding error of A diag(d2) A^T v."""
    return np.abs(A) @ (d2 * (np.abs(A).T @ np.abs(v)))
