"""Failure detection on the GPU: the bounded device-side wait every pipeline
uses (an mbarrier wait with a spin limit) gives up, records the timeout in the
handle's device status word, and the library returns LP_ERR_DEVICE_TIMEOUT;
the handle then keeps working.  The wait is made to run out the allowed way:
on a barrier that nothing completes, with a short limit (10^5 cycles, about
50 microseconds), so no kernel is left waiting and nothing faults."""

import numpy as np
import pytest

import lpgen
from tests.gpu_helpers import EPS32, adat_bound, dev, fp32_lane_columns, host, solver_for, torch_cuda

pytestmark = pytest.mark.gpu


def test_device_wait_times_out_and_the_handle_stays_usable():
    torch = torch_cuda()
    from paper_2209_08722_gb300 import _native as nat
    lp = lpgen.planted_dense(64, 5000, seed=31, storage="f32")
    rng = np.random.default_rng(32)
    d2 = np.exp(rng.uniform(-3, 3, lp.n))
    v = rng.standard_normal(lp.m)
    ref = lp.A @ (d2 * (lp.A.T @ v))
    tol = 4 * (lp.m + fp32_lane_columns(lp.m, lp.n, "f32") + 64) * EPS32 * adat_bound(lp.A, d2, v)
    with solver_for(lp, s=2) as S:
        assert S.wait_probe(1 << 20, complete=True) == nat.LP_OK
        assert S.wait_probe(100_000, complete=False) == nat.LP_ERR_DEVICE_TIMEOUT
        assert "timed out" in S._lib.lp_last_error(S._h).decode()
        # the next calls start from a clear status word and are correct
        u = host(S.adat(dev(torch, d2), dev(torch, v), 0))
        assert np.all(np.abs(u - ref) <= tol)
        assert S.wait_probe(100_000, complete=False) == nat.LP_ERR_DEVICE_TIMEOUT
        x, y, s, info = S.solve(tol=1e-8)
        assert info["status"] == 0
        assert abs(float(lp.c @ x) - lp.objective) <= 1e-7 * (1 + abs(lp.objective))


def test_wait_probe_argument_errors():
    torch_cuda()
    from paper_2209_08722_gb300 import _native as nat
    lp = lpgen.planted_dense(8, 100, seed=33, storage="f32")
    with solver_for(lp, s=2) as S:
        assert S._lib.lp_wait_probe(S._h, 0, 0) == nat.LP_ERR_ARG
        assert S._lib.lp_wait_probe(S._h, (1 << 31) + 1, 0) == nat.LP_ERR_ARG
        assert S._lib.lp_wait_probe(S._h, 1000, 2) == nat.LP_ERR_ARG
        assert S._lib.lp_wait_probe(None, 1000, 0) == nat.LP_ERR_ARG
