"""Guard regions around every device buffer of a handle (lp_options.guard):
the stand-in for a device memory checker.  Solves over the storage formats,
sketches and inner solvers leave every guard intact, and the guarded handle's
results equal the unguarded one's bit for bit."""

import numpy as np
import pytest

import lpgen
from tests.gpu_helpers import solver_for, torch_cuda

pytestmark = pytest.mark.gpu

CASES = [
    ("dense f32, CountSketch, CG", lambda: lpgen.planted_dense(96, 6001, seed=21, storage="f32"), {}),
    ("dense bf16, row-split product", lambda: lpgen.planted_dense(1024, 12288, seed=22, storage="bf16"), {}),
    ("dense f64, Chebyshev", lambda: lpgen.planted_dense(40, 3001, seed=23, storage="f64"), {"inner": 1}),
    ("dense f32, Gaussian tensor-core sketch", lambda: lpgen.planted_dense(130, 5003, seed=24, storage="f32"),
     {"sketch": 1}),
    ("dense f32, two right-hand sides", lambda: lpgen.planted_dense(64, 4001, seed=25, storage="f32"),
     {"sigma_rule": 1}),
    ("CSC f32", lambda: lpgen.planted_sparse(128, 20000, seed=26, storage="f32"), {}),
]


@pytest.mark.parametrize("name,make,opts", CASES, ids=[c[0] for c in CASES])
def test_guards_stay_intact_and_results_are_unchanged(name, make, opts):
    torch_cuda()
    lp = make()
    with solver_for(lp, s=2, guard=0, **opts) as S0:
        x0, y0, _, i0 = S0.solve(tol=1e-8)
    with solver_for(lp, s=2, guard=1, **opts) as S:
        x, y, _, info = S.solve(tol=1e-8)
        checked, damaged, msg = S.check_guards()
        assert checked >= 40 and checked % 2 == 0
        assert damaged == 0, msg
    assert info["status"] == i0["status"] == 0
    assert info["inner_total"] == i0["inner_total"]
    assert np.array_equal(x, x0) and np.array_equal(y, y0)


def test_unguarded_handle_checks_nothing():
    torch_cuda()
    lp = lpgen.planted_dense(16, 500, seed=27, storage="f64")
    with solver_for(lp, guard=0) as S:
        assert S.check_guards() == (0, 0, "")
