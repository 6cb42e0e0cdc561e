"""The learned warm start (lp_mlp_* and lp_set_warm_start): the model's forward
pass, gradients and Adam step against the FP64 NumPy oracle, and warm-started
solves that keep the solution while using fewer inner iterations."""

import numpy as np
import pytest

import lpgen
from oracle import mlp as omlp
from tests.gpu_helpers import solver_for, torch_cuda

pytestmark = pytest.mark.gpu


def test_mlp_forward_gradients_and_adam_match_oracle():
    torch = torch_cuda()
    from paper_2209_08722_gb300 import Mlp
    n_in, hid, n_out, B = 24, 16, 8, 5
    M = Mlp(n_in, hid, n_out, seed=3)
    rng = np.random.default_rng(0)
    flat = (rng.standard_normal(M.num_params) * 0.3).astype(np.float32)
    M.set_params(flat)
    X = rng.standard_normal((B, n_in)).astype(np.float32)
    T = rng.standard_normal((B, n_out)).astype(np.float32)
    Xd, Td = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
    P = omlp.unflatten(flat.astype(np.float64), n_in, hid, n_out)
    Yo, _ = omlp.forward(P, X.T.astype(np.float64))
    Y = M.forward(Xd).cpu().numpy()
    assert np.abs(Y - Yo.T).max() <= 1e-5 * np.abs(Yo).max()
    loss = M.loss_grad(Xd, Td)
    lo, go = omlp.loss_and_grads(P, X.T.astype(np.float64), T.T.astype(np.float64))
    gof = omlp.flatten(go)
    assert abs(loss - lo) <= 1e-5 * lo
    assert np.abs(M.grads() - gof).max() <= 1e-5 * np.abs(gof).max()
    M.train_step(Xd, Td, 1e-2)
    po, _, _ = omlp.adam_step(flat.astype(np.float64), gof, np.zeros_like(gof), np.zeros_like(gof), 1, 1e-2)
    assert np.abs(M.params() - po).max() <= 1e-5


def test_mlp_tensor_core_contractions_at_several_tiles_match_oracle():
    # widths that span several 128 x 128 tiles of the tcgen05 GEMM with ragged
    # edges, and K lengths over many 16-wide chunks, in all three operand forms
    # (forward NN, weight gradients NT, input gradients TN): the FP32-class
    # split-TF32 products against the FP64 oracle; the bound grows with the
    # contraction length (FP32 accumulation over K = B for the weight gradients)
    torch = torch_cuda()
    from paper_2209_08722_gb300 import Mlp
    n_in, hid, n_out, B = 300, 200, 150, 333
    M = Mlp(n_in, hid, n_out, seed=4)
    rng = np.random.default_rng(1)
    flat = (rng.standard_normal(M.num_params) * 0.1).astype(np.float32)
    M.set_params(flat)
    X = rng.standard_normal((B, n_in)).astype(np.float32)
    T = rng.standard_normal((B, n_out)).astype(np.float32)
    Xd, Td = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
    P = omlp.unflatten(flat.astype(np.float64), n_in, hid, n_out)
    Yo, _ = omlp.forward(P, X.T.astype(np.float64))
    Y = M.forward(Xd).cpu().numpy()
    assert np.abs(Y - Yo.T).max() <= 1e-5 * np.abs(Yo).max()
    loss = M.loss_grad(Xd, Td)
    lo, go = omlp.loss_and_grads(P, X.T.astype(np.float64), T.T.astype(np.float64))
    gof = omlp.flatten(go)
    assert abs(loss - lo) <= 1e-5 * lo
    g = M.grads()
    # per block (W1, b1, W2, b2, W3, b3): within 4e-5 of the block's largest gradient
    sizes = [hid * n_in, hid, hid * hid, hid, n_out * hid, n_out]
    off = 0
    for size in sizes:
        blk, ref = g[off:off + size], gof[off:off + size]
        assert np.abs(blk - ref).max() <= 4e-5 * np.abs(ref).max(), off
        off += size


def test_learned_warm_start_keeps_the_solution_and_saves_inner_iterations():
    torch = torch_cuda()
    from paper_2209_08722_gb300 import Mlp
    m, n = 64, 8192
    train = [lpgen.planted_dense(m, n, seed=s, storage="bf16") for s in range(1, 13)]
    test = [lpgen.planted_dense(m, n, seed=s, storage="bf16") for s in range(1000, 1004)]
    recX = torch.zeros(2000, 3 * m, device="cuda")
    recT = torch.zeros(2000, m, device="cuda")
    total = 0
    for lp in train:
        with solver_for(lp, s=2) as S:
            S.set_warm_start("none", None, recX[total:], recT[total:])
            S.solve(tol=1e-8)
            total += S.warm_start_stats()["recorded"]
    assert total > 300
    net = Mlp(3 * m, 1024, m, seed=7)
    X, T = recX[:total].contiguous(), recT[:total].contiguous()
    first = net.train_step(X, T, 1e-3)
    for it in range(1500):
        last = net.train_step(X, T, 1e-3 if it < 1000 else 3e-4)
    assert last < 1e-2 * first
    counts = {}
    for mode in ("none", "previous", "model"):
        inner, accepted = 0, 0
        for lp in test:
            with solver_for(lp, s=2) as S:
                S.set_warm_start(mode, net if mode == "model" else None)
                x, y, s, info = S.solve(tol=1e-8)
                assert info["status"] == 0, (mode, info)
                assert abs(lp.c @ x - lp.objective) <= 1e-7 * (1 + abs(lp.objective))
                inner += info["inner_total"]
                accepted += S.warm_start_stats()["accepted"]
        counts[mode] = (inner, accepted)
    # the Galerkin-combined proposals are used on most outer iterations and
    # save a clear share of the inner iterations (about a quarter here)
    assert counts["model"][1] > 0.5 * 4 * 30, counts
    assert counts["previous"][0] <= 0.9 * counts["none"][0], counts
    assert counts["model"][0] <= 0.9 * counts["none"][0], counts
