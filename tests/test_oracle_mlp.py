"""Pins for oracle.mlp (the warm-start model): gradients against central finite
differences, layout round trip, Adam's first step."""

import numpy as np

from oracle import mlp


def _setup(seed=0, n_in=7, hid=5, n_out=3, B=4):
    rng = np.random.default_rng(seed)
    flat = rng.standard_normal(hid * n_in + hid + hid * hid + hid + n_out * hid + n_out) * 0.5
    X = rng.standard_normal((n_in, B))
    T = rng.standard_normal((n_out, B))
    return flat, X, T, (n_in, hid, n_out)


def test_gradients_match_finite_differences():
    flat, X, T, dims = _setup()
    _, grads = mlp.loss_and_grads(mlp.unflatten(flat, *dims), X, T)
    g = mlp.flatten(grads)
    h = 1e-6
    num = np.empty_like(flat)
    for i in range(flat.size):
        e = np.zeros_like(flat)
        e[i] = h
        lp, _ = mlp.loss_and_grads(mlp.unflatten(flat + e, *dims), X, T)
        lm, _ = mlp.loss_and_grads(mlp.unflatten(flat - e, *dims), X, T)
        num[i] = (lp - lm) / (2 * h)
    assert np.max(np.abs(num - g)) <= 1e-6 * (1 + np.max(np.abs(g)))


def test_flatten_is_the_inverse_of_unflatten_and_column_major():
    flat, _, _, dims = _setup(1)
    params = mlp.unflatten(flat, *dims)
    assert np.array_equal(mlp.flatten(params), flat)
    n_in, hid, _ = dims
    # W1 is column-major: its (1, 0) entry is the second stored value
    assert params[0][1, 0] == flat[1] and params[0][0, 1] == flat[hid]


def test_gelu_special_values():
    assert mlp.gelu(np.array([0.0]))[0] == 0.0
    big = mlp.gelu(np.array([10.0, -10.0]))
    assert abs(big[0] - 10.0) < 1e-12 and abs(big[1]) < 1e-12
    assert abs(mlp.gelu_grad(np.array([0.0]))[0] - 0.5) < 1e-15


def test_adam_first_step_moves_each_weight_by_lr_against_the_gradient_sign():
    rng = np.random.default_rng(2)
    w = rng.standard_normal(10)
    g = rng.standard_normal(10)
    w1, m, v = mlp.adam_step(w, g, np.zeros(10), np.zeros(10), 1, 1e-3)
    # bias-corrected m/sqrt(v) = g/|g| at step 1
    assert np.allclose(w1, w - 1e-3 * np.sign(g) * (np.abs(g) / (np.abs(g) + 1e-8)))
