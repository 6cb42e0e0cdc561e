"""The warm-start MLP in FP64 NumPy (test infrastructure; see package docstring).

in -> H -> H -> out with GELU after both hidden layers; loss
L = 1/(2B) sum_b ||Y_b - T_b||^2; Adam (beta1 0.9, beta2 0.999, eps 1e-8).
Parameter order and layout (column-major weights, rows = outputs) are those of
the library's flat parameter vector: W1 (H x in), b1, W2 (H x H), b2,
W3 (out x H), b3.  Samples are columns of X (in x B).
"""

from __future__ import annotations

import math

import numpy as np

_erf = np.vectorize(math.erf)


def gelu(z):
    return 0.5 * z * (1.0 + _erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + _erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def unflatten(flat, n_in, hid, n_out):
    f = np.asarray(flat, dtype=np.float64)
    o = 0

    def take(rows, cols):
        nonlocal o
        a = f[o:o + rows * cols].reshape(cols, rows).T   # column-major
        o += rows * cols
        return a

    def vec(k):
        nonlocal o
        v = f[o:o + k]
        o += k
        return v
    W1 = take(hid, n_in); b1 = vec(hid)
    W2 = take(hid, hid); b2 = vec(hid)
    W3 = take(n_out, hid); b3 = vec(n_out)
    return [W1, b1, W2, b2, W3, b3]


def flatten(params):
    out = []
    for p in params:
        out.append(p.T.reshape(-1) if p.ndim == 2 else p)
    return np.concatenate(out)


def forward(params, X):
    W1, b1, W2, b2, W3, b3 = params
    Z1 = W1 @ X + b1[:, None]
    A1 = gelu(Z1)
    Z2 = W2 @ A1 + b2[:, None]
    A2 = gelu(Z2)
    Y = W3 @ A2 + b3[:, None]
    return Y, (Z1, A1, Z2, A2)


def loss_and_grads(params, X, T):
    W1, b1, W2, b2, W3, b3 = params
    B = X.shape[1]
    Y, (Z1, A1, Z2, A2) = forward(params, X)
    R = Y - T
    loss = 0.5 * float(np.sum(R * R)) / B
    d3 = R / B
    gW3, gb3 = d3 @ A2.T, d3.sum(axis=1)
    d2 = (W3.T @ d3) * gelu_grad(Z2)
    gW2, gb2 = d2 @ A1.T, d2.sum(axis=1)
    d1 = (W2.T @ d2) * gelu_grad(Z1)
    gW1, gb1 = d1 @ X.T, d1.sum(axis=1)
    return loss, [gW1, gb1, gW2, gb2, gW3, gb3]


def adam_step(flat, grad, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return flat - lr * mh / (np.sqrt(vh) + eps), m, v
