"""Float64 reference of the planner network, for the GPU kernels' tests.

TEST INFRASTRUCTURE ONLY (tests, smoke, benchmark baseline).  The planner is
a multilayer perceptron 4 -> 64 -> 64 -> S with ReLU after the two hidden
layers and a linear output (one predicted log-time per scan strategy),
trained by mean-squared error with Adam.  This module restates those
textbook definitions plainly in numpy float64:

  forward:   Z1 = X W1 + b1, A1 = relu(Z1); Z2 = A1 W2 + b2, A2 = relu(Z2);
             Y = A2 W3 + b3                  (W_l has shape (fan_in, fan_out))
  loss:      L = mean over samples and outputs of (Y - T)^2
  backward:  dY = 2 (Y - T) / (batch * S); dW3 = A2^T dY; db3 = sum_rows dY;
             dZ2 = (dY W3^T) * [Z2 > 0]; dW2 = A1^T dZ2; ...; dW1 = X^T dZ1
  Adam:      m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
             p -= lr * (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps)

Pins: tests/test_mlp_ref.py (finite differences, a hand-worked network,
Adam's first-step closed form).
"""
from __future__ import annotations

import numpy as np

SIZES = (4, 64, 64, 4)


def init(seed: int, sizes=SIZES):
    """He-uniform weights, zero biases; list of (W, b) per layer, float64."""
    rng = np.random.default_rng(seed)
    params = []
    for fan_in, fan_out in zip(sizes[:-1], sizes[1:]):
        lim = np.sqrt(6.0 / fan_in)
        params.append((rng.uniform(-lim, lim, size=(fan_in, fan_out)), np.zeros(fan_out)))
    return params


def forward(params, X):
    """Returns (Y, cache); cache holds each layer's input and pre-activation."""
    a = np.asarray(X, dtype=np.float64)
    cache = []
    for i, (W, b) in enumerate(params):
        z = a @ W + b
        cache.append((a, z))
        a = np.maximum(z, 0.0) if i + 1 < len(params) else z
    return a, cache


def loss(Y, T):
    return float(np.mean((Y - T) ** 2))


def backward(params, cache, Y, T):
    """Gradients [(dW, db)] of the mean-squared error."""
    d = 2.0 * (Y - T) / Y.size
    grads = [None] * len(params)
    for i in range(len(params) - 1, -1, -1):
        a_in, z = cache[i]
        if i + 1 < len(params):
            d = d * (z > 0.0)
        W = params[i][0]
        grads[i] = (a_in.T @ d, d.sum(axis=0))
        d = d @ W.T
    return grads


def adam_state(params):
    return [(np.zeros_like(W), np.zeros_like(b)) for W, b in params], \
           [(np.zeros_like(W), np.zeros_like(b)) for W, b in params]


def adam_step(params, grads, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (step number t >= 1); returns new (params, m, v)."""
    out_p, out_m, out_v = [], [], []
    for (W, b), (gW, gb), (mW, mb), (vW, vb) in zip(params, grads, m, v):
        new = []
        for p, g, mm, vv in ((W, gW, mW, vW), (b, gb, mb, vb)):
            mm = b1 * mm + (1 - b1) * g
            vv = b2 * vv + (1 - b2) * g * g
            mhat = mm / (1 - b1 ** t)
            vhat = vv / (1 - b2 ** t)
            new.append((p - lr * mhat / (np.sqrt(vhat) + eps), mm, vv))
        out_p.append((new[0][0], new[1][0]))
        out_m.append((new[0][1], new[1][1]))
        out_v.append((new[0][2], new[1][2]))
    return out_p, out_m, out_v


def flatten(params):
    """Concatenate [W1, b1, W2, b2, ...] row-major (the layout the GPU kernels use)."""
    return np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in params])


def unflatten(vec, sizes=SIZES):
    params, off = [], 0
    for fan_in, fan_out in zip(sizes[:-1], sizes[1:]):
        W = np.asarray(vec[off:off + fan_in * fan_out], dtype=np.float64).reshape(fan_in, fan_out)
        off += fan_in * fan_out
        b = np.asarray(vec[off:off + fan_out], dtype=np.float64)
        off += fan_out
        params.append((W, b))
    return params
