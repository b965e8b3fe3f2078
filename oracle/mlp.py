"""Three-layer ReLU MLP, MSE loss and Adam in FP64 (oracle; test-only).

The paper has no learned component; this is the reference for the library's
BF16 warm-start network (flattened A_1..A_l -> start iterate).  Plain
definitions, written out:

    Z1 = X W1^T + b1,  A1 = relu(Z1)
    Z2 = A1 W2^T + b2, A2 = relu(Z2)
    Y  = A2 W3^T + b3
    loss = mean over batch and outputs of (Y - T)^2

backward() applies the chain rule to exactly these lines; adam() is Kingma &
Ba's update with bias correction.  Pinned by central finite differences in
tests/test_oracle_mlp.py.
"""

from __future__ import annotations

import numpy as np


def init(sizes, seed: int = 0):
    """He-normal weights W_i (out x in), zero biases."""
    rng = np.random.default_rng(seed)
    params = []
    for fan_in, fan_out in zip(sizes[:-1], sizes[1:]):
        W = rng.normal(0.0, np.sqrt(2.0 / fan_in), size=(fan_out, fan_in))
        params.append([W, np.zeros(fan_out)])
    return params


def forward(params, X):
    acts = [X]
    zs = []
    h = X
    for i, (W, b) in enumerate(params):
        z = h @ W.T + b
        zs.append(z)
        h = np.maximum(z, 0.0) if i < len(params) - 1 else z
        acts.append(h)
    return h, (acts, zs)


def loss(Y, T):
    return float(np.mean((Y - T) ** 2))


def backward(params, cache, Y, T):
    """Gradients of loss(Y, T) with respect to every W_i, b_i."""
    acts, zs = cache
    g = 2.0 * (Y - T) / Y.size
    grads = [None] * len(params)
    for i in range(len(params) - 1, -1, -1):
        W, _ = params[i]
        grads[i] = [g.T @ acts[i], g.sum(axis=0)]
        if i > 0:
            g = (g @ W) * (zs[i - 1] > 0.0)
    return grads


def adam(p, g, m, v, t: int, lr: float, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
    m[:] = b1 * m + (1.0 - b1) * g
    v[:] = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    p -= lr * mh / (np.sqrt(vh) + eps)
