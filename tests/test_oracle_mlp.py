"""Pins of the oracle MLP: central finite differences of the loss, the
one-layer closed form, and one Adam step by hand."""

import numpy as np

from oracle import mlp


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(0)
    params = mlp.init([7, 6, 5, 4], seed=1)
    X = rng.normal(size=(9, 7))
    T = rng.normal(size=(9, 4))
    Y, cache = mlp.forward(params, X)
    grads = mlp.backward(params, cache, Y, T)
    h = 1e-6
    for li in range(3):
        for pi in range(2):
            P = params[li][pi]
            flat = P.reshape(-1)
            for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
                old = flat[idx]
                flat[idx] = old + h
                lp = mlp.loss(mlp.forward(params, X)[0], T)
                flat[idx] = old - h
                lm = mlp.loss(mlp.forward(params, X)[0], T)
                flat[idx] = old
                fd = (lp - lm) / (2 * h)
                assert abs(fd - grads[li][pi].reshape(-1)[idx]) <= 1e-6 * (1 + abs(fd))


def test_single_linear_layer_closed_form():
    rng = np.random.default_rng(2)
    params = mlp.init([3, 2], seed=3)
    X = rng.normal(size=(5, 3))
    T = rng.normal(size=(5, 2))
    Y, cache = mlp.forward(params, X)
    W, b = params[0]
    assert np.allclose(Y, X @ W.T + b)
    gW, gb = mlp.backward(params, cache, Y, T)[0]
    R = 2.0 * (X @ W.T + b - T) / T.size
    assert np.allclose(gW, R.T @ X) and np.allclose(gb, R.sum(0))


def test_adam_first_step_is_signed_lr():
    p = np.array([1.0, -2.0, 3.0])
    g = np.array([0.5, -4.0, 1e-3])
    m, v = np.zeros(3), np.zeros(3)
    mlp.adam(p, g, m, v, t=1, lr=0.01)
    # with bias correction the first step is lr * g / (|g| + eps)
    assert np.allclose(p, np.array([1.0, -2.0, 3.0]) - 0.01 * g / (np.abs(g) + 1e-8))
