"""Pins of the FP64 network reference (oracle/mlp.py): central finite
differences of the loss, and a closed form for a network with one active
path."""
import numpy as np

import mpk_inputs as mi
from oracle import mlp


def _rand(shape, seed):
    n_in, n_h, n_out = shape
    npar = n_h * n_in + n_h + n_h * n_h + n_h + n_out * n_h + n_out
    return mi.uniform(seed, npar, -0.5, 0.5)


def test_gradient_matches_central_differences():
    shape = (7, 6, 3)
    p = _rand(shape, 3)
    X = mi.uniform(4, 11 * 7).reshape(11, 7)
    T = mi.uniform(5, 11 * 3).reshape(11, 3)
    M = (mi.uniform01(6, 33) > 0.3).astype(np.float64).reshape(11, 3)
    f, g = mlp.loss_grad(p, X, T, M, shape)
    assert abs(f - mlp.loss(p, X, T, M, shape)) < 1e-15
    h = 1e-6
    for i in range(p.size):
        e = np.zeros_like(p)
        e[i] = h
        fd = (mlp.loss(p + e, X, T, M, shape) - mlp.loss(p - e, X, T, M, shape)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(fd)), i


def test_single_path_closed_form():
    """One input, one hidden unit per layer, identity-like weights: y = w3 *
    relu(w2 * relu(w1 x + b1) + b2) + b3 and the loss is a plain square."""
    shape = (1, 1, 1)
    w1, b1, w2, b2, w3, b3 = 2.0, 0.5, -1.5, 4.0, 3.0, -1.0
    p = np.array([w1, b1, w2, b2, w3, b3])
    x, t = 0.75, 2.0
    h1 = max(w1 * x + b1, 0)
    h2 = max(w2 * h1 + b2, 0)
    y = w3 * h2 + b3
    f, g = mlp.loss_grad(p, np.array([[x]]), np.array([[t]]), np.ones((1, 1)), shape)
    assert f == (y - t) ** 2
    d = 2 * (y - t)
    assert np.allclose(g, [d * w3 * w2 * x, d * w3 * w2, d * w3 * h1, d * w3, d * h2, d], rtol=1e-15, atol=0)
