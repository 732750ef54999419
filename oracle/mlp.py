"""FP64 reference of the planner's multilayer perceptron (test infrastructure
only, like the rest of oracle/).

Network: x -> h1 = relu(W1 x + b1) -> h2 = relu(W2 h1 + b2) -> y = W3 h2 + b3.
Loss: sum_ij M_ij (y_ij - t_ij)^2 / sum_ij M_ij over a batch.
Parameters are one flat vector in the order W1 (n_hidden x n_in, row-major),
b1, W2 (n_hidden x n_hidden), b2, W3 (n_out x n_hidden), b3.

The backward pass is written from the chain rule and pinned by central
finite differences in tests/test_oracle_mlp.py.
"""
import numpy as np


def split(params, n_in, n_hidden, n_out):
    p = np.asarray(params, dtype=np.float64)
    sizes = [n_hidden * n_in, n_hidden, n_hidden * n_hidden, n_hidden, n_out * n_hidden, n_out]
    out, o = [], 0
    for s in sizes:
        out.append(p[o:o + s])
        o += s
    assert o == p.size
    W1, b1, W2, b2, W3, b3 = out
    return W1.reshape(n_hidden, n_in), b1, W2.reshape(n_hidden, n_hidden), b2, W3.reshape(n_out, n_hidden), b3


def forward(params, X, shape):
    W1, b1, W2, b2, W3, b3 = split(params, *shape)
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ W1.T + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0.0)
    y = h2 @ W3.T + b3
    return y, (X, z1, h1, z2, h2)


def loss(params, X, T, M, shape):
    y, _ = forward(params, X, shape)
    M = np.asarray(M, dtype=np.float64)
    return float(np.sum(M * (y - T) ** 2) / np.sum(M))


def loss_grad(params, X, T, M, shape):
    """Loss and the gradient of all parameters (flat, same layout)."""
    W1, b1, W2, b2, W3, b3 = split(params, *shape)
    y, (X, z1, h1, z2, h2) = forward(params, X, shape)
    M = np.asarray(M, dtype=np.float64)
    msum = np.sum(M)
    dy = 2.0 * M * (y - T) / msum
    gW3 = dy.T @ h2
    gb3 = dy.sum(0)
    dh2 = (dy @ W3) * (z2 > 0)
    gW2 = dh2.T @ h1
    gb2 = dh2.sum(0)
    dh1 = (dh2 @ W2) * (z1 > 0)
    gW1 = dh1.T @ X
    gb1 = dh1.sum(0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return float(np.sum(M * (y - T) ** 2) / msum), g
