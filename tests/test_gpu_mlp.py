"""The planner network's CUDA kernels (forward, loss, backward, Adam)
against the FP64 reference: outputs and gradients within 1e-4 relative."""
import numpy as np
import pytest
import torch

import mpk_inputs as mi
import paper_2205_01598_gb300 as mpk
from oracle import mlp

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("shape,B", [((25, 64, 16), 300), ((7, 5, 3), 9), ((25, 64, 16), 1)])
def test_forward_and_gradient_match_reference(shape, B):
    mpk.build()
    net = mpk.Mlp(*shape, seed=11)
    p = net.get_params().astype(np.float64)
    X = mi.uniform(1, B * shape[0]).reshape(B, shape[0])
    T = mi.uniform(2, B * shape[2]).reshape(B, shape[2])
    M = (mi.uniform01(3, B * shape[2]) > 0.2).astype(np.float64).reshape(B, shape[2])
    M[0, 0] = 1.0
    Xd, Td, Md = (torch.from_numpy(a).float().cuda() for a in (X, T, M))
    y_ref, _ = mlp.forward(p, X.astype(np.float32).astype(np.float64), shape)
    y = net.forward(Xd).cpu().numpy()
    assert np.max(np.abs(y - y_ref)) <= 1e-4 * max(1.0, np.max(np.abs(y_ref)))
    f_ref, g_ref = mlp.loss_grad(p, X.astype(np.float32).astype(np.float64), T.astype(np.float32).astype(np.float64),
                                 M, shape)
    f, g = net.loss_grad(Xd, Td, Md, want_grad=True)
    assert abs(f - f_ref) <= 1e-4 * max(1e-3, abs(f_ref))
    assert np.max(np.abs(g - g_ref)) <= 1e-4 * max(1e-3, np.max(np.abs(g_ref)))


def test_adam_training_reduces_loss_on_a_smooth_target():
    net = mpk.Mlp(4, 32, 2, seed=5)
    X = torch.from_numpy(mi.uniform(7, 512 * 4).reshape(512, 4)).float().cuda()
    T = torch.stack([X[:, 0] * X[:, 1], X[:, 2] - X[:, 3] ** 2], 1).contiguous()
    M = torch.ones_like(T)
    first = net.loss_grad(X, T, M)
    for _ in range(400):
        net.loss_grad(X, T, M)
        net.adam_step(3e-3)
    last = net.loss_grad(X, T, M)
    assert last < 0.1 * first
