"""GPU parity of the multi-step Chebyshev propagation (mpk_cheb_steps): T
time steps y = U^T x whose sweeps run across the steps -- the node of a
step's last power hands its row of the step's result to the next step as
v_0 -- against T applications of the FP64 oracle's propagator.  Sweeps of a
length that does not divide M (so that sweeps straddle step boundaries), a
plan whose p holds the whole propagation (one launch), and the
one-power-per-launch form must all give the same bits."""
import numpy as np
import pytest
import torch

import mpk_inputs as mi
import oracle
import paper_2205_01598_gb300 as mpk
from gpu_helpers import plan_of

pytestmark = pytest.mark.gpu


def _schroedinger(A, M, rdt):
    lo, hi = oracle.gershgorin(A)
    c, r = (hi + lo) / 2, (hi - lo) / 2
    return oracle.cheb_coeffs_schroedinger(M, c, r, rdt / r), c, r


def _run_steps(A, prec, p, coef, c, r, T, x, one=False):
    G = 2 if np.iscomplexobj(coef) else 1
    plan = plan_of(A, p, prec=prec, nrhs=G)
    dt = torch.float64 if prec == "f64" else torch.float32
    xd = torch.from_numpy(np.ascontiguousarray(x)).to(dt).cuda()
    yd = torch.empty(tuple(xd.shape), dtype=torch.float64, device="cuda")
    mpk.mpk_cheb_steps(plan, coef, c, r, T, xd, yd, one_power_per_launch=one)
    return plan, yd


@pytest.mark.parametrize("p", [8, 5, 48])          # divides M, straddles steps, whole propagation in one launch
def test_complex_steps_match_oracle(p):
    A = mi.anderson3d(12, W=16.5, seed=42)
    M, T = 16, 3
    coef, c, r = _schroedinger(A, M, 12.0)
    psi = mi.uniform(1234, A.n) + 1j * mi.uniform(4321, A.n)
    psi /= np.linalg.norm(psi)
    ref = psi
    for _ in range(T):
        ref = oracle.cheb(A, coef, c, r, ref)
    _, yd = _run_steps(A, "f64", p, coef, c, r, T, np.stack([psi.real, psi.imag], 1))
    y = yd.cpu().numpy()
    assert np.max(np.abs(y[:, 0] + 1j * y[:, 1] - ref)) / np.max(np.abs(ref)) <= 1e-12


@pytest.mark.parametrize("p", [16, 7])
def test_real_steps_match_oracle(p):
    A = mi.star3d(14, 2)
    M, T = 20, 2
    lo, hi = oracle.gershgorin(A)
    lo = max(lo, 0.0)
    c, r = (hi + lo) / 2, (hi - lo) / 2
    coef = oracle.cheb_coeffs_heat(M, c, r, 8.0 / r)
    x = mi.random_vector(A.n, 9)
    ref = x
    for _ in range(T):
        ref = oracle.cheb_real(A, coef, c, r, ref)
    _, yd = _run_steps(A, "f64", p, coef, c, r, T, x)
    assert np.max(np.abs(yd.cpu().numpy() - ref)) / np.max(np.abs(x)) <= 1e-12


@pytest.mark.parametrize("prec", ["f64", "bf16val"])
def test_sweep_splits_give_the_same_bits(prec):
    A = mi.anderson3d(10, W=16.5, seed=42)
    M, T = 12, 3
    coef, c, r = _schroedinger(A, M, 10.0)
    psi = mi.uniform(5, A.n) + 1j * mi.uniform(6, A.n)
    x = np.stack([psi.real, psi.imag], 1)
    _, y8 = _run_steps(A, prec, 8, coef, c, r, T, x)
    _, y1 = _run_steps(A, prec, 8, coef, c, r, T, x, one=True)
    _, y36 = _run_steps(A, prec, 36, coef, c, r, T, x)
    assert torch.equal(y8, y1) and torch.equal(y8, y36)


def test_one_step_equals_mpk_cheb():
    A = mi.anderson3d(10, W=16.5, seed=42)
    coef, c, r = _schroedinger(A, 20, 10.0)
    psi = mi.uniform(7, A.n) + 1j * mi.uniform(8, A.n)
    x = np.stack([psi.real, psi.imag], 1)
    plan, y_steps = _run_steps(A, "bf16val", 8, coef, c, r, 1, x)
    y = torch.empty_like(y_steps)
    mpk.mpk_cheb(plan, coef, c, r, torch.from_numpy(x).float().cuda(), y)
    assert torch.equal(y, y_steps)


def test_reduced_precision_steps_within_bound():
    """BF16 hoppings, FP32 vectors: T = 4 steps of degree 32, each step's
    result handed on in FP32; error against T oracle steps within T times
    the one-step bound."""
    A = mi.anderson3d(16, W=16.5, seed=42)
    M, T = 32, 4
    coef, c, r = _schroedinger(A, M, 25.0)
    psi = mi.uniform(1234, A.n) + 1j * mi.uniform(4321, A.n)
    psi /= np.linalg.norm(psi)
    ref = psi
    for _ in range(T):
        ref = oracle.cheb(A, coef, c, r, ref)
    _, yd = _run_steps(A, "bf16val", 8, coef, c, r, T, np.stack([psi.real, psi.imag], 1))
    y = yd.cpu().numpy()
    assert np.max(np.abs(y[:, 0] + 1j * y[:, 1] - ref)) / np.max(np.abs(ref)) <= T * 2e-5
