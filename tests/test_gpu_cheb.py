"""GPU parity of the Chebyshev propagation (mpk_cheb, Sec. 7 Eq. 7-9) against
the FP64 oracle, including sweeps with a remainder (M not a multiple of p)."""
import numpy as np
import pytest
import torch

import mpk_inputs as mi
import oracle
import paper_2205_01598_gb300 as mpk
from gpu_helpers import plan_of

pytestmark = pytest.mark.gpu


def _run(A, prec, p, M, permuted=False, rdt=50.0):
    plan = plan_of(A, p, prec=prec, nrhs=2)
    lo, hi = mpk.mpk_gershgorin(plan)
    olo, ohi = oracle.gershgorin(A)
    if prec == "f64":
        assert (lo, hi) == (olo, ohi)
    c, r = (ohi + olo) / 2, (ohi - olo) / 2
    coef = oracle.cheb_coeffs_schroedinger(M, c, r, rdt / r)
    psi = mi.uniform(1234, A.n) + 1j * mi.uniform(4321, A.n)
    psi /= np.linalg.norm(psi)
    ref = oracle.cheb(A, coef, c, r, psi)
    dt = torch.float64 if prec == "f64" else torch.float32
    x = np.stack([psi.real, psi.imag], 1)
    if permuted:
        perm = mpk.mpk_plan_perm(plan)[0].cpu().numpy()
        x = x[perm]
        ref = ref[perm]
    xd = torch.from_numpy(np.ascontiguousarray(x)).to(dt).cuda()
    yd = torch.empty(A.n, 2, dtype=torch.float64, device="cuda")
    mpk.mpk_cheb(plan, coef, c, r, xd, yd, permuted=permuted)
    y = yd.cpu().numpy()
    got = y[:, 0] + 1j * y[:, 1]
    return np.max(np.abs(got - ref)) / np.max(np.abs(ref))


@pytest.mark.parametrize("p,M", [(8, 64), (5, 17), (1, 6), (16, 12)])
def test_f64_cheb_matches_oracle(p, M):
    A = mi.anderson3d(12, W=16.5, seed=42)
    assert _run(A, "f64", p, M) <= 1e-12


def test_f64_cheb_permuted_io():
    A = mi.anderson3d(10, W=16.5, seed=42)
    assert _run(A, "f64", 8, 64, permuted=True) <= 1e-12


@pytest.mark.parametrize("prec", ["f32", "bf16val"])
def test_reduced_precision_cheb_error_bound(prec):
    """FP32 storage (BF16 hoppings for bf16val, exact for -1), FP64 scaling and
    coefficient sum: relative error against the FP64 oracle <= 2e-5 for the
    degree-64 Anderson propagation."""
    A = mi.anderson3d(16, W=16.5, seed=42)
    err = _run(A, prec, 8, 64)
    print(prec, err)
    assert err <= 2e-5


def test_staged_cheb_matches_oracle():
    A = mi.anderson3d(12, W=16.5, seed=42)
    plan = plan_of(A, 8, prec="f64", nrhs=2, tune=mpk.MPK_TUNE_STAGE)
    assert mpk.mpk_plan_info(plan)["staged"] == 1
    c, r = 0.5, 14.0
    coef = oracle.cheb_coeffs_schroedinger(21, c, r, 2.0)
    psi = mi.uniform(5, A.n) + 1j * mi.uniform(6, A.n)
    ref = oracle.cheb(A, coef, c, r, psi)
    xd = torch.from_numpy(np.stack([psi.real, psi.imag], 1).copy()).cuda()
    yd = torch.empty(A.n, 2, dtype=torch.float64, device="cuda")
    mpk.mpk_cheb(plan, coef, c, r, xd, yd)
    y = yd.cpu().numpy()
    assert np.max(np.abs(y[:, 0] + 1j * y[:, 1] - ref)) / np.max(np.abs(ref)) <= 1e-12


@pytest.mark.parametrize("prec", ["f64", "bf16val"])
def test_one_power_per_launch_is_bitwise_equal(prec):
    """The back-to-back form (MPK_SWEEP_ONE) runs the same node arithmetic, so
    it must reproduce the level-blocked sweeps bit for bit."""
    A = mi.anderson3d(14, W=16.5, seed=42)
    plan = plan_of(A, 8, prec=prec, nrhs=2)
    c, r = 0.1, 14.25
    coef = oracle.cheb_coeffs_schroedinger(30, c, r, 50.0 / r)
    psi = mi.uniform(9, A.n) + 1j * mi.uniform(10, A.n)
    dt = torch.float64 if prec == "f64" else torch.float32
    xd = torch.from_numpy(np.stack([psi.real, psi.imag], 1).copy()).to(dt).cuda()
    y1 = torch.empty(A.n, 2, dtype=torch.float64, device="cuda")
    y2 = torch.empty_like(y1)
    mpk.mpk_cheb(plan, coef, c, r, xd, y1)
    mpk.mpk_cheb(plan, coef, c, r, xd, y2, one_power_per_launch=True)
    assert torch.equal(y1, y2)


def test_anderson_200_full_size_bf16():
    """The 200^3 Anderson workload (N = 8M, nnz = 56M), degree 64 in sweeps of
    p = 8, BF16 hoppings, in the benchmark's launch configuration (level
    order): error against the FP64 oracle on every output within the
    reduced-precision bound."""
    A = mi.anderson3d(200, W=16.5, seed=42)
    assert A.nnz == 56_000_000
    plan = plan_of(A, 8, prec="bf16val", nrhs=2)
    assert mpk.mpk_plan_info(plan)["val_bytes"] == 2
    lo, hi = mpk.mpk_gershgorin(plan)
    c, r = (hi + lo) / 2, (hi - lo) / 2
    coef = mpk.mpk_cheb_coeffs_schroedinger(64, c, r, 50.0 / r)
    psi = mi.uniform(1234, A.n) + 1j * mi.uniform(4321, A.n)
    psi /= np.linalg.norm(psi)
    ref = oracle.cheb(A, coef, c, r, psi)
    perm = mpk.mpk_plan_perm(plan)[0].cpu().numpy()
    x = np.stack([psi.real, psi.imag], 1)[perm]
    xd = torch.from_numpy(np.ascontiguousarray(x)).float().cuda()
    yd = torch.empty(A.n, 2, dtype=torch.float64, device="cuda")
    mpk.mpk_cheb(plan, coef, c, r, xd, yd, permuted=True)
    y = yd.cpu().numpy()
    got = y[:, 0] + 1j * y[:, 1]
    assert np.max(np.abs(got - ref[perm])) / np.max(np.abs(ref)) <= 2e-5
