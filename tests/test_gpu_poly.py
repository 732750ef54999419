"""GPU parity of the approximate inverse applied by Chebyshev propagation
(mpk_cheb_real with mpk_cheb_coeffs_inverse, a polynomial preconditioner
or fixed-degree solve): against the FP64 oracle's propagation (FP64 <=
1e-12, FP32 <= 2e-5, relative to the result), and as a solve, the residual
of A y = b (oracle SpMV) within the truncation bound."""
import numpy as np
import pytest
import torch

import mpk_inputs as mi
import oracle
import paper_2205_01598_gb300 as mpk
from gpu_helpers import plan_of

pytestmark = pytest.mark.gpu


def _shifted(A, sigma):
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    val = A.val.copy()
    val[A.col == rows] += sigma
    return mi.CSR(A.n, A.rowptr, A.col, val)


def _solve(A, sigma, prec, p, M):
    plan = plan_of(A, p, prec=prec, nrhs=1)
    lo, hi = mpk.mpk_gershgorin(plan)
    lo = max(lo, sigma)   # shifted -Laplacian: spectrum in [sigma, hi]
    c, r = (hi + lo) / 2, (hi - lo) / 2
    coef = mpk.mpk_cheb_coeffs_inverse(M, c, r)
    b = mi.random_vector(A.n, 2024)
    dt = torch.float64 if prec == "f64" else torch.float32
    y = torch.empty(A.n, dtype=torch.float64, device="cuda")
    mpk.mpk_cheb_real(plan, coef, c, r, torch.from_numpy(b).to(dt).cuda(), y)
    return y.cpu().numpy(), b, coef, c, r


@pytest.mark.parametrize("make,sigma", [(lambda: mi.laplace3d(24), 1.0), (lambda: mi.laplace2d(80, 60), 0.3),
                                        (lambda: mi.star3d(18, 2), 2.0)], ids=["lap3d", "lap2d", "order4"])
@pytest.mark.parametrize("p,M", [(8, 64), (5, 47)])
def test_inverse_f64_matches_oracle_and_solves(make, sigma, p, M):
    A = _shifted(make(), sigma)
    y, b, coef, c, r = _solve(A, sigma, "f64", p, M)
    ref = oracle.cheb_real(A, coef, c, r, b)
    assert np.max(np.abs(y - ref)) <= 1e-12 * np.max(np.abs(ref))
    s = np.sqrt(c * c - r * r)
    q = r / (c + s)
    bound = 2 * q ** (M + 1) / (s * (1 - q)) * np.linalg.norm(b)
    resid = oracle.mpk(A, y, 1)[0] - b
    # ||A y - b|| <= ||A|| ||y - A^-1 b|| with ||A|| <= c + r
    assert np.max(np.abs(resid)) <= (c + r) * bound + 1e-11 * np.max(np.abs(b))


def test_inverse_f32():
    A = _shifted(mi.laplace3d(20), 1.0)
    y, b, coef, c, r = _solve(A, 1.0, "f32", 8, 64)
    ref = oracle.cheb_real(A, coef, c, r, b.astype(np.float32).astype(np.float64))
    assert np.max(np.abs(y - ref)) <= 2e-5 * np.max(np.abs(ref))


def test_inverse_full_size_160():
    """The 160^3 7-point Laplacian shifted by 1 (spectrum in [1, 13]), degree 64:
    the truncation error is below 1e-15, so the result is A^{-1} b to rounding."""
    A = _shifted(mi.laplace3d(160), 1.0)
    y, b, coef, c, r = _solve(A, 1.0, "f64", 8, 64)
    ref = oracle.cheb_real(A, coef, c, r, b)
    assert np.max(np.abs(y - ref)) <= 1e-12 * np.max(np.abs(ref))
    assert np.max(np.abs(oracle.mpk(A, y, 1)[0] - b)) <= 1e-10 * np.max(np.abs(b))
