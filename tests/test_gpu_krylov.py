"""GPU parity of the Krylov consumers of the MPK (mpk_cg, mpk_sstep_cg)
against the FP64 oracle's CG and s-step CG: both solve A x = b to the
tolerance (checked with the true residual), agree with the oracle's
solution, and s-step CG, CG in exact arithmetic, takes the same number of
steps as the oracle's s-step CG up to one."""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

import mpk_inputs as mi
import oracle
import paper_2205_01598_gb300 as mpk
from gpu_helpers import plan_of

pytestmark = pytest.mark.gpu


def _shifted(n, shift, star=0):
    A = mi.laplace3d(n) if not star else mi.star3d(n, star)
    S = (sp.csr_matrix((A.val, A.col, A.rowptr), shape=(A.n, A.n)) + shift * sp.eye(A.n)).tocsr()
    S.sort_indices()
    return mi.CSR(A.n, S.indptr.astype(np.int32), S.indices.astype(np.int32), S.data.astype(np.float64)), S


def _true_relres(S, x, b):
    return np.linalg.norm(S @ x - b) / np.linalg.norm(b)


@pytest.mark.parametrize("n,shift", [(20, 2.0), (24, 0.5)])
@pytest.mark.parametrize("permuted", [False, True])
def test_cg_matches_oracle(n, shift, permuted):
    A, S = _shifted(n, shift)
    b = mi.random_vector(A.n, 7)
    xo, steps_o, _ = oracle.cg(A, b, tol=1e-10)
    plan = plan_of(A, 1, prec="f64", nrhs=1)
    perm = mpk.mpk_plan_perm(plan)[0].cpu().numpy() if permuted else np.arange(A.n)
    bd = torch.from_numpy(b[perm].copy()).cuda()
    xd = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    steps, rel = mpk.mpk_cg(plan, bd, xd, tol=1e-10, permuted=permuted)
    x = np.empty(A.n)
    x[perm] = xd.cpu().numpy()
    assert rel <= 1e-10 and _true_relres(S, x, b) <= 2e-10
    assert steps_o <= steps <= steps_o + 8          # the norm is read every 8 steps
    assert np.max(np.abs(x - xo)) / np.max(np.abs(xo)) <= 1e-8


@pytest.mark.parametrize("s", [1, 2, 4, 6, 8])
@pytest.mark.parametrize("permuted", [False, True])
def test_sstep_cg_matches_oracle(s, permuted):
    A, S = _shifted(20, 2.0)
    b = mi.random_vector(A.n, 9)
    rho = 14.0
    xo, steps_o, _ = oracle.sstep_cg(A, b, s, rho, tol=1e-10)
    xc, _, _ = oracle.cg(A, b, tol=1e-10)
    plan = plan_of(A, s, prec="f64", nrhs=2)
    perm = mpk.mpk_plan_perm(plan)[0].cpu().numpy() if permuted else np.arange(A.n)
    bd = torch.from_numpy(b[perm].copy()).cuda()
    xd = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    steps, rel = mpk.mpk_sstep_cg(plan, bd, xd, tol=1e-10, rho=rho, permuted=permuted)
    x = np.empty(A.n)
    x[perm] = xd.cpu().numpy()
    assert abs(steps - steps_o) <= 1
    assert rel <= 1e-10 and _true_relres(S, x, b) <= 5e-10
    assert np.max(np.abs(x - xo)) / np.max(np.abs(xo)) <= 1e-8
    assert np.max(np.abs(x - xc)) / np.max(np.abs(xc)) <= 1e-8


def test_sstep_cg_nonzero_guess_and_wide_stencil():
    """A nonzero initial guess, the order-4 star stencil (shifted), rho from
    the Gershgorin bound (rho = 0)."""
    A, S = _shifted(16, 1.0, star=2)
    b = mi.random_vector(A.n, 2)
    x0 = mi.random_vector(A.n, 3)
    plan = plan_of(A, 4, prec="f64", nrhs=2)
    xd = torch.from_numpy(x0.copy()).cuda()
    steps, rel = mpk.mpk_sstep_cg(plan, torch.from_numpy(b).cuda(), xd, tol=1e-9)
    x = xd.cpu().numpy()
    assert rel <= 1e-9 and _true_relres(S, x, b) <= 5e-9
    xo, _, _ = oracle.cg(A, b, tol=1e-12)
    assert np.max(np.abs(x - xo)) / np.max(np.abs(xo)) <= 1e-7


def test_solver_refusals_and_zero_rhs():
    A, _ = _shifted(8, 1.0)
    b = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    p1 = plan_of(A, 3, prec="f64", nrhs=1)
    with pytest.raises(mpk.MpkError) as e:
        mpk.mpk_sstep_cg(p1, b, x)
    assert e.value.code == mpk.MPK_ERR_INVALID
    p2 = plan_of(A, 3, prec="f64", nrhs=2)
    with pytest.raises(mpk.MpkError) as e:
        mpk.mpk_cg(p2, b, x)
    assert e.value.code == mpk.MPK_ERR_INVALID
    with pytest.raises(mpk.MpkError) as e:
        mpk.mpk_sstep_cg(plan_of(A, 17, prec="f64", nrhs=2), b, x)
    assert e.value.code == mpk.MPK_ERR_INVALID
    assert mpk.mpk_sstep_cg(p2, b, x) == (0, 0.0)
    assert mpk.mpk_cg(p1, b, x) == (0, 0.0)
    assert torch.count_nonzero(x) == 0
