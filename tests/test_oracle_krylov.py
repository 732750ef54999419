"""Pins of the oracle's Krylov consumers of the MPK (conjugate gradients and
s-step CG with the monomial basis from one MPK per s steps), checked
against properties fixed by the mathematics:
  - CG on a symmetric positive definite matrix with k distinct eigenvalues
    reaches the solution in k steps (finite termination);
  - both solve A x = b to the tolerance, agreeing with a direct sparse solve;
  - s-step CG is CG in exact arithmetic: the same number of steps and the
    same solution up to rounding, for every s;
  - a zero right-hand side needs no step."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import mpk_inputs as mi
import oracle


def _shifted_laplacian(n, shift):
    A = mi.laplace3d(n)
    S = (sp.csr_matrix((A.val, A.col, A.rowptr), shape=(A.n, A.n)) + shift * sp.eye(A.n)).tocsr()
    S.sort_indices()
    return mi.CSR(A.n, S.indptr.astype(np.int32), S.indices.astype(np.int32), S.data.astype(np.float64)), S


def test_cg_finite_termination_on_distinct_eigenvalues():
    d = np.repeat([1.0, 2.5, 4.0, 7.0, 11.0], 40)          # five distinct eigenvalues
    A = mi.diagonal(d)
    b = mi.random_vector(A.n, 3)
    x, steps, rel = oracle.cg(A, b, tol=1e-13)
    assert steps == 5 and rel <= 1e-13
    assert np.allclose(x, b / d, rtol=1e-13, atol=0)
    for s in (1, 2, 3, 5):
        # the same five steps reach the solution, up to rounding amplified
        # by the conditioning of the monomial basis (it grows with s: 1e-14
        # at s = 1, 4e-11 at s = 5 here); the residual norm of the s-step form
        # comes from the Gram matrix (r'^T G r'), whose rounding can hold the
        # estimate above 1e-13, so the steps are capped at five
        xs, steps_s, _ = oracle.sstep_cg(A, b, s, 11.0, tol=1e-13, max_steps=5)
        assert steps_s == 5
        assert np.allclose(xs, b / d, rtol=1e-9, atol=0)


@pytest.mark.parametrize("n,shift", [(10, 2.0), (14, 0.5)])
def test_cg_matches_direct_solve(n, shift):
    A, S = _shifted_laplacian(n, shift)
    b = mi.random_vector(A.n, 11)
    ref = spla.spsolve(S.tocsc(), b)
    x, steps, rel = oracle.cg(A, b, tol=1e-12)
    assert rel <= 1e-12
    assert np.linalg.norm(S @ x - b) / np.linalg.norm(b) <= 2e-12
    kappa = (12.0 + shift) / shift
    assert np.max(np.abs(x - ref)) / np.max(np.abs(ref)) <= 1e-12 * kappa


@pytest.mark.parametrize("s", [1, 2, 4, 6, 8])
def test_sstep_cg_is_cg(s):
    A, S = _shifted_laplacian(12, 2.0)
    b = mi.random_vector(A.n, 5)
    x, steps, _ = oracle.cg(A, b, tol=1e-11)
    xs, steps_s, rel_s = oracle.sstep_cg(A, b, s, 14.0, tol=1e-11)
    assert abs(steps_s - steps) <= 1
    assert np.linalg.norm(S @ xs - b) / np.linalg.norm(b) <= 2e-11
    assert np.max(np.abs(xs - x)) / np.max(np.abs(x)) <= 1e-9


def test_zero_right_hand_side():
    A, _ = _shifted_laplacian(6, 1.0)
    b = np.zeros(A.n)
    x, steps, rel = oracle.cg(A, b)
    assert steps == 0 and np.all(x == 0)
    xs, steps_s, _ = oracle.sstep_cg(A, b, 4, 14.0)
    assert steps_s == 0 and np.all(xs == 0)
