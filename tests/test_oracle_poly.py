"""Pins for the approximate inverse applied by Chebyshev propagation (a
polynomial preconditioner, Sec. 8): the oracle's quadrature coefficients
against the closed-form geometric series of 1/(c + r t), the truncated
series against 1/(c + r t) within its bound, the oracle's propagation
against a dense solve, and the library's coefficients (host code, no GPU)
against the oracle."""
import numpy as np
import pytest
import scipy.linalg as sla

import mpk_inputs as mi
import oracle
import paper_2205_01598_gb300 as mpk


@pytest.fixture(scope="module")
def lib():
    mpk.build()
    return mpk.load()


def _bound(c, r, M):
    s = np.sqrt(c * c - r * r)
    q = r / (c + s)
    return 2 * q ** (M + 1) / (s * (1 - q))


@pytest.mark.parametrize("c,r,M", [(7.0, 6.0, 64), (2.0, 1.0, 30), (1.0, 0.0, 5), (13.0, 12.9, 200)])
def test_quadrature_matches_geometric_series(c, r, M):
    got = oracle.cheb_coeffs_inverse(M, c, r, nodes=max(4096, 8 * M))
    s = np.sqrt(c * c - r * r)
    q = (c - s) / r if r > 0 else 0.0
    k = np.arange(M + 1)
    want = np.where(k == 0, 1.0, 2.0) * (-q) ** k / s
    assert np.max(np.abs(got - want)) <= 1e-13 * np.abs(want).max()


@pytest.mark.parametrize("c,r,M", [(7.0, 6.0, 40), (2.0, 1.9, 120)])
def test_truncated_series_approximates_the_inverse(c, r, M):
    coef = oracle.cheb_coeffs_inverse(M, c, r, nodes=8192)
    t = np.linspace(-1, 1, 501)
    series = (coef[None, :] * np.cos(np.outer(np.arccos(t), np.arange(M + 1)))).sum(1)
    assert np.max(np.abs(series - 1.0 / (c + r * t))) <= _bound(c, r, M) + 1e-13 * coef[0] * (M + 1)


def _shifted(A, sigma):
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    val = A.val.copy()
    val[A.col == rows] += sigma
    return mi.CSR(A.n, A.rowptr, A.col, val)


def test_propagation_solves_a_dense_system():
    A = _shifted(mi.laplace2d(9, 7), 0.5)
    lo, hi = oracle.gershgorin(A)
    lo = max(lo, 0.5)   # the shifted Laplacian's spectrum starts above the shift
    c, r, M = (hi + lo) / 2, (hi - lo) / 2, 80
    b = mi.random_vector(A.n, 12)
    y = oracle.cheb_real(A, oracle.cheb_coeffs_inverse(M, c, r), c, r, b)
    D = np.zeros((A.n, A.n))
    for i in range(A.n):
        D[i, A.col[A.rowptr[i]:A.rowptr[i + 1]]] = A.val[A.rowptr[i]:A.rowptr[i + 1]]
    want = sla.solve(D, b)
    assert np.max(np.abs(y - want)) <= _bound(c, r, M) * np.linalg.norm(b) + 1e-12 * np.abs(want).max()


@pytest.mark.parametrize("c,r,M", [(7.0, 6.0, 64), (3.5, 0.25, 9), (1.0, 0.0, 3)])
def test_library_coefficients_match_the_oracle(lib, c, r, M):
    got = mpk.mpk_cheb_coeffs_inverse(M, c, r)
    want = oracle.cheb_coeffs_inverse(M, c, r)
    assert np.max(np.abs(got - want)) <= 1e-14 * want[0]


@pytest.mark.parametrize("c,r", [(1.0, 1.0), (1.0, 2.0), (-1.0, 0.5), (1.0, -0.1)])
def test_library_rejects_intervals_that_reach_zero(lib, c, r):
    with pytest.raises(mpk.MpkError) as e:
        mpk.mpk_cheb_coeffs_inverse(8, c, r)
    assert e.value.code == mpk.MPK_ERR_INVALID
