"""Pins for the oracle's heat-equation propagation (Sec. 7, modified-Bessel
coefficients; Eq. 7-9 with real vectors): scipy's scaled modified Bessel
function, the generating function, the decay of a Laplacian eigenmode, a
diagonal operator, a dense matrix exponential, and agreement with the
complex recurrence."""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.special as sps

import mpk_inputs as mi
import oracle


def _dense(A):
    D = np.zeros((A.n, A.n))
    for i in range(A.n):
        D[i, A.col[A.rowptr[i]:A.rowptr[i + 1]]] = A.val[A.rowptr[i]:A.rowptr[i + 1]]
    return D


def _tail(c, r, tau, M):
    """Truncation bound sum_{k>M} |c_k| = 2 e^{-tau c} sum_{k>M} I_k(tau r)."""
    k = np.arange(M + 1, M + 400)
    return 2 * np.exp(-tau * (c - r)) * sps.ive(k, tau * r).sum()


@pytest.mark.parametrize("c,r,tau,M", [(6.0, 6.0, 50 / 6.0, 64), (2.0, 1.5, 3.0, 30), (0.5, 0.5, 0.1, 8),
                                       (12.0, 12.0, 20 / 12.0, 48)])
def test_coefficients_match_scaled_bessel(c, r, tau, M):
    coef = oracle.cheb_coeffs_heat(M, c, r, tau)
    k = np.arange(M + 1)
    want = np.where(k == 0, 1.0, 2.0) * (-1.0) ** k * np.exp(-tau * (c - r)) * sps.ive(k, tau * r)
    assert np.max(np.abs(coef - want)) <= 1e-14 * max(1.0, np.abs(want).max())


@pytest.mark.parametrize("c,r,tau,M", [(6.0, 6.0, 50 / 6.0, 64), (1.0, 3.0, 0.7, 20)])
def test_generating_function(c, r, tau, M):
    """sum_k c_k cos(k t) = exp(-tau (c + r cos t)): the expansion of exp(-tau A)
    at the eigenvalue c + r cos t."""
    coef = oracle.cheb_coeffs_heat(M, c, r, tau)
    t = np.linspace(0, np.pi, 97)
    lhs = (coef[None, :] * np.cos(np.outer(t, np.arange(M + 1)))).sum(1)
    rhs = np.exp(-tau * (c + r * np.cos(t)))
    assert np.max(np.abs(lhs - rhs)) <= _tail(c, r, tau, M) + 1e-15 * (M + 1) * np.abs(coef).sum()


def test_laplacian_eigenmode_decays_exactly():
    """A = 3D 7-point Laplacian (Dirichlet), v = product of sines with
    eigenvalue lam: exp(-tau A) v = exp(-tau lam) v."""
    n = 10
    A = mi.laplace3d(n)
    lo, hi = oracle.gershgorin(A)
    c, r = (hi + lo) / 2, (hi - lo) / 2
    tau, M = 40.0 / r, 64
    coef = oracle.cheb_coeffs_heat(M, c, r, tau)
    idx = np.arange(1, n + 1, dtype=np.float64)
    for m in [(1, 1, 1), (3, 7, 2), (9, 10, 10)]:
        s = [np.sin(mm * np.pi * idx / (n + 1)) for mm in m]
        v = (s[2][:, None, None] * s[1][None, :, None] * s[0][None, None, :]).ravel()
        lam = sum(2 - 2 * np.cos(mm * np.pi / (n + 1)) for mm in m)
        y = oracle.cheb_real(A, coef, c, r, v)
        want = np.exp(-tau * lam) * v
        assert np.max(np.abs(y - want)) <= 1e-12 * np.max(np.abs(v)) + _tail(c, r, tau, M)


def test_diagonal_operator():
    d = mi.uniform(8, 50, 0.0, 4.0)
    A = mi.diagonal(d)
    c, r = 2.0, 2.0
    tau, M = 5.0, 40
    x = mi.uniform(9, 50)
    y = oracle.cheb_real(A, oracle.cheb_coeffs_heat(M, c, r, tau), c, r, x)
    assert np.max(np.abs(y - np.exp(-tau * d) * x)) <= 1e-13 + _tail(c, r, tau, M)


def test_dense_expm():
    A = mi.laplace2d(9, 7)
    lo, hi = oracle.gershgorin(A)
    c, r = (hi + lo) / 2, (hi - lo) / 2
    tau, M = 2.5, 40
    x = mi.random_vector(A.n, 3)
    y = oracle.cheb_real(A, oracle.cheb_coeffs_heat(M, c, r, tau), c, r, x)
    want = sla.expm(-tau * _dense(A)) @ x
    assert np.max(np.abs(y - want)) <= 1e-12 * np.max(np.abs(x)) + _tail(c, r, tau, M)


def test_real_recurrence_agrees_with_complex_one():
    """The real and the complex recurrences of the oracle are separate code;
    with real coefficients and a real vector they must give the same values."""
    A = mi.anderson3d(6, seed=42)
    lo, hi = oracle.gershgorin(A)
    c, r = (hi + lo) / 2, (hi - lo) / 2
    coef = oracle.cheb_coeffs_heat(20, c, r, 0.3)
    x = mi.random_vector(A.n, 5)
    yr = oracle.cheb_real(A, coef, c, r, x)
    yc = oracle.cheb(A, coef.astype(np.complex128), c, r, x.astype(np.complex128))
    assert np.array_equal(yr, yc.real) and np.all(yc.imag == 0)
