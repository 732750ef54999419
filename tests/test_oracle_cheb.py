"""Pins for the oracle's Chebyshev time propagation (Sec. 7, Eq. 7-9), its
coefficients and the Gershgorin scaling: trigonometric closed forms of T_k,
the generating function of the Bessel coefficients, diagonal Hamiltonians,
a dense matrix exponential from scipy, and unitarity."""
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


def _tail(z, M):
    """Truncation bound sum_{k>M} 2|J_k(z)| (terms decay super-exponentially)."""
    k = np.arange(M + 1, M + 200)
    return 2 * np.abs(sps.jv(k, z)).sum()


def test_gershgorin_diagonal_and_dense():
    d = mi.uniform(3, 40, -5, 7)
    lo, hi = oracle.gershgorin(mi.diagonal(d))
    assert (lo, hi) == (d.min(), d.max())
    A = mi.anderson3d(5, W=16.5, seed=42)
    lo, hi = oracle.gershgorin(A)
    ev = np.linalg.eigvalsh(_dense(A))
    assert lo <= ev.min() and ev.max() <= hi
    eps = A.val[A.col == np.repeat(np.arange(A.n), np.diff(A.rowptr))]
    assert np.isclose(lo, eps.min() - 6) and np.isclose(hi, eps.max() + 6)


@pytest.mark.parametrize("c,r,dt,M", [(0.0, 14.25, 50 / 14.25, 64), (0.3, 2.0, 1.5, 20),
                                      (-1.0, 5.0, 0.7, 16)])
def test_coefficient_generating_function(c, r, dt, M):
    """sum_k coef_k T_k(cos t) = exp(-i (c + r cos t) dt): the Jacobi-Anger
    expansion evaluated where T_k(cos t) = cos(k t) is known in closed form."""
    coef = oracle.cheb_coeffs_schroedinger(M, c, r, dt)
    bound = _tail(r * dt, M) + 1e-13 * M
    for t in np.linspace(0, np.pi, 9):
        got = np.sum(coef * np.cos(np.arange(M + 1) * t))
        want = np.exp(-1j * (c + r * np.cos(t)) * dt)
        assert abs(got - want) <= bound, t
    # J_0 + 2 sum J_2k = 1 is the t = 0, c = 0 case of the same identity
    z = r * dt
    assert abs(sps.jv(0, z) + 2 * sum(sps.jv(2 * k, z) for k in range(1, 200)) - 1) < 1e-12


def test_truncation_at_degree_64_with_rdt_50():
    """Degree 64 with r*dt = 50 keeps the discarded coefficients below the
    1e-4 cut-off used for the Schroedinger runs (Sec. 7)."""
    k = np.arange(65, 200)
    assert np.max(2 * np.abs(sps.jv(k, 50.0))) < 1e-4


@pytest.mark.parametrize("K", [0, 1, 2, 5, 9])
def test_eigenvector_gives_cos_k_theta(K):
    """For A v = lambda v and Ahat = (A - c)/r = cos(theta): v_k = cos(k theta) v.
    With coefficients e_K the oracle must return cos(K theta) v."""
    n = 16
    A = mi.laplace1d(n)
    i = np.arange(n)
    kmode = 5
    v = np.sin(kmode * np.pi * (i + 1) / (n + 1))
    lam = 2 - 2 * np.cos(kmode * np.pi / (n + 1))
    c, r = 2.0, 2.0
    theta = np.arccos((lam - c) / r)
    coef = np.zeros(12, dtype=complex)
    coef[K] = 1.0
    y = oracle.cheb(A, coef, c, r, v.astype(complex))
    assert np.max(np.abs(y - np.cos(K * theta) * v)) < 1e-13


def test_diagonal_hamiltonian_phase():
    d = mi.uniform(8, 64, -3, 4)
    A = mi.diagonal(d)
    lo, hi = oracle.gershgorin(A)
    c, r = (hi + lo) / 2, (hi - lo) / 2
    dt = 50.0 / r
    M = 64
    coef = oracle.cheb_coeffs_schroedinger(M, c, r, dt)
    psi = mi.uniform(1, 64) + 1j * mi.uniform(2, 64)
    y = oracle.cheb(A, coef, c, r, psi)
    assert np.max(np.abs(y - np.exp(-1j * d * dt) * psi)) <= _tail(r * dt, M) * np.max(np.abs(psi)) + 1e-12


def test_anderson_vs_dense_expm_and_unitarity():
    A = mi.anderson3d(4, W=16.5, seed=42)
    lo, hi = oracle.gershgorin(A)
    c, r = (hi + lo) / 2, (hi - lo) / 2
    dt = 50.0 / r
    M = 64
    coef = oracle.cheb_coeffs_schroedinger(M, c, r, dt)
    psi = mi.uniform(1234, A.n) + 1j * mi.uniform(4321, A.n)
    psi /= np.linalg.norm(psi)
    y = oracle.cheb(A, coef, c, r, psi)
    want = sla.expm(-1j * dt * _dense(A)) @ psi
    bound = _tail(r * dt, M) * np.sqrt(A.n)
    assert np.linalg.norm(y - want) <= bound + 1e-11
    assert abs(np.linalg.norm(y) - 1.0) <= bound + 1e-11
