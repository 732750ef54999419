"""Pins for the oracle's SpMV / baseline MPK (Sec. 3.1, Fig. 1) and its
level-blocked traversal (Fig. 5), checked against facts that do not come
from the oracle itself: dense brute force, eigen-pairs in closed form,
exact integer arithmetic, diagonal matrices and permutation invariance."""
import numpy as np
import pytest

import mpk_inputs as mi
import oracle


def _dense(A):
    D = np.zeros((A.n, A.n))
    for i in range(A.n):
        np.add.at(D[i], A.col[A.rowptr[i]:A.rowptr[i + 1]], A.val[A.rowptr[i]:A.rowptr[i + 1]])
    return D


@pytest.mark.parametrize("seed", [1, 2, 3])
@pytest.mark.parametrize("nrhs", [1, 3])
def test_mpk_vs_dense_brute_force(seed, nrhs):
    n = 17 + 11 * seed
    A = mi.random_sparse(n, 0.15, seed, symmetric=(seed != 2))
    x = mi.random_vector(n, 1234 + seed, nrhs)
    pm = 6
    Y = oracle.mpk(A, x, pm)
    D = _dense(A).astype(np.longdouble)
    y = x.astype(np.longdouble)
    for k in range(pm):
        y = D @ y
        ref = y.astype(np.float64)
        err = np.max(np.abs(Y[k] - ref)) / np.max(np.abs(ref))
        assert err <= 1e-13, (k, err)


def _eig_check(A, v_ld, lam_ld, pm):
    """A^k v = lam^k v for an exact eigenpair given in extended precision:
    the oracle gets v rounded to FP64; the error allowed is the forward
    error of k rounded SpMVs plus the propagated rounding of v itself."""
    v = v_ld.astype(np.float64)
    Y = oracle.mpk(A, v, pm)
    norm_a = np.max(np.add.reduceat(np.abs(A.val), A.rowptr[:-1]))
    nnzr = np.max(np.diff(A.rowptr))
    u = 2.0 ** -53
    for k in range(1, pm + 1):
        want = (lam_ld ** k * v_ld).astype(np.float64)
        tol = (2 * k * nnzr + 2) * u * norm_a ** k * np.max(np.abs(v))
        err = np.max(np.abs(Y[k - 1] - want))
        assert err <= tol, (k, err, tol)
        # and the check is sharp: a wrong power is far outside the tolerance
        assert np.max(np.abs(Y[k - 1] - lam_ld.astype(np.float64) ** (k - 1) * v)) > 1e3 * tol or abs(lam_ld - 1) < 1e-3


_PI = np.pi if np.finfo(np.longdouble).eps >= 1e-16 else np.longdouble("3.141592653589793238462643383279502884")


def _sin_mode(k, i, n):
    return np.sin(np.longdouble(k) * _PI * (i + 1).astype(np.longdouble) / np.longdouble(n + 1))


def _lam(k, n):
    return np.longdouble(2) - 2 * np.cos(np.longdouble(k) * _PI / np.longdouble(n + 1))


@pytest.mark.parametrize("kmode", [10, 15, 20])  # modes away from the bottom: low modes amplify rounding by (|A|/lambda)^k
def test_laplace1d_sine_eigenmodes(kmode):
    n = 20
    A = mi.laplace1d(n)
    i = np.arange(n)
    _eig_check(A, _sin_mode(kmode, i, n), _lam(kmode, n), 8)


@pytest.mark.parametrize("k1,k2", [(64, 64), (32, 40), (1, 64)])
def test_laplace2d_sine_eigenmodes_config_grid(k1, k2):
    n = 64
    A = mi.laplace2d(n)
    ix = np.arange(n * n) % n
    iy = np.arange(n * n) // n
    v = _sin_mode(k1, ix, n) * _sin_mode(k2, iy, n)
    _eig_check(A, v, _lam(k1, n) + _lam(k2, n), 4)


def test_laplace3d_sine_eigenmode():
    n = 12
    A = mi.laplace3d(n)
    idx = np.arange(n ** 3)
    c = [idx % n, (idx // n) % n, idx // (n * n)]
    v = np.ones(n ** 3, dtype=np.longdouble)
    lam = np.longdouble(0)
    for kd, cd in zip((12, 11, 6), c):
        v = v * _sin_mode(kd, cd, n)
        lam = lam + _lam(kd, n)
    _eig_check(A, v, lam, 8)


def test_diagonal_powers_exact():
    n = 50
    z = mi.splitmix64(5, n)
    d = 2.0 ** ((z % np.uint64(9)).astype(np.int64) - 4)        # powers of two
    d *= np.where((z >> np.uint64(8)) % np.uint64(2) == 0, 1.0, -1.0)
    x = 2.0 ** (((z >> np.uint64(16)) % np.uint64(7)).astype(np.int64) - 3)
    A = mi.diagonal(d)
    Y = oracle.mpk(A, x, 7)
    for k in range(1, 8):
        assert np.array_equal(Y[k - 1], d ** k * x)


@pytest.mark.parametrize("make,pm", [(lambda: mi.laplace3d(9), 6), (lambda: mi.laplace2d(30), 10),
                                     (lambda: mi.box27(6), 5)])
def test_integer_valued_exact(make, pm):
    """Integer matrix and x in {-1,0,1}: every partial sum is an integer below
    2^53, so FP64 must agree exactly with int64 arithmetic."""
    A = make()
    x = mi.integer_vector(A.n, 77)
    Y = oracle.mpk(A, x, pm)
    ai = A.val.astype(np.int64)
    assert np.array_equal(ai.astype(np.float64), A.val)
    y = x.astype(np.int64)
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    for k in range(pm):
        nxt = np.zeros(A.n, dtype=np.int64)
        np.add.at(nxt, rows, ai * y[A.col])
        y = nxt
        assert np.max(np.abs(y)) < 2 ** 53
        assert np.array_equal(Y[k], y.astype(np.float64)), k


def test_permutation_invariance():
    """oracle(P A P^T, P x) == P oracle(A, x): exact on integer data, within
    rounding on random data (the row sums change order)."""
    A = mi.laplace3d(8)
    lev, L = oracle.bfs_levels(A)
    perm, iperm, _ = oracle.level_perm(lev, L)
    Ap = oracle.permute_csr(A, perm, iperm)
    xi = mi.integer_vector(A.n, 3)
    Y = oracle.mpk(A, xi, 5)
    Yp = oracle.mpk(Ap, xi[perm], 5)
    assert np.array_equal(Yp, Y[:, perm])
    xr = mi.random_vector(A.n, 1234)
    Y = oracle.mpk(A, xr, 5)
    Yp = oracle.mpk(Ap, xr[perm], 5)
    for k in range(5):
        assert np.max(np.abs(Yp[k] - Y[k][perm])) <= 1e-14 * np.max(np.abs(Y[k]))


@pytest.mark.parametrize("make", [lambda: mi.stencil2d_7pt(8), lambda: mi.laplace2d(24),
                                  lambda: mi.laplace3d(7), lambda: mi.random_sparse(60, 0.08, 9)])
@pytest.mark.parametrize("pm", [1, 3, 5])
def test_level_blocked_order_equals_baseline(make, pm):
    """Fig. 5 (levels) and the level-group traversal give bit-identical
    results to pm back-to-back SpMVs: same operands, same row sums.  Y starts
    as NaN, so a node that read a value before it was computed would show."""
    A = make()
    lev, L = oracle.bfs_levels(A, symmetrize=True)
    perm, iperm, lp = oracle.level_perm(lev, L)
    Ap = oracle.permute_csr(A, perm, iperm)
    x = mi.random_vector(A.n, 1234)[perm]
    ref = oracle.mpk(Ap, x, pm)
    got = oracle.lb_mpk(Ap, lp, x, pm)
    assert np.array_equal(got, ref)
    w = np.diff(lp).astype(np.float64)
    gp = oracle.level_groups(w, pm, 0.5, 4.0 * (pm + 1) * max(w))
    rows_of_groups = lp[gp]
    got = oracle.lb_mpk(Ap, rows_of_groups, x, pm)
    assert np.array_equal(got, ref)


def test_level_blocked_order_detects_bad_units():
    """Counter-check of the NaN sentinel: with units that are not BFS levels
    (an odd/even interleaving of a 1D chain, which breaks Eq. 4) the same
    traversal reads entries of y_{p-1} that are not computed yet."""
    A = mi.laplace1d(100)
    x = mi.random_vector(A.n, 1)
    P = np.concatenate([np.arange(0, 100, 2), np.arange(1, 100, 2)]).astype(np.int32)
    IP = np.empty_like(P)
    IP[P] = np.arange(100, dtype=np.int32)
    Ab = oracle.permute_csr(A, P, IP)
    units = np.array([0, 25, 50, 75, 100], dtype=np.int32)
    assert np.isnan(oracle.lb_mpk(Ab, units, x[P], 3)).any()
    # while the true levels of the same chain work
    lev, L = oracle.bfs_levels(A)
    perm, iperm, lp = oracle.level_perm(lev, L)
    Ap = oracle.permute_csr(A, perm, iperm)
    assert np.array_equal(oracle.lb_mpk(Ap, lp, x[perm], 3), oracle.mpk(Ap, x[perm], 3))
