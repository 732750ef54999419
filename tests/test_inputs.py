"""Pins for the synthetic input generators (CPU only)."""
import numpy as np
import pytest

import mpk_inputs as mi
from conftest import read_golden


def test_splitmix64_published_vector():
    # Reference output of SplitMix64 for seed 1234567 (Steele et al. 2014;
    # the widely used test vector of the splitmix64.c reference code).
    want = [6457827717110365317, 3203168211198807973, 9817491932198370423,
            4593380528125082431, 16408922859458223821]
    assert [int(v) for v in mi.splitmix64(1234567, 5)] == want


def test_uniform_counter_based_and_in_range():
    a = mi.uniform(1234, 1000)
    b = mi.uniform(1234, 2000)[:1000]
    assert np.array_equal(a, b)
    assert a.min() >= -1.0 and a.max() < 1.0
    assert abs(a.mean()) < 0.1


def _star_nnz(n, r):
    # each of the 3 axes contributes, per grid line of n points, 2*(r*n - r(r+1)/2)
    # off-diagonal entries; there are n^2 lines per axis; plus N diagonal entries
    return n ** 3 + 3 * n * n * 2 * (r * n - r * (r + 1) // 2)


@pytest.mark.parametrize("n", [5, 9, 12])
@pytest.mark.parametrize("r", [1, 2, 3])
def test_star_stencil_nnz_closed_form(n, r):
    A = mi.star3d(n, r) if r > 1 else mi.laplace3d(n)
    assert A.nnz == _star_nnz(n, r)
    # symmetric pattern and values
    dense = np.zeros((A.n, A.n))
    for i in range(A.n):
        dense[i, A.col[A.rowptr[i]:A.rowptr[i + 1]]] = A.val[A.rowptr[i]:A.rowptr[i + 1]]
    assert np.array_equal(dense, dense.T)


def test_tab3_heat_sizes_follow_closed_form():
    g = read_golden("matrix_sizes.txt")
    n = g["heat_n"][0]
    assert [_star_nnz(n, r) for r in (1, 2, 3)] == g["heat_nnz"]


def test_anderson_and_hpcg_sizes():
    g = read_golden("matrix_sizes.txt")
    n = g["anderson_n"][0]
    assert 7 * n ** 3 - 6 * n ** 2 == g["anderson_nnz"][0]      # open boundaries
    for m in (4, 7):
        assert mi.anderson3d(m, periodic=False).nnz == 7 * m ** 3 - 6 * m ** 2
        assert mi.anderson3d(m, periodic=True).nnz == 7 * m ** 3
    h = g["hpcg_n"][0]
    assert (3 * h - 2) ** 3 == g["hpcg_nnz"][0]
    for m in (3, 6):
        assert mi.box27(m).nnz == (3 * m - 2) ** 3


def test_laplace2d_64_config_size():
    A = mi.laplace2d(64)
    assert (A.n, A.nnz) == (4096, 20224)
    assert np.all(np.diff(A.rowptr) <= 5)


def test_rows_sorted_and_diagonal_values():
    A = mi.anderson3d(6, W=16.5, seed=42)
    for i in range(A.n):
        cs = A.col[A.rowptr[i]:A.rowptr[i + 1]]
        assert np.all(np.diff(cs) > 0)
        vs = A.val[A.rowptr[i]:A.rowptr[i + 1]]
        assert np.count_nonzero(vs == -1.0) == 6
        d = vs[cs == i][0]
        assert -8.25 <= d <= 8.25
