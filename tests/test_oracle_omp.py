"""The multicore comparator of the benchmark (p back-to-back SpMVs, rows split
statically over OpenMP threads) agrees with the sequential oracle bit for bit:
both sum every row in stored order without FMA contraction."""
import numpy as np
import pytest

import mpk_inputs as mi
import oracle


@pytest.mark.parametrize("make,p", [(lambda: mi.laplace3d(20), 8), (lambda: mi.zipf_graph(5000, 3), 3),
                                    (lambda: mi.random_sparse(64, 0.2, 5), 5)])
def test_openmp_pxspmv_equals_the_oracle(make, p):
    try:
        oracle.omp_pxspmv(mi.laplace2d(4), np.ones(16), 1)
    except RuntimeError:
        pytest.skip("gcc without OpenMP")
    A = make()
    x = mi.random_vector(A.n, 9)
    Y, threads = oracle.omp_pxspmv(A, x, p)
    assert threads >= 1
    assert np.array_equal(Y, oracle.mpk(A, x, p))
