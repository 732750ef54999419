"""Degenerate and extreme inputs of the level-blocked MPK against the FP64
oracle: a single row (with and without its diagonal), rows without entries,
the all-zero matrix (no stored entries, NULL index and value arrays), the
largest power (p = 255), the widest block vector (nrhs = 64), one very wide
row, and a dense block; in both schedules where they apply."""
import numpy as np
import pytest
import torch

import mpk_inputs as mi
import oracle
import paper_2205_01598_gb300 as mpk
from gpu_helpers import plan_of, rel_errors, run_mpk

pytestmark = pytest.mark.gpu


def _csr(n, rows):
    """CSR from a list of (row, col, value) triples."""
    rows = sorted(rows)
    rowptr = np.zeros(n + 1, dtype=np.int32)
    for r, _, _ in rows:
        rowptr[r + 1] += 1
    rowptr = np.cumsum(rowptr).astype(np.int32)
    col = np.array([c for _, c, _ in rows], dtype=np.int32)
    val = np.array([v for _, _, v in rows], dtype=np.float64)
    return mi.CSR(n, rowptr, col, val, name="edge")


def _check(A, p, tol=0.0, **kw):
    x = mi.random_vector(A.n, 31)
    ref = oracle.mpk(A, x, p)
    got = run_mpk(plan_of(A, p, prec="f64", **kw), x)
    scale = max(1e-300, np.max(np.abs(ref)))
    assert np.max(np.abs(got - ref)) <= tol * scale, (np.max(np.abs(got - ref)), scale)


def test_single_row():
    _check(_csr(1, [(0, 0, 0.5)]), 6)          # y_k = 0.5^k x exactly
    _check(_csr(1, []), 3)                      # no entries: all zero


def test_rows_without_entries():
    # a chain with every third row empty: several components, zero rows
    trip = []
    for i in range(301):
        if i % 3 == 2:
            continue
        trip.append((i, i, 2.0))
        if i + 1 < 301 and (i + 1) % 3 != 2:
            trip += [(i, i + 1, -1.0), (i + 1, i, -1.0)]
    A = _csr(301, trip)
    _check(A, 5, tol=1e-12)
    _check(A, 5, tol=1e-12, tune=mpk.MPK_TUNE_RESIDENT)


def test_all_zero_matrix_with_null_arrays():
    n = 100
    rp = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
    cl = torch.zeros(0, dtype=torch.int32, device="cuda")
    va = torch.zeros(0, dtype=torch.float64, device="cuda")
    plan = mpk.mpk_plan(rp, cl, va, 4)
    info = mpk.mpk_plan_info(plan)
    assert info["n_levels"] == n and info["nnz"] == 0
    x = torch.from_numpy(mi.random_vector(n, 2)).cuda()
    Y = torch.full((4, n), float("nan"), dtype=torch.float64, device="cuda")
    mpk.mpk_run(plan, x, Y)
    assert torch.count_nonzero(Y).item() == 0


def test_largest_power():
    A = mi.laplace2d(20)
    x = mi.random_vector(A.n, 5)
    # scale so that 255 powers stay in range: the spectral radius of A/8 is < 1
    A8 = mi.CSR(A.n, A.rowptr, A.col, A.val / 8.0)
    ref = oracle.mpk(A8, x, 255)
    got = run_mpk(plan_of(A8, 255, prec="f64"), x)
    assert np.all(rel_errors(got, ref) <= 1e-11)
    with pytest.raises(mpk.MpkError):
        plan_of(A8, 256, prec="f64")


def test_widest_block_vector():
    A = mi.laplace3d(10)
    x = mi.random_vector(A.n, 6, 64)
    ref = oracle.mpk(A, x, 3)
    got = run_mpk(plan_of(A, 3, prec="f64", nrhs=64), x)
    assert np.all(rel_errors(got, ref) <= 1e-12)
    with pytest.raises(mpk.MpkError):
        plan_of(A, 3, prec="f64", nrhs=65)


def test_one_very_wide_row_and_dense_block():
    n = 3000
    trip = [(i, i, 4.0) for i in range(n)]
    trip += [(0, j, 1e-3) for j in range(1, n)] + [(j, 0, 1e-3) for j in range(1, n)]   # arrow matrix
    _check(_csr(n, trip), 4, tol=1e-12)
    D = mi.random_sparse(64, 1.0, 9)   # fully dense 64 x 64
    _check(D, 5, tol=1e-12)
    _check(D, 5, tol=1e-12, tune=mpk.MPK_TUNE_RESIDENT)


def test_binding_rejects_mismatched_cuda_tensors():
    """A CUDA tensor of the wrong size or dtype never reaches a kernel: the
    binding raises before the launch, and the plan stays usable."""
    A = mi.laplace2d(16)
    plan = plan_of(A, 3, prec="f64")
    x = torch.rand(A.n, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        mpk.mpk_run(plan, x[:-1], torch.empty(3, A.n, dtype=torch.float64, device="cuda"))
    with pytest.raises(ValueError):
        mpk.mpk_run(plan, x, torch.empty(2, A.n, dtype=torch.float64, device="cuda"))
    with pytest.raises(TypeError):
        mpk.mpk_run(plan, x.float(), torch.empty(3, A.n, dtype=torch.float32, device="cuda"))
    Y = torch.empty(3, A.n, dtype=torch.float64, device="cuda")
    mpk.mpk_run(plan, x, Y)
    ref = oracle.mpk(A, x.cpu().numpy(), 3)
    assert np.all(rel_errors(Y.cpu().numpy(), ref) <= 1e-12)
