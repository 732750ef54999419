"""GPU parity of the double-float FP64 form (MPK_F64_DF: FP64 x and Y, the
arithmetic on the FP32 pipe in pairs of FP32 numbers with compensated row
sums) against the FP64 oracle, through the C ABI.

Bars: the FP64 bar (relative infinity-norm error <= 1e-12 per power) on
matrices with FP32-exact values (stored as FP32) and with general FP64
values (stored as hi/lo pairs); integer-valued runs bit-identical to the
oracle while the results stay below 2^47; the wavefront and the baseline
(same row arithmetic) bit-identical; the range guard refuses inputs the pairs
cannot hold; the calls the form does not serve say so."""
import numpy as np
import pytest
import torch

import mpk_inputs as mi
import oracle
import paper_2205_01598_gb300 as mpk
from gpu_helpers import plan_of, rel_errors, run_mpk

pytestmark = pytest.mark.gpu

MATS = {
    "laplace2d-64": (lambda: mi.laplace2d(64), 4),           # FP32-exact values: stored as FP32
    "laplace3d-40": (lambda: mi.laplace3d(40), 4),
    "box27-14": (lambda: mi.box27(14), 4),
    "star3d-r3-18": (lambda: mi.star3d(18, 3), 8),           # order-6 weights: (hi, lo) pairs
    "anderson-16": (lambda: mi.anderson3d(16, seed=42), 8),  # random diagonal: pairs
    "randsym-3000": (lambda: mi.random_sparse(3000, 4.0 / 3000, 3), 8),
    "zipf-20000": (lambda: mi.zipf_graph(20000, 1001), 8),
}


@pytest.mark.parametrize("name", list(MATS))
@pytest.mark.parametrize("p", [1, 4, 8])
def test_df_matches_oracle(name, p):
    make, vbytes = MATS[name]
    A = make()
    x = mi.random_vector(A.n, 1234)
    ref = oracle.mpk(A, x, p)
    plan = plan_of(A, p, prec="f64df")
    info = mpk.mpk_plan_info(plan)
    assert info["prec"] == mpk.MPK_F64_DF and info["val_bytes"] == vbytes
    got = run_mpk(plan, x)
    err = rel_errors(got, ref)
    assert np.all(err <= 1e-12), err


def test_df_wavefront_equals_baseline_and_repeats():
    A = mi.anderson3d(20, seed=42)
    p = 7
    plan = plan_of(A, p, prec="f64df", tile_rows=128)
    perm = mpk.mpk_plan_perm(plan)[0].cpu().numpy()
    x = mi.random_vector(A.n, 5)[perm]
    y = run_mpk(plan, x, permuted=True)
    assert np.array_equal(y, run_mpk(plan, x, permuted=True, baseline=True))
    assert np.array_equal(y, run_mpk(plan, x, permuted=True))


def test_df_integer_valued_bit_exact():
    """x in {-1, 0, 1} on the 3D 7-point stencil: |y_p| <= 12^p < 2^47 for
    p <= 13, so every pair holds its integers exactly and the FP64 outputs
    equal the oracle's bit for bit."""
    A = mi.laplace3d(26)
    x = mi.integer_vector(A.n, 5)
    p = 12
    ref = oracle.mpk(A, x, p)
    assert np.max(np.abs(ref)) < 2.0 ** 47
    got = run_mpk(plan_of(A, p, prec="f64df"), x)
    assert np.array_equal(got, ref)


def test_df_unpermuted_io_and_host_buffers():
    A = mi.star3d(16, 2)
    p = 5
    plan = plan_of(A, p, prec="f64df")
    x = mi.random_vector(A.n, 17)
    ref = oracle.mpk(A, x, p)
    y = run_mpk(plan, x)
    assert np.all(rel_errors(y, ref) <= 1e-12)
    xh = torch.from_numpy(x).pin_memory()
    Yh = torch.empty(p, A.n, dtype=torch.float64).pin_memory()
    mpk.mpk_run_host(plan, xh, Yh)
    assert np.array_equal(Yh.numpy(), y)


def test_df_range_guard():
    """Values outside [2^-60, 2^60] are refused at planning time; an x whose
    powers would leave the pairs' range makes the call report
    MPK_ERR_UNSUPPORTED, and the plan serves the next valid call."""
    A = mi.laplace2d(12)
    big = mi.CSR(A.n, A.rowptr, A.col, A.val * 2.0 ** 70)
    with pytest.raises(mpk.MpkError) as e:
        plan_of(big, 2, prec="f64df")
    assert e.value.code == mpk.MPK_ERR_UNSUPPORTED
    p = 4
    plan = plan_of(A, p, prec="f64df")
    x = mi.random_vector(A.n, 3)
    xd = torch.from_numpy(x * 2.0 ** 95).cuda()
    Y = torch.empty(p, A.n, dtype=torch.float64, device="cuda")
    with pytest.raises(mpk.MpkError) as e:
        mpk.mpk_run(plan, xd, Y)
    assert e.value.code == mpk.MPK_ERR_UNSUPPORTED
    with pytest.raises(mpk.MpkError) as e:
        mpk.mpk_baseline_run(plan, xd, Y)
    assert e.value.code == mpk.MPK_ERR_UNSUPPORTED
    assert np.all(rel_errors(run_mpk(plan, x), oracle.mpk(A, x, p)) <= 1e-12)


def test_df_unserved_calls():
    A = mi.laplace3d(8)
    with pytest.raises(mpk.MpkError) as e:
        plan_of(A, 2, prec="f64df", nrhs=2)
    assert e.value.code == mpk.MPK_ERR_UNSUPPORTED
    plan = plan_of(A, 2, prec="f64df")
    with pytest.raises(mpk.MpkError) as e:
        mpk.mpk_batch_create([plan])
    assert e.value.code == mpk.MPK_ERR_UNSUPPORTED
    x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    y = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    with pytest.raises(mpk.MpkError) as e:
        mpk.mpk_cheb_real(plan, np.ones(3), 6.0, 6.0, x, y)
    assert e.value.code == mpk.MPK_ERR_UNSUPPORTED
    lo, hi = mpk.mpk_gershgorin(plan)
    assert (lo, hi) == oracle.gershgorin(A)


def test_df_config_3d_160_p8_full_size():
    """The 3D 7-point 160^3 workload (N = 4,096,000, nnz = 28,518,400, p = 8)
    in the double-float form, in the launch configuration the benchmark times
    (level order): every output against the oracle."""
    A = mi.laplace3d(160)
    p = 8
    plan = plan_of(A, p, prec="f64df")
    assert mpk.mpk_plan_info(plan)["val_bytes"] == 4
    perm = mpk.mpk_plan_perm(plan)[0].cpu().numpy()
    x = mi.random_vector(A.n, 1234)
    got = run_mpk(plan, x[perm], permuted=True)
    err = rel_errors(got, oracle.mpk(A, x, p)[:, perm])
    assert np.all(err <= 1e-12), err
