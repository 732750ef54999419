"""GPU parity of the level-blocked MPK (mpk_run) and of the baseline
(mpk_baseline_run) against the FP64 oracle, through the C ABI.

Bars: FP64 relative infinity-norm error <= 1e-12 per power; integer-valued
runs bit-identical (FP64 and FP32); FP32 <= 1e-5 per power on the stencil
workloads; baseline and wavefront bit-identical to each other (same row
kernel, same summation order); repeated runs bit-identical."""
import numpy as np
import pytest
import torch

import mpk_inputs as mi
import oracle
import paper_2205_01598_gb300 as mpk
from gpu_helpers import plan_of, rel_errors, run_mpk

pytestmark = pytest.mark.gpu

MATS = {
    "laplace2d-64": lambda: mi.laplace2d(64),              # 2D 5-point 64x64 workload
    "laplace3d-40": lambda: mi.laplace3d(40),
    "anderson-16": lambda: mi.anderson3d(16, seed=42),
    "box27-14": lambda: mi.box27(14),
    "randsym-3000": lambda: mi.random_sparse(3000, 4.0 / 3000, 3),
    "star3d-r3-18": lambda: mi.star3d(18, 3),
}


@pytest.mark.parametrize("name", list(MATS))
@pytest.mark.parametrize("p", [1, 4, 8])
def test_f64_matches_oracle(name, p):
    A = MATS[name]()
    x = mi.random_vector(A.n, 1234)
    ref = oracle.mpk(A, x, p)
    plan = plan_of(A, p, prec="f64")
    got = run_mpk(plan, x)
    assert np.all(rel_errors(got, ref) <= 1e-12)


@pytest.mark.parametrize("nrhs", [2, 3, 4, 8, 11])
def test_f64_block_vectors(nrhs):
    A = mi.laplace3d(20)
    x = mi.random_vector(A.n, 99, nrhs)
    ref = oracle.mpk(A, x, 5)
    plan = plan_of(A, 5, prec="f64", nrhs=nrhs)
    got = run_mpk(plan, x)
    assert np.all(rel_errors(got, ref) <= 1e-12)


@pytest.mark.parametrize("tile_rows,ctas,cache", [(32, 1, 50_000.0), (64, 8, 300_000.0), (1024, 2, 1e6),
                                                  (96, 3, 0.0)])
def test_wavefront_stress_many_groups(tile_rows, ctas, cache):
    """Small caches (many level groups), tiny or large tiles and few or many
    resident CTAs: every schedule must give the oracle's result."""
    A = mi.laplace3d(32)
    p = 7
    x = mi.random_vector(A.n, 7)
    ref = oracle.mpk(A, x, p)
    plan = plan_of(A, p, prec="f64", tile_rows=tile_rows, ctas_per_sm=ctas, cache_bytes=cache)
    info = mpk.mpk_plan_info(plan)
    if cache and cache < 1e6:
        assert info["n_groups"] > 10
    got = run_mpk(plan, x)
    assert np.all(rel_errors(got, ref) <= 1e-12)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_integer_valued_bit_exact(prec):
    """Integer matrix, x in {-1,0,1}: all partial sums are exact integers
    (< 2^24 for p <= 6 on the 7-point stencil), so any order of the sums gives
    the oracle's values exactly."""
    A = mi.laplace3d(26)
    x = mi.integer_vector(A.n, 5)
    ref = oracle.mpk(A, x, 6)
    assert np.max(np.abs(ref)) < 2 ** 24
    got = run_mpk(plan_of(A, 6, prec=prec), x)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("name", ["laplace2d-64", "laplace3d-40", "anderson-16"])
def test_f32_within_1e5(name):
    A = MATS[name]()
    x = mi.random_vector(A.n, 1234)
    ref = oracle.mpk(A, x, 8)
    got = run_mpk(plan_of(A, 8, prec="f32"), x.astype(np.float32))
    err = rel_errors(got, ref)
    assert np.all(err <= 1e-5), err


def test_permuted_io_and_baseline_bitwise():
    A = mi.anderson3d(14, seed=42)
    p = 6
    plan = plan_of(A, p, prec="f64", tile_rows=64)
    perm = mpk.mpk_plan_perm(plan)[0].cpu().numpy()
    x = mi.random_vector(A.n, 3)
    y_orig = run_mpk(plan, x)
    y_perm = run_mpk(plan, x[perm], permuted=True)
    assert np.array_equal(y_perm, y_orig[:, perm])
    y_base = run_mpk(plan, x[perm], permuted=True, baseline=True)
    assert np.array_equal(y_base, y_perm)
    y_again = run_mpk(plan, x[perm], permuted=True)
    assert np.array_equal(y_again, y_perm)
    # and the permuted result is the oracle on P A P^T (Sec. 4.1)
    level, L = oracle.bfs_levels(A)
    operm, oiperm, _ = oracle.level_perm(level, L)
    Ap = oracle.permute_csr(A, operm, oiperm)
    assert np.all(rel_errors(y_perm, oracle.mpk(Ap, x[perm], p)) <= 1e-12)


def test_permute_vectors_roundtrip():
    A = mi.laplace2d(30)
    plan = plan_of(A, 2, prec="f32", nrhs=3)
    perm = mpk.mpk_plan_perm(plan)[0].cpu().numpy()
    src = torch.arange(A.n * 3 * 2, dtype=torch.float32, device="cuda").reshape(2, A.n, 3)
    dst = torch.empty_like(src)
    mpk.mpk_permute_vectors(plan, src, dst, 2, True)
    assert torch.equal(dst.cpu(), src.cpu()[:, perm])
    back = torch.empty_like(src)
    mpk.mpk_permute_vectors(plan, dst, back, 2, False)
    assert torch.equal(back, src)


def test_timeout_is_reported_and_plan_recovers():
    """A completion flag that nothing sets (test hook) makes the dependent
    waits expire: the call returns MPK_ERR_TIMEOUT within the limit, names the
    node, and the next launch of the same plan is correct."""
    import time
    A = mi.laplace3d(24)
    p = 4
    plan = plan_of(A, p, prec="f64", tile_rows=64, timeout_s=0.25)
    info = mpk.mpk_plan_info(plan)
    x = mi.random_vector(A.n, 11)
    xd = torch.from_numpy(x).cuda()
    Y = torch.empty(p, A.n, dtype=torch.float64, device="cuda")
    t_drop = info["n_tiles"] // 2
    mpk.mpk_plan_debug_drop_flag(plan, t_drop, 2)
    t0 = time.time()
    with pytest.raises(mpk.MpkError) as e:
        mpk.mpk_run(plan, xd, Y)
    assert e.value.code == mpk.MPK_ERR_TIMEOUT
    assert time.time() - t0 < 10.0
    mpk.mpk_run(plan, xd, Y)   # recovered
    assert np.all(rel_errors(Y.cpu().numpy(), oracle.mpk(A, x, p)) <= 1e-12)


def test_config_3d_160_p8_full_size():
    """The 3D 7-point 160^3 workload (N = 4,096,000, nnz = 28,518,400, p = 8),
    FP64, in the launch configuration the benchmark times (level order),
    compared with the oracle on every output."""
    A = mi.laplace3d(160)
    assert A.nnz == 28_518_400
    p = 8
    plan = plan_of(A, p, prec="f64")
    perm = mpk.mpk_plan_perm(plan)[0].cpu().numpy()
    x = mi.random_vector(A.n, 1234)
    got = run_mpk(plan, x[perm], permuted=True)
    ref = oracle.mpk(A, x, p)
    assert np.all(rel_errors(got, ref[:, perm]) <= 1e-12)
    got32 = run_mpk(plan_of(A, p, prec="f32"), x[perm].astype(np.float32), permuted=True)
    assert np.all(rel_errors(got32, ref[:, perm]) <= 1e-5)


@pytest.mark.parametrize("prec", ["f64", "f32", "bf16val"])
@pytest.mark.parametrize("tile_rows", [128, 512])
def test_staged_slices_match_oracle(prec, tile_rows):
    """Opt-in form that stages each item's matrix slice in shared memory with
    bulk copies (MPK_TUNE_STAGE, with the evict-last hint)."""
    A = mi.anderson3d(18, seed=42) if prec == "bf16val" else mi.laplace3d(36)
    p = 6
    x = mi.random_vector(A.n, 21)
    ref = oracle.mpk(A, x, p)
    plan = plan_of(A, p, prec=prec, tile_rows=tile_rows, tune=mpk.MPK_TUNE_STAGE | mpk.MPK_TUNE_EVICT_LAST)
    assert mpk.mpk_plan_info(plan)["staged"] == 1
    xin = x if prec == "f64" else x.astype(np.float32)
    err = rel_errors(run_mpk(plan, xin), ref)
    assert np.all(err <= (1e-12 if prec == "f64" else 1e-5)), err


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 1e-5)])
def test_irregular_rows_sorted_by_length(prec, tol):
    """Zipf-degree rows: the plan sorts rows by length inside each work item
    (SELL-C-sigma); results match the oracle and, bit for bit, the unsorted
    packing (the same entries are summed in the same order)."""
    A = mi.zipf_graph(30000, 1003)
    x = mi.random_vector(A.n, 8, 3)
    ref = oracle.mpk(A, x, 5)
    ps = plan_of(A, 5, prec=prec, nrhs=3, tile_rows=512)
    pu = plan_of(A, 5, prec=prec, nrhs=3, tile_rows=512, tune=mpk.MPK_TUNE_NO_SORT)
    i_s, i_u = mpk.mpk_plan_info(ps), mpk.mpk_plan_info(pu)
    assert i_s["sorted"] == 1 and i_u["sorted"] == 0
    assert i_s["packed_entries"] < 0.8 * i_u["packed_entries"]
    xin = x if prec == "f64" else x.astype(np.float32)
    ys = run_mpk(ps, xin)
    assert np.all(rel_errors(ys, ref) <= tol)
    assert np.array_equal(ys, run_mpk(pu, xin))
    assert np.array_equal(ys, run_mpk(ps, xin, baseline=True))
