"""GPU parity of the resident schedule (MPK_TUNE_RESIDENT): every CTA keeps a
tile's packed slice in shared memory for all p powers.  Same bars as the
work-list schedule: FP64 <= 1e-12 relative per power, FP32 <= 1e-5, the
baseline's bits (same row arithmetic, same summation order), Chebyshev FP64
<= 1e-12; plans that cannot run it (rows too wide for a stage, or a grid too
small to rule out a cycle of waits) fall back and stay correct."""
import numpy as np
import pytest
import torch

import mpk_inputs as mi
import oracle
import paper_2205_01598_gb300 as mpk
from gpu_helpers import plan_of, rel_errors, run_mpk

pytestmark = pytest.mark.gpu
RES = mpk.MPK_TUNE_RESIDENT

MATS = {
    "laplace2d-64": lambda: mi.laplace2d(64),
    "laplace3d-40": lambda: mi.laplace3d(40),
    "anderson-16": lambda: mi.anderson3d(16, seed=42),
    "box27-14": lambda: mi.box27(14),
    "star3d-r3-18": lambda: mi.star3d(18, 3),
}


@pytest.mark.parametrize("name", list(MATS))
@pytest.mark.parametrize("p", [1, 4, 8])
def test_resident_f64_matches_oracle(name, p):
    A = MATS[name]()
    x = mi.random_vector(A.n, 1234)
    ref = oracle.mpk(A, x, p)
    plan = plan_of(A, p, prec="f64", tune=RES)
    assert mpk.mpk_plan_info(plan)["resident"] == 1
    assert np.all(rel_errors(run_mpk(plan, x), ref) <= 1e-12)


@pytest.mark.parametrize("tile_rows,ctas", [(32, 1), (64, 2), (96, 1)])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_resident_many_tiles_per_cta(tile_rows, ctas, prec):
    """Small explicit tiles: each CTA runs many tiles in turn, both stages
    alternate, and the grid is far below the tile count."""
    A = mi.laplace2d(300, 200)
    p = 8
    x = mi.random_vector(A.n, 5)
    ref = oracle.mpk(A, x, p)
    plan = plan_of(A, p, prec=prec, tile_rows=tile_rows, ctas_per_sm=ctas, tune=RES)
    info = mpk.mpk_plan_info(plan)
    assert info["resident"] == 1 and info["n_tiles"] > 1.5 * info["grid_ctas"]
    assert info["grid_ctas"] > (p - 1) * info["dep_span"]
    xin = x if prec == "f64" else x.astype(np.float32)
    got = run_mpk(plan, xin)
    assert np.all(rel_errors(got, ref) <= (1e-12 if prec == "f64" else 1e-5))
    assert np.array_equal(got, run_mpk(plan, xin, baseline=True))


@pytest.mark.parametrize("prec", ["f64", "f32", "bf16val"])
def test_resident_bitwise_equal_to_baseline(prec):
    A = mi.anderson3d(20, seed=42)
    p = 8
    plan = plan_of(A, p, prec=prec, tune=RES)
    assert mpk.mpk_plan_info(plan)["resident"] == 1
    x = mi.random_vector(A.n, 17)
    xin = x if prec == "f64" else x.astype(np.float32)
    got = run_mpk(plan, xin)
    assert np.array_equal(got, run_mpk(plan, xin, baseline=True))
    assert np.array_equal(got, run_mpk(plan, xin))   # repeatable
    assert np.all(rel_errors(got, oracle.mpk(A, x, p)) <= (1e-12 if prec == "f64" else 1e-5))


def test_resident_block_vectors_of_two():
    A = mi.laplace3d(24)
    x = mi.random_vector(A.n, 99, 2)
    plan = plan_of(A, 6, prec="f64", nrhs=2, tune=RES)
    assert mpk.mpk_plan_info(plan)["resident"] == 1
    assert np.all(rel_errors(run_mpk(plan, x), oracle.mpk(A, x, 6)) <= 1e-12)


def test_rows_too_wide_fall_back():
    """Zipf-degree rows up to 500 wide: a stage cannot hold 32 such rows in
    FP64, so the plan keeps the work-list schedule."""
    A = mi.zipf_graph(20000, 77)
    plan = plan_of(A, 4, prec="f64", tune=RES)
    assert mpk.mpk_plan_info(plan)["resident"] == 0
    x = mi.random_vector(A.n, 3)
    assert np.all(rel_errors(run_mpk(plan, x), oracle.mpk(A, x, 4)) <= 1e-12)


def test_wide_dependency_span_falls_back():
    """Tiny tiles on a 3D grid: a tile's columns reach about a level (dozens
    of tiles) ahead, so (p-1) * span exceeds the grid and the plan keeps the
    work-list schedule."""
    A = mi.laplace3d(40)
    p = 8
    plan = plan_of(A, p, prec="f64", tile_rows=32, tune=RES)
    info = mpk.mpk_plan_info(plan)
    assert (p - 1) * info["dep_span"] >= 152 and info["resident"] == 0
    x = mi.random_vector(A.n, 4)
    assert np.all(rel_errors(run_mpk(plan, x), oracle.mpk(A, x, p)) <= 1e-12)


def test_resident_timeout_is_reported_and_plan_recovers():
    import time
    A = mi.laplace2d(200, 150)
    p = 4
    plan = plan_of(A, p, prec="f64", tile_rows=64, timeout_s=0.25, tune=RES)
    info = mpk.mpk_plan_info(plan)
    assert info["resident"] == 1
    x = mi.random_vector(A.n, 11)
    xd = torch.from_numpy(x).cuda()
    Y = torch.empty(p, A.n, dtype=torch.float64, device="cuda")
    mpk.mpk_plan_debug_drop_flag(plan, info["n_tiles"] // 2, 2)
    t0 = time.time()
    with pytest.raises(mpk.MpkError) as e:
        mpk.mpk_run(plan, xd, Y)
    assert e.value.code == mpk.MPK_ERR_TIMEOUT
    assert time.time() - t0 < 10.0
    mpk.mpk_run(plan, xd, Y)
    assert np.all(rel_errors(Y.cpu().numpy(), oracle.mpk(A, x, p)) <= 1e-12)


def _cheb_err(A, prec, p, M, tune, one=False):
    plan = plan_of(A, p, prec=prec, nrhs=2, tune=tune)
    assert mpk.mpk_plan_info(plan)["resident"] == (1 if tune & RES else 0)
    olo, ohi = oracle.gershgorin(A)
    c, r = (ohi + olo) / 2, (ohi - olo) / 2
    coef = oracle.cheb_coeffs_schroedinger(M, c, r, 50.0 / r)
    psi = mi.uniform(1234, A.n) + 1j * mi.uniform(4321, A.n)
    psi /= np.linalg.norm(psi)
    ref = oracle.cheb(A, coef, c, r, psi)
    dt = torch.float64 if prec == "f64" else torch.float32
    xd = torch.from_numpy(np.stack([psi.real, psi.imag], 1).copy()).to(dt).cuda()
    yd = torch.empty(A.n, 2, dtype=torch.float64, device="cuda")
    mpk.mpk_cheb(plan, coef, c, r, xd, yd, one_power_per_launch=one)
    y = yd.cpu().numpy()
    return np.max(np.abs(y[:, 0] + 1j * y[:, 1] - ref)) / np.max(np.abs(ref)), yd


@pytest.mark.parametrize("p,M", [(8, 64), (5, 17), (1, 6)])
def test_resident_cheb_f64(p, M):
    err, _ = _cheb_err(mi.anderson3d(12, W=16.5, seed=42), "f64", p, M, RES)
    assert err <= 1e-12


@pytest.mark.parametrize("prec", ["f32", "bf16val"])
def test_resident_cheb_reduced_precision(prec):
    A = mi.anderson3d(16, W=16.5, seed=42)
    err, y_res = _cheb_err(A, prec, 8, 64, RES)
    assert err <= 2e-5
    _, y_one = _cheb_err(A, prec, 8, 64, RES, one=True)
    assert torch.equal(y_res, y_one)   # same node arithmetic, one power per launch


def test_resident_full_size_160():
    """The 160^3 workload (p = 8) on the resident schedule, level order, as
    the benchmark runs it: FP64 <= 1e-12 and FP32 <= 1e-5 on every output."""
    A = mi.laplace3d(160)
    p = 8
    x = mi.random_vector(A.n, 1234)
    ref = oracle.mpk(A, x, p)
    for prec, tol in (("f64", 1e-12), ("f32", 1e-5)):
        plan = plan_of(A, p, prec=prec, tune=RES)
        assert mpk.mpk_plan_info(plan)["resident"] == 1
        perm = mpk.mpk_plan_perm(plan)[0].cpu().numpy()
        xin = x[perm] if prec == "f64" else x[perm].astype(np.float32)
        got = run_mpk(plan, xin, permuted=True)
        assert np.all(rel_errors(got, ref[:, perm]) <= tol)
        del plan
