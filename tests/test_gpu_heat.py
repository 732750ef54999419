"""GPU parity of the real Chebyshev propagation (the heat equation of Sec. 7,
mpk_cheb_real) and of the library's modified-Bessel coefficients, against
the FP64 oracle, relative to the input's magnitude (the v_k carry rounding
of that size, summed with sum|c_k| ~ 1 over M = 64 steps, while the result
is damped far below it): FP64 <= 1e-12, FP32 <= 2e-5; the
one-power-per-launch form bit for bit; both schedules."""
import numpy as np
import pytest
import scipy.special as sps
import torch

import mpk_inputs as mi
import oracle
import paper_2205_01598_gb300 as mpk
from gpu_helpers import plan_of

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("c,r,tau,M", [(6.0, 6.0, 50 / 6.0, 64), (2.0, 1.5, 3.0, 30), (0.5, 0.5, 0.1, 8),
                                       (12.0, 12.0, 400 / 12.0, 120), (1.0, 1.0, 0.0, 4)])
def test_heat_coefficients(c, r, tau, M):
    mpk.build()
    got = mpk.mpk_cheb_coeffs_heat(M, c, r, tau)
    k = np.arange(M + 1)
    want = np.where(k == 0, 1.0, 2.0) * (-1.0) ** k * np.exp(-tau * (c - r)) * sps.ive(k, tau * r)
    scale = max(1.0, np.abs(want).max())
    assert np.max(np.abs(got - want)) <= 1e-14 * scale
    if tau > 0:
        assert np.max(np.abs(got - oracle.cheb_coeffs_heat(M, c, r, tau))) <= 1e-14 * scale


def _heat(A, prec, p, M, tune=0, permuted=False, one=False, rtau=50.0):
    plan = plan_of(A, p, prec=prec, nrhs=1, tune=tune)
    olo, ohi = oracle.gershgorin(A)
    lo, hi = mpk.mpk_gershgorin(plan)
    if prec == "f64":   # same bounds up to the order of the row sums
        assert abs(lo - olo) <= 1e-14 * max(1.0, abs(olo)) and abs(hi - ohi) <= 1e-14 * max(1.0, abs(ohi))
    # -Delta of any order is positive semi-definite: its spectrum lies in
    # [0, hi], tighter than Gershgorin's lower bound for the wider stencils
    olo = max(olo, 0.0)
    c, r = (ohi + olo) / 2, (ohi - olo) / 2
    assert np.abs(oracle.cheb_coeffs_heat(M, c, r, rtau / r)).sum() <= 1.0 + 1e-12
    coef = oracle.cheb_coeffs_heat(M, c, r, rtau / r)
    x = mi.random_vector(A.n, 77)
    ref = oracle.cheb_real(A, coef, c, r, x)
    if permuted:
        perm = mpk.mpk_plan_perm(plan)[0].cpu().numpy()
        x, ref = x[perm], ref[perm]
    dt = torch.float64 if prec == "f64" else torch.float32
    xd = torch.from_numpy(np.ascontiguousarray(x)).to(dt).cuda()
    yd = torch.empty(A.n, dtype=torch.float64, device="cuda")
    mpk.mpk_cheb_real(plan, coef, c, r, xd, yd, permuted=permuted, one_power_per_launch=one)
    info = mpk.mpk_plan_info(plan)
    diff = np.max(np.abs(yd.cpu().numpy() - ref))
    # relative to the input: the propagator (norm <= 1) damps the result far
    # below the v_k, whose rounding (of the input's magnitude) it sums with
    # sum|c_k| ~ 1, so ||error|| <~ M eps ||x|| in either precision.  The
    # result-relative error is reported beside it (HEAT_ERRORS) and bounded
    # loosely in FP64.
    err_in, err_out = diff / np.max(np.abs(x)), diff / np.max(np.abs(ref))
    HEAT_ERRORS.append((A.n, prec, p, M, err_in, err_out))
    return err_in, yd, info, err_out


HEAT_ERRORS = []


@pytest.mark.parametrize("make", [lambda: mi.laplace3d(24), lambda: mi.star3d(18, 2), lambda: mi.laplace2d(70, 50)],
                         ids=["order2-24", "order4-18", "lap2d"])
@pytest.mark.parametrize("p,M", [(8, 64), (5, 17), (1, 6)])
def test_heat_f64_matches_oracle(make, p, M):
    err, _, _, err_out = _heat(make(), "f64", p, M)
    assert err <= 1e-12, (err, err_out)
    assert err_out <= 1e-10, (err, err_out)


def test_heat_permuted_io_and_resident():
    A = mi.star3d(20, 3)   # order-6 stencil
    err, _, _, err_out = _heat(A, "f64", 8, 64, permuted=True)
    assert err <= 1e-12 and err_out <= 1e-10, (err, err_out)
    err, _, info, err_out = _heat(A, "f64", 8, 64, tune=mpk.MPK_TUNE_RESIDENT)
    assert info["resident"] == 1 and err <= 1e-12 and err_out <= 1e-10, (err, err_out)


@pytest.mark.parametrize("prec", ["f32", "bf16val"])
def test_heat_reduced_precision(prec):
    A = mi.star3d(20, 2)
    err, y, _, err_out = _heat(A, prec, 8, 64)
    assert err <= 2e-5, (err, err_out)
    _, y1, _, _ = _heat(A, prec, 8, 64, one=True)
    assert torch.equal(y, y1)


def test_heat_rejects_complex_plan():
    A = mi.laplace3d(8)
    plan = plan_of(A, 4, prec="f64", nrhs=2)
    x = torch.zeros(A.n, 2, dtype=torch.float64, device="cuda")
    y = torch.zeros(A.n, 2, dtype=torch.float64, device="cuda")
    with pytest.raises(mpk.MpkError) as e:
        mpk.mpk_cheb_real(plan, np.ones(5), 0.0, 1.0, x, y)
    assert e.value.code == mpk.MPK_ERR_INVALID


def test_heat_order4_160_full_size():
    """The order-4 160^3 heat workload (nnz = 52,787,200, Tab. 3), degree 64
    in sweeps of 8, FP64, level order as the benchmark runs it."""
    A = mi.star3d(160, 2)
    assert A.nnz == 52_787_200
    plan = plan_of(A, 8, prec="f64", nrhs=1)
    lo, hi = mpk.mpk_gershgorin(plan)
    lo = max(lo, 0.0)
    c, r = (hi + lo) / 2, (hi - lo) / 2
    coef = mpk.mpk_cheb_coeffs_heat(64, c, r, 50.0 / r)
    x = mi.random_vector(A.n, 1234)
    ref = oracle.cheb_real(A, coef, c, r, x)
    perm = mpk.mpk_plan_perm(plan)[0].cpu().numpy()
    xd = torch.from_numpy(np.ascontiguousarray(x[perm])).cuda()
    yd = torch.empty(A.n, dtype=torch.float64, device="cuda")
    mpk.mpk_cheb_real(plan, coef, c, r, xd, yd, permuted=True)
    diff = np.max(np.abs(yd.cpu().numpy() - ref[perm]))
    err_in, err_out = diff / np.max(np.abs(x)), diff / np.max(np.abs(ref))
    assert err_in <= 1e-12 and err_out <= 1e-10, (err_in, err_out)


def test_heat_errors_report():
    """Both errors of every heat case above, input-relative (the bar) and
    result-relative, printed (pytest -s)."""
    lines = ["n prec p M err/|x| err/|y|"] + [f"{n} {pr} {p} {M} {a:.2e} {b:.2e}" for n, pr, p, M, a, b in HEAT_ERRORS]
    print("\n".join(lines))
    assert all(np.isfinite(a) and np.isfinite(b) for _, _, _, _, a, b in HEAT_ERRORS)
