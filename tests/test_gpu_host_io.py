"""GPU parity of the host-buffer entry points (the device work between two
copies, so the results equal the device forms' bit for bit):
- mpk_run_host: the MPK, the copies overlapped with the reordering of each
  power; also against the oracle within the usual bars, with pinned and
  pageable memory, both vector orders, the asynchronous form and repeated
  calls (the staging blocks alternate between powers and calls);
- mpk_cheb_host / mpk_cheb_real_host: the Chebyshev propagations."""
import numpy as np
import pytest
import torch

import mpk_inputs as mi
import oracle
import paper_2205_01598_gb300 as mpk
from gpu_helpers import plan_of, rel_errors

pytestmark = pytest.mark.gpu
TOL = {"f64": 1e-12, "f32": 1e-5, "bf16val": 1e-5}


def _host(a, dt, pinned):
    t = torch.from_numpy(np.ascontiguousarray(a)).to(dt)
    return t.pin_memory() if pinned else t


@pytest.mark.parametrize("prec", ["f64", "f32", "bf16val"])
@pytest.mark.parametrize("nrhs,p", [(1, 8), (1, 1), (2, 5), (4, 3)])
@pytest.mark.parametrize("permuted", [False, True])
def test_host_io_equals_device_run(prec, nrhs, p, permuted):
    A = mi.anderson3d(12, seed=3) if prec == "bf16val" else mi.laplace3d(22)
    plan = plan_of(A, p, prec=prec, nrhs=nrhs)
    dt = plan.vec_dtype
    x = mi.random_vector(A.n, 31, nrhs) if nrhs > 1 else mi.random_vector(A.n, 31)
    shape = (A.n, nrhs) if nrhs > 1 else (A.n,)
    xd = torch.from_numpy(np.ascontiguousarray(x)).to(dt).cuda()
    Yd = torch.empty((p,) + shape, dtype=dt, device="cuda")
    mpk.mpk_run(plan, xd, Yd, permuted=permuted)
    xh = _host(x, dt, True)
    Yh = torch.full((p,) + shape, float("nan"), dtype=dt).pin_memory()
    mpk.mpk_run_host(plan, xh, Yh, permuted=permuted)
    assert torch.equal(Yh, Yd.cpu())
    if not permuted:
        ref = oracle.mpk(A, xh.double().numpy(), p)
        assert np.all(rel_errors(Yh.double().numpy(), ref) <= TOL[prec])


def test_pageable_async_and_repeated_calls():
    A = mi.laplace2d(150, 90)
    p = 6
    plan = plan_of(A, p, prec="f64")
    x = mi.random_vector(A.n, 8)
    ref = oracle.mpk(A, x, p)
    xh = torch.from_numpy(x)                        # pageable
    Yh = torch.empty(p, A.n, dtype=torch.float64)   # pageable
    mpk.mpk_run_host(plan, xh, Yh)
    assert np.all(rel_errors(Yh.numpy(), ref) <= 1e-12)
    first = Yh.clone()
    Yp = torch.empty(p, A.n, dtype=torch.float64).pin_memory()
    for _ in range(3):   # asynchronous: the plan's stream covers the copies
        Yp.fill_(float("nan"))
        mpk.mpk_run_host(plan, xh.pin_memory(), Yp, asynchronous=True)
        torch.cuda.current_stream().synchronize()
        assert torch.equal(Yp, first)
    Yd = torch.empty(p, A.n, dtype=torch.float64, device="cuda")   # device runs in between keep working
    mpk.mpk_run(plan, xh.cuda(), Yd)
    assert torch.equal(Yd.cpu(), first)


def test_unaligned_vectors_permute_with_narrow_words():
    """Vectors at an offset of one element: the reordering falls back to
    4-byte words and stays exact."""
    A = mi.laplace3d(14)
    plan = plan_of(A, 3, prec="f32")
    x = mi.random_vector(A.n, 4).astype(np.float32)
    xbuf = torch.zeros(A.n + 1, dtype=torch.float32, device="cuda")
    xbuf[1:] = torch.from_numpy(x).cuda()
    ybuf = torch.zeros(3 * A.n + 1, dtype=torch.float32, device="cuda")
    Y = ybuf[1:].view(3, A.n)
    mpk.mpk_run(plan, xbuf[1:], Y)
    ref = oracle.mpk(A, x.astype(np.float64), 3)
    assert np.all(rel_errors(Y.cpu().double().numpy(), ref) <= 1e-5)


@pytest.mark.parametrize("prec", ["f64", "bf16val"])
@pytest.mark.parametrize("permuted", [False, True])
def test_cheb_host_equals_device(prec, permuted):
    """mpk_cheb_host / mpk_cheb_real_host: the device propagation between a
    host-to-device and a device-to-host copy, bit-identical to the device form."""
    A = mi.anderson3d(10, seed=8)
    for G in (2, 1):
        plan = plan_of(A, 4, prec=prec, nrhs=G)
        lo, hi = mpk.mpk_gershgorin(plan)
        c, r = (hi + lo) / 2, (hi - lo) / 2
        dt = plan.vec_dtype
        shape = (A.n, 2) if G == 2 else (A.n,)
        x = torch.from_numpy(mi.uniform(5, A.n * G).reshape(shape)).to(dt)
        yd = torch.empty(shape, dtype=torch.float64, device="cuda")
        yh = torch.full(shape, float("nan"), dtype=torch.float64).pin_memory()
        if G == 2:
            coef = mpk.mpk_cheb_coeffs_schroedinger(21, c, r, 3.0 / r)
            mpk.mpk_cheb(plan, coef, c, r, x.cuda(), yd, permuted=permuted)
            mpk.mpk_cheb_host(plan, coef, c, r, x.pin_memory(), yh, permuted=permuted)
        else:
            coef = mpk.mpk_cheb_coeffs_heat(21, c, r, 3.0 / r)
            mpk.mpk_cheb_real(plan, coef, c, r, x.cuda(), yd, permuted=permuted)
            mpk.mpk_cheb_real_host(plan, coef, c, r, x, yh, permuted=permuted)   # pageable input
        assert torch.equal(yh, yd.cpu())
