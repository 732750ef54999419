"""GPU parity of mpk_run_host: the MPK with x and Y in host memory, the
copies overlapped with the reordering of each power.  The device work is
that of mpk_run, so the results equal mpk_run's bit for bit, and the
oracle's within the usual bars; pinned and pageable host memory, both
orders of the vectors, the asynchronous form, and repeated calls (the
staging buffers alternate between powers and calls)."""
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
