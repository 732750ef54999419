"""Batched level-blocked MPK: several plans of different sizes, block widths
and powers in one persistent launch (mpk_batch_run), also captured in a CUDA
graph and replayed (mpk_batch_graph_capture / _launch).  Each result must
equal the oracle (FP64 <= 1e-12, FP32 <= 1e-5 per power) and, bit for bit,
the result of running the same plan on its own."""
import numpy as np
import pytest
import torch

import mpk_inputs as mi
import oracle
import paper_2205_01598_gb300 as mpk
from gpu_helpers import plan_of, rel_errors

pytestmark = pytest.mark.gpu

CASES = [  # matrix, nrhs, p
    (lambda: mi.laplace3d(22), 1, 8),
    (lambda: mi.zipf_graph(6000, 1001), 3, 4),
    (lambda: mi.anderson3d(12, seed=42), 2, 10),
    (lambda: mi.zipf_graph(20000, 1002), 16, 2),
    (lambda: mi.random_sparse(900, 0.01, 4), 5, 6),
    (lambda: mi.laplace2d(64), 8, 3),
]


def _setup(prec):
    mats, plans, xs, Ys, xh = [], [], [], [], []
    dt = torch.float64 if prec == "f64" else torch.float32
    for i, (make, nrhs, p) in enumerate(CASES):
        A = make()
        plan = plan_of(A, p, prec=prec, nrhs=nrhs, tile_rows=128)
        perm = mpk.mpk_plan_perm(plan)[0].cpu().numpy()
        x = mi.random_vector(A.n, 500 + i, nrhs)
        mats.append((A, perm, p))
        plans.append(plan)
        xh.append(x)
        xs.append(torch.from_numpy(np.ascontiguousarray(x[perm])).to(dt).cuda())
        Ys.append(torch.full((p,) + tuple(xs[-1].shape), float("nan"), dtype=dt, device="cuda"))
    return mats, plans, xs, Ys, xh


def _check(mats, Ys, xh, tol):
    for (A, perm, p), Y, x in zip(mats, Ys, xh):
        ref = oracle.mpk(A, x, p)
        got = Y.cpu().numpy().astype(np.float64)
        assert np.all(rel_errors(got, ref[:, perm]) <= tol)


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 1e-5)])
def test_batched_run_matches_oracle_and_single_runs(prec, tol):
    mats, plans, xs, Ys, xh = _setup(prec)
    batch = mpk.mpk_batch_create(plans)
    info = mpk.mpk_batch_info(batch)
    assert info["n_items"] == sum(mpk.mpk_plan_info(pl)["n_tiles"] * p for pl, (_, _, p) in zip(plans, mats))
    mpk.mpk_batch_run(batch, xs, Ys)
    _check(mats, Ys, xh, tol)
    for plan, x, Y in zip(plans, xs, Ys):      # each plan alone: bit-identical
        Y1 = torch.empty_like(Y)
        mpk.mpk_run(plan, x, Y1, permuted=True)
        assert torch.equal(Y1, Y)
    mpk.mpk_batch_run(batch, xs, Ys)           # and again (epochs advance)
    _check(mats, Ys, xh, tol)


def test_batched_cuda_graph_replay():
    mats, plans, xs, Ys, xh = _setup("f32")
    batch = mpk.mpk_batch_create(plans)
    mpk.mpk_batch_graph_capture(batch, xs, Ys)
    for rep in range(3):
        for Y in Ys:
            Y.fill_(float("nan"))
        mpk.mpk_batch_graph_launch(batch)
        _check(mats, Ys, xh, 1e-5)
    # a single plan still runs on its own between graph replays
    Y0 = torch.empty_like(Ys[0])
    mpk.mpk_run(plans[0], xs[0], Y0, permuted=True)
    assert torch.equal(Y0, Ys[0])


def test_batch_rejects_mixed_precision():
    A = mi.laplace2d(16)
    p64 = plan_of(A, 2, prec="f64")
    p32 = plan_of(A, 2, prec="f32")
    with pytest.raises(mpk.MpkError) as e:
        mpk.mpk_batch_create([p64, p32])
    assert e.value.code == mpk.MPK_ERR_UNSUPPORTED
