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


def _zipf_member(spec):
    """Matrix of one batch member (module level, for the spawned pool)."""
    m, seed, n = spec
    return m, mi.zipf_graph(n, seed)


def batch_specs(count=64, n_lo=20_000, n_hi=2_000_000):
    """Members of the batched workload: (m, seed, N, nrhs, p) with N ~ U[n_lo, n_hi],
    nrhs ~ U{1..16} and p ~ U{2..10} from SplitMix64 seed 1000 + m."""
    specs = []
    for m in range(count):
        z = mi.splitmix64(1000 + m, 3)
        n = n_lo + int(z[0] % np.uint64(n_hi - n_lo + 1))
        specs.append((m, 1000 + m, n, 1 + int(z[1] % np.uint64(16)), 2 + int(z[2] % np.uint64(9))))
    return specs


def spmv_ref(A, v):
    """A v in FP64 for v (n,) or (n, nrhs): the multicore comparator (bit-identical
    to the oracle) one column at a time, else the oracle itself."""
    cols = v.reshape(A.n, -1)
    out = np.empty_like(cols)
    for q in range(cols.shape[1]):
        c = np.ascontiguousarray(cols[:, q])
        try:
            out[:, q] = oracle.omp_pxspmv(A, c, 1)[0][0]
        except RuntimeError:
            out[:, q] = oracle.mpk(A, c, 1)[0]
    return out.reshape(v.shape)


def check_powers(A, x, Y, tol):
    """Every power of Y (p, n[, nrhs], original numbering) against an FP64 SpMV
    of the previous one (the first against x): Y[k] = A Y[k-1] at any size."""
    prev = x.astype(np.float64)
    for k in range(Y.shape[0]):
        ref = spmv_ref(A, prev)
        got = Y[k].astype(np.float64)
        assert np.max(np.abs(got - ref)) <= tol * max(np.max(np.abs(ref)), 1e-300), (k, A.n)
        prev = got


def test_batched_full_size_zipf64():
    """The batched workload at full size in the benchmark's launch configuration:
    64 Zipf-degree matrices, N ~ U[20k, 2M], nrhs ~ U{1..16}, p ~ U{2..10}, FP32,
    one persistent launch replayed from a CUDA graph.  The oracle cannot run all
    790M entries x powers in seconds, so every power of every member is checked
    by the property that holds at any size, against FP64 SpMVs."""
    import multiprocessing as mp
    import os
    specs = batch_specs()
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        mats = dict(pool.map(_zipf_member, [(m, seed, n) for m, seed, n, _, _ in specs]))
    plans, xs, Ys, perms, xh = [], [], [], [], []
    for m, seed, n, nrhs, p in specs:
        A = mats[m]
        plan = plan_of(A, p, prec="f32", nrhs=nrhs)
        perm = mpk.mpk_plan_perm(plan)[0].cpu().numpy()
        x = mi.random_vector(A.n, 3000 + m, nrhs).astype(np.float32)
        plans.append(plan)
        perms.append(perm)
        xh.append(x)
        xs.append(torch.from_numpy(np.ascontiguousarray(x[perm])).cuda())
        Ys.append(torch.full((p,) + x.shape, float("nan"), dtype=torch.float32, device="cuda"))
    batch = mpk.mpk_batch_create(plans)
    mpk.mpk_batch_graph_capture(batch, xs, Ys)
    mpk.mpk_batch_graph_launch(batch)
    torch.cuda.synchronize()
    for (m, seed, n, nrhs, p), perm, x, Y in zip(specs, perms, xh, Ys):
        Yl = Y.cpu().numpy()
        Yo = np.empty_like(Yl)
        Yo[:, perm] = Yl
        check_powers(mats[m], x, Yo, 1e-5)
