"""The MPK in sweeps of q < p powers inside one launch (mpk_opts.sweep):
results equal the FP64 oracle per power and, bit for bit, the back-to-back
SpMV comparator of the same plan (the row arithmetic does not depend on the
issue order); the batch runs members planned with different work-item
sizes, f and sweep lengths in one launch, each equal to its own run."""
import numpy as np
import pytest
import torch

import mpk_inputs as mi
import oracle
import paper_2205_01598_gb300 as mpk
from gpu_helpers import plan_of, rel_errors, run_mpk

pytestmark = pytest.mark.gpu

MATS = {
    "laplace3d-40": lambda: mi.laplace3d(40),
    "zipf-20000": lambda: mi.zipf_graph(20000, 1007),
    "rgg3d-8000": lambda: mi.random_geometric_graph(8000, 3, 14.0, 9),
}


@pytest.mark.parametrize("name", list(MATS))
@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 1e-5)])
@pytest.mark.parametrize("p,q", [(8, 1), (8, 4), (9, 2)])
def test_sweeps_match_oracle_and_comparator(name, prec, tol, p, q):
    A = MATS[name]()
    plan = plan_of(A, p, prec=prec, sweep=q, tile_rows=128)
    x = mi.random_vector(A.n, 77)
    xin = x if prec == "f64" else x.astype(np.float32)
    got = run_mpk(plan, xin)
    assert np.all(rel_errors(got, oracle.mpk(A, x, p)) <= tol)
    assert np.array_equal(got, run_mpk(plan, xin, baseline=True))


def test_sweep_with_recursion():
    A = mi.zipf_graph(30000, 1005)
    w = np.diff(A.rowptr).astype(np.float64) * 12.0
    plan = plan_of(A, 8, prec="f64", sweep=3, cache_bytes=0.8 * w.sum(), safety_f=0.5, recursion=3,
                   tile_rows=64)
    assert mpk.mpk_plan_info(plan)["rec_stages"] >= 1
    x = mi.random_vector(A.n, 5)
    assert np.all(rel_errors(run_mpk(plan, x), oracle.mpk(A, x, 8)) <= 1e-12)


def test_chebyshev_on_a_swept_plan():
    """The Chebyshev launches share the plan's issue order: sweeps inside a
    launch leave the propagation unchanged, bit for bit."""
    A = mi.anderson3d(12, W=16.5, seed=42)
    lo, hi = oracle.gershgorin(A)
    c, r = (hi + lo) / 2, (hi - lo) / 2
    coef = oracle.cheb_coeffs_schroedinger(24, c, r, 2.0)
    psi = mi.uniform(3, A.n) + 1j * mi.uniform(4, A.n)
    xd = torch.from_numpy(np.stack([psi.real, psi.imag], 1).copy()).cuda()
    ys = []
    for sweep in (0, 3, 1):
        plan = plan_of(A, 8, prec="f64", nrhs=2, sweep=sweep, tile_rows=64)
        y = torch.empty(A.n, 2, dtype=torch.float64, device="cuda")
        mpk.mpk_cheb(plan, coef, c, r, xd, y)
        ys.append(y)
    assert torch.equal(ys[0], ys[1]) and torch.equal(ys[0], ys[2])
    ref = oracle.cheb(A, coef, c, r, psi)
    y = ys[0].cpu().numpy()
    assert np.max(np.abs(y[:, 0] + 1j * y[:, 1] - ref)) / np.max(np.abs(ref)) <= 1e-12


def test_batch_members_with_their_own_options():
    """Per-member options in one batch launch: work-item rows, f and sweep
    length differ between members; each member equals the oracle and its own
    plan run alone."""
    members = [  # matrix, nrhs, p, options
        (lambda: mi.zipf_graph(20000, 1011), 3, 6, {"tile_rows": 64, "safety_f": 0.25, "sweep": 1}),
        (lambda: mi.zipf_graph(9000, 1012), 1, 10, {"tile_rows": 256, "safety_f": 0.5, "sweep": 5}),
        (lambda: mi.laplace3d(24), 2, 8, {"tile_rows": 512, "safety_f": 0.5}),
        (lambda: mi.zipf_graph(30000, 1013), 16, 2, {"tile_rows": 128, "safety_f": 0.25, "sweep": 1}),
        (lambda: mi.laplace2d(80), 4, 7, {"tile_rows": 1024, "safety_f": 0.25, "sweep": 4}),
    ]
    mats, plans, xs, Ys, xh = [], [], [], [], []
    for i, (make, nrhs, p, opts) in enumerate(members):
        A = make()
        plan = plan_of(A, p, prec="f32", nrhs=nrhs, **opts)
        perm = mpk.mpk_plan_perm(plan)[0].cpu().numpy()
        x = mi.random_vector(A.n, 900 + i, nrhs)
        mats.append((A, perm, p))
        plans.append(plan)
        xh.append(x)
        xs.append(torch.from_numpy(np.ascontiguousarray(x[perm])).float().cuda())
        Ys.append(torch.full((p,) + tuple(xs[-1].shape), float("nan"), dtype=torch.float32, device="cuda"))
    batch = mpk.mpk_batch_create(plans)
    mpk.mpk_batch_graph_capture(batch, xs, Ys)
    mpk.mpk_batch_graph_launch(batch)
    for (A, perm, p), plan, x, xd, Y in zip(mats, plans, xh, xs, Ys):
        ref = oracle.mpk(A, x, p)
        assert np.all(rel_errors(Y.cpu().numpy().astype(np.float64), ref[:, perm]) <= 1e-5)
        Y1 = torch.empty_like(Y)
        mpk.mpk_run(plan, xd, Y1, permuted=True)
        assert torch.equal(Y1, Y)
