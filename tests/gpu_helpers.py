"""Shared helpers of the GPU parity tests (the CUDA path through the C ABI vs the oracle)."""
import numpy as np
import torch

import oracle
import paper_2205_01598_gb300 as mpk


def ensure_built():
    mpk.build()
    mpk.load()


def plan_of(A, p, **kw):
    ensure_built()
    rp, cl, va = mpk.csr_to_device(A)
    kw.setdefault("assume_symmetric", True)
    return mpk.mpk_plan(rp, cl, va, p, **kw)


def rel_errors(got, ref):
    """Per-power relative infinity-norm errors ||got_k - ref_k|| / ||ref_k||."""
    out = []
    for k in range(ref.shape[0]):
        den = np.max(np.abs(ref[k]))
        out.append(np.max(np.abs(got[k] - ref[k])) / (den if den > 0 else 1e-300))
    return np.array(out)


def run_mpk(plan, x, permuted=False, baseline=False):
    """x: host array (n,) or (n, nrhs) in the precision of the plan."""
    dt = plan.vec_dtype
    xd = torch.from_numpy(np.ascontiguousarray(x)).to(dtype=dt, device="cuda")
    Y = torch.full((plan.p,) + tuple(xd.shape), float("nan"), dtype=dt, device="cuda")
    (mpk.mpk_baseline_run if baseline else mpk.mpk_run)(plan, xd, Y, permuted=permuted)
    return Y.cpu().numpy().astype(np.float64)


def oracle_levels(A, root=0, symmetrize=False):
    level, L = oracle.bfs_levels(A, root=root, symmetrize=symmetrize)
    perm, iperm, lp = oracle.level_perm(level, L)
    return level, L, perm, iperm, lp
