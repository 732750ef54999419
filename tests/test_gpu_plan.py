"""GPU plan parity: levels (Eq. 3), the level renumbering, level_ptr and the
Eq. 5 level groups from mpk_plan must equal the oracle's bit for bit."""
import numpy as np
import pytest

import mpk_inputs as mi
import oracle
import paper_2205_01598_gb300 as mpk
from gpu_helpers import oracle_levels, plan_of

pytestmark = pytest.mark.gpu


def _chain(n):
    return mi.laplace1d(n)


CASES = [
    ("2d7pt-8x8", lambda: mi.stencil2d_7pt(8), {}),
    ("laplace2d-64", lambda: mi.laplace2d(64), {}),
    ("laplace3d-24", lambda: mi.laplace3d(24), {}),
    ("anderson-12-pbc", lambda: mi.anderson3d(12), {}),
    ("box27-10", lambda: mi.box27(10), {}),
    ("chain-3000", lambda: _chain(3000), {}),                       # 3000 levels: two radix passes
    ("randsym-700", lambda: mi.random_sparse(700, 1.5 / 700, 5), {}),  # many components
    ("diag-300", lambda: mi.diagonal(np.arange(1.0, 301.0)), {}),   # 300 singleton levels
    ("root-17", lambda: mi.laplace2d(40, 33), {"root": 17}),
    ("nonsym", lambda: mi.random_sparse(400, 0.01, 8, symmetric=False), {"assume_symmetric": False}),
]


@pytest.mark.parametrize("name,make,kw", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_levels_perm_groups_bit_exact(name, make, kw, prec):
    A = make()
    p = 4
    kw = dict(kw)
    root = kw.get("root", 0)
    sym = kw.get("assume_symmetric", True)
    plan = plan_of(A, p, prec=prec, **kw)
    info = mpk.mpk_plan_info(plan)
    perm, lp, gp, lev = (t.cpu().numpy() for t in mpk.mpk_plan_perm(plan))
    level, L, operm, _, olp = oracle_levels(A, root=root, symmetrize=not sym)
    assert info["n_levels"] == L
    assert np.array_equal(lev, level)
    assert np.array_equal(perm, operm)
    assert np.array_equal(lp, olp)
    # Eq. 5 groups with the plan's own C, f and bytes per stored entry
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    lnnz = np.bincount(level[rows], minlength=L).astype(np.float64)
    bpe = 8 + 4 if prec == "f64" else 4 + 4
    ogp = oracle.level_groups(lnnz * bpe, p, 0.5, info["cache_bytes"])
    assert np.array_equal(gp, ogp)


def test_small_cache_gives_many_groups_matching_oracle():
    A = mi.laplace3d(30)
    p = 6
    C = 200_000.0
    plan = plan_of(A, p, cache_bytes=C, safety_f=0.7)
    info = mpk.mpk_plan_info(plan)
    _, _, gp, lev = (t.cpu().numpy() for t in mpk.mpk_plan_perm(plan))
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    lnnz = np.bincount(lev[rows], minlength=info["n_levels"]).astype(np.float64)
    ogp = oracle.level_groups(lnnz * 12, p, 0.7, C)
    assert np.array_equal(gp, ogp)
    assert info["n_groups"] > 20


def test_invalid_inputs_are_rejected():
    import torch
    A = mi.laplace2d(8)
    rp, cl, va = mpk.csr_to_device(A)
    with pytest.raises(mpk.MpkError) as e:
        mpk.mpk_plan(rp, cl, va, 0)
    assert e.value.code == mpk.MPK_ERR_INVALID
    bad = cl.clone()
    bad[5] = A.n + 3                          # column out of range: found on the device
    with pytest.raises(mpk.MpkError) as e:
        mpk.mpk_plan(rp, bad, va, 2)
    assert e.value.code == mpk.MPK_ERR_INVALID
    rbad = rp.clone()
    rbad[3] = rbad[4] + 1                     # row pointer not monotone
    with pytest.raises(mpk.MpkError) as e:
        mpk.mpk_plan(rbad, cl, va, 2)
    assert e.value.code == mpk.MPK_ERR_INVALID
    with pytest.raises(mpk.MpkError):
        mpk.mpk_plan(rp, cl, va, 2, nrhs=0)
    torch.cuda.synchronize()
