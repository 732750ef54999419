"""GPU parity of the recursion of Sec. 4.4 (mpk_opts.recursion = s_m): the
permutation, the finest levels and the level groups of the GPU plan equal
the oracle's recursive construction bit for bit; the MPK with those groups
matches the FP64 oracle; and the issue order that places each item by its
latest dependency (the diamond around a refined subgraph) holds every item
once with every dependency earlier."""
import numpy as np
import pytest

import mpk_inputs as mi
import oracle
import paper_2205_01598_gb300 as mpk
from gpu_helpers import plan_of, rel_errors, run_mpk

pytestmark = pytest.mark.gpu

# (matrix, p, cache fraction of the matrix bytes, s_m): the cache is chosen
# so that only part of the level groups are bulky (one level over Eq. 5)
CASES = {
    "laplace3d-14": (lambda: mi.laplace3d(14), 8, 0.5, 1),
    "laplace3d-14-s3": (lambda: mi.laplace3d(14), 4, 0.12, 3),
    "laplace3d-40": (lambda: mi.laplace3d(40), 8, 0.15, 2),
    "zipf-4000": (lambda: mi.zipf_graph(4000, 1003), 6, 2.0, 2),
    "zipf-30000": (lambda: mi.zipf_graph(30000, 1005), 4, 0.8, 3),
    "box27-10": (lambda: mi.box27(10), 8, 0.4, 2),
    "rgg2d-3000": (lambda: mi.random_geometric_graph(3000, 2, 10.0, 5), 5, 0.05, 2),
}


def _plan_and_oracle(name, prec="f64", **kw):
    make, p, frac, s_max = CASES[name]
    A = make()
    bpe = 12.0 if prec == "f64" else 8.0
    w = np.diff(A.rowptr).astype(np.float64) * bpe
    C = frac * w.sum()
    plan = plan_of(A, p, prec=prec, cache_bytes=C, safety_f=0.5, recursion=s_max, **kw)
    ref = oracle.recursive_levels(A, w, p, 0.5, C, s_max)
    return A, p, plan, ref


@pytest.mark.parametrize("name", list(CASES))
def test_recursive_levels_match_oracle(name):
    A, p, plan, (operm, olp, ogp, ogs, ostages) = _plan_and_oracle(name)
    info = mpk.mpk_plan_info(plan)
    perm, lp, gp, level = (t.cpu().numpy() for t in mpk.mpk_plan_perm(plan))
    assert ostages >= 1 and info["rec_stages"] == ostages
    assert np.array_equal(perm, operm)
    assert np.array_equal(lp, olp)
    assert np.array_equal(gp, ogp)
    # the per-vertex levels stay those of Eq. 3 on the whole graph
    assert np.array_equal(level, oracle.bfs_levels(A)[0])


@pytest.mark.parametrize("name", ["laplace3d-40", "zipf-30000", "box27-10", "rgg2d-3000"])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_mpk_with_recursion_matches_oracle(name, prec):
    A, p, plan, _ = _plan_and_oracle(name, prec=prec, tile_rows=64)
    x = mi.random_vector(A.n, 31)
    ref = oracle.mpk(A, x, p)
    got = run_mpk(plan, x if prec == "f64" else x.astype(np.float32))
    err = rel_errors(got, ref)
    assert np.all(err <= (1e-12 if prec == "f64" else 1e-5)), err
    assert np.array_equal(got, run_mpk(plan, x if prec == "f64" else x.astype(np.float32), baseline=True))


@pytest.mark.parametrize("name", ["laplace3d-40", "zipf-30000", "rgg2d-3000"])
def test_diamond_order_is_complete_and_dependency_ordered(name):
    A, p, plan, _ = _plan_and_oracle(name, tile_rows=32)
    info = mpk.mpk_plan_info(plan)
    work, lo, hi = mpk.mpk_plan_schedule(plan)
    T = info["n_tiles"]
    t, k = work >> 8, work & 255
    assert work.shape == (T * p,)
    assert np.array_equal(np.sort(t * 256 + k),
                          np.sort(np.repeat(np.arange(T), p) * 256 + np.tile(np.arange(1, p + 1), T)))
    pos = np.empty((T, p + 1), dtype=np.int64)
    pos[t, k] = np.arange(T * p)
    for j in range(T * p):
        if k[j] > 1:
            assert pos[lo[t[j]]:hi[t[j]] + 1, k[j] - 1].max() < j


def test_chebyshev_with_recursion():
    A = mi.anderson3d(14, W=16.5, seed=42)
    w = np.diff(A.rowptr).astype(np.float64) * 12.0
    plan = plan_of(A, 8, prec="f64", nrhs=2, cache_bytes=0.3 * w.sum(), recursion=2, tile_rows=64)
    assert mpk.mpk_plan_info(plan)["rec_stages"] >= 1
    lo, hi = oracle.gershgorin(A)
    c, r = (hi + lo) / 2, (hi - lo) / 2
    coef = oracle.cheb_coeffs_schroedinger(20, c, r, 1.5)
    psi = mi.uniform(3, A.n) + 1j * mi.uniform(4, A.n)
    ref = oracle.cheb(A, coef, c, r, psi)
    import torch
    xd = torch.from_numpy(np.stack([psi.real, psi.imag], 1).copy()).cuda()
    yd = torch.empty(A.n, 2, dtype=torch.float64, device="cuda")
    mpk.mpk_cheb(plan, coef, c, r, xd, yd)
    y = yd.cpu().numpy()
    assert np.max(np.abs(y[:, 0] + 1j * y[:, 1] - ref)) / np.max(np.abs(ref)) <= 1e-12
