"""The wavefront's schedule (mpk_plan_schedule) against the oracle's view of
the matrix: every tile's dependency range covers the tiles of all columns
of its rows and every tile that reads it (the ring of the Chebyshev node
relies on the second), the issue order holds every (tile, power) item once,
and every dependency of an item comes before it -- the property the
in-order dealing of the persistent launch needs to be free of deadlock."""
import numpy as np
import pytest

import mpk_inputs as mi
import oracle
import paper_2205_01598_gb300 as mpk
from gpu_helpers import plan_of

pytestmark = pytest.mark.gpu

CASES = {
    "laplace3d-30": (lambda: mi.laplace3d(30), {}),
    "laplace3d-30-tiny-tiles": (lambda: mi.laplace3d(30), {"tile_rows": 32, "cache_bytes": 200_000.0}),
    "anderson-torus-16": (lambda: mi.anderson3d(16, seed=42), {"tile_rows": 64}),
    "zipf-8000": (lambda: mi.zipf_graph(8000, 7), {"tile_rows": 128}),
    "rgg2d-6000": (lambda: mi.random_geometric_graph(6000, 2, 10.0, 3), {"tile_rows": 64}),
    "box27-12": (lambda: mi.box27(12), {"tile_rows": 96}),
    "diag-500": (lambda: mi.diagonal(np.arange(1.0, 501.0)), {}),
}


def _tiles(level_ptr, group_ptr, n, tile_rows):
    """First row of every tile: tiles of tile_rows rows inside each level group."""
    starts = []
    for g in range(len(group_ptr) - 1):
        r0, r1 = level_ptr[group_ptr[g]], level_ptr[group_ptr[g + 1]]
        starts += list(range(r0, r1, tile_rows))
    return np.array(starts + [n])


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("p", [1, 4, 8])
def test_schedule_is_complete_and_dependency_ordered(name, p):
    make, kw = CASES[name]
    A = make()
    plan = plan_of(A, p, prec="f64", **kw)
    info = mpk.mpk_plan_info(plan)
    perm, lp, gp, _ = (t.cpu().numpy() for t in mpk.mpk_plan_perm(plan))
    work, lo, hi = mpk.mpk_plan_schedule(plan)
    T = info["n_tiles"]
    starts = _tiles(lp, gp, A.n, info["tile_rows"])
    assert len(starts) == T + 1
    tile_of = np.repeat(np.arange(T), np.diff(starts))

    # dependency ranges cover the columns of each tile's rows, and every reader
    level, L = oracle.bfs_levels(A)
    operm, oiperm, _ = oracle.level_perm(level, L)
    assert np.array_equal(operm, perm)
    Ap = oracle.permute_csr(A, operm, oiperm)
    rows = np.repeat(np.arange(A.n), np.diff(Ap.rowptr))
    tr, tc = tile_of[rows], tile_of[Ap.col]
    assert np.all(lo <= np.arange(T)) and np.all(np.arange(T) <= hi)
    assert np.all(lo[tr] <= tc) and np.all(tc <= hi[tr])      # what a tile reads
    assert np.all(lo[tc] <= tr) and np.all(tr <= hi[tc])      # who reads a tile

    # every item once, every dependency earlier
    assert work.shape == (T * p,)
    t, k = work >> 8, work & 255
    assert np.array_equal(np.sort(t * 256 + k), np.sort(np.repeat(np.arange(T), p) * 256 + np.tile(np.arange(1, p + 1), T)))
    pos = np.empty((T, p + 1), dtype=np.int64)
    pos[t, k] = np.arange(T * p)
    for j in range(T * p):
        if k[j] > 1:
            assert pos[lo[t[j]]:hi[t[j]] + 1, k[j] - 1].max() < j


@pytest.mark.parametrize("name", ["laplace3d-30", "zipf-8000", "box27-12"])
@pytest.mark.parametrize("p,q", [(8, 1), (8, 3), (10, 5), (7, 4)])
def test_sweeps_in_one_launch_are_ordered_by_sweep(name, p, q):
    """mpk_opts.sweep = q: every item of sweep s (powers s*q+1 .. (s+1)*q)
    is issued after every item of sweep s-1, each dependency still earlier,
    and the level groups are those of Eq. 5 for q powers (a plan for p = q
    has the same groups)."""
    make, kw = CASES[name]
    A = make()
    plan = plan_of(A, p, prec="f64", sweep=q, **kw)
    info = mpk.mpk_plan_info(plan)
    assert info["sweep"] == q and info["resident"] == 0
    work, lo, hi = mpk.mpk_plan_schedule(plan)
    T = info["n_tiles"]
    t, k = work >> 8, work & 255
    assert work.shape == (T * p,)
    s = (k - 1) // q
    assert np.all(np.diff(s) >= 0)
    pos = np.empty((T, p + 1), dtype=np.int64)
    pos[t, k] = np.arange(T * p)
    for j in range(T * p):
        if k[j] > 1:
            assert pos[lo[t[j]]:hi[t[j]] + 1, k[j] - 1].max() < j
    gp = mpk.mpk_plan_perm(plan)[2].cpu().numpy()
    gq = mpk.mpk_plan_perm(plan_of(A, q, prec="f64", **kw))[2].cpu().numpy()
    assert np.array_equal(gp, gq)


@pytest.mark.parametrize("name", ["laplace3d-30", "laplace3d-30-tiny-tiles", "zipf-8000", "box27-12", "diag-500"])
@pytest.mark.parametrize("p,q", [(8, 8), (8, 3), (5, 1)])
def test_issue_order_is_the_sorted_wavefront(name, p, q):
    """The plan's issue order (placed on the GPU) is exactly the sort of the
    items by (key, k, t) within each sweep, key = v(t) + slope * (k - k0):
    v(t) = group index + the fraction of the group's rows before tile t, the
    slope as the plan reports it, k0 the sweep's first power."""
    make, kw = CASES[name]
    A = make()
    plan = plan_of(A, p, prec="f64", sweep=q, **kw)
    info = mpk.mpk_plan_info(plan)
    assert info["rec_stages"] == 0
    _, lp, gp, _ = (t.cpu().numpy() for t in mpk.mpk_plan_perm(plan))
    work, _, _ = mpk.mpk_plan_schedule(plan)
    tr = info["tile_rows"]
    v, T = [], 0
    for g in range(len(gp) - 1):
        r0, r1 = int(lp[gp[g]]), int(lp[gp[g + 1]])
        for a in range(r0, r1, tr):
            v.append(g + float(a - r0) / float(r1 - r0))
    T = len(v)
    assert T == info["n_tiles"]
    sigma = info["slope"]
    items = []
    for k in range(1, p + 1):
        s = (k - 1) // q
        k0 = s * q + 1
        for t in range(T):
            items.append((s, v[t] + sigma * (k - k0), k, t))
    items.sort()
    want = np.array([(t << 8) | k for _, _, k, t in items], dtype=np.int32)
    assert np.array_equal(work, want)
