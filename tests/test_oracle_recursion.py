"""Pins of the oracle's recursive level construction (Sec. 4.4), checked
against the paper's worked example (Fig. 8), the stage-0 construction it
must reduce to, and properties that any correct refinement has, verified
with code that shares nothing with the oracle's search:
  - the renumbering is a permutation, identical to stage 0 outside the
    refined runs, and each refined run holds the same vertices as before;
  - inside a refined run the sub-levels are a breadth-first certificate of
    the induced subgraph (Eq. 4 and a parent one sub-level lower, component
    roots at the lowest unvisited position);
  - the groups are Eq. 5's greedy groups over the finest levels' weights."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.csgraph as csg

import mpk_inputs as mi
import oracle
from conftest import read_golden


def _stage0(A, w, pm, f, C):
    level, L = oracle.bfs_levels(A)
    perm, iperm, lp = oracle.level_perm(level, L)
    lw = np.array([w[perm[lp[l]:lp[l + 1]]].sum() for l in range(L)])
    gp = oracle.level_groups(lw, pm, f, C)
    return perm, lp, gp, lw


def test_fig8_subgraph_levels():
    """Sec. 4.4, Fig. 8: on the 8x8 2d-7pt graph with a cache that admits
    groups of at most six vertices, the bulky groups T(4)..T(6) (one level
    each) induce a subgraph with eight BFS levels, whose groups satisfy the
    bound, and the process stops."""
    g = read_golden("groups_fig8.txt")
    A = mi.stencil2d_7pt(8)
    w = np.ones(A.n)
    budget = g["budget"][0]
    perm0, lp0, gp0, _ = _stage0(A, w, 0, 1.0, budget)
    perm, lp, gp, gs, stages = oracle.recursive_levels(A, w, 0, 1.0, budget, 4)
    assert stages == 1                                   # stage 1 already fits: the process stops
    l6, l9 = g["bulky_levels"][0], g["bulky_levels"][-1] + 1
    refined = gs == 1
    assert int(refined.sum()) >= 1
    # levels before and after the subgraph are those of stage 0
    assert np.array_equal(lp[:l6 + 1], lp0[:l6 + 1])
    nsub = g["subgraph_levels"][0]
    assert len(lp) - 1 == (len(lp0) - 1) - (l9 - l6) + nsub
    assert np.array_equal(lp[l6 + nsub:], lp0[l9:])
    # every group of the refined subgraph satisfies Eq. 5 (at most six vertices)
    sizes = np.diff(lp)
    for q in range(len(gp) - 1):
        tot = sizes[gp[q]:gp[q + 1]].sum()
        assert tot < budget or gp[q + 1] - gp[q] == 1
        if gs[q] == 1:
            assert tot < budget
    # the subgraph's vertices are the same set, renumbered inside its range
    a, b = lp0[l6], lp0[l9]
    assert sorted(perm[a:b]) == sorted(perm0[a:b])
    assert np.array_equal(perm[:a], perm0[:a]) and np.array_equal(perm[b:], perm0[b:])


@pytest.mark.parametrize("make", [lambda: mi.laplace3d(12), lambda: mi.zipf_graph(3000, 1002),
                                  lambda: mi.random_sparse(800, 6.0 / 800, 4)])
def test_no_recursion_is_stage_zero(make):
    A = make()
    w = np.diff(A.rowptr).astype(np.float64) * 12.0
    C = 0.02 * w.sum() * 9
    perm0, lp0, gp0, _ = _stage0(A, w, 8, 0.5, C)
    perm, lp, gp, gs, stages = oracle.recursive_levels(A, w, 8, 0.5, C, 0)
    assert stages == 0 and np.all(gs == 0)
    assert np.array_equal(perm, perm0) and np.array_equal(lp, lp0) and np.array_equal(gp, gp0)


def _certify_run(A, perm, iperm, lp, l0, l1):
    """Breadth-first certificate of the sub-levels l0..l1-1 (rows lp[l0] ..
    lp[l1]-1) on the subgraph induced by those rows, with component roots at
    the lowest unvisited position."""
    a, b = lp[l0], lp[l1]
    M = sp.csr_matrix((np.ones(A.nnz), A.col, A.rowptr), shape=(A.n, A.n))
    sub = M[perm[a:b]][:, perm[a:b]].tocsr()       # induced subgraph, positions a..b-1
    lev = np.repeat(np.arange(l1 - l0), np.diff(lp[l0:l1 + 1]))
    rows = np.repeat(np.arange(b - a), np.diff(sub.indptr))
    assert np.all(np.abs(lev[rows] - lev[sub.indices]) <= 1)   # Eq. 4 inside the subgraph
    assert np.all(np.diff(lev) >= 0)                           # sub-levels consecutive
    ncomp, comp = csg.connected_components(sub, directed=False)
    for i in range(b - a):
        parents = lev[sub.indices[sub.indptr[i]:sub.indptr[i + 1]]]
        if not np.any(parents == lev[i] - 1):
            # a component root: the lowest position of its component, one
            # level above everything numbered before it
            assert i == np.flatnonzero(comp == comp[i])[0]
            assert i == 0 or lev[i] == lev[i - 1] + 1
    # inside one sub-level, the previous numbering is kept (stable)
    return ncomp


@pytest.mark.parametrize("make,pm,frac,s_max", [
    (lambda: mi.laplace3d(14), 8, 0.5, 1),       # the middle levels bulky: 18 of 28 groups
    (lambda: mi.laplace3d(14), 4, 0.12, 3),
    (lambda: mi.zipf_graph(4000, 1003), 6, 2.0, 2),
    (lambda: mi.zipf_graph(4000, 1003), 3, 0.6, 1),
    (lambda: mi.box27(10), 8, 0.4, 2),
    (lambda: mi.random_geometric_graph(3000, 2, 10.0, 5), 5, 0.05, 1),
])
def test_refinement_properties(make, pm, frac, s_max):
    A = make()
    w = np.diff(A.rowptr).astype(np.float64) * 12.0
    C = frac * w.sum()
    f = 0.5
    perm0, lp0, gp0, lw0 = _stage0(A, w, pm, f, C)
    perm, lp, gp, gs, stages = oracle.recursive_levels(A, w, pm, f, C, s_max)
    n = A.n
    assert np.array_equal(np.sort(perm), np.arange(n))
    iperm = np.empty(n, dtype=np.int64)
    iperm[perm] = np.arange(n)
    budget = f * C
    bulky0 = [q for q in range(len(gp0) - 1)
              if gp0[q + 1] - gp0[q] == 1 and (pm + 1) * lw0[gp0[q]] >= budget]
    assert bulky0 and stages >= 1 and not np.array_equal(perm, perm0)   # the case refines something
    # each maximal run of stage-0 bulky groups keeps its vertex set
    q = 0
    while q < len(bulky0):
        r = q
        while r + 1 < len(bulky0) and bulky0[r + 1] == bulky0[r] + 1:
            r += 1
        a, b = lp0[gp0[bulky0[q]]], lp0[gp0[bulky0[r] + 1]]
        assert sorted(perm[a:b]) == sorted(perm0[a:b])
        # the finest levels inside the run, at the first stage, certify a BFS
        # of the induced subgraph when this run was refined once only
        lo = int(np.searchsorted(lp, a)); hi = int(np.searchsorted(lp, b))
        assert lp[lo] == a and lp[hi] == b
        if s_max == 1:
            _certify_run(A, perm, iperm, lp, lo, hi)
        q = r + 1
    # outside the runs, stage 0 is untouched
    inside = np.zeros(n, dtype=bool)
    for q in bulky0:
        inside[lp0[gp0[q]]:lp0[gp0[q] + 1]] = True
    assert np.array_equal(perm[~inside], perm0[~inside])
    # every multi-level group satisfies Eq. 5, and no group of a stage could
    # have taken the next level of the same stage (the greedy's maximality)
    lw = np.array([w[perm[lp[l]:lp[l + 1]]].sum() for l in range(len(lp) - 1)])
    for g in range(len(gp) - 1):
        tot = lw[gp[g]:gp[g + 1]].sum()
        if gp[g + 1] - gp[g] > 1:
            assert (pm + 1) * tot < budget
        if g + 1 < len(gp) - 1 and gs[g + 1] == gs[g]:
            assert not ((pm + 1) * (tot + lw[gp[g + 1]]) < budget)


def test_edgeless_subgraph_gives_singletons():
    """A star: the centre is level 0, every leaf level 1.  The leaves induce a
    subgraph without edges, so each leaf is a component of its own and the
    restart rule makes every leaf a sub-level, in the order of the stage-0
    numbering."""
    n = 41
    rows = [np.arange(1, n)] + [np.array([0]) for _ in range(1, n)]
    rp = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int32)
    A = mi.CSR(n, rp, np.concatenate(rows).astype(np.int32), np.ones(rp[-1]))
    w = np.ones(n)
    perm, lp, gp, gs, stages = oracle.recursive_levels(A, w, 0, 1.0, 10.0, 1)
    assert stages == 1
    assert np.array_equal(lp, np.arange(n + 1))          # level 0, then 40 singleton sub-levels
    assert np.array_equal(perm, np.arange(n))
    assert np.all(gs[gp[:-1] >= 1] == 1)


def test_paper_statement_on_boundary_locality():
    """Sec. 4.4 (Fig. 9): refining a subgraph renumbers it without regard to
    the vertices outside, so the bandwidth of the boundary rows grows; the
    rows outside the subgraph keep their stage-0 neighbours."""
    A = mi.stencil2d_7pt(8)
    w = np.ones(A.n)
    perm0, lp0, gp0, _ = _stage0(A, w, 0, 1.0, 7.0)
    perm, lp, gp, gs, _ = oracle.recursive_levels(A, w, 0, 1.0, 7.0, 1)
    def bandwidth(p):
        ip = np.empty(A.n, dtype=np.int64)
        ip[p] = np.arange(A.n)
        rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
        return np.max(np.abs(ip[rows] - ip[A.col]))
    assert bandwidth(perm) > bandwidth(perm0)
