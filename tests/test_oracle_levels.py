"""Pins for the oracle's levels (Eq. 3), renumbering (Sec. 4.1), level
groups (Eq. 5) and Lp traversal (Fig. 5): the paper's worked examples,
closed forms on grids, a BFS certificate that shares no code with the
oracle, a library shortest-path routine, and brute-force properties."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.csgraph as csg

import mpk_inputs as mi
import oracle
from conftest import read_golden


def _sym_adj(A):
    M = sp.csr_matrix((np.ones(A.nnz), A.col, A.rowptr), shape=(A.n, A.n))
    return ((M + M.T) != 0).astype(np.int8).tocsr()


def certify_levels(A, level, root=0):
    """Independent check that `level` is the Eq. 3 level map with the
    component-restart reading: (1) root at 0; (2) every edge joins levels
    that differ by <= 1 (Eq. 4); (3) every vertex that is not a component
    root has a neighbour exactly one level lower; (4) component roots are,
    in order, the chosen root and then the lowest-numbered vertex not yet
    reached, each one level above the previous component's last level."""
    M = _sym_adj(A).tocoo()
    assert level[root] == 0
    assert np.all(np.abs(level[M.row] - level[M.col]) <= 1)
    has_lower = np.zeros(A.n, dtype=bool)
    lower = level[M.col] == level[M.row] - 1
    has_lower[M.row[lower]] = True
    ncomp, comp = csg.connected_components(_sym_adj(A), directed=False)
    roots = [root]
    seen = np.zeros(ncomp, dtype=bool)
    seen[comp[root]] = True
    for v in range(A.n):
        if not seen[comp[v]]:
            seen[comp[v]] = True
            roots.append(v)
    prev_max = -1
    for r in roots:
        members = comp == comp[r]
        assert level[r] == prev_max + 1
        assert level[members].min() == level[r]
        assert np.all(has_lower[members] | (np.arange(A.n)[members] == r))
        prev_max = level[members].max()
    return prev_max + 1


def test_worked_example_levels_and_level_ptr():
    g = read_golden("worked_example_2d7pt_8x8.txt")
    A = mi.stencil2d_7pt(8)
    level, L = oracle.bfs_levels(A, root=0)
    assert L == g["nlevels"][0]
    perm, iperm, lp = oracle.level_perm(level, L)
    assert list(lp) == g["level_ptr"]
    assert (lp[6], lp[7] - 1) == tuple(g["L6_rows"])
    assert (lp[5], lp[8] - 1) == tuple(g["L5_to_L7_rows"])
    assert certify_levels(A, level) == L


def _grid_levels(dims, periodic):
    idx = np.arange(int(np.prod(dims)))
    tot = np.zeros_like(idx)
    rem = idx
    for d in dims:
        c = rem % d
        rem = rem // d
        tot = tot + (np.minimum(c, d - c) if periodic else c)
    return tot


@pytest.mark.parametrize("make,dims,periodic", [
    (lambda: mi.laplace2d(64), (64, 64), False),
    (lambda: mi.laplace3d(17), (17, 17, 17), False),
    (lambda: mi.box27(9), None, False),
    (lambda: mi.anderson3d(12), (12, 12, 12), True),
    (lambda: mi.anderson3d(7), (7, 7, 7), True),
])
def test_grid_levels_closed_form(make, dims, periodic):
    A = make()
    level, L = oracle.bfs_levels(A)
    if dims is None:   # 27-point: Chebyshev (max-norm) distance from the corner
        n = round(A.n ** (1 / 3))
        i = np.arange(A.n)
        want = np.maximum(np.maximum(i % n, (i // n) % n), i // (n * n))
    else:
        want = _grid_levels(dims, periodic)
    assert np.array_equal(level, want)
    assert L == want.max() + 1


def _level_sizes_by_convolution(n, d, periodic):
    one = np.ones(n, dtype=np.int64)
    if periodic:
        one = np.bincount(np.minimum(np.arange(n), n - np.arange(n)))
    h = np.array([1], dtype=np.int64)
    for _ in range(d):
        h = np.convolve(h, one)
    return h


def test_config_level_counts():
    """Level counts and largest levels of the three stencil workloads
    (2D 64^2, 3D 160^3, periodic 200^3), from the distance histograms."""
    h = _level_sizes_by_convolution(64, 2, False)
    assert (len(h), h.max()) == (127, 64)
    h = _level_sizes_by_convolution(160, 3, False)
    assert (len(h), h.max(), h.sum()) == (478, 19200, 160 ** 3)
    h = _level_sizes_by_convolution(200, 3, True)
    assert (len(h), h.max(), h.sum()) == (301, 59996, 200 ** 3)
    # and the oracle agrees with the same histogram on a smaller grid
    level, L = oracle.bfs_levels(mi.laplace3d(21))
    assert np.array_equal(np.bincount(level), _level_sizes_by_convolution(21, 3, False))


@pytest.mark.parametrize("seed", range(6))
def test_random_graphs_certificate_and_scipy_distances(seed):
    n = 40 + 13 * seed
    A = mi.random_sparse(n, 2.5 / n, seed, symmetric=True, diag=(seed % 2 == 0))
    root = (seed * 7) % n
    level, L = oracle.bfs_levels(A, root=root)
    assert certify_levels(A, level, root) == L
    dist = csg.shortest_path(_sym_adj(A), unweighted=True, indices=root)
    reach = np.isfinite(dist)
    assert np.array_equal(level[reach], dist[reach].astype(np.int32))


def test_disconnected_restart_rule():
    # components {0,1,2} (path 2-0-1) and {3,4}; vertex 5 isolated
    D = np.zeros((6, 6))
    for a, b in [(0, 1), (0, 2), (3, 4)]:
        D[a, b] = D[b, a] = 1.0
    A = mi.from_dense(D)
    level, L = oracle.bfs_levels(A, root=0)
    assert list(level) == [0, 1, 1, 2, 3, 4] and L == 5
    level, L = oracle.bfs_levels(A, root=4)
    assert list(level) == [2, 3, 3, 1, 0, 4] and L == 5


def test_diagonal_matrix_singleton_levels():
    A = mi.diagonal(np.arange(1.0, 31.0))
    level, L = oracle.bfs_levels(A)
    assert L == 30 and np.array_equal(level, np.arange(30))


def test_nonsymmetric_pattern_symmetrized():
    A = mi.random_sparse(50, 0.05, 11, symmetric=False, diag=False)
    level, L = oracle.bfs_levels(A, root=3, symmetrize=True)
    S = _sym_adj(A)
    B = mi.CSR(A.n, S.indptr, S.indices, np.ones(S.nnz))
    level2, L2 = oracle.bfs_levels(B, root=3)
    assert np.array_equal(level, level2) and L == L2
    assert certify_levels(A, level, 3) == L


def test_level_perm_is_stable_sort():
    A = mi.anderson3d(9)
    level, L = oracle.bfs_levels(A)
    perm, iperm, lp = oracle.level_perm(level, L)
    assert np.array_equal(perm, np.lexsort((np.arange(A.n), level)))
    assert np.array_equal(iperm[perm], np.arange(A.n))
    assert np.array_equal(lp, np.concatenate([[0], np.cumsum(np.bincount(level))]))


def test_permuted_matrix_is_level_banded():
    """After the renumbering, rows of L(i) only reference L(i-1..i+1) (Eq. 4)."""
    A = mi.laplace3d(10)
    level, L = oracle.bfs_levels(A)
    perm, iperm, lp = oracle.level_perm(level, L)
    Ap = oracle.permute_csr(A, perm, iperm)
    lev_new = level[perm]
    rows = np.repeat(np.arange(A.n), np.diff(Ap.rowptr))
    assert np.all(np.abs(lev_new[rows] - lev_new[Ap.col]) <= 1)
    for r in range(A.n):
        assert np.all(np.diff(Ap.col[Ap.rowptr[r]:Ap.rowptr[r + 1]]) > 0)


# ------------------------------------------------------------------ groups
def test_fig8_grouping_example():
    g = read_golden("groups_fig8.txt")
    A = mi.stencil2d_7pt(8)
    level, L = oracle.bfs_levels(A)
    perm, iperm, lp = oracle.level_perm(level, L)
    sizes = np.diff(lp).astype(np.float64)          # vertices per level
    gp = oracle.level_groups(sizes, 0, 1.0, g["budget"][0])   # (pm+1) = 1
    gsize = np.add.reduceat(sizes, gp[:-1])
    bulky = [i for i in range(len(gp) - 1) if gsize[i] > 6]
    assert bulky == g["bulky_groups"]
    assert [int(gp[i]) for i in bulky] == g["bulky_levels"]
    assert all(gp[i + 1] - gp[i] == 1 for i in bulky)
    # the subgraph induced by the bulky levels has eight BFS levels (Fig. 8b)
    Ap = oracle.permute_csr(A, perm, iperm)
    lo, hi = lp[g["bulky_levels"][0]], lp[g["bulky_levels"][-1] + 1]
    S = sp.csr_matrix((Ap.val, Ap.col, Ap.rowptr), shape=(A.n, A.n))[lo:hi, lo:hi].tocsr()
    sub = mi.CSR(hi - lo, S.indptr, S.indices, S.data)
    _, Ls = oracle.bfs_levels(sub, root=0)
    assert Ls == g["subgraph_levels"][0]


@pytest.mark.parametrize("seed", range(20))
def test_groups_greedy_properties(seed):
    """Brute-force characterisation of Eq. 5's greedy: groups are consecutive,
    cover all levels; a multi-level group satisfies the bound; a single-level
    group either satisfies it or its level alone violates it; and no group
    could have taken the next level."""
    z = mi.splitmix64(seed, 40)
    nl = int(z[0] % np.uint64(30)) + 1
    w = (z[1:nl + 1] % np.uint64(50)).astype(np.float64) + 1.0
    pm = int(z[-1] % np.uint64(8)) + 1
    budget = float(z[-2] % np.uint64(400)) + 20.0
    gp = oracle.level_groups(w, pm, 0.5, 2.0 * budget)   # f*C = budget
    assert gp[0] == 0 and gp[-1] == nl and np.all(np.diff(gp) >= 1)
    for a, b in zip(gp[:-1], gp[1:]):
        tot = w[a:b].sum()
        if b - a > 1:
            assert (pm + 1) * tot < budget
        if b < nl:
            assert not ((pm + 1) * (tot + w[b]) < budget)


# ------------------------------------------------------------------ Lp order
def test_fig4_step_numbers():
    g = read_golden("lp_order_15x5.txt")
    L, pm = g["nlevels"][0], g["pm"][0]
    ni, npw = oracle.lp_order(L, pm)
    step = {(int(i), int(p)): s for s, (i, p) in enumerate(zip(ni, npw))}
    assert step[(10, 1)] == g["node_10_1_step"][0]
    assert step[(10, 2)] == g["node_10_2_step"][0]
    # steady-state reuse distance of a level between consecutive powers
    for i in range(pm, L - pm):
        for p in range(1, pm):
            assert step[(i, p + 1)] - step[(i, p)] == g["reuse_distance"][0]


@pytest.mark.parametrize("L,pm", [(15, 5), (3, 8), (1, 4), (40, 1), (7, 7)])
def test_lp_order_covers_and_respects_dependencies(L, pm):
    ni, npw = oracle.lp_order(L, pm)
    assert len(ni) == L * pm
    step = {(int(i), int(p)): s for s, (i, p) in enumerate(zip(ni, npw))}
    assert len(step) == L * pm
    for (i, p), s in step.items():
        for j in (i - 1, i, i + 1):
            if p > 1 and 0 <= j < L:
                assert step[(j, p - 1)] < s
