"""Planner features, autotuner and learned planner on the GPU.

The features are checked against a host computation over the oracle's BFS
levels and permuted matrix; the autotuner's table against its own contract;
the learned planner (trained weights shipped with the package) against the
library's default options on freshly generated matrices outside its
training range.
"""
import math
import os

import numpy as np
import pytest

import mpk_inputs as mi
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import paper_2205_01598_gb300 as mpk
    mpk.build()
    return mpk.load()


def _host_features(A):
    """The 25 features of mpk_plan_features, from the oracle's levels."""
    lev, L = oracle.bfs_levels(A, root=0)
    perm, iperm, level_ptr = oracle.level_perm(lev, L)
    Ap = oracle.permute_csr(A, perm, iperm)
    rp, cl, n = Ap.rowptr, Ap.col, A.n
    lens = np.diff(rp).astype(np.float64)
    rows = np.repeat(np.arange(n), np.diff(rp))
    dist = np.abs(cl.astype(np.int64) - rows)
    sizes = np.diff(level_ptr)
    f = [math.log10(n), lens.mean(), math.sqrt(max(0.0, (lens ** 2).mean() - lens.mean() ** 2)),
         math.log10(1 + lens.max()), dist.sum() / max(1, lens.sum()) / n, dist.max() / n,
         math.log10(L), sizes.max() / n, n / L / sizes.max()]
    for q in range(16):
        l0, l1 = L * q // 16, L * (q + 1) // 16
        f.append((level_ptr[l1] - level_ptr[l0]) / n)
    return np.array(f)


@pytest.mark.parametrize("make", [lambda: mi.laplace2d(50, 37), lambda: mi.box27(12),
                                  lambda: mi.zipf_graph(3000, 5), lambda: mi.random_geometric_graph(4000, 3, 12.0, 9)],
                         ids=["lap2d", "box27", "zipf", "rgg3d"])
def test_features_match_host(lib, make):
    A = make()
    from paper_2205_01598_gb300 import csr_to_device, mpk_plan, mpk_plan_features
    plan = mpk_plan(*csr_to_device(A), 4, prec="f32")
    got = mpk_plan_features(plan)
    want = _host_features(A)
    assert got.shape == (25,)
    np.testing.assert_allclose(got, want, rtol=2e-6, atol=1e-7)


def test_default_grid_layout(lib):
    from paper_2205_01598_gb300 import mpk_tune_default_grid
    g = mpk_tune_default_grid(8)
    assert g[0] == {"tile_rows": 0, "safety_f": 0.5, "tune": 0, "p_sweep": 8}
    assert [c["tune"] for c in g[1:3]] == [8, 8] and [c["p_sweep"] for c in g[1:3]] == [8, 4]
    assert len(g) == 1 + 2 + 5 * 2 * 3
    assert {c["p_sweep"] for c in g} == {8, 4, 1}
    assert len(mpk_tune_default_grid(1)) == 1 + 1 + 5 * 2


def test_autotune_table(lib):
    from paper_2205_01598_gb300 import csr_to_device, mpk_autotune, mpk_tune_default_grid
    A = mi.laplace3d(24)
    g = mpk_tune_default_grid(5)
    best, ms = mpk_autotune(*csr_to_device(A), 5, g, prec="f32", min_time_s=0.002)
    assert len(ms) == len(g)
    assert all(t > 0 for t in ms)
    assert 0 <= best < len(g) and ms[best] == min(ms)


def test_autotune_split_runs_remainder(lib):
    """Sweeps of 3 for k = 7 run as one plan (sweeps 3, 3, 1 in one launch);
    a candidate with p_sweep > k is clamped to k; a resident candidate with
    p_sweep < k times one plan per sweep and one for the remainder."""
    from paper_2205_01598_gb300 import csr_to_device, mpk_autotune
    A = mi.laplace2d(40)
    cands = [{"tile_rows": 64, "safety_f": 0.5, "p_sweep": 3}, {"tile_rows": 64, "safety_f": 0.5, "p_sweep": 99},
             {"tile_rows": 0, "safety_f": 0.5, "p_sweep": 3, "tune": 8}]
    best, ms = mpk_autotune(*csr_to_device(A), 7, cands, prec="f64", min_time_s=0.002)
    assert all(t > 0 for t in ms) and best in (0, 1, 2)


def test_planner_beats_default(lib):
    """On matrices outside the training range (corpus indices 90000+), the
    learned planner's choice has a lower mean regret against the best of the
    grid than the library's default options."""
    from paper_2205_01598_gb300 import planner as P
    if not os.path.exists(P.WEIGHTS):
        pytest.skip("no trained planner weights in the package")
    net = P.Planner.load()
    F, MS = [], []
    for i in range(90000, 90010):
        A = P.corpus_matrix(i, 20_000, 200_000)
        f, ms, _ = P.measure(A, min_time_s=0.01)
        F.append(f)
        MS.append(ms)
    F, MS = np.array(F), np.array(MS)
    r_mlp = P.regret(MS, net.choose(F))
    r_def = P.regret(MS, np.zeros(len(MS), dtype=int))
    assert r_mlp.mean() <= r_def.mean(), (r_mlp, r_def)
    assert r_mlp.mean() <= 0.10, r_mlp   # within 10 % of the autotuner's best on average


def test_plan_options_network_and_fallbacks(lib):
    """plan_options: the network's pick when weights ship; the full
    autotuner without weights, or when the network names no grid entry."""
    from paper_2205_01598_gb300 import csr_to_device
    from paper_2205_01598_gb300 import planner as P
    A = mi.laplace3d(30)
    rp, cl, va = csr_to_device(A)
    g = P.grid()
    keys = ("tile_rows", "safety_f", "tune", "sweep")
    if os.path.exists(P.WEIGHTS):
        opt = P.plan_options(rp, cl, va)
        assert opt["source"] == "mlp" and {k: opt[k] for k in keys} == P.member_options(g[opt["grid_index"]], 8)
        opt = P.plan_options(rp, cl, va, p=5, nrhs=3)      # a member of another p and width
        assert {k: opt[k] for k in keys} == P.member_options(g[opt["grid_index"]], 5)
    opt = P.plan_options(rp, cl, va, p=6, use_weights=False)
    g6 = P.mpk_tune_default_grid(6)
    assert opt["source"] == "autotuner" and {k: opt[k] for k in keys} == P.member_options(g6[opt["grid_index"]], 6, 6)

    class Broken:
        def choose(self, feats):
            return np.array([len(g) + 5])
    assert P.plan_options(rp, cl, va, planner=Broken())["source"] == "autotuner"
