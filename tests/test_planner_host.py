"""Host-side checks of the learned planner's shipped artefacts (no GPU): the
weights file matches the network shape the planner builds (25 features, two
hidden layers of 64, one output per entry of the default grid for k = 8:
the library defaults, 2 resident candidates and 5 x 2 x 3 work-list ones),
its feature standardisation is finite, and the corpus generator is
deterministic."""
import os

import numpy as np
import pytest

from paper_2205_01598_gb300 import planner as P


def test_weights_match_network_shape():
    if not os.path.exists(P.WEIGHTS):
        pytest.skip("no trained planner weights in the package")
    d = np.load(P.WEIGHTS)
    n_in, n_h, n_out = (int(v) for v in d["shape"])
    assert (n_in, n_h, n_out) == (25, P.HIDDEN, 1 + 2 + 5 * 2 * 3)
    assert d["params"].shape == (n_h * n_in + n_h + n_h * n_h + n_h + n_out * n_h + n_out,)
    assert np.all(np.isfinite(d["params"]))
    assert d["mean"].shape == d["std"].shape == (n_in,)
    assert np.all(np.isfinite(d["mean"])) and np.all(d["std"] > 0)


def test_corpus_is_deterministic_and_spans_families():
    fams = [P.corpus_spec(i)[0] for i in range(10000, 10010)]
    assert sorted(set(fams)) == sorted(P.FAMILIES)
    for i in (10000, 10003, 10004):
        a, b = P.corpus_matrix(i, 2000, 6000), P.corpus_matrix(i, 2000, 6000)
        assert a.n == b.n and np.array_equal(a.col, b.col) and np.array_equal(a.val, b.val)
        fam, n, _ = P.corpus_spec(i, 2000, 6000)
        assert 2000 <= n <= 6000


def test_regret_and_targets():
    ms = np.array([[2.0, 1.0, -1.0, 4.0], [3.0, 3.0, 6.0, 1.5]])
    y, m = P.targets(ms)
    assert np.allclose(y[0], [np.log(2.0), 0.0, 0.0, np.log(4.0)]) and list(m[0]) == [1, 1, 0, 1]
    assert np.allclose(P.regret(ms, np.array([1, 1])), [0.0, 1.0])
    assert np.allclose(P.regret(ms, np.array([2, 3])), [3.0, 0.0])   # a failed pick counts as the worst


def test_member_options_carry_the_sweep_kind():
    """A grid entry tuned for k = 8 maps to a member of p powers by its sweep
    kind: all powers in one sweep, two sweeps, or single-power sweeps."""
    base = {"tile_rows": 128, "safety_f": 0.25, "tune": 0}
    for p in range(1, 11):
        assert P.member_options(dict(base, p_sweep=8), p)["sweep"] == p
        assert P.member_options(dict(base, p_sweep=4), p)["sweep"] == (p + 1) // 2
        assert P.member_options(dict(base, p_sweep=1), p)["sweep"] == 1
    o = P.member_options(dict(base, p_sweep=4), 7)
    assert o == {"tile_rows": 128, "safety_f": 0.25, "tune": 0, "sweep": 4}
    assert P.member_options({"tile_rows": 0, "safety_f": 0.5, "tune": 0, "p_sweep": 6}, 6, 6)["sweep"] == 6


def test_regret_matrix_and_load_sets(tmp_path):
    ms = np.array([[2.0, 1.0, -1.0], [3.0, 6.0, 1.5]])
    R = P.regret_matrix(ms)
    assert np.allclose(R, [[1.0, 0.0, 1.0], [1.0, 3.0, 0.0]])
    for i, part in enumerate((ms[:1], ms[1:])):
        np.savez(tmp_path / f"s{i}.npz", features=np.full((1, 25), i, np.float32), ms=part,
                 names=np.array([f"m{i}"]))
    F, MS, names = P.load_sets([tmp_path / "s0.npz", tmp_path / "s1.npz"])
    assert F.shape == (2, 25) and np.array_equal(MS, ms) and names == ["m0", "m1"]
