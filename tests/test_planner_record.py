"""The committed evaluation record of the learned planner
(paper_2205_01598_gb300/planner_eval.json) is reproducible from committed
files alone: the timing sets it names (held-out corpus matrices and the two
headline matrices), the shipped weights, and the FP64 network reference of
the oracle.  The network's picks, recomputed on
the host, are the recorded ones (up to near-ties of the FP32 forward pass),
and every recorded regret and summary follows from the timings."""
import json
import os

import numpy as np
import pytest

from oracle import mlp
from paper_2205_01598_gb300 import planner as P

RECORD = os.path.join(os.path.dirname(P.WEIGHTS), "planner_eval.json")
DATA = os.path.join(os.path.dirname(P.WEIGHTS), "planner_data")


@pytest.fixture(scope="module")
def record():
    if not os.path.exists(RECORD):
        pytest.skip("no planner record committed")
    with open(RECORD) as f:
        return json.load(f)


def test_record_follows_from_committed_data(record):
    F, MS, names = P.load_sets([os.path.join(DATA, d) for d in record["data"]])
    rows = record["matrices"]
    assert [r["matrix"] for r in rows] == names
    d = np.load(P.WEIGHTS)
    shape = tuple(int(s) for s in d["shape"])
    X = (F.astype(np.float64) - d["mean"]) / d["std"]
    pred, _ = mlp.forward(d["params"].astype(np.float64), X, shape)
    chosen = np.array([r["chosen"] for r in rows])
    host = np.argmin(pred, axis=1)
    gap = pred[np.arange(len(rows)), chosen] - pred[np.arange(len(rows)), host]
    assert np.all(gap <= 1e-4), np.flatnonzero(gap > 1e-4)      # the same pick, or a near-tie
    r = P.regret(MS, chosen)
    assert np.allclose(r, [row["regret"] for row in rows], rtol=0, atol=1e-12)
    assert np.allclose([row["best_ms"] for row in rows], np.where(MS > 0, MS, np.inf).min(1))


def test_record_summaries(record):
    rows = record["matrices"]
    reg = np.array([r["regret"] for r in rows])
    n = np.array([r["n"] for r in rows])
    assert record["all"]["matrices"] == len(rows)
    assert abs(record["all"]["regret_mlp_mean"] - reg.mean()) < 1e-12
    small, large = n <= 2_000_000, n > 2_000_000
    assert abs(record["n_up_to_2M"]["regret_mlp_mean"] - reg[small].mean()) < 1e-12
    assert abs(record["n_above_2M"]["regret_mlp_mean"] - reg[large].mean()) < 1e-12
    assert record["n_above_2M"]["matrices"] >= 40 and max(n) >= 7_000_000
    assert sum(r["matrix"].endswith("-headline") for r in rows) == 2
