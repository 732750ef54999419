"""The replica path of bench.py (several GPUs as independent replicas, no
data-path collective) on the CPU: two gloo ranks take the max of their step
times, the whole-job value counts every rank's work, and the reference arm
does no work outside rank 0."""
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update({"RANK": str(rank), "LOCAL_RANK": str(rank), "WORLD_SIZE": "2",
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import bench
    r, ws, dist = bench.dist_setup(2, backend="gloo")
    assert (r, ws) == (rank, 2)
    dist.barrier()
    ms = bench.max_over_ranks(1.5 if rank == 0 else 4.0, dist, device="cpu")
    out[rank] = ms
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(port, out), nprocs=2, join=True)
        assert dict(out) == {0: 4.0, 1: 4.0}


def test_whole_job_value_counts_every_rank():
    import bench
    assert bench.whole_job_value(2e9, 1, 1000.0) == pytest.approx(2.0)
    assert bench.whole_job_value(2e9, 4, 1000.0) == pytest.approx(8.0)   # weak scaling: 4x the work, same time


def test_reference_arm_idles_outside_rank_zero(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")
    args = type("A", (), {"steps": 1, "warmup": 0})()
    assert bench.run_reference(args, "laplace2d", 64, 4, {}) is None
    assert capsys.readouterr().out == ""


def test_reference_arm_times_exactly_k_steps(monkeypatch, capsys):
    """Rank 0 runs W untimed warm-up steps and exactly K timed ones, and
    prints one JSON line with the keys the reference arm carries."""
    import json
    import bench
    import oracle
    calls = []
    real = oracle.mpk
    monkeypatch.setattr(oracle, "mpk", lambda A, x, p: calls.append(p) or real(A, x, p))
    monkeypatch.setenv("RANK", "0")
    args = type("A", (), {"steps": 4, "warmup": 3})()
    bench.run_reference(args, "laplace2d", 64, 4, {"workload": "2D 64^2"})
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert calls == [4] * 7
    assert line["impl"] == "reference" and line["steps"] == 4 and line["warmup"] == 3
    assert line["config"]["nnz"] == 20224 and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
