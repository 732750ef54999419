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
    assert bench.run_reference(args, "laplace2d", 64, 4, "f64", "2D 64^2") is None
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
    bench.run_reference(args, "laplace2d", 64, 4, "f64", "2D 64^2")
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert calls == [4] * 7
    assert line["impl"] == "reference" and line["steps"] == 4 and line["warmup"] == 3
    assert line["config"]["nnz"] == 20224 and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]


def test_both_arms_print_the_same_config():
    """The config dicts come from the host matrix alone, so the reference arm
    and the GPU arm print identical ones (MPK, Chebyshev and batch lines)."""
    import bench
    import mpk_inputs as mi
    A = mi.laplace2d(64)
    c1 = bench.mpk_config("2D", A, 4, "f64")
    assert c1 == bench.mpk_config("2D", mi.laplace2d(64), 4, "f64")
    assert c1["l2"].startswith("L2 flushed")        # 0.4 MB working set
    big = type("M", (), {"n": 4_096_000, "nnz": 28_518_400})()
    assert bench.mpk_config("3D", big, 8, "f64")["l2"].startswith("inputs larger than L2")
    specs = [(0, 1000, 25_000, 3, 4), (1, 1001, 30_000, 1, 2)]
    assert bench.batch_config("b", specs) == {"workload": "b", "matrices": 2, "rows": 55_000, "rhs": 4,
                                              "powers": 6, "data": "synthetic"}


def test_algorithmic_bytes_of_the_headline_workload():
    """The one-read and p x SpMV bytes of the 3D 160^3 p = 8 workload
    (653.5 MB and 3.39 GB in FP64, 392 MB and 2.22 GB in FP32), and the
    Anderson sweep (about 833 MB with BF16 hoppings)."""
    import bench
    n, nnz = 4_096_000, 28_518_400
    assert bench.one_read_bytes(nnz, n, 8, "f64") == pytest.approx(653.5e6, rel=1e-3)
    assert bench.pxspmv_bytes(nnz, n, 8, "f64") == pytest.approx(3.393e9, rel=1e-3)
    assert bench.one_read_bytes(nnz, n, 8, "f32") == pytest.approx(392.0e6, rel=2e-3)
    assert bench.pxspmv_bytes(nnz, n, 8, "f32") == pytest.approx(2.218e9, rel=1e-3)
    sweep = bench.cheb_sweep_bytes("anderson3d", 56_000_000, 8_000_000, "bf16val", 2)
    assert sweep == pytest.approx(833e6, rel=0.01)


def test_per_power_errors():
    import numpy as np
    import bench
    ref = np.array([[1.0, -2.0], [0.0, 0.0]])
    got = np.array([[1.0, -2.0 + 1e-3], [0.0, 1e-310]])
    e = bench.per_power_errors(got, ref)
    assert e[0] == pytest.approx(5e-4) and e[1] > 0
