"""Benchmark of the level-blocked matrix-power kernel on one GB300 (or N replicas).

Default workload: 3D 7-point Laplacian on a 160^3 grid (N = 4,096,000,
nnz = 28,518,400), FP64, p = 8.  One step = one level-blocked MPK
(y_k = A^k x, k = 1..8) in a single persistent wavefront launch, vectors in
the plan's level order (the paper times in permuted space).  The plan
(levels, groups, packing) is built once before timing and reported apart,
as the paper reports preprocessing apart.

The JSON line carries: GFLOP/s (2 nnz p / t) for the whole job, the same
metric end to end through the public API with host buffers, the baseline of
p back-to-back SpMVs on the same GPU and the speedup over it, the FP32 form,
the roofline of the dominant kernel, the CPU oracle timed on the host and the
SM clocks sampled during the timed region.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--config NAME]
"""
import argparse
import ctypes
import json
import os
import statistics
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

# Inputs whose working set is below this many bytes (twice the 136 MB L2 of a
# GB300) get an L2 flush before every timed iteration.  The rule reads the
# host matrix only, so both arms of the benchmark print the same config.
L2_FLUSH_BELOW = 2 * 136_000_000

CONFIGS = {
    # name: (generator, size, p, precision, description)
    "laplace3d-160-p8-f64": ("laplace3d", 160, 8, "f64", "3D 7-point Laplacian 160^3, p=8, FP64"),
    "laplace3d-160-p8-f32": ("laplace3d", 160, 8, "f32", "3D 7-point Laplacian 160^3, p=8, FP32"),
    "laplace3d-160-p8-f64df": ("laplace3d", 160, 8, "f64df",
                               "3D 7-point Laplacian 160^3, p=8, FP64 inputs and outputs, double-float arithmetic "
                               "on the FP32 pipe"),
    "laplace3d-160-p8-bf16val": ("laplace3d", 160, 8, "bf16val",
                                 "3D 7-point Laplacian 160^3, p=8, FP32 vectors and accumulation, the BF16-exact "
                                 "off-diagonal values (-1) in BF16 and the diagonal (6) in FP32"),
    "laplace2d-64-p4-f64": ("laplace2d", 64, 4, "f64", "2D 5-point Laplacian 64^2, p=4, FP64"),
    "anderson200-cheb64-p8-bf16val": ("anderson3d", 200, 8, "bf16val",
                                      "3D Anderson 200^3 periodic (W=16.5), Chebyshev degree 64 in sweeps of "
                                      "p=8, FP32 vectors, BF16 hoppings, FP64 scaling and coefficient sum"),
    "heat160-o4-cheb64-p8-f64": ("heat", 160, 8, "f64",
                                 "3D heat equation, order-4 star stencil on 160^3 (Tab. 3: nnz 52,787,200), "
                                 "Chebyshev degree 64 (modified Bessel, tau*r = 50) in sweeps of p=8, FP64"),
}
BATCH_CONFIGS = {
    # name: (count, N low, N high, description)
    "batched-zipf64-f32": (64, 20_000, 2_000_000,
                           "64 random symmetric Zipf-degree matrices, N ~ U[20k, 2M], nrhs ~ U{1..16}, "
                           "p ~ U{2..10}, FP32, one persistent launch replayed from a CUDA graph"),
    "batched-zipf64-small-f32": (64, 2_000, 200_000, "as batched-zipf64-f32 with N ~ U[2k, 200k]"),
}
CHEB_M = 64
CHEB_RDT = 50.0
DEFAULT = "laplace3d-160-p8-f64"


def make_matrix(kind, size):
    import mpk_inputs as mi
    if kind == "heat":
        return mi.star3d(size, 2)   # order-4 star stencil (Tab. 3)
    if kind == "anderson3d":
        return mi.anderson3d(size, W=16.5, seed=42)
    return getattr(mi, kind)(size)


def vec_bytes(prec):
    """Bytes of a vector element and of a matrix value in the workload's
    definition (FP64 for the FP64 workloads, whatever form computes them)."""
    return 8 if prec in ("f64", "f64df") else 4


def mpk_config(desc, A, p, prec):
    """The config dict of an MPK line, computed from the host matrix alone
    (identical in both arms)."""
    ws = A.nnz * (vec_bytes(prec) + 4) + (p + 1) * A.n * vec_bytes(prec)
    l2 = (f"inputs larger than L2 (working set {ws / 1e6:.0f} MB)" if ws > L2_FLUSH_BELOW else
          "L2 flushed before every timed iteration (256 MB write outside the timing)")
    return {"workload": desc, "n": A.n, "nnz": A.nnz, "p": p, "prec": prec, "io": "level order (permuted space)",
            "l2": l2, "data": "synthetic"}


def cheb_config(desc, A, p, prec):
    return {"workload": desc, "n": A.n, "nnz": A.nnz, "p": p, "prec": prec, "M": CHEB_M, "r_dt": CHEB_RDT,
            "io": "level order (permuted space)", "l2": "inputs larger than L2", "data": "synthetic"}


def one_read_bytes(nnz, n, p, prec, nrhs=1):
    """Algorithmic bytes of one MPK (the one-matrix-read lower bound): the
    packed matrix once (value + 32-bit column per entry; with BF16 values, 2
    bytes per off-diagonal value and the FP32 diagonal apart), the row
    pointers, x and the p outputs."""
    vb = vec_bytes(prec)
    if prec == "bf16val":
        return (nnz - n) * (2 + 4) + 4 * n + 4 * (n + 1) + vb * n * nrhs * (1 + p)
    return nnz * (vb + 4) + 4 * (n + 1) + vb * n * nrhs * (1 + p)


def pxspmv_bytes(nnz, n, p, prec, nrhs=1):
    """Algorithmic bytes of p back-to-back SpMVs: the matrix, the row pointers,
    the input and the output once per power."""
    vb = vec_bytes(prec)
    return p * (nnz * (vb + 4) + 4 * n + 2 * vb * n * nrhs)


def cheb_sweep_bytes(kind, nnz, n, prec, cols):
    """Algorithmic bytes of one Chebyshev sweep of p powers: the matrix once
    (BF16 off-diagonal values, 32-bit columns and the FP32 diagonal in the
    BF16 form; value + column per entry otherwise), the two state vectors
    read at the start and the two written at the end, and the FP64
    coefficient sum read and written once."""
    vb = vec_bytes(prec)
    if prec == "bf16val":
        off = nnz - n
        matrix = off * (2 + 4) + n * 4
    else:
        matrix = nnz * (vb + 4)
    return matrix + 4 * n * cols * vb + 2 * n * cols * 8


def fma_rate(mpk, torch, prec, iters):
    """Sustained FMA rate (TFLOP/s) of the library's FMA-chain probe in `prec`,
    timed with CUDA events on the current stream (best of 3 after a warm-up)."""
    sink = torch.zeros(2, dtype=torch.float64, device="cuda")
    st = torch.cuda.current_stream()
    mpk.mpk_probe_fma(prec, sink, iters=iters)
    best = None
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        fl = mpk.mpk_probe_fma(prec, sink, iters=iters)
        e1.record(st)
        torch.cuda.synchronize()
        rate = fl / (e0.elapsed_time(e1) * 1e-3) / 1e12
        best = rate if best is None else max(best, rate)
    return best


def per_power_errors(got, ref):
    """Relative infinity-norm error of every power: ||got_k - ref_k|| / ||ref_k||."""
    out = []
    for k in range(ref.shape[0]):
        den = float(np.max(np.abs(ref[k])))
        out.append(float(np.max(np.abs(got[k] - ref[k]))) / (den if den > 0 else 1e-300))
    return out


def kernel_sources_hash():
    """sha256 prefix of the sources that define the MPK kernels and the plan's
    data layout (mpk_exec.cu, mpk_plan.cu, mpk_internal.cuh, in that order):
    a change to any of them invalidates a recorded ncu capture."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2205_01598_gb300", "csrc")
    for name in ("mpk_exec.cu", "mpk_plan.cu", "mpk_internal.cuh"):
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def recorded_traffic(summary, prec):
    """DRAM bytes (read + write) per launch of the dominant kernel from the
    committed ncu summary, or None once the kernel sources have changed since
    the capture (or no capture covers this precision)."""
    path = os.path.join(ROOT, "profiles", summary)
    try:
        with open(path) as f:
            line = next(l for l in f if l.startswith("traffic-bytes-per-launch:"))
    except (OSError, StopIteration):
        return None
    fields = dict(kv.split("=", 1) for kv in line.split(":", 1)[1].split())
    if fields.get("sources") != kernel_sources_hash() or prec not in fields:
        return None
    return int(fields[prec])


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# ---------------------------------------------------------------- clocks (NVML, read only)
class ClockSampler:
    """Samples the SM clock and the clock-event reasons through NVML while
    running (read-only queries; nothing is set)."""

    HW_SLOWDOWN, SW_THERMAL, HW_THERMAL, SW_POWER_CAP = 0x8, 0x20, 0x40, 0x4

    def __init__(self, index=0, period_s=0.002):
        self.period = period_s
        self.samples, self.reasons = [], 0
        self.max_mhz = None
        self.ok = False
        try:
            self.nvml = ctypes.CDLL("libnvidia-ml.so.1")
            if self.nvml.nvmlInit_v2() != 0:
                return
            self.h = ctypes.c_void_p()
            if self.nvml.nvmlDeviceGetHandleByIndex_v2(index, ctypes.byref(self.h)) != 0:
                return
            mx = ctypes.c_uint()
            if self.nvml.nvmlDeviceGetMaxClockInfo(self.h, 1, ctypes.byref(mx)) == 0:
                self.max_mhz = mx.value
            self.ok = True
        except OSError:
            pass

    def _one(self):
        clk = ctypes.c_uint()
        rs = ctypes.c_ulonglong()
        if self.nvml.nvmlDeviceGetClockInfo(self.h, 1, ctypes.byref(clk)) == 0:
            self.samples.append(clk.value)
        fn = getattr(self.nvml, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            getattr(self.nvml, "nvmlDeviceGetCurrentClocksThrottleReasons")
        if fn(self.h, ctypes.byref(rs)) == 0:
            self.reasons |= rs.value

    def __enter__(self):
        self._stop = threading.Event()
        if self.ok:
            self._t = threading.Thread(target=self._run, daemon=True)
            self._t.start()
        return self

    def _run(self):
        while not self._stop.is_set():
            self._one()
            time.sleep(self.period)

    def __exit__(self, *a):
        self._stop.set()
        if self.ok:
            self._t.join()
            self._one()

    def summary(self):
        names = []
        if self.reasons & self.HW_SLOWDOWN:
            names.append("hw_slowdown")
        if self.reasons & self.HW_THERMAL:
            names.append("hw_thermal_slowdown")
        if self.reasons & self.SW_THERMAL:
            names.append("sw_thermal_slowdown")
        if self.reasons & self.SW_POWER_CAP:
            names.append("sw_power_cap")
        return {"sm_mhz": statistics.median(self.samples) if self.samples else None,
                "sm_max_mhz": self.max_mhz, "reasons": names, "samples": len(self.samples),
                "source": "nvml" if self.ok else "unavailable"}


# ---------------------------------------------------------------- CPU oracle timing
def time_oracle(A, x, p, budget_s=12.0):
    """The FP64 CPU oracle (sequential C, one core) on the full matrix,
    repeated until `budget_s` of work; returns (GFLOP/s, reps, seconds)."""
    import oracle
    oracle.mpk(A, x, 1)
    reps, t0 = 0, time.perf_counter()
    while True:
        oracle.mpk(A, x, p)
        reps += 1
        el = time.perf_counter() - t0
        if el >= budget_s:
            break
    return 2.0 * A.nnz * p * reps / el / 1e9, reps, el


def time_omp(A, x, p, budget_s=5.0):
    """The multicore comparator: p back-to-back FP64 SpMVs with the rows split
    statically over all OpenMP threads of the host (a reported baseline,
    not the target), repeated until `budget_s`."""
    import oracle
    try:
        _, threads = oracle.omp_pxspmv(A, x, 1)
    except RuntimeError as e:
        return {"unavailable": str(e)}
    reps, t0 = 0, time.perf_counter()
    while True:
        oracle.omp_pxspmv(A, x, p)
        reps += 1
        el = time.perf_counter() - t0
        if el >= budget_s:
            break
    return {"value": round(2.0 * A.nnz * p * reps / el / 1e9, 4), "unit": "GFLOP/s", "cores": threads,
            "kind": "p x SpMV, OpenMP static schedule, FP64 CRS",
            "sample": f"full matrix, p={p}, {reps} runs in {el:.1f} s on {threads} threads"}


def dist_setup(n_gpus, backend="nccl"):
    """Replicas under torchrun: one process per GPU (RANK / LOCAL_RANK /
    WORLD_SIZE / MASTER_* from the environment), no data-path collective;
    the group only carries the barrier and the max-over-ranks timing."""
    import torch
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
        return rank, ws, dist
    return 0, 1, None


def max_over_ranks(ms, dist, device="cuda"):
    """The slowest rank's time: the whole job is done when every replica is."""
    if not dist:
        return ms
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(work_per_rank, world_size, ms):
    """Throughput of the whole job: every rank did work_per_rank units
    (weak scaling) in ms milliseconds; in units per second / 1e9."""
    return world_size * work_per_rank / (ms * 1e-3) / 1e9


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default=DEFAULT, choices=sorted(CONFIGS) + sorted(BATCH_CONFIGS))
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle leg")
    args = ap.parse_args()
    if args.config in BATCH_CONFIGS:
        return run_batch(args)
    kind, size, p, prec, desc = CONFIGS[args.config]
    if args.impl == "reference":
        return run_reference(args, kind, size, p, prec, desc)
    if kind in ("anderson3d", "heat"):
        return run_cheb(args, kind, size, p, prec, desc)

    import torch
    import mpk_inputs as mi
    import paper_2205_01598_gb300 as mpk
    rank, ws, dist = dist_setup(args.gpus)
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    mpk.build()
    mpk.load()

    A = make_matrix(kind, size)
    cfg = mpk_config(desc, A, p, prec)
    flops = 2.0 * A.nnz * p
    rp, cl, va = mpk.csr_to_device(A)
    # the first plan of a process also pays the one-time loading of the
    # library's kernels; the plan that is used (and whose time is reported
    # as the preprocessing cost) is the second
    first = mpk.mpk_plan(rp, cl, va, p, prec=prec)
    first_ms = mpk.mpk_plan_info(first)["plan_ms"]
    del first
    plan = mpk.mpk_plan(rp, cl, va, p, prec=prec)
    info = mpk.mpk_plan_info(plan)
    perm = mpk.mpk_plan_perm(plan)[0]
    vdt = torch.float64 if vec_bytes(prec) == 8 else torch.float32
    x_host = mi.random_vector(A.n, 1234)
    x = torch.from_numpy(x_host).to(vdt).cuda()[perm.long()].contiguous()
    Y = torch.empty(p, A.n, dtype=vdt, device="cuda")
    st = torch.cuda.current_stream()

    # inputs smaller than twice the L2: every timed iteration starts from a
    # flushed L2 (a 256 MB write outside the iteration's events)
    l2 = torch.cuda.get_device_properties(0).L2_cache_size
    ws_bytes = A.nnz * (vec_bytes(prec) + 4) + (p + 1) * A.n * vec_bytes(prec)
    need_flush = ws_bytes <= L2_FLUSH_BELOW or ws_bytes <= 2 * l2
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda") if need_flush else None

    def timed(fn, steps, warmup, sampler=None):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        ctx = sampler if sampler is not None else _Null()
        if flush is None:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with ctx:
                e0.record(st)
                for _ in range(steps):
                    fn()
                e1.record(st)
                torch.cuda.synchronize()
            total = e0.elapsed_time(e1)
        else:
            evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
            with ctx:
                for b, e in evs:
                    flush.fill_(1)
                    b.record(st)
                    fn()
                    e.record(st)
                torch.cuda.synchronize()
            total = sum(b.elapsed_time(e) for b, e in evs)
        if dist:
            dist.barrier()
        return max_over_ranks(total / steps, dist)

    # headline: level-blocked MPK, one persistent launch per step
    sampler = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    ms = timed(lambda: mpk.mpk_run(plan, x, Y, permuted=True, asynchronous=True), args.steps, args.warmup, sampler)
    mpk.mpk_run(plan, x, Y, permuted=True)   # synchronous call: surfaces any device-side error
    value = whole_job_value(flops, ws, ms)
    Y_level = Y.cpu().numpy().astype(np.float64)

    # baseline: p back-to-back SpMVs over the same packed matrix, same GPU
    ms_base = timed(lambda: mpk.mpk_baseline_run(plan, x, Y, permuted=True, asynchronous=True),
                    args.steps, args.warmup)
    base_detail = {"ms_per_step": round(ms_base, 5), "value": round(whole_job_value(flops, ws, ms_base), 3),
                   "gpu_launches_per_step": p}
    if prec == "f64df":
        # the double-float form against both p x SpMV comparators: the same
        # arithmetic (above) and native FP64 SpMVs; the faster one counts
        plan64 = mpk.mpk_plan(rp, cl, va, p, prec="f64")
        perm64 = mpk.mpk_plan_perm(plan64)[0]
        x64 = torch.from_numpy(x_host).cuda()[perm64.long()].contiguous()
        ms_base64 = timed(lambda: mpk.mpk_baseline_run(plan64, x64, Y, permuted=True, asynchronous=True),
                          args.steps, args.warmup)
        base_detail = {"same_arithmetic": base_detail,
                       "native_fp64": {"ms_per_step": round(ms_base64, 5),
                                       "value": round(whole_job_value(flops, ws, ms_base64), 3),
                                       "gpu_launches_per_step": p},
                       "speedup_vs_same_arithmetic": round(ms_base / ms, 4),
                       "speedup_vs_native_fp64": round(ms_base64 / ms, 4)}
        ms_base = min(ms_base, ms_base64)
        del plan64, x64

    # end to end through the C ABI with host buffers (mpk_run_host): x copied
    # in, the MPK in the caller's numbering, every power copied out (the
    # copies overlap the reordering of the next power)
    xh = torch.from_numpy(x_host).to(vdt).pin_memory()
    Yh = torch.empty(p, A.n, dtype=vdt).pin_memory()

    def e2e_step():
        mpk.mpk_run_host(plan, xh, Yh, asynchronous=True)

    ms_e2e = timed(e2e_step, max(3, min(args.steps, 20)), 2)
    value_e2e = whole_job_value(flops, ws, ms_e2e)

    # roofline of the dominant kernel (the wavefront, one launch per step):
    # the one-read algorithmic bytes per launch over the launch time, against
    # the measured HBM copy bandwidth; the FP64 pipe's share beside it,
    # against the FP64 FMA rate measured in this process
    peaks, peak_src = load_peaks()
    traffic = recorded_traffic("k_wave_laplace3d160_p8.md", prec) if (kind, size, p) == ("laplace3d", 160, 8) else None
    alg = one_read_bytes(info["nnz"], A.n, p, prec)
    achieved = alg / (ms * 1e-3) / 1e9
    fp64_rate = fma_rate(mpk, torch, "f64", 1 << 13)
    fp32_rate = fma_rate(mpk, torch, "f32", 1 << 19)
    pipe_rate = fp64_rate if prec == "f64" else fp32_rate   # the double-float form runs on the FP32 pipe
    roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": round(achieved / peaks["hbm_gbs"], 4), "traffic": traffic,
            "peak_source": f"{peak_src} HBM copy bandwidth (MEASURED_PEAKS.json)",
            "algorithmic_bytes_per_launch": int(alg),
            "pipe": {"unit": "TFLOP/s", "achieved": round(flops / (ms * 1e-3) / 1e12, 4),
                     "peak": round(pipe_rate, 4), "frac": round(flops / (ms * 1e-3) / 1e12 / pipe_rate, 4),
                     "peak_source": f"measured in this run: {'FP64' if prec == 'f64' else 'FP32'} FMA-chain probe "
                                    "(mpk_probe_fma), best of 3, CUDA events",
                     "note": ("one FMA (2 flops) per stored entry and power" if prec != "f64df" else
                              "2 flops per stored entry and power counted; the double-float form spends about "
                              "11 FP32-pipe operations on each")}}

    # the two HBM bounds of the method: p back-to-back SpMVs streaming the
    # matrix p times, and one read of the matrix per MPK
    bytes_pxspmv = pxspmv_bytes(info["nnz"], A.n, p, prec)
    gbs = peaks["hbm_gbs"] * 1e9
    bounds = {"pxspmv_hbm_gflops": round(flops / (bytes_pxspmv / gbs) / 1e9, 1),
              "one_read_hbm_gflops": round(flops / (alg / gbs) / 1e9, 1),
              "frac_of_pxspmv_bound": round(value / (flops / (bytes_pxspmv / gbs) / 1e9), 4),
              "frac_of_one_read_bound": round(value / (flops / (alg / gbs) / 1e9), 4),
              "dram_bytes_per_nnz_per_power": round(traffic / (info["nnz"] * p), 3) if traffic else None,
              "hbm_gbs": peaks["hbm_gbs"], "peak_source": peak_src,
              "fp64_fma_tflops_measured": round(fp64_rate, 4), "fp32_fma_tflops_measured": round(fp32_rate, 3)}
    cpu = cpu_omp = err = None
    if rank == 0:
        import oracle
        ref = oracle.mpk(A, x_host, p)
        got = np.empty_like(Y_level)
        got[:, perm.cpu().numpy().astype(np.int64)] = Y_level
        err = [float("%.3e" % e) for e in per_power_errors(got, ref)]
        if not args.no_cpu:
            gf, reps, el = time_oracle(A, x_host, p)
            cpu = {"value": round(gf, 4), "unit": "GFLOP/s", "cores": 1, "kind": "oracle",
                   "sample": f"full matrix, p={p}, {reps} MPK runs in {el:.1f} s (sequential FP64 C)"}
            cpu_omp = time_omp(A, x_host, p)

    clocks = sampler.summary()
    out = {
        "metric": "MPK GFLOP/s (2*nnz*p/t)",
        "value": round(value, 3),
        "unit": "GFLOP/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms, 5),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": {"f64": "f64", "f32": "f32", "f64df": "f32x2", "bf16val": "f32"}[prec],
        "arithmetic": {"f64": "FP64", "f32": "FP32",
                       "bf16val": "FP32 (BF16-exact off-diagonal values widened to FP32, FP32 diagonal)",
                       "f64df": "double-float (pairs of FP32, compensated row sums) on the FP32 pipe; FP64 x and Y, "
                                "every output rounded once to FP64"}[prec],
        "data": "synthetic",
        "config": cfg,
        "error_vs_fp64_oracle": {"per_power": err, "max": max(err) if err else None,
                                 "norm": "relative infinity norm, ||Y_k - A^k x|| / ||A^k x|| per power k"},
        "speedup_vs_pxspmv": round(ms_base / ms, 4),
        "baseline_pxspmv": base_detail,
        "e2e": {"value": round(value_e2e, 3), "unit": "GFLOP/s",
                "h2d_bytes_per_step": A.n * x.element_size(),
                "d2h_bytes_per_step": p * A.n * Y.element_size(), "ms_per_step": round(ms_e2e, 4)},
        "gpu_launches": args.steps * (2 if prec == "f64df" else 1),
        "roofline": roof,
        "bounds": bounds,
        "cpu_baseline": cpu,
        "cpu_pxspmv_openmp": cpu_omp,
        "clocks": clocks,
        "l2_flush": {"flushed": flush is not None, "device_l2_bytes": l2},
        "plan": {"ms": round(info["plan_ms"], 2), "spmv_equiv": round(info["plan_ms"] / (ms_base / p), 1),
                 "phases_ms": {k: round(v, 3) for k, v in zip(mpk.PLAN_PHASES, info["phase_ms"])},
                 "first_plan_of_process_ms": round(first_ms, 2),
                 "levels": info["n_levels"], "groups": info["n_groups"], "tiles": info["n_tiles"],
                 "tile_rows": info["tile_rows"], "grid_ctas": info["grid_ctas"],
                 "cache_bytes": info["cache_bytes"], "matrix_bytes": info["matrix_bytes"]},
    }
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


def batch_config(desc, specs):
    """Config of a batched line (identical in both arms): the matrix count and
    the total rows, right-hand sides and powers of the members."""
    return {"workload": desc, "matrices": len(specs), "rows": int(sum(s[2] for s in specs)),
            "rhs": int(sum(s[3] for s in specs)), "powers": int(sum(s[4] for s in specs)), "data": "synthetic"}


def _gen_batch_member(spec):
    import mpk_inputs as mi
    m, seed, n = spec
    return m, mi.zipf_graph(n, seed)


def run_batch(args):
    """Batched workload: all matrices' MPKs in one persistent launch replayed
    from a CUDA graph; metric = sum_m 2 nnz_m nrhs_m p_m / t."""
    import multiprocessing as mp
    count, n_lo, n_hi, desc = BATCH_CONFIGS[args.config]
    import mpk_inputs as mi
    specs = []
    for m in range(count):
        z = mi.splitmix64(1000 + m, 3)
        n = n_lo + int(z[0] % np.uint64(n_hi - n_lo + 1))
        specs.append((m, 1000 + m, n, 1 + int(z[1] % np.uint64(16)), 2 + int(z[2] % np.uint64(9))))
    # matrices are generated on the host cores before the first CUDA call (spawned workers)
    if args.impl == "reference":
        return run_batch_reference(args, specs, desc, count)
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        mats = dict(pool.map(_gen_batch_member, [(m, seed, n) for m, seed, n, _, _ in specs]))
    t_gen = time.perf_counter() - t0
    import torch
    import paper_2205_01598_gb300 as mpk
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    mpk.build()
    mpk.load()
    from paper_2205_01598_gb300 import planner as pln
    net = pln.Planner.load() if os.path.exists(pln.WEIGHTS) else None
    g8 = pln.grid()
    plans, plans_unsorted, plans_tuned, xs, Ys, flops, nnz_total, rows_total = [], [], [], [], [], 0.0, 0, 0
    options = []
    t0 = time.perf_counter()
    for m, seed, n, nrhs, p in specs:
        A = mats[m]
        rp, cl, va = mpk.csr_to_device(A)
        plan = mpk.mpk_plan(rp, cl, va, p, prec="f32", nrhs=nrhs)
        plans.append(plan)
        plans_unsorted.append(mpk.mpk_plan(rp, cl, va, p, prec="f32", nrhs=nrhs, tune=mpk.MPK_TUNE_NO_SORT))
        # the member's own options: the learned planner's pick from the
        # features of its default plan (the autotuner, searched for this p
        # and width, without weights); the batch runs the work-list schedule,
        # so a resident pick keeps its f and sweep with automatic work items
        if net is not None:
            i = int(net.choose(mpk.mpk_plan_features(plan))[0])
            o = dict(pln.member_options(g8[i], p), source="mlp", grid_index=i)
        else:
            o = pln.plan_options(rp, cl, va, p, prec="f32", nrhs=nrhs, use_weights=False)
        if o["tune"] & mpk.MPK_TUNE_RESIDENT:
            o["tune"] &= ~mpk.MPK_TUNE_RESIDENT
            o["tile_rows"], o["resident_pick"] = 0, True
        options.append(o)
        plans_tuned.append(mpk.mpk_plan(rp, cl, va, p, prec="f32", nrhs=nrhs, tile_rows=o["tile_rows"],
                                        safety_f=o["safety_f"], tune=o["tune"], sweep=o["sweep"]))
        xs.append(torch.rand(A.n, nrhs, dtype=torch.float32, device="cuda"))
        Ys.append(torch.empty(p, A.n, nrhs, dtype=torch.float32, device="cuda"))
        flops += 2.0 * A.nnz * nrhs * p
        nnz_total += A.nnz
        rows_total += A.n
        del rp, cl, va
    t_plan = time.perf_counter() - t0
    batch = mpk.mpk_batch_create(plans_tuned)
    binfo = mpk.mpk_batch_info(batch)
    mpk.mpk_batch_graph_capture(batch, xs, Ys)
    batch_def = mpk.mpk_batch_create(plans)
    mpk.mpk_batch_graph_capture(batch_def, xs, Ys)
    st = torch.cuda.current_stream()

    def timed(fn, steps, warmup, sampler=None):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ctx = sampler if sampler is not None else _Null()
        with ctx:
            e0.record(st)
            for _ in range(steps):
                fn()
            e1.record(st)
            torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    sampler = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    ms = timed(lambda: mpk.mpk_batch_graph_launch(batch, asynchronous=True), args.steps, args.warmup, sampler)
    mpk.mpk_batch_graph_launch(batch)   # synchronous: surfaces device-side errors

    def baseline(ps):
        for plan, x, Y in zip(ps, xs, Ys):
            mpk.mpk_baseline_run(plan, x, Y, permuted=True, asynchronous=True)

    def separate(ps):
        for plan, x, Y in zip(ps, xs, Ys):
            mpk.mpk_run(plan, x, Y, permuted=True, asynchronous=True)

    ms_def = timed(lambda: mpk.mpk_batch_graph_launch(batch_def, asynchronous=True), max(3, args.steps // 4), 2)
    mpk.mpk_batch_graph_launch(batch_def)
    ms_sep = timed(lambda: separate(plans_tuned), max(3, args.steps // 4), 2)
    # the comparator gets the best of the packings (rows sorted by length
    # inside a work item cut padding but scatter single-vector writes; the
    # members' own work-item sizes)
    ms_base = min(timed(lambda: baseline(ps), max(3, args.steps // 4), 2)
                  for ps in (plans, plans_unsorted, plans_tuned))
    kinds = {"one sweep": 0, "two sweeps": 0, "single-power sweeps": 0}
    for o, (_, _, _, _, p) in zip(options, specs):
        kinds["one sweep" if o["sweep"] == p else ("single-power sweeps" if o["sweep"] == 1 else "two sweeps")] += 1
    out = {
        "metric": "batched MPK GFLOP/s (sum 2*nnz*nrhs*p / t)", "value": round(flops / (ms * 1e-3) / 1e9, 3),
        "unit": "GFLOP/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": batch_config(desc, specs),
        "batch": {"nnz": nnz_total, "gen_s": round(t_gen, 1), "plan_s": round(t_plan, 1), "items": binfo["n_items"],
                  "grid_ctas": binfo["grid_ctas"]},
        "speedup_vs_separate_launches": round(ms_sep / ms, 4),
        "speedup_vs_pxspmv": round(ms_base / ms, 4),
        "member_options": {
            "source": options[0]["source"] if options else None,
            "sweep_kinds": kinds, "resident_picks_run_as_work_list": sum(1 for o in options if o.get("resident_pick")),
            "per_member": [[o["tile_rows"], o["safety_f"], o["sweep"]] for o in options],
            "per_member_fields": ["tile_rows (0 = automatic)", "safety_f", "sweep"]},
        "default_options_batch": {"ms_per_step": round(ms_def, 4), "speedup_of_member_options": round(ms_def / ms, 4)},
        "separate_launches": {"ms_per_step": round(ms_sep, 4), "gpu_launches_per_step": count},
        "baseline_pxspmv": {"ms_per_step": round(ms_base, 4),
                            "gpu_launches_per_step": int(sum(s[4] for s in specs))},
        "gpu_launches": args.steps, "clocks": sampler.summary(),
    }
    print(json.dumps(out), flush=True)


def run_cheb(args, kind, size, p, prec, desc):
    """Chebyshev time propagation (Sec. 7): one step = y = sum_k c_k T_k(Ahat) psi
    with M = 64 moments in sweeps of p powers.  Schroedinger (Anderson
    Hamiltonian, complex psi, Bessel coefficients) or heat equation (order-4
    star stencil, real psi, modified-Bessel coefficients); metric = SpMV
    GFLOP/s (2 nnz x columns x M per step, columns = 2 complex / 1 real)."""
    import torch
    import mpk_inputs as mi
    import paper_2205_01598_gb300 as mpk
    rank, ws, dist = dist_setup(args.gpus)
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    mpk.build()
    mpk.load()
    heat = kind == "heat"
    G = 1 if heat else 2
    A = make_matrix(kind, size)
    cfg = cheb_config(desc, A, p, prec)
    flops = 2.0 * A.nnz * G * CHEB_M
    rp, cl, va = mpk.csr_to_device(A)
    plan = mpk.mpk_plan(rp, cl, va, p, prec=prec, nrhs=G)
    info = mpk.mpk_plan_info(plan)
    lo, hi = mpk.mpk_gershgorin(plan)
    if heat:   # -Delta is positive semi-definite: spectrum in [0, hi]
        lo = max(lo, 0.0)
    c, r = (hi + lo) / 2, (hi - lo) / 2
    vdt = torch.float64 if prec == "f64" else torch.float32
    perm = mpk.mpk_plan_perm(plan)[0].long()
    if heat:
        coef = mpk.mpk_cheb_coeffs_heat(CHEB_M, c, r, CHEB_RDT / r)
        psi = mi.random_vector(A.n, 1234)
        xh = psi
        run = mpk.mpk_cheb_real
        y = torch.empty(A.n, dtype=torch.float64, device="cuda")
    else:
        coef = mpk.mpk_cheb_coeffs_schroedinger(CHEB_M, c, r, CHEB_RDT / r)
        psi = mi.uniform(1234, A.n) + 1j * mi.uniform(4321, A.n)
        psi /= np.linalg.norm(psi)
        xh = np.stack([psi.real, psi.imag], 1)
        run = mpk.mpk_cheb
        y = torch.empty(A.n, 2, dtype=torch.float64, device="cuda")
    x = torch.from_numpy(xh).to(vdt).cuda()[perm].contiguous()
    st = torch.cuda.current_stream()

    def timed(fn, steps, warmup, sampler=None):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ctx = sampler if sampler is not None else _Null()
        with ctx:
            e0.record(st)
            for _ in range(steps):
                fn()
            e1.record(st)
            torch.cuda.synchronize()
        if dist:
            dist.barrier()
        return max_over_ranks(e0.elapsed_time(e1) / steps, dist)

    sampler = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    ms = timed(lambda: run(plan, coef, c, r, x, y, permuted=True, asynchronous=True), args.steps, args.warmup, sampler)
    run(plan, coef, c, r, x, y, permuted=True)
    y_gpu = torch.empty_like(y)
    y_gpu[perm] = y
    ms_base = timed(lambda: run(plan, coef, c, r, x, y, permuted=True, asynchronous=True, one_power_per_launch=True),
                    max(3, args.steps // 2), 2)
    # end to end through the C ABI with host buffers (mpk_cheb[_real]_host)
    xh_t = torch.from_numpy(xh).to(vdt).pin_memory()
    yh_t = torch.empty(tuple(y.shape), dtype=torch.float64).pin_memory()
    run_host = mpk.mpk_cheb_real_host if heat else mpk.mpk_cheb_host

    def e2e_step():
        run_host(plan, coef, c, r, xh_t, yh_t, asynchronous=True)

    ms_e2e = timed(e2e_step, max(3, min(args.steps, 10)), 2)
    # roofline of the dominant kernel (the sweep, ceil(M/p) launches per
    # step): the algorithmic bytes of a sweep times the sweeps of a step,
    # over the step time, against the measured HBM copy bandwidth
    peaks, peak_src = load_peaks()
    sweeps = -(-CHEB_M // p)
    alg = sweeps * cheb_sweep_bytes(kind, A.nnz, A.n, prec, G)
    achieved = alg / (ms * 1e-3) / 1e9
    # DRAM bytes of one sweep launch (one ncu capture of the same workload),
    # while the kernel sources are those of the capture
    traffic = recorded_traffic("k_cheb_wave_anderson200_m64.md", prec) if (kind, size) == ("anderson3d", 200) else None
    roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": round(achieved / peaks["hbm_gbs"], 4), "traffic": traffic,
            "traffic_unit": "DRAM bytes (read + write) per sweep launch",
            "algorithmic_bytes_per_launch": int(alg / sweeps),
            "peak_source": f"{peak_src} HBM copy bandwidth (MEASURED_PEAKS.json)",
            "algorithmic_bytes_per_step": int(alg),
            "note": f"{sweeps} sweeps per step; per sweep the matrix once, two state vectors read and two "
                    "written, the FP64 coefficient sum read and written"}
    if prec == "f64":
        fp64_rate = fma_rate(mpk, torch, "f64", 1 << 13)
        tf = 2.0 * A.nnz * G * CHEB_M / (ms * 1e-3) / 1e12
        roof["pipe"] = {"unit": "TFLOP/s", "achieved": round(tf, 4), "peak": round(fp64_rate, 4),
                        "frac": round(tf / fp64_rate, 4),
                        "peak_source": "measured in this run: FP64 FMA-chain probe (mpk_probe_fma)",
                        "note": "SpMV flops only (2 per stored entry, column and power)"}
    cpu, err = None, None
    if rank == 0 and not args.no_cpu:
        import oracle
        t0 = time.perf_counter()
        if heat:
            ref = oracle.cheb_real(A, coef, c, r, psi)
        else:
            ref = oracle.cheb(A, coef, c, r, psi)
        el = time.perf_counter() - t0
        yg = y_gpu.cpu().numpy()
        got = yg if heat else yg[:, 0] + 1j * yg[:, 1]
        err = {"result_relative": float("%.3e" % (np.max(np.abs(got - ref)) / np.max(np.abs(ref)))),
               "input_relative": float("%.3e" % (np.max(np.abs(got - ref)) / np.max(np.abs(psi)))),
               "norm": "infinity norm of y - y_oracle over that of y_oracle (result) and of the input (input)"}
        cpu = {"value": round(flops / el / 1e9, 4), "unit": "GFLOP/s", "cores": 1, "kind": "oracle",
               "sample": f"one full Chebyshev step (M={CHEB_M}) in {el:.1f} s (sequential FP64 C)"}
    out = {
        "metric": "Chebyshev propagation SpMV GFLOP/s (2*nnz*cols*M/t)", "value": round(whole_job_value(flops, ws, ms), 3),
        "unit": "GFLOP/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": {"f64": "f64"}.get(prec, "f32"),
        "data": "synthetic", "config": cfg, "error_vs_fp64_oracle": err,
        "speedup_vs_one_power_per_launch": round(ms_base / ms, 4),
        "baseline_one_power_per_launch": {"ms_per_step": round(ms_base, 4), "gpu_launches_per_step": CHEB_M},
        "e2e": {"value": round(whole_job_value(flops, ws, ms_e2e), 3), "unit": "GFLOP/s",
                "h2d_bytes_per_step": int(np.prod(x.shape)) * xh_t.element_size(),
                "d2h_bytes_per_step": int(np.prod(y.shape)) * 8, "ms_per_step": round(ms_e2e, 4)},
        "gpu_launches": args.steps * (-(-CHEB_M // p) + 2), "roofline": roof, "cpu_baseline": cpu,
        "clocks": sampler.summary(),
        "plan": {"ms": round(info["plan_ms"], 2), "levels": info["n_levels"], "groups": info["n_groups"],
                 "tiles": info["n_tiles"], "val_bytes": info["val_bytes"], "matrix_bytes": info["matrix_bytes"]},
    }
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


class _Null:
    def __enter__(self):
        return self

    def __exit__(self, *a):
        return False


def _reference_line(args, metric, work, el, steps, warm, cfg, sample):
    value = work / el / 1e9
    return {"impl": "reference", "metric": metric, "value": round(value, 4), "unit": "GFLOP/s",
            "n_gpus": int(os.environ.get("WORLD_SIZE", "1")), "steps": steps, "warmup": warm,
            "ms_per_step": round(el / steps * 1e3, 3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": round(value, 4), "unit": "GFLOP/s", "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(value, 4), "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_reference(args, kind, size, p, prec, desc):
    """Reference arm: the FP64 CPU oracle (sequential C) on the host cores,
    rank 0 only; W untimed warm-up steps, then exactly K timed steps, each a
    bounded sample of the workload: one full MPK (MPK configs) or one sweep
    of 8 Chebyshev steps (the first 8 terms of the expansion; Chebyshev
    configs)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import mpk_inputs as mi
    import oracle
    oracle.build()
    A = make_matrix(kind, size)
    cfg = cheb_config(desc, A, p, prec) if kind in ("anderson3d", "heat") else mpk_config(desc, A, p, prec)
    if kind in ("anderson3d", "heat"):
        lo, hi = oracle.gershgorin(A)
        if kind == "heat":   # -Delta is positive semi-definite: spectrum in [0, hi]
            lo = max(lo, 0.0)
        c, r = (hi + lo) / 2, (hi - lo) / 2
        cols, terms = (1 if kind == "heat" else 2), p
        if kind == "heat":
            coef = oracle.cheb_coeffs_heat(CHEB_M, c, r, CHEB_RDT / r)[:terms + 1]
            x = mi.random_vector(A.n, 1234)
            step = lambda: oracle.cheb_real(A, coef, c, r, x)   # noqa: E731
        else:
            coef = oracle.cheb_coeffs_schroedinger(CHEB_M, c, r, CHEB_RDT / r)[:terms + 1]
            x = mi.uniform(1234, A.n) + 1j * mi.uniform(4321, A.n)
            step = lambda: oracle.cheb(A, coef, c, r, x)   # noqa: E731
        work = 2.0 * A.nnz * cols * terms
        metric = "Chebyshev propagation SpMV GFLOP/s (2*nnz*cols*M/t)"
        sample = f"one sweep of {terms} Chebyshev steps (of M={CHEB_M}) of the full workload per step"
    else:
        x = mi.random_vector(A.n, 1234)
        step = lambda: oracle.mpk(A, x, p)   # noqa: E731
        work, metric = 2.0 * A.nnz * p, "MPK GFLOP/s (2*nnz*p/t)"
        sample = f"one full MPK (p={p}) of the workload per step"
    steps, warm = max(1, args.steps), max(0, args.warmup)
    for _ in range(warm):
        step()
    t0 = time.perf_counter()
    for _ in range(steps):
        step()
    el = time.perf_counter() - t0
    out = _reference_line(args, metric, work * steps, el, steps, warm, cfg,
                          f"{steps} timed steps after {warm} warm-up; {sample} (sequential FP64 C)")
    print(json.dumps(out), flush=True)


def run_batch_reference(args, specs, desc, count):
    """Reference arm of the batched workload: the FP64 CPU oracle, rank 0
    only; step i is the MPK of batch member i mod count (its own nrhs and p),
    W untimed warm-up steps, then exactly K timed steps."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import multiprocessing as mp
    import oracle
    import mpk_inputs as mi
    oracle.build()
    steps, warm = max(1, args.steps), max(0, args.warmup)
    used = sorted({i % count for i in range(warm + steps)})
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        mats = dict(pool.map(_gen_batch_member, [(specs[m][0], specs[m][1], specs[m][2]) for m in used]))
    xs = {m: np.stack([mi.random_vector(mats[m].n, 2000 + 17 * m + q) for q in range(specs[m][3])], axis=1)
          for m in used}

    def step(i):
        m = i % count
        oracle.mpk(mats[m], xs[m], specs[m][4])
        return 2.0 * mats[m].nnz * specs[m][3] * specs[m][4]

    for i in range(warm):
        step(i)
    work = 0.0
    t0 = time.perf_counter()
    for i in range(warm, warm + steps):
        work += step(i)
    el = time.perf_counter() - t0
    cfg = batch_config(desc, specs)
    out = _reference_line(args, "batched MPK GFLOP/s (sum 2*nnz*nrhs*p / t)", work, el, steps, warm, cfg,
                          f"{steps} timed steps after {warm} warm-up; step i = the MPK of batch member i mod "
                          f"{count} with its nrhs and p (sequential FP64 C)")
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
