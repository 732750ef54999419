"""Cost of the preprocessing (mpk_plan) by phase, as the paper reports the
preprocessing apart from the kernel (Sec. 6.3: its cost in units of SpMV).

  python -m paper_2205_01598_gb300.plancost --matrix laplace3d-160 --p 8 --prec f64 --repeat 3

prints one JSON line: for every repeat the wall time of mpk_plan split into
the phases of mpk_plan_stats.phase_ms (the first repeat also pays the
first-touch costs of the process), and the time of one SpMV of the same plan
(the back-to-back comparator with one power) as the unit.
"""
from __future__ import annotations

import argparse
import json
import time

from . import PLAN_PHASES, csr_to_device, mpk_baseline_run, mpk_plan, mpk_plan_info


def matrix(name: str):
    import mpk_inputs as mi
    kind, size = name.rsplit("-", 1)
    size = int(size)
    makers = {"laplace3d": mi.laplace3d, "laplace2d": mi.laplace2d, "box27": mi.box27,
              "anderson3d": lambda k: mi.anderson3d(k, W=16.5, seed=42),
              "zipf": lambda k: mi.zipf_graph(k, 1000)}
    return makers[kind](size)


def spmv_ms(plan, nrhs=1, reps=20):
    """Mean time of one SpMV (mpk_baseline_run of a p = 1 plan)."""
    import torch
    x = torch.rand(plan.n, nrhs, dtype=plan.vec_dtype, device="cuda").squeeze(1)
    Y = torch.empty((1,) + tuple(x.shape), dtype=plan.vec_dtype, device="cuda")
    for _ in range(3):
        mpk_baseline_run(plan, x, Y, permuted=True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        mpk_baseline_run(plan, x, Y, permuted=True, asynchronous=True)
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--matrix", default="laplace3d-160")
    ap.add_argument("--p", type=int, default=8)
    ap.add_argument("--prec", default="f64")
    ap.add_argument("--repeat", type=int, default=3)
    a = ap.parse_args()
    import torch
    A = matrix(a.matrix)
    rp, cl, va = csr_to_device(A)
    torch.cuda.synchronize()
    runs = []
    for _ in range(a.repeat):
        t0 = time.perf_counter()
        plan = mpk_plan(rp, cl, va, a.p, prec=a.prec)
        wall = (time.perf_counter() - t0) * 1e3
        info = mpk_plan_info(plan)
        runs.append({"wall_ms": round(wall, 3), "plan_ms": round(info["plan_ms"], 3),
                     "phases_ms": {k: round(v, 3) for k, v in zip(PLAN_PHASES, info["phase_ms"])},
                     "levels": info["n_levels"], "tiles": info["n_tiles"]})
        del plan
    unit = spmv_ms(mpk_plan(rp, cl, va, 1, prec=a.prec))
    best = min(r["plan_ms"] for r in runs)
    print(json.dumps({"matrix": a.matrix, "n": A.n, "nnz": int(A.nnz), "p": a.p, "prec": a.prec,
                      "spmv_ms": round(unit, 4), "plan_ms_best": best,
                      "spmv_equivalents_best": round(best / unit, 1), "runs": runs}))


if __name__ == "__main__":
    main()
