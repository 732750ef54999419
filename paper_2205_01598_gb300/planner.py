"""Learned planner of the level-blocked MPK.

The paper chooses p_m, the cache size C and the recursion depth by search
(Sec. 5, Sec. 6.1).  Here a small multilayer perceptron, given features of a
matrix (computed on the GPU by mpk_plan, see mpk_plan_features), predicts for
every candidate configuration of the autotuner's grid (work-item rows, f of
Eq. 5, and the split of k powers into sweeps) its time relative to the best
candidate, log(t_c / t_best); the planner picks the argmin.  The network is
trained on the GPU with the library's own kernels (mpk_mlp_*) on timings the
autotuner (mpk_autotune) measured on generated matrices.  The autotuner is
the fallback (no weights, or a predicted configuration that fails) and the
yardstick of regret, regret = t(chosen) / t(best) - 1.

A candidate's sweep length for k = 8 powers carries over to an MPK of p
powers by its kind: one sweep of all powers, two sweeps (ceil(p/2)), or
single-power sweeps (member_options); the batch takes each member's options
that way.

Command line (GPU):
  python -m paper_2205_01598_gb300.planner collect --first 10000 --count 2000 --out train.npz
  python -m paper_2205_01598_gb300.planner train --data train.npz --data train_large.npz --out planner_weights.npz
  python -m paper_2205_01598_gb300.planner evaluate --data heldout.npz --weights planner_weights.npz
  python -m paper_2205_01598_gb300.planner collect-headline --out headline.npz
  python -m paper_2205_01598_gb300.planner record --data heldout.npz --data heldout_large.npz --data headline.npz --out planner_eval.json
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time

import numpy as np

from . import MPK_TUNE_RESIDENT, Mlp, csr_to_device, mpk_autotune, mpk_plan, mpk_plan_features, mpk_tune_default_grid

HERE = os.path.dirname(os.path.abspath(__file__))
WEIGHTS = os.path.join(HERE, "planner_weights.npz")
K_POWERS = 8            # the MPK the planner is trained for
HIDDEN = 64
FAMILIES = ("laplace2d", "laplace3d", "box27", "rgg", "zipf")
N_LO, N_HI = 10_000, 2_000_000


# ---------------------------------------------------------------- corpus
def corpus_spec(i: int, n_lo: int = N_LO, n_hi: int = N_HI):
    """Matrix i of the corpus: family i mod 5, N log-uniform in [n_lo, n_hi]
    from SplitMix64 seed i."""
    import mpk_inputs as mi
    u = mi.uniform01(i, 2)
    n = int(round(math.exp(math.log(n_lo) + (math.log(n_hi) - math.log(n_lo)) * u[0])))
    return FAMILIES[i % len(FAMILIES)], n, float(u[1])


def corpus_matrix(i: int, n_lo: int = N_LO, n_hi: int = N_HI):
    """Builds matrix i of the corpus (host CRS)."""
    import mpk_inputs as mi
    fam, n, u = corpus_spec(i, n_lo, n_hi)
    if fam == "laplace2d":
        return mi.laplace2d(max(8, int(round(math.sqrt(n)))))
    if fam == "laplace3d":
        return mi.laplace3d(max(4, int(round(n ** (1 / 3)))))
    if fam == "box27":
        return mi.box27(max(4, int(round(n ** (1 / 3)))))
    if fam == "rgg":
        return mi.random_geometric_graph(n, 2 if u < 0.5 else 3, 8.0 + 22.0 * u, seed=i)
    return mi.zipf_graph(n, i)


def headline_matrix(name: str):
    """The two headline workloads as planner test matrices: the 3D 7-point
    Laplacian on 160^3 and the 3D Anderson Hamiltonian on 200^3 (W = 16.5,
    seed 42)."""
    import mpk_inputs as mi
    if name == "laplace3d-160":
        return mi.laplace3d(160)
    if name == "anderson3d-200":
        return mi.anderson3d(200, W=16.5, seed=42)
    raise ValueError(name)


HEADLINE = ("laplace3d-160", "anderson3d-200")


def _corpus_worker(args):
    i, n_lo, n_hi = args
    return corpus_matrix(i, n_lo, n_hi)


def corpus(indices, n_lo=N_LO, n_hi=N_HI, workers=None, chunk=None):
    """Yields (i, matrix) over `indices`, built on the host cores by a spawned
    pool one chunk ahead of the consumer (bounded host memory: chunks of 32
    matrices up to 2M rows, 8 above)."""
    import multiprocessing as mp
    indices = list(indices)
    chunk = chunk or (32 if n_hi <= 2_000_000 else 8)
    workers = workers or min(16 if n_hi <= 2_000_000 else 8, os.cpu_count() or 1)
    chunks = [indices[s:s + chunk] for s in range(0, len(indices), chunk)]
    with mp.get_context("spawn").Pool(workers) as pool:
        submit = lambda c: pool.map_async(_corpus_worker, [(i, n_lo, n_hi) for i in c])
        pending = submit(chunks[0]) if chunks else None
        for j, c in enumerate(chunks):
            mats = pending.get()
            pending = submit(chunks[j + 1]) if j + 1 < len(chunks) else None
            yield from zip(c, mats)


# ---------------------------------------------------------------- data
def grid():
    return mpk_tune_default_grid(K_POWERS)


def measure(A, prec="f32", min_time_s=0.02):
    """Features and the autotuner's timing of every grid candidate for A."""
    rp, cl, va = csr_to_device(A)
    plan = mpk_plan(rp, cl, va, K_POWERS, prec=prec)
    feats = mpk_plan_features(plan)
    del plan
    best, ms = mpk_autotune(rp, cl, va, K_POWERS, grid(), prec=prec, min_time_s=min_time_s)
    return feats, np.array(ms, dtype=np.float64), best


def collect(first, count, out, n_lo=N_LO, n_hi=N_HI, prec="f32", min_time_s=0.01):
    """Features and grid timings of corpus matrices first .. first+count-1,
    saved to `out` (npz)."""
    F, MS, names, ns = [], [], [], []
    t0 = time.time()
    for i, A in corpus(range(first, first + count), n_lo, n_hi):
        f, ms, _ = measure(A, prec=prec, min_time_s=min_time_s)
        F.append(f)
        MS.append(ms)
        names.append(f"{corpus_spec(i, n_lo, n_hi)[0]}-{A.n}")
        ns.append(A.n)
    np.savez(out, features=np.array(F, dtype=np.float32), ms=np.array(MS), names=np.array(names),
             n=np.array(ns, dtype=np.int64), grid=json.dumps(grid()), seconds=time.time() - t0)
    return out


def targets(ms):
    """Relative log-times log(t_c / t_best) and the mask of candidates that ran."""
    ok = ms > 0
    best = np.where(ok, ms, np.inf).min(1, keepdims=True)
    y = np.where(ok, np.log(np.where(ok, ms, 1.0) / best), 0.0)
    return y.astype(np.float32), ok.astype(np.float32)


# ---------------------------------------------------------------- model
class Planner:
    """Trained network + feature standardisation."""

    def __init__(self, params, mean, std, shape):
        self.params, self.mean, self.std, self.shape = params, mean, std, tuple(int(s) for s in shape)
        self.net = Mlp(*self.shape)
        self.net.set_params(params)

    @classmethod
    def load(cls, path=WEIGHTS):
        d = np.load(path)
        return cls(d["params"], d["mean"], d["std"], d["shape"])

    def save(self, path):
        np.savez(path, params=self.net.get_params(), mean=self.mean, std=self.std, shape=np.array(self.shape))

    def predict(self, feats):
        import torch
        X = (np.atleast_2d(feats) - self.mean) / self.std
        return self.net.forward(torch.from_numpy(X.astype(np.float32)).cuda()).cpu().numpy()

    def choose(self, feats):
        return np.argmin(self.predict(feats), axis=1)


def train(F, MS, epochs=3000, lr=3e-3, batch=128, seed=7):
    """Trains the network on the GPU kernels (mpk_mlp_loss_grad / _adam_step)."""
    import torch
    Y, M = targets(MS)
    mean, std = F.mean(0), F.std(0) + 1e-6
    X = ((F - mean) / std).astype(np.float32)
    shape = (X.shape[1], HIDDEN, Y.shape[1])
    net = Mlp(*shape, seed=seed)
    planner = Planner.__new__(Planner)
    planner.mean, planner.std, planner.shape, planner.net = mean, std, shape, net
    Xd, Yd, Md = (torch.from_numpy(a).cuda() for a in (X, Y, M))
    rng = np.random.default_rng(seed)
    history = []
    for ep in range(epochs):
        idx = torch.from_numpy(rng.permutation(X.shape[0])[:batch]).cuda()
        loss = net.loss_grad(Xd[idx].contiguous(), Yd[idx].contiguous(), Md[idx].contiguous())
        net.adam_step(lr)
        if ep % 100 == 0:
            history.append(loss)
    planner.params = net.get_params()
    return planner, history


def regret(ms, choice):
    """Per-matrix regret t(choice) / t(best) - 1 (a failed choice counts as the worst candidate)."""
    ok = ms > 0
    best = np.where(ok, ms, np.inf).min(1)
    worst = np.where(ok, ms, -np.inf).max(1)
    t = ms[np.arange(ms.shape[0]), choice]
    t = np.where(t > 0, t, worst)
    return t / best - 1.0


def default_index():
    """Grid entry 0 is the library's default options."""
    return 0


def evaluate(planner, F, MS):
    r_mlp = regret(MS, planner.choose(F))
    r_def = regret(MS, np.full(MS.shape[0], default_index()))
    return {"matrices": int(MS.shape[0]), "regret_mlp_mean": float(r_mlp.mean()),
            "regret_mlp_median": float(np.median(r_mlp)), "regret_default_mean": float(r_def.mean()),
            "regret_default_median": float(np.median(r_def)),
            "within_10pct_mlp": float(np.mean(r_mlp <= 0.10)), "within_10pct_default": float(np.mean(r_def <= 0.10))}


def member_options(entry, p, k=K_POWERS):
    """mpk_plan options for p powers from a grid entry tuned for k: the sweep
    kind carries over (all k powers -> all p, ceil(k/2) -> ceil(p/2), one ->
    one)."""
    q = int(entry["p_sweep"])
    sweep = p if q >= k else (1 if q == 1 else (p + 1) // 2)
    return {"tile_rows": int(entry["tile_rows"]), "safety_f": float(entry["safety_f"]),
            "tune": int(entry.get("tune", 0)), "sweep": sweep}


def plan_options(rowptr, col, val, p=K_POWERS, prec="f32", nrhs=1, planner=None, use_weights=True, features=None):
    """Options for the MPK of a matrix with p powers: the network's choice,
    or the autotuner's (searched for p powers) when there is no network or
    the choice fails to plan.  Returns a dict of mpk_plan keyword options
    plus "source" and "grid_index"."""
    if planner is None and use_weights and os.path.exists(WEIGHTS):
        planner = Planner.load()
    if planner is not None:
        if features is None:
            probe = mpk_plan(rowptr, col, val, K_POWERS, prec=prec)
            features = mpk_plan_features(probe)
            del probe
        g = grid()
        i = int(planner.choose(features)[0])
        if 0 <= i < len(g):
            o = member_options(g[i], p)
            try:
                mpk_plan(rowptr, col, val, p, prec=prec, nrhs=nrhs, **o)
                return dict(o, source="mlp", grid_index=i)
            except RuntimeError:
                pass
    g = mpk_tune_default_grid(p)
    best, _ = mpk_autotune(rowptr, col, val, p, g, prec=prec, nrhs=nrhs, min_time_s=0.01)
    return dict(member_options(g[best], p, p), source="autotuner", grid_index=best)


def load_sets(paths):
    """Concatenated features, timings and names of one or more collected sets."""
    F, MS, names = [], [], []
    for path in paths:
        d = np.load(path)
        F.append(d["features"])
        MS.append(d["ms"])
        names += [str(x) for x in d["names"]]
    return np.concatenate(F), np.concatenate(MS), names


def collect_headline(out, min_time_s=0.01):
    """Features and grid timings of the two headline matrices, saved to `out`
    in the format of collect()."""
    F, MS, names, ns = [], [], [], []
    t0 = time.time()
    for name in HEADLINE:
        A = headline_matrix(name)
        f, ms, _ = measure(A, min_time_s=min_time_s)
        F.append(f)
        MS.append(ms)
        names.append(f"{name}-headline")
        ns.append(A.n)
    np.savez(out, features=np.array(F, dtype=np.float32), ms=np.array(MS), names=np.array(names),
             n=np.array(ns, dtype=np.int64), grid=json.dumps(grid()), seconds=time.time() - t0)
    return out


def set_sizes(paths):
    """Rows N of the matrices of collected sets (from the feature log10 N
    where a set does not store them)."""
    out = []
    for path in paths:
        d = np.load(path)
        out.append(d["n"] if "n" in d.files else np.rint(10.0 ** d["features"][:, 0].astype(np.float64)))
    return np.concatenate(out).astype(np.int64)


def record(planner, paths):
    """Evaluation record of the planner on collected sets (held-out corpus
    matrices, the headline matrices): regret per matrix and in summary, split
    at N = 2M."""
    F, MS, names = load_sets(paths)
    choice = planner.choose(F)
    r_mlp = regret(MS, choice)
    r_def = regret(MS, np.full(MS.shape[0], default_index()))
    best_fixed = int(np.argmin(regret_matrix(MS).mean(0)))
    r_fix = regret(MS, np.full(MS.shape[0], best_fixed))
    n = set_sizes(paths)
    rows = [{"matrix": nm, "n": int(nn), "best_ms": float(np.where(m > 0, m, np.inf).min()),
             "chosen": int(c), "chosen_ms": float(m[c]), "regret": float(r)}
            for nm, nn, m, c, r in zip(names, n, MS, choice, r_mlp)]

    def summary(mask):
        if not np.any(mask):
            return None
        return {"matrices": int(mask.sum()), "regret_mlp_mean": float(r_mlp[mask].mean()),
                "regret_mlp_median": float(np.median(r_mlp[mask])),
                "within_10pct_mlp": float(np.mean(r_mlp[mask] <= 0.10)),
                "regret_best_fixed_entry_mean": float(r_fix[mask].mean()),
                "regret_default_mean": float(r_def[mask].mean())}

    return {"grid": grid(), "best_fixed_entry": best_fixed, "data": [os.path.basename(p) for p in paths],
            "all": summary(np.ones(len(n), bool)), "n_up_to_2M": summary(n <= 2_000_000),
            "n_above_2M": summary(n > 2_000_000), "matrices": rows}


def regret_matrix(ms):
    """Regret of every grid entry on every matrix (failed entries: the worst)."""
    return np.stack([regret(ms, np.full(ms.shape[0], j)) for j in range(ms.shape[1])], 1)


def main():
    ap = argparse.ArgumentParser()
    sub = ap.add_subparsers(dest="cmd", required=True)
    c = sub.add_parser("collect")
    c.add_argument("--first", type=int, default=10000)
    c.add_argument("--count", type=int, default=2000)
    c.add_argument("--n-lo", type=int, default=N_LO)
    c.add_argument("--n-hi", type=int, default=N_HI)
    c.add_argument("--out", required=True)
    t = sub.add_parser("train")
    t.add_argument("--data", required=True, action="append")
    t.add_argument("--out", default=WEIGHTS)
    t.add_argument("--epochs", type=int, default=4000)
    e = sub.add_parser("evaluate")
    e.add_argument("--data", required=True, action="append")
    e.add_argument("--weights", default=WEIGHTS)
    h = sub.add_parser("collect-headline")
    h.add_argument("--out", required=True)
    r = sub.add_parser("record")
    r.add_argument("--data", required=True, action="append")
    r.add_argument("--weights", default=WEIGHTS)
    r.add_argument("--out", required=True)
    a = ap.parse_args()
    if a.cmd == "collect":
        collect(a.first, a.count, a.out, n_lo=a.n_lo, n_hi=a.n_hi)
    elif a.cmd == "train":
        F, MS, _ = load_sets(a.data)
        planner, hist = train(F, MS, epochs=a.epochs)
        planner.save(a.out)
        print(json.dumps({"train": evaluate(planner, F, MS), "loss": hist[::5]}))
    elif a.cmd == "collect-headline":
        collect_headline(a.out)
    elif a.cmd == "evaluate":
        F, MS, _ = load_sets(a.data)
        print(json.dumps(evaluate(Planner.load(a.weights), F, MS)))
    else:
        rec = record(Planner.load(a.weights), a.data)
        with open(a.out, "w") as f:
            json.dump(rec, f, indent=1)
        print(json.dumps({k: rec[k] for k in ("all", "n_up_to_2M", "n_above_2M")}))


if __name__ == "__main__":
    main()
