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

Command line (GPU):
  python -m paper_2205_01598_gb300.planner collect --first 7000 --count 300 --out data.npz
  python -m paper_2205_01598_gb300.planner train --data data.npz --out planner_weights.npz
  python -m paper_2205_01598_gb300.planner evaluate --data heldout.npz --weights planner_weights.npz
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time

import numpy as np

from . import Mlp, csr_to_device, mpk_autotune, mpk_plan, mpk_plan_features, mpk_tune_default_grid

HERE = os.path.dirname(os.path.abspath(__file__))
WEIGHTS = os.path.join(HERE, "planner_weights.npz")
K_POWERS = 8            # the MPK the planner is trained for
HIDDEN = 64
FAMILIES = ("laplace2d", "laplace3d", "box27", "rgg", "zipf")
N_LO, N_HI = 10_000, 500_000


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


def _corpus_worker(args):
    i, n_lo, n_hi = args
    return corpus_matrix(i, n_lo, n_hi)


def corpus(indices, n_lo=N_LO, n_hi=N_HI, workers=None, chunk=32):
    """Yields (i, matrix) over `indices`, built on the host cores by a spawned
    pool one chunk ahead of the consumer (bounded host memory)."""
    import multiprocessing as mp
    indices = list(indices)
    workers = workers or min(16, os.cpu_count() or 1)
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
    F, MS, names = [], [], []
    t0 = time.time()
    for i, A in corpus(range(first, first + count), n_lo, n_hi):
        f, ms, _ = measure(A, prec=prec, min_time_s=min_time_s)
        F.append(f)
        MS.append(ms)
        names.append(f"{corpus_spec(i, n_lo, n_hi)[0]}-{A.n}")
    np.savez(out, features=np.array(F, dtype=np.float32), ms=np.array(MS), names=np.array(names),
             grid=json.dumps(grid()), seconds=time.time() - t0)
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


def plan_options(rowptr, col, val, prec="f32", planner=None, use_weights=True):
    """Options for the MPK of a matrix: the network's choice, or the
    autotuner's when there is no network or the choice fails to plan."""
    g = grid()
    if planner is None and use_weights and os.path.exists(WEIGHTS):
        planner = Planner.load()
    if planner is not None:
        probe = mpk_plan(rowptr, col, val, K_POWERS, prec=prec)
        i = int(planner.choose(mpk_plan_features(probe))[0])
        del probe
        if 0 <= i < len(g):
            c = g[i]
            try:
                mpk_plan(rowptr, col, val, c["p_sweep"], prec=prec, tile_rows=c["tile_rows"],
                         safety_f=c["safety_f"], tune=c.get("tune", 0))
                return dict(c, source="mlp")
            except RuntimeError:
                pass
    best, _ = mpk_autotune(rowptr, col, val, K_POWERS, g, prec=prec)
    return dict(g[best], source="autotuner")


def main():
    ap = argparse.ArgumentParser()
    sub = ap.add_subparsers(dest="cmd", required=True)
    c = sub.add_parser("collect")
    c.add_argument("--first", type=int, default=7000)
    c.add_argument("--count", type=int, default=300)
    c.add_argument("--n-hi", type=int, default=N_HI)
    c.add_argument("--out", required=True)
    t = sub.add_parser("train")
    t.add_argument("--data", required=True)
    t.add_argument("--out", default=WEIGHTS)
    t.add_argument("--epochs", type=int, default=3000)
    e = sub.add_parser("evaluate")
    e.add_argument("--data", required=True)
    e.add_argument("--weights", default=WEIGHTS)
    a = ap.parse_args()
    if a.cmd == "collect":
        collect(a.first, a.count, a.out, n_hi=a.n_hi)
    elif a.cmd == "train":
        d = np.load(a.data)
        planner, hist = train(d["features"], d["ms"], epochs=a.epochs)
        planner.save(a.out)
        print(json.dumps({"train": evaluate(planner, d["features"], d["ms"]), "loss": hist[::5]}))
    else:
        d = np.load(a.data)
        print(json.dumps(evaluate(Planner.load(a.weights), d["features"], d["ms"])))


if __name__ == "__main__":
    main()
