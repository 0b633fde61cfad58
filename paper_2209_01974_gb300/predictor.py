"""Training and use of the learned filter-parameter predictor.

The interval heuristic of fd_solve has three free parameters: the degree
constant c_n (degree = c_n pi / dtheta) and the window margins m_l, m_r.  A
64-128-128-3 perceptron (FP32, GELU; kernels in csrc/fd_mlp.cu) predicts them
from the kernel-polynomial DOS moments of the matrix and the target window
(fd_filter_features).  Labels come from FD runs the library itself makes: for
every training problem, batched solves (fd_solve_batched) over a small grid of
(c_n, m) values record the SpMMV count to reach the tolerance, and the cheapest
grid points, weighted by how close their cost is to the cheapest, give the
label (log c_n, m_l, m_r).  Training runs on the GPU with the
project's forward/backward/Adam kernels (fd_mlp_train_step).

Everything numeric runs in libfd; this module only loops over problems and
grid points and keeps the logs.
"""
import json
import math
import os

import numpy as np

from . import (fd_build_matrix, fd_filter_features, fd_mlp_num_params, fd_mlp_train_step,
               fd_predict_filter_params, fd_solve, fd_solve_batched)

HERE = os.path.dirname(os.path.abspath(__file__))
WEIGHTS = os.path.join(HERE, "predictor_weights.npy")
GRID_CN = (2.0, 2.5, 3.25, 4.0)
GRID_M = (0.25, 0.4, 0.55)


def _uniform(seed, stream, i):
    # counter-based draw for problem generation (SplitMix64 mix of seed/stream/i)
    z = (seed * 0x9E3779B97F4A7C15 + stream * 0xBF58476D1CE4E5B9 + i * 0x94D049BB133111EB) % 2 ** 64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) % 2 ** 64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) % 2 ** 64
    z ^= z >> 31
    return (z >> 11) * 2.0 ** -53


def training_problems(n, seed=1000):
    """Anderson (L 14..22, W 2..16) and Hubbard (8 sites) problems with windows
    inside the spectrum: list of (spec, a, b, n_target, seed)."""
    probs = []
    for k in range(n):
        u = [_uniform(seed, s, k) for s in range(6)]
        if u[0] < 0.7:
            L = 14 + int(9 * u[1])
            W = 2.0 + 14.0 * u[2]
            spec = f"anderson3d:L={L},W={W!r},seed={seed + k}"
            half = 6.0 + W / 2
            c = (u[3] - 0.5) * 0.8 * half
        else:
            nu = 3 + int(2 * u[1])
            U = 2.0 + 6.0 * u[2]
            spec = f"hubbard:n_sites=8,n_up={nu},n_dn={nu},t=1,U={U!r},bc=open"
            c = U * nu * nu / 8.0 + (u[3] - 0.5) * 4.0
        w = 0.02 + 0.1 * u[4]
        nt = (8, 12, 16)[int(3 * u[5])]
        probs.append((spec, c - w, c + w, nt, seed + k))
    return probs


def features(ctx, problems, nb):
    X = []
    for spec, a, b, nt, sd in problems:
        A = fd_build_matrix(ctx, spec)
        ns = nb * math.ceil(4 * nt / nb)
        X.append(fd_filter_features(ctx, A, a, b, nt, nb, ns, sd))
    return np.stack(X)


def label_problems(ctx, problems, nb, degree, tol, max_outer=25, n_max=3000, verbose=False):
    """SpMMV counts on the (c_n, m) grid; returns (labels, cost table, log)."""
    import time
    mats = [fd_build_matrix(ctx, p[0]) for p in problems]
    probs = [(a, b, nt, sd) for (_, a, b, nt, sd) in problems]
    cost = np.full((len(problems), len(GRID_CN), len(GRID_M)), np.inf)
    log = []
    for i, cn in enumerate(GRID_CN):
        for j, m in enumerate(GRID_M):
            t0 = time.time()
            out, res = fd_solve_batched(ctx, mats, probs, nb, degree, tol, raise_noconv=False,
                                        c_n=cn, m_l=m, m_r=m, max_outer=max_outer, n_max=n_max)
            if verbose:
                print(f"grid c_n={cn} m={m}: {sum(r['converged'] for r in res)}/{len(res)} converged "
                      f"in {time.time() - t0:.1f}s", flush=True)
            for k, r in enumerate(res):
                if r["converged"]:
                    cost[k, i, j] = r["n_spmmv"]
                log.append({"problem": k, "c_n": cn, "m": m, "converged": r["converged"],
                            "n_spmmv": r["n_spmmv"], "iterations": r["iterations"],
                            "degree": r["final_degree"]})
    return soft_labels(cost), cost, log


def soft_labels(cost, temperature=0.05):
    """Cost-weighted average of the grid parameters: weight exp(-(c/c_min - 1)/T),
    so grid points within a few percent of the cheapest share the label (the
    SpMMV counts of neighbouring grid points differ by noise of that order)."""
    lc = np.log(np.array(GRID_CN))
    gm = np.array(GRID_M)
    labels = []
    for k in range(cost.shape[0]):
        c = cost[k]
        cmin = c.min()
        if not np.isfinite(cmin):
            labels.append((math.log(4.0), 0.5, 0.5))
            continue
        w = np.where(np.isfinite(c), np.exp(-(c / cmin - 1.0) / temperature), 0.0)
        w /= w.sum()
        x = float(np.sum(w * lc[:, None]))
        m = float(np.sum(w * gm[None, :]))
        labels.append((x, m, m))
    return np.array(labels, dtype=np.float32)


def train(ctx, X, T, steps=3000, lr=2e-3, seed=0, val_frac=0.0):
    """Full-batch Adam on the GPU; returns (params tensor, loss history).  With
    val_frac > 0 a random share of the rows is held back and the parameters with
    the lowest validation loss (checked every 25 steps) are returned."""
    import torch

    from . import fd_mlp_gradient
    rng = np.random.default_rng(seed)
    Xv = Tv = None
    if val_frac > 0:
        perm = rng.permutation(len(X))
        nv = max(1, int(val_frac * len(X)))
        Xv, Tv = X[perm[:nv]], T[perm[:nv]]
        X, T = X[perm[nv:]], T[perm[nv:]]
    sizes = [(64, 128), (128, 128), (128, 3)]
    parts = []
    for i, o in sizes:
        parts.append(rng.standard_normal(i * o) * math.sqrt(2.0 / i))
        parts.append(np.zeros(o))
    p0 = np.concatenate(parts).astype(np.float32)
    assert p0.size == fd_mlp_num_params()
    params = torch.from_numpy(p0).cuda()
    m = torch.zeros_like(params)
    v = torch.zeros_like(params)
    Xd = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).cuda()
    Td = torch.from_numpy(np.ascontiguousarray(T, dtype=np.float32)).cuda()
    hist = []
    best, best_val = params.clone(), float("inf")
    if Xv is not None:
        Xvd = torch.from_numpy(np.ascontiguousarray(Xv, dtype=np.float32)).cuda()
        Tvd = torch.from_numpy(np.ascontiguousarray(Tv, dtype=np.float32)).cuda()
    for k in range(1, steps + 1):
        loss = fd_mlp_train_step(ctx, params, m, v, Xd, Td, k, lr)
        if Xv is not None and k % 25 == 0:
            _, vl = fd_mlp_gradient(ctx, params, Xvd, Tvd)
            if vl < best_val:
                best_val, best = vl, params.clone()
        if k % 100 == 0 or k == 1:
            hist.append((k, loss, best_val if Xv is not None else None))
    return (best if Xv is not None else params), hist


def save(params, path=WEIGHTS):
    np.save(path, params.cpu().numpy())


def load(path=WEIGHTS):
    import torch
    return torch.from_numpy(np.load(path).astype(np.float32)).cuda()


def solve_with(ctx, params, A, a, b, nt, nb, degree, tol, seed=0, **opts):
    """fd_solve with the predicted (c_n, m_l, m_r); the heuristic when params is None.

    The plain heuristic is the fallback twice over: a non-finite network output
    selects it (fd_predict_filter_params), and a learned solve that does not
    converge within max_outer is repeated with it; the returned SpMMV count and
    time then include both runs."""
    ns = nb * math.ceil(4 * nt / nb)
    pred = {"c_n": 4.0, "m_l": 0.5, "m_r": 0.5, "fallback": 1}
    if params is not None:
        f = fd_filter_features(ctx, A, a, b, nt, nb, ns, seed)
        pred = fd_predict_filter_params(ctx, params, f)
    th, rho, res = fd_solve(ctx, A, a, b, nt, nb, degree, tol, seed=seed, raise_noconv=False,
                            c_n=pred["c_n"], m_l=pred["m_l"], m_r=pred["m_r"], **opts)
    if params is not None and not res["converged"]:
        th, rho, r2 = fd_solve(ctx, A, a, b, nt, nb, degree, tol, seed=seed, raise_noconv=False, **opts)
        r2 = dict(r2)
        r2["n_spmmv"] += res["n_spmmv"]
        r2["t_total"] += res["t_total"]
        res = r2
        pred = dict(pred, fallback=2)
    return th, rho, res, pred


def dump_log(path, obj):
    with open(path, "w") as f:
        json.dump(obj, f, indent=1)


def main(argv=None):
    """Generate FD logs on the GPU, train the predictor on them, write the weights."""
    import argparse
    import time

    from . import fd_create
    ap = argparse.ArgumentParser()
    ap.add_argument("--problems", type=int, default=300)
    ap.add_argument("--holdout", type=int, default=40)
    ap.add_argument("--nb", type=int, default=16)
    ap.add_argument("--degree", type=int, default=40)
    ap.add_argument("--tol", type=float, default=1e-9)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--out", default=WEIGHTS)
    ap.add_argument("--log", default=os.path.join(HERE, "predictor_log.json"),
                    help="the training run's metadata (read by the held-out test)")
    ap.add_argument("--runs-log", default="predictor_runs.json",
                    help="every labelling run and held-out solve (large; kept out of the package)")
    a = ap.parse_args(argv)
    ctx = fd_create(0)
    t0 = time.time()
    probs = training_problems(a.problems + a.holdout)
    train_p, hold_p = probs[:a.problems], probs[a.problems:]
    X = features(ctx, probs, a.nb)
    print(f"features of {len(probs)} problems: {time.time() - t0:.1f}s", flush=True)
    T, cost, runs = label_problems(ctx, train_p, a.nb, a.degree, a.tol, verbose=True)
    t_label = time.time() - t0
    ok = np.isfinite(cost.reshape(len(train_p), -1)).any(axis=1)
    print(f"labels: {int(ok.sum())}/{len(train_p)} problems converged somewhere on the grid; "
          f"{time.time() - t0:.1f}s", flush=True)
    params, hist = train(ctx, X[:a.problems][ok], T[ok], steps=a.steps, val_frac=0.2)
    print(f"training loss {hist[0][1]:.4f} -> {hist[-1][1]:.4f}, best validation {hist[-1][2]:.4f}",
          flush=True)
    save(params, a.out)
    # held-out comparison: SpMMV counts of the heuristic and of the predictor
    evals = []
    for (spec, lo, hi, nt, sd) in hold_p:
        A = fd_build_matrix(ctx, spec)
        r0 = solve_with(ctx, None, A, lo, hi, nt, a.nb, a.degree, a.tol, sd, max_outer=40, n_max=3000)
        r1 = solve_with(ctx, params, A, lo, hi, nt, a.nb, a.degree, a.tol, sd, max_outer=40, n_max=3000)
        evals.append({"spec": spec, "window": [lo, hi], "n_target": nt,
                      "heuristic": {"n_spmmv": r0[2]["n_spmmv"], "converged": r0[2]["converged"],
                                    "seconds": r0[2]["t_total"]},
                      "learned": {"n_spmmv": r1[2]["n_spmmv"], "converged": r1[2]["converged"],
                                  "seconds": r1[2]["t_total"], "params": r1[3]}})
    h = sum(e["heuristic"]["n_spmmv"] for e in evals)
    l = sum(e["learned"]["n_spmmv"] for e in evals)
    dump_log(a.log, {"problems": len(train_p), "holdout_problems": len(hold_p), "runs": len(runs),
                     "label_seconds": t_label, "nb": a.nb, "degree": a.degree, "tol": a.tol,
                     "grid": {"c_n": GRID_CN, "m": GRID_M}, "loss": hist,
                     "labelled": int(ok.sum()),
                     "holdout_summary": {"problems": len(evals), "heuristic_spmmv": h, "learned_spmmv": l,
                                         "learned_converged": sum(e["learned"]["converged"] for e in evals)}})
    dump_log(a.runs_log, {"holdout": evals, "runs_log": runs})
    print(f"runs {len(runs)} in {t_label:.1f}s; held-out SpMMVs heuristic {h} learned {l} "
          f"({100 * (1 - l / max(1, h)):.1f}% fewer)")


if __name__ == "__main__":
    main()
