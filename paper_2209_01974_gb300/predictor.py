"""Training and use of the learned filter-parameter predictor.

The interval heuristic of fd_solve has three free parameters: the degree
constant c_n (degree = c_n pi / dtheta) and the window margins m_l, m_r.  A
64-128-128-3 perceptron (FP32, GELU; kernels in csrc/fd_mlp.cu) predicts them
from the kernel-polynomial DOS moments of the matrix and the target window
(fd_filter_features).  Labels come from FD runs the library itself makes: for
every training problem, batched solves (fd_solve_batched) over a small grid of
(c_n, m) values record the SpMMV count to reach the tolerance, and the cheapest
grid point is the label (log c_n, m_l, m_r).  Training runs on the GPU with the
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
GRID_CN = (2.5, 4.0, 6.0)
GRID_M = (0.3, 0.5, 0.7)


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


def label_problems(ctx, problems, nb, degree, tol, max_outer=40):
    """SpMMV counts on the (c_n, m) grid; returns (labels, cost table, log)."""
    mats = [fd_build_matrix(ctx, p[0]) for p in problems]
    probs = [(a, b, nt, sd) for (_, a, b, nt, sd) in problems]
    cost = np.full((len(problems), len(GRID_CN), len(GRID_M)), np.inf)
    log = []
    for i, cn in enumerate(GRID_CN):
        for j, m in enumerate(GRID_M):
            out, res = fd_solve_batched(ctx, mats, probs, nb, degree, tol, raise_noconv=False,
                                        c_n=cn, m_l=m, m_r=m, max_outer=max_outer)
            for k, r in enumerate(res):
                if r["converged"]:
                    cost[k, i, j] = r["n_spmmv"]
                log.append({"problem": k, "c_n": cn, "m": m, "converged": r["converged"],
                            "n_spmmv": r["n_spmmv"], "iterations": r["iterations"],
                            "degree": r["final_degree"]})
    labels = []
    for k in range(len(problems)):
        i, j = np.unravel_index(np.argmin(cost[k]), cost[k].shape)
        labels.append((math.log(GRID_CN[i]), GRID_M[j], GRID_M[j]))
    return np.array(labels, dtype=np.float32), cost, log


def train(ctx, X, T, steps=3000, lr=2e-3, seed=0):
    """Full-batch Adam on the GPU; returns (params tensor, loss history)."""
    import torch
    rng = np.random.default_rng(seed)
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
    for k in range(1, steps + 1):
        loss = fd_mlp_train_step(ctx, params, m, v, Xd, Td, k, lr)
        if k % 100 == 0 or k == 1:
            hist.append((k, loss))
    return params, hist


def save(params, path=WEIGHTS):
    np.save(path, params.cpu().numpy())


def load(path=WEIGHTS):
    import torch
    return torch.from_numpy(np.load(path).astype(np.float32)).cuda()


def solve_with(ctx, params, A, a, b, nt, nb, degree, tol, seed=0, **opts):
    """fd_solve with the predicted (c_n, m_l, m_r); the heuristic when params is None."""
    ns = nb * math.ceil(4 * nt / nb)
    pred = {"c_n": 4.0, "m_l": 0.5, "m_r": 0.5, "fallback": 1}
    if params is not None:
        f = fd_filter_features(ctx, A, a, b, nt, nb, ns, seed)
        pred = fd_predict_filter_params(ctx, params, f)
    th, rho, res = fd_solve(ctx, A, a, b, nt, nb, degree, tol, seed=seed, raise_noconv=False,
                            c_n=pred["c_n"], m_l=pred["m_l"], m_r=pred["m_r"], **opts)
    return th, rho, res, pred


def dump_log(path, obj):
    with open(path, "w") as f:
        json.dump(obj, f, indent=1)
