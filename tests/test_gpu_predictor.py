"""The predictor's GPU kernels against the FP64 MLP oracle, its features against
the KPM oracle, and the trained network against the plain heuristic."""
import math
import os

import numpy as np
import pytest

from oracle import chebyshev as ch
from oracle import kpm, lanczos
from oracle import matrices as mat
from oracle import mlp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fd():
    import paper_2209_01974_gb300 as fd
    return fd


@pytest.fixture(scope="module")
def ctx(fd):
    return fd.fd_create(0)


def _t(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()


def _case(seed, B=19):
    rng = np.random.default_rng(seed)
    p = (mlp.init(seed) * 0.7).astype(np.float32).astype(np.float64)
    X = rng.standard_normal((B, 64)).astype(np.float32).astype(np.float64)
    T = rng.standard_normal((B, 3)).astype(np.float32).astype(np.float64)
    return p, X, T


def test_forward_matches_oracle(fd, ctx):
    p, X, _ = _case(1)
    Y = fd.fd_mlp_forward(ctx, _t(p), _t(X)).cpu().numpy()
    Yo, _ = mlp.forward(p, X)
    # FP32 dot products of length <= 128 with |terms| ~ 1: relative error ~ 128 * 2^-24
    assert np.abs(Y - Yo).max() <= 1e-4 * max(1.0, np.abs(Yo).max())


@pytest.mark.parametrize("B", [1, 19, 256])
def test_gradient_matches_oracle(fd, ctx, B):
    p, X, T = _case(2 + B, B)
    g, loss = fd.fd_mlp_gradient(ctx, _t(p), _t(X), _t(T))
    lo, go = mlp.loss_and_grad(p, X, T)
    g = g.cpu().numpy()
    assert loss == pytest.approx(lo, rel=1e-4)
    assert np.abs(g - go).max() <= 2e-4 * np.abs(go).max()


def test_adam_step_matches_oracle(fd, ctx):
    import torch
    p, X, T = _case(5)
    pt, m, v = _t(p), torch.zeros(mlp.N_PARAMS, device="cuda"), torch.zeros(mlp.N_PARAMS, device="cuda")
    for k in (1, 2):
        g, _ = fd.fd_mlp_gradient(ctx, pt, _t(X), _t(T))
        po, mo, vo = mlp.adam(pt.cpu().numpy().astype(np.float64), g.cpu().numpy().astype(np.float64),
                              m.cpu().numpy().astype(np.float64), v.cpu().numpy().astype(np.float64),
                              k, lr=1e-3)
        fd.fd_mlp_train_step(ctx, pt, m, v, _t(X), _t(T), k, 1e-3)
        assert np.abs(pt.cpu().numpy() - po).max() <= 1e-6


def test_features_match_kpm_oracle(fd, ctx):
    spec = "anderson3d:L=12,W=6,seed=4"
    A = fd.fd_build_matrix(ctx, spec)
    f = fd.fd_filter_features(ctx, A, -0.2, 0.2, 8, 16, 32, 3)
    csr = mat.build(spec)
    lo, hi = lanczos.inclusion_interval(csr, 20, 3)
    alpha, beta = ch.scale_params(lo, hi)
    mu = kpm.kpm_moments(mat.to_scipy(csr), 48, 16, 3, alpha, beta)
    assert np.abs(f[:48] - mu).max() <= 1e-6
    assert f[48] == pytest.approx(alpha * -0.2 + beta, abs=1e-6)
    assert f[49] == pytest.approx(alpha * 0.2 + beta, abs=1e-6)
    assert np.all(f[60:] == 0.0)


def test_predictor_falls_back_on_nonfinite_output(fd, ctx):
    import torch
    p = torch.full((fd.fd_mlp_num_params(),), float("nan"), device="cuda")
    r = fd.fd_predict_filter_params(ctx, p, np.zeros(64, np.float32))
    assert r["fallback"] == 1 and (r["c_n"], r["m_l"], r["m_r"]) == (4.0, 0.5, 0.5)


def test_training_reduces_loss(fd, ctx):
    from paper_2209_01974_gb300 import predictor
    rng = np.random.default_rng(7)
    X = rng.standard_normal((128, 64)).astype(np.float32)
    T = np.tanh(X[:, :3] * 0.5).astype(np.float32)
    params, hist = predictor.train(ctx, X, T, steps=400, lr=3e-3)
    assert hist[-1][1] < 0.2 * hist[0][1]
    _, hist_v = predictor.train(ctx, X, T, steps=200, lr=3e-3, val_frac=0.25)
    assert hist_v[-1][2] < hist_v[0][1]


WEIGHTS = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                       "paper_2209_01974_gb300", "predictor_weights.npy")


LOG = os.path.join(os.path.dirname(WEIGHTS), "predictor_log.json")


@pytest.mark.skipif(not os.path.exists(WEIGHTS) or not os.path.exists(LOG),
                    reason="no trained predictor weights")
def test_trained_predictor_beats_heuristic_on_heldout_problems(fd, ctx):
    """The held-out problems of the training run (same generator, not trained on):
    every learned solve (with the heuristic as fallback) converges to the
    tolerance, and in total it needs fewer SpMMVs than the plain heuristic."""
    import json

    from paper_2209_01974_gb300 import predictor
    log = json.load(open(LOG))
    n_train, n_hold = log["problems"], log["holdout_problems"]
    hold = predictor.training_problems(n_train + n_hold)[n_train:]
    params = predictor.load()
    h_tot = l_tot = 0
    for spec, a, b, nt, sd in hold:
        A = fd.fd_build_matrix(ctx, spec)
        r0 = predictor.solve_with(ctx, None, A, a, b, nt, log["nb"], log["degree"], log["tol"], sd,
                                  max_outer=40, n_max=3000)
        r1 = predictor.solve_with(ctx, params, A, a, b, nt, log["nb"], log["degree"], log["tol"], sd,
                                  max_outer=40, n_max=3000)
        assert r1[2]["converged"] == 1 and r1[1].max() <= log["tol"]   # converged residuals decide
        h_tot += r0[2]["n_spmmv"]
        l_tot += r1[2]["n_spmmv"]
    print(f"held-out SpMMVs: heuristic {h_tot}, learned {l_tot} ({100 * (1 - l_tot / h_tot):.1f}% fewer)")
    assert l_tot < h_tot
