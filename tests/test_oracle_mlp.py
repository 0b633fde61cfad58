"""Pins of the MLP oracle: gradients against central finite differences, GELU
against its definition's limits, Adam against its closed form for a constant gradient."""
import numpy as np
import pytest

from oracle import mlp


def test_parameter_count():
    assert mlp.N_PARAMS == 64 * 128 + 128 + 128 * 128 + 128 + 128 * 3 + 3


def test_gelu_limits_and_derivative():
    x = np.linspace(-6, 6, 1201)
    g = mlp.gelu(x)
    assert g[0] == pytest.approx(0.0, abs=1e-7) and g[-1] == pytest.approx(6.0, rel=1e-7)
    assert mlp.gelu(np.array([0.0]))[0] == 0.0
    h = 1e-6
    fd = (mlp.gelu(x + h) - mlp.gelu(x - h)) / (2 * h)
    assert np.abs(fd - mlp.gelu_grad(x)).max() < 1e-8


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(0)
    p = mlp.init(1) * 0.5
    X = rng.standard_normal((7, 64))
    T = rng.standard_normal((7, 3))
    loss, g = mlp.loss_and_grad(p, X, T)
    idx = rng.choice(mlp.N_PARAMS, 60, replace=False)
    idx = np.concatenate([idx, [0, 64 * 128, mlp.N_PARAMS - 1, mlp.N_PARAMS - 4]])
    h = 1e-5
    for i in idx:
        e = np.zeros(mlp.N_PARAMS); e[i] = h
        num = (mlp.loss_and_grad(p + e, X, T)[0] - mlp.loss_and_grad(p - e, X, T)[0]) / (2 * h)
        assert num == pytest.approx(g[i], rel=1e-5, abs=1e-9)


def test_adam_constant_gradient_closed_form():
    # with a constant gradient g the bias-corrected moments are exactly g and g^2,
    # so every step moves each parameter by lr * g / (|g| + eps)
    p = np.zeros(5); g = np.array([1.0, -2.0, 0.5, 3.0, -0.25])
    m = np.zeros(5); v = np.zeros(5)
    for k in range(1, 6):
        p, m, v = mlp.adam(p, g, m, v, k, lr=0.1)
    assert np.allclose(p, -5 * 0.1 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-14)


def test_training_reduces_loss_on_a_learnable_map():
    rng = np.random.default_rng(3)
    X = rng.standard_normal((256, 64))
    Wt = rng.standard_normal((64, 3)) * 0.2
    T = np.tanh(X @ Wt)
    p = mlp.init(2)
    m = np.zeros_like(p); v = np.zeros_like(p)
    l0 = mlp.loss_and_grad(p, X, T)[0]
    for k in range(1, 201):
        l, g = mlp.loss_and_grad(p, X, T)
        p, m, v = mlp.adam(p, g, m, v, k, lr=3e-3)
    assert mlp.loss_and_grad(p, X, T)[0] < 0.1 * l0
