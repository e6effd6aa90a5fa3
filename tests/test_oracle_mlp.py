"""Pins of the FP64 warm-start network reference: gradients vs central finite differences."""
import numpy as np

from oracle import mlp


def test_gradients_match_finite_differences():
    n_in, n_h, n_out = 7, 5, 3
    rng = np.random.default_rng(0)
    p = mlp.init_params(n_in, n_h, n_out, 1) + 0.05 * rng.standard_normal(mlp.param_count(n_in, n_h, n_out))
    X = rng.standard_normal((11, n_in))
    T = rng.standard_normal((11, n_out))
    L, g = mlp.loss_and_grad(p, X, T, n_in, n_h, n_out)
    h = 1e-6
    for k in range(p.size):
        e = np.zeros_like(p)
        e[k] = h
        lp, _ = mlp.loss_and_grad(p + e, X, T, n_in, n_h, n_out)
        lm, _ = mlp.loss_and_grad(p - e, X, T, n_in, n_h, n_out)
        assert abs((lp - lm) / (2 * h) - g[k]) < 1e-8


def test_adam_reduces_loss():
    n_in, n_h, n_out = 6, 16, 2
    rng = np.random.default_rng(2)
    X = rng.standard_normal((64, n_in))
    T = np.stack([np.sin(X[:, 0]), X[:, 1] * X[:, 2]], axis=1)
    p = mlp.init_params(n_in, n_h, n_out, 3)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    L0, _ = mlp.loss_and_grad(p, X, T, n_in, n_h, n_out)
    for t in range(1, 301):
        L, g = mlp.loss_and_grad(p, X, T, n_in, n_h, n_out)
        p, m, v = mlp.adam_step(p, g, m, v, t, 1e-2)
    assert L < 0.2 * L0
