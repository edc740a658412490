"""Pins of the cost-model oracle (oracle/mlp.py): central finite differences
of the float64 loss, closed forms, and one Adam step worked out by hand."""
import numpy as np

import synth
from oracle import mlp


def _case(in_dim=7, n=50, seed=3):
    p = synth.uniform(seed, (mlp.n_params(in_dim),)) * 0.3
    X = synth.uniform(seed + 1, (n, in_dim))
    y = synth.uniform(seed + 2, (n,))
    return p, X, y


def test_gradient_matches_central_differences():
    p, X, y = _case()
    _, g = mlp.loss_grad(p, X, y, 7)
    rng_idx = (synth.splitmix64(9, 40) % np.uint64(p.size)).astype(int)
    for i in list(rng_idx) + [p.size - 1, 0, 7 * 64 + 3]:
        h = 1e-6
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (mlp.loss_grad(pp, X, y, 7)[0] - mlp.loss_grad(pm, X, y, 7)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), i


def test_zero_weights_closed_form():
    # all weights zero: f(x) = b3, so loss = mean((b3 - y)^2), d/db3 = 2 mean(b3 - y),
    # and the hidden layers see z = b; with b1 = b2 = 0 every ReLU gradient is 0
    in_dim = 5
    p = np.zeros(mlp.n_params(in_dim))
    p[-1] = 0.25
    X = synth.uniform(1, (20, in_dim))
    y = synth.uniform(2, (20,))
    loss, g = mlp.loss_grad(p, X, y, in_dim)
    assert np.isclose(loss, np.mean((0.25 - y) ** 2), rtol=1e-14)
    assert np.isclose(g[-1], 2 * np.mean(0.25 - y), rtol=1e-14)
    assert np.all(g[:-1] == 0)


def test_first_adam_step_moves_each_parameter_by_lr():
    # at t = 1, m/(1-b1) = g and v/(1-b2) = g^2, so the step is lr * g / (|g| + eps)
    p, X, y = _case(in_dim=4, n=16)
    _, g = mlp.loss_grad(p, X, y, 4)
    p1 = mlp.adam_train(p, X, y, 4, steps=1, batch=16, lr=1e-3)
    want = p - 1e-3 * g / (np.abs(g) + 1e-8)
    assert np.allclose(p1, want, rtol=0, atol=1e-15)


def test_training_reduces_loss():
    p, X, y = _case(in_dim=6, n=256)
    p = p * 0.3
    l0 = mlp.loss_grad(p, X, y, 6)[0]
    p2 = mlp.adam_train(p, X, y, 6, steps=200, batch=64, lr=3e-3)
    assert mlp.loss_grad(p2, X, y, 6)[0] < 0.5 * l0
