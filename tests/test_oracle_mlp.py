"""Pins of the learned-guess MLP oracle: analytic backprop vs central finite
differences, Adam against its closed-form first step, bf16 rounding."""
import numpy as np

from oracle import mlp


def test_backprop_matches_finite_differences():
    rng = np.random.default_rng(0)
    theta = mlp.init(3)
    theta += 0.05 * rng.standard_normal(theta.size)  # leave the near-zero last layer
    X = rng.standard_normal((40, 16))
    Y = rng.standard_normal((40, 3))
    loss, g = mlp.loss_grad(theta, X, Y)
    idx = rng.choice(theta.size, 60, replace=False)
    for i in idx:
        e = np.zeros_like(theta)
        h = 1e-6 * max(1.0, abs(theta[i]))
        e[i] = h
        fd = (mlp.loss_grad(theta + e, X, Y)[0] - mlp.loss_grad(theta - e, X, Y)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])) + 1e-9, i
    assert mlp.N_PARAMS == 5443


def test_adam_first_step_is_lr_times_sign():
    g = np.array([0.3, -2.0, 1e-3])
    th, m, v = mlp.adam(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, lr=0.01)
    np.testing.assert_allclose(th, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)


def test_bf16_rounding():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 2 ** -7, 3.14159265, -2.5e-3])
    r = mlp.bf16(x)
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1.0 + 2 ** -7  # tie to even, exact
    assert abs(r[3] - 3.140625) < 1e-12
    assert np.all(np.abs(r - x) <= np.abs(x) * 2 ** -8)
