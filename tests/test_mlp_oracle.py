"""Pins for the fp64 MLP reference: backpropagation against central finite differences, the
closed-form gradient of a linear special case, and Adam against a hand-computed first step."""
import numpy as np

from oracle import mlp


def _data(rng, B=32):
    X = rng.standard_normal((B, 16))
    t = rng.standard_normal(B)
    theta = rng.standard_normal(mlp.n_params()) * 0.2
    return theta, X, t


def test_parameter_count():
    assert mlp.n_params() == 16 * 64 + 64 + 64 * 64 + 64 + 64 * 64 + 64 + 64 + 1 == 9473


def test_backprop_matches_finite_differences():
    rng = np.random.default_rng(0)
    theta, X, t = _data(rng)
    _, g = mlp.gradient(theta, X, t)
    idx = rng.choice(theta.size, size=60, replace=False)
    fd = mlp.finite_difference(theta, X, t, idx)
    assert np.allclose(g[idx], fd, rtol=1e-5, atol=1e-8)


def test_linear_special_case_closed_form():
    # one linear layer: L = mean((X w + b - t)^2) -> dL/dw = 2/B X^T r, dL/db = 2/B sum r
    rng = np.random.default_rng(1)
    sizes = (5, 1)
    X = rng.standard_normal((20, 5))
    t = rng.standard_normal(20)
    theta = rng.standard_normal(6)
    r = X @ theta[:5] + theta[5] - t
    _, g = mlp.gradient(theta, X, t, sizes)
    assert np.allclose(g[:5], 2 / 20 * X.T @ r, atol=1e-12)
    assert np.isclose(g[5], 2 / 20 * r.sum(), atol=1e-12)


def test_adam_first_step_is_sign_scaled():
    # with m = v = 0, the first bias-corrected step is lr * g / (|g| + eps) per coordinate
    g = np.array([0.5, -2.0, 1e-3])
    th, m, v = mlp.adam_step(np.zeros(3), np.zeros(3), np.zeros(3), g, 1, lr=0.01)
    assert np.allclose(th, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-9)


def test_planted_sign_error_is_caught():
    rng = np.random.default_rng(2)
    theta, X, t = _data(rng)
    _, g = mlp.gradient(theta, X, t)
    idx = np.arange(0, theta.size, 97)
    fd = mlp.finite_difference(theta, X, t, idx)
    assert not np.allclose(-g[idx], fd, rtol=1e-3, atol=1e-6)
