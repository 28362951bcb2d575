"""Pins of the oracle's MLP gradient and Adam step (no GPU)."""
import numpy as np

from oracle import mlp


def _problem(nf=10, B=40, seed=0):
    rng = np.random.default_rng(seed)
    p = rng.standard_normal(mlp.n_params(nf)) * 0.3
    X = rng.standard_normal((B, nf))
    T = rng.standard_normal(B)
    return p, X, T


def test_gradient_matches_central_differences():
    p, X, T = _problem()
    _, g = mlp.loss_grad(p, X, T)
    rng = np.random.default_rng(1)
    idx = rng.choice(p.size, 60, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        fd = (mlp.loss(p + e, X, T) - mlp.loss(p - e, X, T)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])), i


def test_loss_is_mean_squared_error_of_forward():
    p, X, T = _problem(B=7)
    y, _ = mlp.forward(p, X)
    assert mlp.loss(p, X, T) == np.mean((y - T) ** 2)
    # a single-sample, hand-built net: y = W3 relu(W2 relu(W1 x))
    nf = 2
    q = np.zeros(mlp.n_params(nf))
    W1, b1, W2, b2, W3, b3 = mlp.unpack(q, nf)
    q[:mlp.H * nf].reshape(mlp.H, nf)[0] = [1.0, -1.0]          # unit 0 of layer 1: x0 - x1
    off = mlp.H * nf + mlp.H
    q[off:off + mlp.H * mlp.H].reshape(mlp.H, mlp.H)[0, 0] = 2.0  # unit 0 of layer 2: 2 h1_0
    q[off + mlp.H * mlp.H + mlp.H] = 3.0                           # y = 3 h2_0
    assert mlp.forward(q, np.array([[5.0, 2.0]]))[0][0] == 18.0
    assert mlp.forward(q, np.array([[2.0, 5.0]]))[0][0] == 0.0     # ReLU cuts it


def test_adam_first_step_moves_by_lr_times_sign():
    p = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 1e-3])
    p1, m, v = mlp.adam_step(p, g, np.zeros(3), np.zeros(3), 1, lr=0.01)
    # with bias correction the first step is lr * g / (|g| + eps) ~ lr * sign(g)
    np.testing.assert_allclose(p - p1, 0.01 * np.sign(g), rtol=1e-4)
