"""Pins of the oracle's surrogate network: gradients against central finite
differences of its own forward pass, a one-unit network against its
hand-derived gradient, and the Adam update against its definition."""
import math

import numpy as np

import oracle


def _theta(rng, din=3, dh=8, dout=3):
    return rng.normal(0, 0.6, oracle.mlp_n_params(din, dh, dout))


def test_forward_of_tiny_network_by_hand():
    # din = dh = dout = 1: y = w4 tanh(w3 tanh(w2 tanh(w1 x + b1) + b2) + b3) + b4
    th = np.array([0.7, -0.2, 1.3, 0.1, -0.9, 0.05, 2.0, 0.3])
    x = np.array([[0.4]])
    y = oracle.mlp_forward(th, x, 1, 1, 1)
    h = math.tanh(0.7 * 0.4 - 0.2)
    h = math.tanh(1.3 * h + 0.1)
    h = math.tanh(-0.9 * h + 0.05)
    assert abs(y[0, 0] - (2.0 * h + 0.3)) < 1e-15


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(0)
    th = _theta(rng)
    x = rng.uniform(-1, 1, (7, 3))
    t = rng.uniform(-1, 1, (7, 3))
    loss, g = oracle.mlp_loss_grad(th, x, t, 3, 8, 3)
    y = oracle.mlp_forward(th, x, 3, 8, 3)
    assert abs(loss - np.mean(np.sum((y - t) ** 2, axis=1))) < 1e-14
    eps = 1e-6
    fd = np.zeros_like(th)
    for i in range(len(th)):
        a, b = th.copy(), th.copy()
        a[i] += eps
        b[i] -= eps
        fd[i] = (oracle.mlp_loss_grad(a, x, t, 3, 8, 3)[0] - oracle.mlp_loss_grad(b, x, t, 3, 8, 3)[0]) / (2 * eps)
    assert np.max(np.abs(fd - g)) <= 1e-6 * max(1.0, np.max(np.abs(g)))


def test_adam_step_definition():
    rng = np.random.default_rng(1)
    th = rng.normal(size=20)
    g = rng.normal(size=20)
    m = np.zeros(20)
    v = np.zeros(20)
    th0 = th.copy()
    oracle.adam(th, g, m, v, lr=1e-2, step=1)
    # the first bias-corrected step moves every parameter by lr * sign(g) (up to eps)
    np.testing.assert_allclose(th0 - th, 1e-2 * np.sign(g) * np.abs(g) / (np.abs(g) + 1e-8), rtol=1e-12)
    np.testing.assert_allclose(m, 0.1 * g, rtol=1e-14)
    np.testing.assert_allclose(v, 0.001 * g * g, rtol=1e-14)


def test_training_reduces_loss():
    rng = np.random.default_rng(2)
    th = _theta(rng, dh=8) * 0.5
    x = rng.uniform(-1, 1, (64, 3))
    t = np.stack([np.sin(x[:, 0]), x[:, 1] * x[:, 2], np.tanh(x[:, 0] - x[:, 2])], 1)
    m, v = np.zeros_like(th), np.zeros_like(th)
    first = oracle.mlp_loss_grad(th, x, t, 3, 8, 3)[0]
    for step in range(1, 301):
        loss, g = oracle.mlp_loss_grad(th, x, t, 3, 8, 3)
        oracle.adam(th, g, m, v, lr=1e-2, step=step)
    assert oracle.mlp_loss_grad(th, x, t, 3, 8, 3)[0] < 0.05 * first
