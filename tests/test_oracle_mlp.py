"""Pins of the FP64 cost-model oracle (oracle/mlp.py) that do not use the oracle's
own formulas: finite differences, a hand-built network with a closed-form output,
the variance identity of the mean squared error, and Adam's constant-gradient step."""
import numpy as np
import pytest

from oracle import mlp
from paper_2102_08463_gb300 import workloads as wl


def _theta(seed, scale=0.3):
    return scale * wl.normal(seed, mlp.NPARAM, stream=7)


def _data(seed, B):
    X = wl.uniform01(seed, B * mlp.NFEAT, stream=8).reshape(B, mlp.NFEAT) * 2.0 - 1.0
    T = wl.normal(seed, B, stream=9)
    return X, T


def test_layout_size():
    assert mlp.NPARAM == 64 * 12 + 64 + 64 * 64 + 64 + 64 + 1 == 5057
    th = np.arange(mlp.NPARAM, dtype=np.float64)
    assert np.array_equal(mlp.pack(*mlp.unpack(th)), th)


def test_gradient_matches_central_differences():
    theta = _theta(11)
    X, T = _data(12, 40)
    g = mlp.grad(theta, X, T)
    rng = np.random.default_rng(3)
    # every bias and output weight, plus a sample of the matrix entries
    o1 = 64 * 12
    o2 = o1 + 64 + 64 * 64
    idx = np.concatenate([np.arange(o1, o1 + 64), np.arange(o2, mlp.NPARAM),
                          rng.choice(o1, 60, replace=False),
                          o1 + 64 + rng.choice(64 * 64, 120, replace=False)])
    h = 1e-6
    worst = 0.0
    for i in idx:
        tp = theta.copy()
        tm = theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (mlp.loss(tp, X, T) - mlp.loss(tm, X, T)) / (2 * h)
        worst = max(worst, abs(fd - g[i]) / max(1e-3, abs(g[i])))
    assert worst < 1e-5


def test_closed_form_network():
    # h1 = (relu(x), relu(-x), 0...); the second layer moves unit i of h1 to
    # unit (i + 5) mod 24 (not symmetric, so a transposed W2 fails), and
    # y = sum_k a_k |x_k| + c exactly.
    W1 = np.zeros((64, 12))
    W1[:12] = np.eye(12)
    W1[12:24] = -np.eye(12)
    b1 = np.zeros(64)
    W2 = np.zeros((64, 64))
    for i in range(24):
        W2[(i + 5) % 24, i] = 1.0
    b2 = np.zeros(64)
    a = np.linspace(0.5, 2.0, 12)
    w3 = np.zeros(64)
    for i in range(24):
        w3[(i + 5) % 24] = a[i % 12]
    c = -0.75
    theta = mlp.pack(W1, b1, W2, b2, w3, c)
    X, _ = _data(21, 30)
    y, _ = mlp.forward(theta, X)
    assert np.allclose(y, np.abs(X) @ a + c, rtol=0, atol=1e-13)
    # a transposed first layer would read column k as unit k; check the layout
    X2 = np.zeros((1, 12))
    X2[0, 3] = 2.0
    assert mlp.forward(theta, X2)[0][0] == pytest.approx(2.0 * a[3] + c, abs=1e-14)


def test_constant_network_loss_is_variance():
    X, T = _data(31, 50)
    theta = np.zeros(mlp.NPARAM)
    theta[-1] = np.mean(T)
    assert mlp.loss(theta, X, T) == pytest.approx(np.var(T), rel=1e-13)
    # and its gradient is zero: only b3 could move, and d/db3 = 2 mean(y - T) = 0
    assert np.max(np.abs(mlp.grad(theta, X, T))) < 1e-13


def test_adam_constant_gradient_step():
    g = np.array([0.3, -2.0, 1e-3, 0.0, 5.0])
    th = np.zeros_like(g)
    m = np.zeros_like(g)
    v = np.zeros_like(g)
    lr, eps = 0.01, 1e-8
    for t in range(1, 6):
        new, m, v = mlp.adam_step(th, g, m, v, t, lr, eps=eps)
        step = th - new
        assert np.allclose(step, lr * g / (np.abs(g) + eps), rtol=1e-12, atol=0)
        th = new


def test_training_lowers_loss():
    X, _ = _data(41, 256)
    T = np.sin(2.0 * X[:, 0]) + 0.5 * X[:, 1] ** 2
    theta = _theta(42, 0.2)
    batches = [(X[i:i + 64], T[i:i + 64]) for i in range(0, 256, 64)] * 40
    _, losses = mlp.train_steps(theta, batches, lr=3e-3)
    assert np.mean(losses[-4:]) < 0.2 * np.mean(losses[:4])
