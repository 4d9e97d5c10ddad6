"""FP64 oracle of the tile picker's cost model: a 12 -> 64 -> 64 -> 1 perceptron.

TEST INFRASTRUCTURE ONLY: imported by the tests and by nothing on the product
path.  The cost model is not part of the paper; the paper picks its spreading
method and tiles by hand-tuned rules (Sec. 4.1 remark on bin sizes and M_sub,
and the method recommendations of Sec. 5.4).  What is written here is the plain
textbook definition of each piece:

* network   y(x) = w3 . relu(W2 relu(W1 x + b1) + b2) + b3   (ReLU perceptron)
* loss      L = (1/B) sum_b (y(x_b) - t_b)^2                  (mean squared error)
* gradient  reverse-mode chain rule of L through the three layers
* update    Adam (Kingma and Ba, 2015): m <- b1 m + (1-b1) g, v <- b2 v + (1-b2) g^2,
            theta <- theta - lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)

Flat parameter layout (NPARAM = 5057 numbers, in this order):
  W1[64][12] (row i = hidden unit i), b1[64], W2[64][64] (row j = unit j of the
  second layer), b2[64], w3[64], b3[1].

Pins (tests/test_oracle_mlp.py): the gradient against central finite
differences of the loss; a hand-built network whose output is a closed form
(a weighted sum of |x_k|); the loss of a constant-output network equal to the
variance of the targets; Adam's step under a constant gradient, which bias
correction makes equal to lr g / (|g| + eps) at every step.
"""
from __future__ import annotations

import numpy as np

NFEAT = 12
HIDDEN = 64
NPARAM = HIDDEN * NFEAT + HIDDEN + HIDDEN * HIDDEN + HIDDEN + HIDDEN + 1


def unpack(theta):
    """Views of the flat parameter vector: W1, b1, W2, b2, w3, b3."""
    theta = np.asarray(theta, dtype=np.float64)
    assert theta.shape == (NPARAM,)
    o = 0
    W1 = theta[o:o + HIDDEN * NFEAT].reshape(HIDDEN, NFEAT)
    o += HIDDEN * NFEAT
    b1 = theta[o:o + HIDDEN]
    o += HIDDEN
    W2 = theta[o:o + HIDDEN * HIDDEN].reshape(HIDDEN, HIDDEN)
    o += HIDDEN * HIDDEN
    b2 = theta[o:o + HIDDEN]
    o += HIDDEN
    w3 = theta[o:o + HIDDEN]
    o += HIDDEN
    b3 = theta[o]
    return W1, b1, W2, b2, w3, b3


def pack(W1, b1, W2, b2, w3, b3):
    return np.concatenate([np.ravel(W1), np.ravel(b1), np.ravel(W2), np.ravel(b2),
                           np.ravel(w3), np.atleast_1d(b3)]).astype(np.float64)


def forward(theta, X):
    """Predictions y[B] for inputs X[B][12], and the pre-activations (z1, z2)."""
    W1, b1, W2, b2, w3, b3 = unpack(theta)
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ W1.T + b1                 # [B, 64]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2.T + b2                # [B, 64]
    h2 = np.maximum(z2, 0.0)
    y = h2 @ w3 + b3                   # [B]
    return y, (z1, h1, z2, h2)


def loss(theta, X, T):
    """Mean squared error over the B samples."""
    y, _ = forward(theta, X)
    r = y - np.asarray(T, dtype=np.float64)
    return float(np.mean(r * r))


def grad(theta, X, T):
    """dL/dtheta in the flat layout, by the chain rule layer by layer."""
    W1, b1, W2, b2, w3, b3 = unpack(theta)
    X = np.asarray(X, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    B = X.shape[0]
    y, (z1, h1, z2, h2) = forward(theta, X)
    gy = 2.0 * (y - T) / B             # dL/dy_b
    g_w3 = h2.T @ gy
    g_b3 = np.sum(gy)
    d2 = np.outer(gy, w3) * (z2 > 0)   # dL/dz2 [B, 64]
    g_W2 = d2.T @ h1
    g_b2 = d2.sum(axis=0)
    d1 = (d2 @ W2) * (z1 > 0)          # dL/dz1 [B, 64]
    g_W1 = d1.T @ X
    g_b1 = d1.sum(axis=0)
    return pack(g_W1, g_b1, g_W2, g_b2, g_w3, g_b3)


def adam_step(theta, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update at step t (1-based); returns new (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    theta = theta - lr * mhat / (np.sqrt(vhat) + eps)
    return theta, m, v


def train_steps(theta, batches, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """Adam from zero moments over the given (X, T) minibatches, in order."""
    theta = np.array(theta, dtype=np.float64)
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    losses = []
    for t, (X, T) in enumerate(batches, start=1):
        losses.append(loss(theta, X, T))
        g = grad(theta, X, T)
        theta, m, v = adam_step(theta, g, m, v, t, lr, beta1, beta2, eps)
    return theta, losses
