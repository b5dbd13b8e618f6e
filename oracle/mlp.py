"""Launch-parameter MLP in fp64 numpy -- TEST INFRASTRUCTURE.

The network maps 4 features to 3 regression targets through two hidden
ReLU layers of 64 units:

    z1 = X W1^T + b1,  h1 = relu(z1)
    z2 = h1 W2^T + b2, h2 = relu(z2)
    y  = h2 W3^T + b3

Weights are stored row-major as [out][in].  The loss is the mean of the
squared errors over the batch and the outputs,

    L = 1/(B*O) * sum_{b,o} (y_bo - t_bo)^2,

and relu'(z) is taken as 1 for z > 0 and 0 otherwise.  The optimiser step is
Adam (Kingma and Ba, 2015):

    m <- beta1 m + (1 - beta1) g,   v <- beta2 v + (1 - beta2) g^2,
    theta <- theta - lr * (m / (1 - beta1^t)) / (sqrt(v / (1 - beta2^t)) + eps).

The paper fits its stream models with regression and curve fitting
(Sec. 2.4); this network is the learned replacement that predicts the block
size, the stream count and the chunk size.
"""
from __future__ import annotations

import numpy as np

SHAPES = (("W1", (64, 4)), ("b1", (64,)), ("W2", (64, 64)), ("b2", (64,)), ("W3", (3, 64)),
          ("b3", (3,)))


def init_params(seed=0, dims=(4, 64, 64, 3)):
    rng = np.random.default_rng(seed)
    p = {}
    names = ("1", "2", "3")
    for i, nm in enumerate(names):
        fan_in, fan_out = dims[i], dims[i + 1]
        lim = np.sqrt(6.0 / fan_in)  # He-uniform, suits ReLU
        p["W" + nm] = rng.uniform(-lim, lim, size=(fan_out, fan_in))
        p["b" + nm] = np.zeros(fan_out)
    return p


def forward(p, X):
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ p["W1"].T + p["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(z2, 0.0)
    y = h2 @ p["W3"].T + p["b3"]
    return y, (X, z1, h1, z2, h2)


def loss(p, X, T):
    y, _ = forward(p, X)
    T = np.asarray(T, dtype=np.float64)
    return float(np.mean((y - T) ** 2))


def backward(p, X, T):
    """Returns (loss, grads) with grads keyed like the parameters."""
    y, (X, z1, h1, z2, h2) = forward(p, X)
    T = np.asarray(T, dtype=np.float64)
    B, O = y.shape
    L = float(np.mean((y - T) ** 2))
    dy = 2.0 * (y - T) / (B * O)
    g = {}
    g["W3"] = dy.T @ h2
    g["b3"] = dy.sum(axis=0)
    dh2 = dy @ p["W3"]
    dz2 = dh2 * (z2 > 0.0)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(axis=0)
    dh1 = dz2 @ p["W2"]
    dz1 = dh1 * (z1 > 0.0)
    g["W1"] = dz1.T @ X
    g["b1"] = dz1.sum(axis=0)
    return L, g


def adam_step(p, g, state, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update in place; ``state`` holds m and v per parameter; t >= 1."""
    for k in p:
        m = state.setdefault("m_" + k, np.zeros_like(p[k]))
        v = state.setdefault("v_" + k, np.zeros_like(p[k]))
        m[...] = beta1 * m + (1.0 - beta1) * g[k]
        v[...] = beta2 * v + (1.0 - beta2) * g[k] * g[k]
        mh = m / (1.0 - beta1 ** t)
        vh = v / (1.0 - beta2 ** t)
        p[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)
    return p


def numeric_grad(p, X, T, key, idx, h=1e-6):
    """Central finite difference of the loss in one parameter entry."""
    q = {k: v.copy() for k, v in p.items()}
    q[key][idx] += h
    lp = loss(q, X, T)
    q[key][idx] -= 2 * h
    lm = loss(q, X, T)
    return (lp - lm) / (2 * h)
