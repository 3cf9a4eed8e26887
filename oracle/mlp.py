"""FP64 reference of the warm-start network (test infrastructure only).

The network maps standardized log-hyperparameters to coefficients on a fixed
Nystrom basis; the warm start of PCG is then x0 = K(X, Z | theta) c, the
initial iterate of Algorithm 1.  Architecture: Linear(in, h1) - tanh -
Linear(h1, h2) - tanh - Linear(h2, out); loss = mean squared error over the
batch and outputs; optimiser Adam (Kingma & Ba 2015) with bias correction.

Parameters are a dict of float64 arrays W1 (h1, in), b1 (h1), W2 (h2, h1),
b2 (h2), W3 (out, h2), b3 (out); y = W x + b.  Initial weights are inputs
(drawn by synthetic.mlp_init), so the GPU and this reference start from the
same point.
"""
from __future__ import annotations

import numpy as np

NAMES = ("W1", "b1", "W2", "b2", "W3", "b3")


def forward(params, X):
    """Returns (output, cache) for a batch X of shape (B, in)."""
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ params["W1"].T + params["b1"]
    a1 = np.tanh(z1)
    z2 = a1 @ params["W2"].T + params["b2"]
    a2 = np.tanh(z2)
    out = a2 @ params["W3"].T + params["b3"]
    return out, (X, a1, a2)


def loss(params, X, T):
    out, _ = forward(params, X)
    return float(np.mean((out - np.asarray(T, dtype=np.float64)) ** 2))


def backward(params, X, T):
    """Gradient of the mean squared error, by the chain rule layer by layer."""
    out, (X, a1, a2) = forward(params, X)
    B, O = out.shape
    d3 = 2.0 * (out - T) / (B * O)
    g = {"W3": d3.T @ a2, "b3": d3.sum(axis=0)}
    d2 = (d3 @ params["W3"]) * (1.0 - a2 ** 2)
    g["W2"] = d2.T @ a1
    g["b2"] = d2.sum(axis=0)
    d1 = (d2 @ params["W2"]) * (1.0 - a1 ** 2)
    g["W1"] = d1.T @ X
    g["b1"] = d1.sum(axis=0)
    return g


def adam_step(params, grads, state, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update in place; state holds m, v per parameter and the step t."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    for k in NAMES:
        m = state.setdefault("m_" + k, np.zeros_like(params[k]))
        v = state.setdefault("v_" + k, np.zeros_like(params[k]))
        m[...] = beta1 * m + (1 - beta1) * grads[k]
        v[...] = beta2 * v + (1 - beta2) * grads[k] ** 2
        mhat = m / (1 - beta1 ** t)
        vhat = v / (1 - beta2 ** t)
        params[k] = params[k] - lr * mhat / (np.sqrt(vhat) + eps)
    return params
