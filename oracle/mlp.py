"""FP64 CPU statement of the dispatch MLP (forward, MSE loss, gradients, Adam).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: it checks the CUDA
kernels behind afmm_mlp_forward / afmm_mlp_loss_grad / afmm_mlp_adam and
shares no code with them.  The network (no counterpart in the paper):

    H1 = relu(X W1 + b1),  H2 = relu(H1 W2 + b2),  P = H2 W3 + b3,
    loss = sum M (P - T)^2 / count,

parameters flat and row-major: [W1 (F x H), b1 (H), W2 (H x H), b2 (H),
W3 (H x V), b3 (V)].  Gradients follow the chain rule written out layer by
layer; the pins check them against central finite differences.
"""
from __future__ import annotations

import numpy as np

__all__ = ["unpack", "forward", "loss_and_grads", "adam_step", "param_count"]


def param_count(F: int, H: int, V: int) -> int:
    return F * H + H + H * H + H + H * V + V


def unpack(p, F, H, V):
    p = np.asarray(p, dtype=np.float64)
    o = 0
    W1 = p[o:o + F * H].reshape(F, H); o += F * H
    b1 = p[o:o + H]; o += H
    W2 = p[o:o + H * H].reshape(H, H); o += H * H
    b2 = p[o:o + H]; o += H
    W3 = p[o:o + H * V].reshape(H, V); o += H * V
    b3 = p[o:o + V]; o += V
    assert o == p.size
    return W1, b1, W2, b2, W3, b3


def forward(p, X, F, H, V):
    """Predictions P (rows x V) and the hidden activations."""
    W1, b1, W2, b2, W3, b3 = unpack(p, F, H, V)
    X = np.asarray(X, dtype=np.float64)
    H1 = np.maximum(X @ W1 + b1, 0.0)
    H2 = np.maximum(H1 @ W2 + b2, 0.0)
    return H2 @ W3 + b3, H1, H2


def loss_and_grads(p, X, T, M, count, F, H, V):
    """(loss, flat gradient) of sum M (P - T)^2 / count."""
    W1, b1, W2, b2, W3, b3 = unpack(p, F, H, V)
    X = np.asarray(X, dtype=np.float64)
    P, H1, H2 = forward(p, X, F, H, V)
    D = (P - np.asarray(T, np.float64)) * np.asarray(M, np.float64)
    loss = float(np.sum(D * D) / count)
    dP = 2.0 * D / count
    gW3 = H2.T @ dP
    gb3 = dP.sum(axis=0)
    dH2 = (dP @ W3.T) * (H2 > 0)
    gW2 = H1.T @ dH2
    gb2 = dH2.sum(axis=0)
    dH1 = (dH2 @ W2.T) * (H1 > 0)
    gW1 = X.T @ dH1
    gb1 = dH1.sum(axis=0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return loss, g


def adam_step(p, g, m, v, lr, b1, b2, eps, step):
    """One bias-corrected Adam step; returns new (p, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
