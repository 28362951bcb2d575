"""FP64 reference of the performance-prediction MLP (TEST INFRASTRUCTURE ONLY).

The model the library trains on the GPU, written out with numpy in FP64:
x -> h1 = relu(W1 x + b1) -> h2 = relu(W2 h1 + b2) -> y = W3 h2 + b3 (64 hidden
units per layer), mean squared error L = mean((y - t)^2), its gradient by the
chain rule, and one Adam step (Kingma & Ba 2015: m <- b1 m + (1 - b1) g,
v <- b2 v + (1 - b2) g^2, p <- p - lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)).
The flat parameter order is W1[64][nf], b1[64], W2[64][64], b2[64], W3[64], b3.
Pinned by central finite differences (tests/test_oracle_mlp.py).
"""
from __future__ import annotations

import numpy as np

H = 64


def n_params(nf: int) -> int:
    return H * nf + H + H * H + H + H + 1


def unpack(p: np.ndarray, nf: int):
    p = np.asarray(p, dtype=np.float64)
    o = 0
    W1 = p[o:o + H * nf].reshape(H, nf); o += H * nf
    b1 = p[o:o + H]; o += H
    W2 = p[o:o + H * H].reshape(H, H); o += H * H
    b2 = p[o:o + H]; o += H
    W3 = p[o:o + H]; o += H
    b3 = p[o]
    return W1, b1, W2, b2, W3, b3


def forward(p, X):
    X = np.asarray(X, dtype=np.float64)
    W1, b1, W2, b2, W3, b3 = unpack(p, X.shape[1])
    a1 = X @ W1.T + b1
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ W2.T + b2
    h2 = np.maximum(a2, 0.0)
    return h2 @ W3 + b3, (h1, h2)


def loss(p, X, T) -> float:
    y, _ = forward(p, X)
    return float(np.mean((y - np.asarray(T, dtype=np.float64)) ** 2))


def loss_grad(p, X, T):
    X = np.asarray(X, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    B, nf = X.shape
    W1, b1, W2, b2, W3, b3 = unpack(p, nf)
    y, (h1, h2) = forward(p, X)
    dy = 2.0 * (y - T) / B
    gW3 = h2.T @ dy
    gb3 = dy.sum()
    d2 = np.outer(dy, W3) * (h2 > 0)
    gW2 = d2.T @ h1
    gb2 = d2.sum(axis=0)
    d1 = (d2 @ W2) * (h1 > 0)
    gW1 = d1.T @ X
    gb1 = d1.sum(axis=0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3, [gb3]])
    return float(np.mean((y - T) ** 2)), g


def adam_step(p, g, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    p = p - lr * (m / (1 - b1 ** t)) / (np.sqrt(v / (1 - b2 ** t)) + eps)
    return p, m, v
