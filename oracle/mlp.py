"""CPU oracle of the source-order MLP -- TEST INFRASTRUCTURE.

Plain numpy in float64: y = w3 . relu(W2 relu(W1 x + b1) + b2) + b3 and the
gradient of L = (1/m) sum (y_i - t_i)^2 by the chain rule written out.  The
parameter vector layout is W1[64][5], b1[64], W2[64][64], b2[64], w3[64], b3.
Weights are first rounded to bfloat16 (round to nearest even) to match the
model the library evaluates.  Pinned by central finite differences in
tests/test_oracle_mlp.py.
"""
from __future__ import annotations

import numpy as np

F, H = 5, 64
P = H * F + H + H * H + H + H + 1


def bf16_round(w: np.ndarray) -> np.ndarray:
    """Round float32 values to bfloat16 (nearest, ties to even), returned as float64."""
    b = np.ascontiguousarray(w, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (b >> 16) & 1
    r = ((b + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(p: np.ndarray):
    p = np.asarray(p, dtype=np.float64)
    i = 0
    W1 = p[i:i + H * F].reshape(H, F); i += H * F
    b1 = p[i:i + H]; i += H
    W2 = p[i:i + H * H].reshape(H, H); i += H * H
    b2 = p[i:i + H]; i += H
    w3 = p[i:i + H]; i += H
    b3 = p[i]
    return W1, b1, W2, b2, w3, b3


def forward(p, x):
    W1, b1, W2, b2, w3, b3 = unpack(p)
    a1 = x @ W1.T + b1
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ W2.T + b2
    h2 = np.maximum(a2, 0.0)
    return h2 @ w3 + b3


def loss(p, x, t):
    y = forward(p, x)
    return float(np.mean((y - t) ** 2))


def gradient(p, x, t):
    """dL/dp in the packed layout."""
    W1, b1, W2, b2, w3, b3 = unpack(p)
    m = x.shape[0]
    a1 = x @ W1.T + b1
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ W2.T + b2
    h2 = np.maximum(a2, 0.0)
    y = h2 @ w3 + b3
    dy = 2.0 * (y - t) / m
    g_w3 = h2.T @ dy
    g_b3 = dy.sum()
    d2 = np.outer(dy, w3) * (a2 > 0)
    g_W2 = d2.T @ h1
    g_b2 = d2.sum(axis=0)
    d1 = (d2 @ W2) * (a1 > 0)
    g_W1 = d1.T @ x
    g_b1 = d1.sum(axis=0)
    return np.concatenate([g_W1.ravel(), g_b1, g_W2.ravel(), g_b2, g_w3, [g_b3]])
