"""Oracle for the learned screen's network (test infrastructure only).

The screen is not part of the paper's method: it decides which disks need the
full indicator of Eq. 3.1. The network is 3 -> 64 -> 64 -> 1 with ReLU hidden
layers and a sigmoid output, evaluated at the BF16 rounding of its FP32
parameters. This module restates it in FP64 NumPy: BF16 rounding from its
definition (keep the upper 16 bits of the IEEE single, round to nearest, ties
to even), the forward pass, the class-weighted binary cross-entropy and its
gradient by the chain rule. Parameter order: W1[64][3], b1[64], W2[64][64],
b2[64], W3[64], b3 (4481 values).
"""
from __future__ import annotations

import numpy as np

H = 64
NPARAM = H * 3 + H + H * H + H + H + 1


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round float32 values to bfloat16 (nearest, ties to even), returned as float32."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = (u + 0x7FFF + lsb) & 0xFFFF0000
    return r.astype(np.uint32).view(np.float32)


def unpack(p: np.ndarray):
    p = np.asarray(p, dtype=np.float64)
    o = 0
    W1 = p[o:o + H * 3].reshape(H, 3); o += H * 3
    b1 = p[o:o + H]; o += H
    W2 = p[o:o + H * H].reshape(H, H); o += H * H
    b2 = p[o:o + H]; o += H
    W3 = p[o:o + H]; o += H
    b3 = p[o]
    return W1, b1, W2, b2, W3, b3


def forward(params32: np.ndarray, X: np.ndarray):
    """Logits and hidden activations at the BF16 rounding of the parameters."""
    W1, b1, W2, b2, W3, b3 = unpack(bf16_round(params32))
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ W1.T + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0.0)
    o = h2 @ W3 + b3
    return o, (z1, h1, z2, h2)


def probability(params32, X):
    o, _ = forward(params32, X)
    return 1.0 / (1.0 + np.exp(-o))


def loss_and_grad(params32, X, y, pos_weight):
    """Mean class-weighted BCE on the logits and its gradient w.r.t. the (rounded) parameters."""
    W1, b1, W2, b2, W3, b3 = unpack(bf16_round(params32))
    X = np.asarray(X, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    o, (z1, h1, z2, h2) = forward(params32, X)
    wgt = np.where(y > 0, pos_weight, 1.0)
    loss = np.mean(wgt * (np.logaddexp(0.0, o) - y * o))
    d_o = wgt * (1.0 / (1.0 + np.exp(-o)) - y) / len(y)
    gW3 = h2.T @ d_o
    gb3 = np.sum(d_o)
    d2 = np.outer(d_o, W3) * (z2 > 0)
    gW2 = d2.T @ h1
    gb2 = d2.sum(axis=0)
    d1 = (d2 @ W2) * (z1 > 0)
    gW1 = d1.T @ X
    gb1 = d1.sum(axis=0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3, [gb3]])
    return loss, g


def init_params(rng: np.random.Generator) -> np.ndarray:
    """He-style initial parameters (float32)."""
    W1 = rng.standard_normal((H, 3)) * np.sqrt(2.0 / 3)
    W2 = rng.standard_normal((H, H)) * np.sqrt(2.0 / H)
    W3 = rng.standard_normal(H) * np.sqrt(1.0 / H)
    p = np.concatenate([W1.ravel(), np.zeros(H), W2.ravel(), np.zeros(H), W3, [0.0]])
    return p.astype(np.float32)
