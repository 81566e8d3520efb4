"""FP64 multilayer perceptron for the learned starting guess (oracle; test infrastructure only).

The paper has no learned component; it notes only that the Python implementation suits machine-
learning workflows (PyNOF section). This is the plain reference the GPU kernels are checked
against: x (F) -> relu(W1 x + b1) (H) -> relu(W2 h1 + b2) (H) -> W3 h2 + b3 (O), mean-squared
error over a batch, gradients by back-propagation.

Parameters are packed like the GPU side: W1 [H][F], b1 [H], W2 [H][H], b2 [H], W3 [O][H], b3 [O].
Parity: pinned by central finite differences of the loss in every parameter block.
"""
from __future__ import annotations

import numpy as np


def sizes(F: int, H: int, O: int = 1):
    return [(H, F), (H,), (H, H), (H,), (O, H), (O,)]


def count(F: int, H: int, O: int = 1) -> int:
    return sum(int(np.prod(s)) for s in sizes(F, H, O))


def unpack(theta, F, H, O=1):
    out, k = [], 0
    for s in sizes(F, H, O):
        m = int(np.prod(s))
        out.append(np.asarray(theta[k:k + m], np.float64).reshape(s))
        k += m
    return out


def forward(theta, X, F, H, O=1):
    W1, b1, W2, b2, W3, b3 = unpack(theta, F, H, O)
    Z1 = X @ W1.T + b1
    A1 = np.maximum(Z1, 0.0)
    Z2 = A1 @ W2.T + b2
    A2 = np.maximum(Z2, 0.0)
    Y = A2 @ W3.T + b3
    return Y, (Z1, A1, Z2, A2)


def loss_and_grad(theta, X, T, F, H, O=1):
    """Mean over the batch of sum_o (Y - T)^2 and its gradient (packed like theta)."""
    W1, b1, W2, b2, W3, b3 = unpack(theta, F, H, O)
    Y, (Z1, A1, Z2, A2) = forward(theta, X, F, H, O)
    Bn = X.shape[0]
    R = Y - T
    loss = float(np.sum(R * R) / Bn)
    dY = 2.0 * R / Bn
    gW3 = dY.T @ A2
    gb3 = dY.sum(0)
    dA2 = dY @ W3
    dZ2 = dA2 * (Z2 > 0)
    gW2 = dZ2.T @ A1
    gb2 = dZ2.sum(0)
    dA1 = dZ2 @ W2
    dZ1 = dA1 * (Z1 > 0)
    gW1 = dZ1.T @ X
    gb1 = dZ1.sum(0)
    g = np.concatenate([a.ravel() for a in (gW1, gb1, gW2, gb2, gW3, gb3)])
    return loss, g


def init(F, H, O=1, seed=0):
    """He-style initial weights from the shared input generator's normals."""
    from paper_2512_13550_gb300 import inputs
    parts = []
    k = 0
    for s in sizes(F, H, O):
        m = int(np.prod(s))
        if len(s) == 2:
            parts.append(inputs.normal(seed * 7919 + k, m) * np.sqrt(2.0 / s[1]))
        else:
            parts.append(np.zeros(m))
        k += 1
    return np.concatenate(parts)
