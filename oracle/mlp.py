"""FP64 reference of the local learned smoother network (oracle, test infrastructure).

The network maps the 15-point neighbourhood of s = D^-1 r at a micro-vertex
(centre + 14 lattice neighbours in the order of the stencil directions,
padded with a zero to 16 features) to a correction:
    h1 = relu(W1 x),  h2 = relu(W2 h1),  out = w3 . h2,
with W1 (32 x 16), W2 (32 x 32), w3 (32) and no biases, so N(a s) = a N(s)
for a > 0.  The smoothing step it serves is x <- x + omega s + N(s) and the
training loss on samples (s-neighbourhood X, target t = e - omega s) is the
mean squared error  L = mean_b (out_b - t_b)^2.

``bf16`` rounds to the nearest bfloat16 (ties to even), the rounding the
tensor-core kernels apply to their inputs and weights.

Parity pinned by: finite differences of the loss, homogeneity, and the
closed-form gradient of a one-hidden-unit case (tests).
"""
from __future__ import annotations

import numpy as np

N_IN, N_H = 16, 32


def bf16(a):
    """Round float values to bfloat16 (round to nearest, ties to even); FP64 out."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def init_weights(seed: int, scale: float = 1.0):
    """He-style random weights (W1, W2, w3) from a seeded PCG64 stream (FP64)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    W1 = rng.normal(0, scale * np.sqrt(2.0 / N_IN), size=(N_H, N_IN))
    W2 = rng.normal(0, scale * np.sqrt(2.0 / N_H), size=(N_H, N_H))
    w3 = rng.normal(0, scale * np.sqrt(1.0 / N_H), size=N_H)
    return W1, W2, w3


def forward(W1, W2, w3, X):
    """X (B,16) -> (out (B,), cache)."""
    z1 = X @ W1.T
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2.T
    h2 = np.maximum(z2, 0.0)
    out = h2 @ w3
    return out, (X, z1, h1, z2, h2)


def forward_bf16(W1, W2, w3, X):
    """The network with the rounding points of the BF16 tensor-core kernels:
    inputs, W1, W2 and the first hidden layer rounded to bfloat16, w3 to
    FP32, every sum exact (their FP32 accumulation, emulated in FP64)."""
    Xb = bf16(X)
    z1 = Xb @ bf16(np.asarray(W1, dtype=np.float32)).T
    h1 = bf16(np.maximum(z1, 0.0))
    z2 = h1 @ bf16(np.asarray(W2, dtype=np.float32)).T
    return np.maximum(z2, 0.0) @ np.asarray(w3, dtype=np.float32).astype(np.float64)


def loss_and_grad(W1, W2, w3, X, t):
    """Mean squared error and its gradient by back-propagation."""
    out, (X, z1, h1, z2, h2) = forward(W1, W2, w3, X)
    B = len(t)
    r = out - t
    loss = float(np.mean(r * r))
    g = 2.0 * r / B
    dw3 = h2.T @ g
    dh2 = np.outer(g, w3) * (z2 > 0)
    dW2 = dh2.T @ h1
    dh1 = (dh2 @ W2) * (z1 > 0)
    dW1 = dh1.T @ X
    return loss, dW1, dW2, dw3


def adam_step(params, grads, m, v, step, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015) on lists of arrays, in place."""
    for p, g, mi, vi in zip(params, grads, m, v):
        mi *= b1
        mi += (1 - b1) * g
        vi *= b2
        vi += (1 - b2) * g * g
        mh = mi / (1 - b1 ** step)
        vh = vi / (1 - b2 ** step)
        p -= lr * mh / (np.sqrt(vh) + eps)
