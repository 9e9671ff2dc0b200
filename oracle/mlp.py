"""CPU oracle for the warm-start network (test infrastructure only).

The network maps per-element features f (F values) to a predicted solution element
(re, im): h1 = tanh(f W1 + b1), h2 = tanh(h1 W2 + b2), y = h2 W3 + b3, with
W1 [F, H], W2 [H, H], W3 [H, 2]. The loss over n rows with targets t is
L = sum (y - t)^2 / n. Forward and the analytic gradients (chain rule written
out) in FP64; ``bf16=True`` rounds the weight matrices to bfloat16 (round to
nearest even) before use, as the GPU forward does, the gradients are then those
of the rounded network.

The parameter vector layout (shared with the C ABI) is W1, b1, W2, b2, W3, b3,
each row-major.
"""
import numpy as np


def shapes(F, H):
    return [(F, H), (H,), (H, H), (H,), (H, 2), (2,)]


def n_params(F, H):
    return F * H + H + H * H + H + 2 * H + 2


def unpack(theta, F, H):
    out, pos = [], 0
    for s in shapes(F, H):
        n = int(np.prod(s))
        out.append(theta[pos:pos + n].reshape(s))
        pos += n
    return out


def bf16_round(a):
    """Round float32 values to bfloat16 (nearest, ties to even), returned as float64."""
    x = np.asarray(a, dtype=np.float32).copy()
    u = x.view(np.uint32)
    lsb = (u >> 16) & 1
    u = ((u + 0x7FFF + lsb) & 0xFFFF0000).astype(np.uint32)
    return u.view(np.float32).astype(np.float64)


def forward(theta, F, H, X, bf16=False):
    W1, b1, W2, b2, W3, b3 = unpack(np.asarray(theta, dtype=np.float64), F, H)
    if bf16:
        W1, W2, W3 = bf16_round(W1), bf16_round(W2), bf16_round(W3)
    h1 = np.tanh(X @ W1 + b1)
    h2 = np.tanh(h1 @ W2 + b2)
    y = h2 @ W3 + b3
    return y, (W1, W2, W3, h1, h2)


def loss_and_grad(theta, F, H, X, T, bf16=False):
    n = X.shape[0]
    y, (W1, W2, W3, h1, h2) = forward(theta, F, H, X, bf16)
    r = y - T
    loss = float(np.sum(r * r) / n)
    dy = 2.0 * r / n
    dW3 = h2.T @ dy
    db3 = dy.sum(0)
    dz2 = (dy @ W3.T) * (1.0 - h2 * h2)
    dW2 = h1.T @ dz2
    db2 = dz2.sum(0)
    dz1 = (dz2 @ W2.T) * (1.0 - h1 * h1)
    dW1 = X.T @ dz1
    db1 = dz1.sum(0)
    g = np.concatenate([dW1.ravel(), db1, dW2.ravel(), db2, dW3.ravel(), db3])
    return loss, g


def init_params(F, H, seed):
    """Glorot-uniform weights, zero biases."""
    rng = np.random.default_rng(seed)
    parts = []
    for s in shapes(F, H):
        if len(s) == 2:
            lim = np.sqrt(6.0 / (s[0] + s[1]))
            parts.append(rng.uniform(-lim, lim, size=s).ravel())
        else:
            parts.append(np.zeros(s))
    return np.concatenate(parts)
