"""Test infrastructure only: fp64 CPU reference of the learned merge
priority's training step (the loss, its gradient and an AdamW step), used to
check the CUDA training kernels.  The product path never imports it.

The trainable form is the MLP 16 -> 64 -> 64 -> 1 in floating point on the
scaled features x = f / 256:
    z1 = W1 x + b1, h1 = max(z1, 0), z2 = W2 h1 + b2, h2 = max(z2, 0),
    o = w3 . h2 + b3, loss = mean over rows of BCE(sigmoid(o), y)
with BCE(sigmoid(o), y) = max(o, 0) - o y + log(1 + exp(-|o|)).
Parameters form one flat array: W1[64][16], b1[64], W2[64][64], b2[64],
w3[64], b3 (5313 values).  The gradient is written out by the chain rule,
one layer at a time.
"""
from __future__ import annotations

import numpy as np

NPARAM = 64 * 16 + 64 + 64 * 64 + 64 + 64 + 1
_SPLIT = np.cumsum([64 * 16, 64, 64 * 64, 64, 64])


def unpack(p):
    w1, b1, w2, b2, w3, b3 = np.split(np.asarray(p, dtype=np.float64), _SPLIT)
    return w1.reshape(64, 16), b1, w2.reshape(64, 64), b2, w3, float(b3[0])


def pack(w1, b1, w2, b2, w3, b3):
    return np.concatenate([np.ravel(w1), b1, np.ravel(w2), b2, w3, [b3]]).astype(np.float64)


def bf16(a):
    """a rounded to the nearest bfloat16 (ties to even), from its float32
    value: the top 16 bits of the float32 after adding 0x7FFF plus the lowest
    kept bit (the rounding of the bf16 operands of the tensor-core form)."""
    f = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(p, feat, mixed=False):
    """mixed: the weights W1, W2 and the hidden activations h1 enter the two
    matrix products as bf16 (the tensor-core form); sums stay exact here."""
    w1, b1, w2, b2, w3, b3 = unpack(p)
    x = np.asarray(feat, dtype=np.float64).reshape(-1, 16) / 256.0
    r = bf16 if mixed else (lambda a: a)
    z1 = x @ r(w1).T + b1
    h1 = np.maximum(z1, 0.0)
    z2 = r(h1) @ r(w2).T + b2
    h2 = np.maximum(z2, 0.0)
    o = h2 @ w3 + b3
    return x, z1, h1, z2, h2, o


def loss(p, feat, y):
    o = forward(p, feat)[-1]
    y = np.asarray(y, dtype=np.float64)
    return float(np.mean(np.maximum(o, 0.0) - o * y + np.log1p(np.exp(-np.abs(o))))) if len(y) else 0.0


def loss_and_grad(p, feat, y, mixed=False):
    """Mean loss and its gradient with respect to the flat parameters.
    mixed: the tensor-core form, where every operand of the five matrix
    products (W1, W2, h1, dL/dz2, dL/dz1; x is exact) is rounded to bf16 and
    the bias, w3 and b3 gradients and the output layer stay in full precision."""
    w1, b1, w2, b2, w3, b3 = unpack(p)
    x, z1, h1, z2, h2, o = forward(p, feat, mixed)
    r = bf16 if mixed else (lambda a: a)
    y = np.asarray(y, dtype=np.float64)
    n = len(y)
    if n == 0:
        return 0.0, np.zeros(NPARAM)
    sig = 1.0 / (1.0 + np.exp(-o))
    d_o = (sig - y) / n                      # d loss / d o
    g_w3 = h2.T @ d_o
    g_b3 = d_o.sum()
    d_z2 = np.outer(d_o, w3) * (z2 > 0)      # d loss / d z2
    g_w2 = r(d_z2).T @ r(h1)
    g_b2 = d_z2.sum(axis=0)
    d_z1 = (r(d_z2) @ r(w2)) * (z1 > 0)      # d loss / d z1
    g_w1 = r(d_z1).T @ x
    g_b1 = d_z1.sum(axis=0)
    l = float(np.mean(np.maximum(o, 0.0) - o * y + np.log1p(np.exp(-np.abs(o)))))
    return l, pack(g_w1, g_b1, g_w2, g_b2, g_w3, g_b3)


def adamw_step(p, g, m, v, step, lr, beta1, beta2, eps, wd):
    """One AdamW step (Kingma & Ba 2015; decoupled weight decay,
    Loshchilov & Hutter 2019); returns the new (p, m, v)."""
    p, g, m, v = (np.asarray(a, dtype=np.float64) for a in (p, g, m, v))
    m = beta1 * m + (1 - beta1) * g
    v = beta2 * v + (1 - beta2) * g * g
    mh = m / (1 - beta1 ** step)
    vh = v / (1 - beta2 ** step)
    return p - lr * (mh / (np.sqrt(vh) + eps) + wd * p), m, v


def random_params(seed: int, scale: float = 1.0):
    """He-style uniform initialisation, seeded."""
    r = np.random.default_rng(seed)
    w1 = r.uniform(-1, 1, (64, 16)) * np.sqrt(6 / 16) * scale
    w2 = r.uniform(-1, 1, (64, 64)) * np.sqrt(6 / 64) * scale
    w3 = r.uniform(-1, 1, 64) * np.sqrt(6 / 64) * scale
    return pack(w1, r.uniform(-0.1, 0.1, 64), w2, r.uniform(-0.1, 0.1, 64), w3, 0.05)
