"""Learned Davidson preconditioner, plain numpy FP64 (TEST INFRASTRUCTURE ONLY --
nothing in the GPU product path may import this module).

The diagonal correction t = r / (w - D) of the Davidson method (Sec. III A)
with a learned additive multiplier: t_x = r_x (p_x + m(f_x)), p_x = -1/d_x
(|d_x| clamped to >= 1e-8), d_x = D_x - w, f_x = (d_x, sign(d_x)/max(|d_x|,
0.01), blk_x), m a 3 -> 64 -> 64 -> 1 tanh network with weights W1[64][3],
b1[64], W2[64][64], b2[64], W3[64], b3 (flat, in this order).  Loss over
samples (d, blk, r, t*): L = sum (r (p + m) - t*)^2 / sum t*^2.
"""
from __future__ import annotations

import numpy as np

NF, NH = 3, 64
SIZES = [("W1", (NH, NF)), ("b1", (NH,)), ("W2", (NH, NH)), ("b2", (NH,)), ("W3", (NH,)), ("b3", (1,))]
NW = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(w):
    out, o = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = np.asarray(w[o:o + n], dtype=np.float64).reshape(shape)
        o += n
    return out


def features(d, blk):
    d = np.asarray(d, dtype=np.float64)
    ad = np.abs(d)
    inv = np.where(ad < 0.01, np.where(d < 0, -1.0, 1.0) / 0.01, 1.0 / np.where(ad < 0.01, 1.0, d))
    return np.stack([d, inv, np.asarray(blk, dtype=np.float64)], axis=1)


def diag_mult(d):
    d = np.asarray(d, dtype=np.float64)
    dc = np.where(np.abs(d) < 1e-8, np.where(d < 0, -1e-8, 1e-8), d)
    return -1.0 / dc


def forward(w, f):
    P = unpack(w)
    z1 = f @ P["W1"].T + P["b1"]
    h1 = np.tanh(z1)
    z2 = h1 @ P["W2"].T + P["b2"]
    h2 = np.tanh(z2)
    m = h2 @ P["W3"] + P["b3"][0]
    return m, (h1, h2)


def loss_grad(w, d, blk, r, t):
    """(loss, gradient [NW]) by explicit backpropagation."""
    P = unpack(w)
    f = features(d, blk)
    m, (h1, h2) = forward(w, f)
    r = np.asarray(r, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)
    inv_norm = 1.0 / np.sum(t * t)
    e = r * (diag_mult(d) + m) - t
    loss = np.sum(e * e) * inv_norm
    g = 2.0 * e * r * inv_norm  # dL/dm
    gW3 = g @ h2
    gb3 = np.array([g.sum()])
    g2 = (g[:, None] * P["W3"][None, :]) * (1.0 - h2 * h2)
    gW2 = g2.T @ h1
    gb2 = g2.sum(axis=0)
    g1 = (g2 @ P["W2"]) * (1.0 - h1 * h1)
    gW1 = g1.T @ f
    gb1 = g1.sum(axis=0)
    grad = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3, gb3])
    return loss, grad


def precondition(w, R, omega, D, n1):
    """t = R (p + m) for one residual (the learned Davidson correction)."""
    d = np.asarray(D, dtype=np.float64) - omega
    blk = (np.arange(d.size) < n1).astype(np.float64)
    m, _ = forward(w, features(d, blk))
    return np.asarray(R) * (diag_mult(d) + m)
