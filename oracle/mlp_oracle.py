"""FP64 NumPy oracle of the warm-start network: forward, backward and Adam.

TEST INFRASTRUCTURE ONLY (tests and benchmark baseline); it imports nothing from the CUDA
package.

Network: standardised input x_hat = (x - mu_in) / sd_in, then layers
  h_1 = silu(W_1 x_hat + b_1), h_2 = silu(W_2 h_1 + b_2), y_hat = W_3 h_2 + b_3,
with silu(z) = z / (1 + e^-z); the prediction is y = mu_out + sd_out y_hat and the training
loss is the mean over the batch of (1/2) |y_hat - (t - mu_out)/sd_out|^2 summed over outputs.
The weights W_l are used in BFloat16 (the GPU keeps FP32 master copies and computes with the
BF16-rounded copies), so the oracle rounds them the same way before computing in FP64.
Parameter order of the flattened vector: W_1, b_1, W_2, b_2, W_3, b_3 (row-major W_l, shape
(out, in)).
"""
from __future__ import annotations

import numpy as np


def bf16_round(w):
    """Round FP32 values to BFloat16 (round to nearest even), returned as FP64."""
    a = np.ascontiguousarray(w, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def shapes(n_in, n_hidden, n_out):
    return [(n_hidden, n_in), (n_hidden,), (n_hidden, n_hidden), (n_hidden,), (n_out, n_hidden), (n_out,)]


def unflatten(theta, n_in, n_hidden, n_out):
    out, o = [], 0
    for s in shapes(n_in, n_hidden, n_out):
        k = int(np.prod(s))
        out.append(np.asarray(theta[o:o + k], dtype=np.float64).reshape(s))
        o += k
    return out


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def forward(theta, dims, x_hat):
    W1, b1, W2, b2, W3, b3 = unflatten(theta, *dims)
    W1, W2, W3 = bf16_round(W1), bf16_round(W2), bf16_round(W3)
    z1 = x_hat @ W1.T + b1
    h1 = silu(z1)
    z2 = h1 @ W2.T + b2
    h2 = silu(z2)
    y = h2 @ W3.T + b3
    return y, (x_hat, z1, h1, z2, h2, W1, W2, W3)


def loss_and_grad(theta, dims, x_hat, t_hat):
    """Loss (1/B) sum_b (1/2)|y_hat_b - t_hat_b|^2 and its gradient w.r.t. theta (the BF16
    rounding of the weights is treated as the identity, as in mixed-precision training)."""
    y, (x, z1, h1, z2, h2, W1, W2, W3) = forward(theta, dims, x_hat)
    B = x.shape[0]
    r = y - t_hat
    loss = 0.5 * np.sum(r * r) / B
    dy = r / B
    gW3 = dy.T @ h2
    gb3 = dy.sum(0)
    dz2 = (dy @ W3) * dsilu(z2)
    gW2 = dz2.T @ h1
    gb2 = dz2.sum(0)
    dz1 = (dz2 @ W2) * dsilu(z1)
    gW1 = dz1.T @ x
    gb1 = dz1.sum(0)
    g = np.concatenate([a.reshape(-1) for a in (gW1, gb1, gW2, gb2, gW3, gb3)])
    return loss, g


def adam(theta, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (bias-corrected), step index t >= 1; returns (theta, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
