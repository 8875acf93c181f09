"""FP64 reference of the learned surrogate: a multilayer perceptron with SiLU hidden
activations, mean-squared error on standardised targets, and Adam.

TEST INFRASTRUCTURE ONLY. The CUDA library never imports it; the tests compare the
library's BF16 tensor-core kernels with it. The surrogate is not part of the paper: it
stands in for the substep loop of one control step (the paper's Section 3.2 dynamics),
predicting the 13-d state change from the state, the four RPMs and the 4 nearest
neighbours' relative positions and velocities.

Everything here is plain numpy in float64 written from the definitions:
  forward   z_l = h_{l-1} W_l^T + b_l,  h_l = silu(z_l) = z_l / (1 + exp(-z_l)) (last layer linear)
  loss      L = mean over rows and outputs of (y - t)^2
  backward  dL/dy = 2 (y - t) / (rows * outputs); dW_l = dz_l^T h_{l-1}; db_l = sum_rows dz_l;
            dh_{l-1} = dz_l W_l; dz_{l-1} = dh_{l-1} * silu'(z_{l-1}),
            silu'(z) = s (1 + z (1 - s)), s = 1 / (1 + exp(-z))
  Adam      (Kingma and Ba, 2015) m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
            w -= lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)
With bf16_storage=True the inputs, weights, hidden activations and backpropagated
pre-activation gradients are rounded to bfloat16 (round to nearest even) where the
kernels store them in bfloat16, so that the comparison isolates accumulation order and
special-function rounding.
"""
from __future__ import annotations

import numpy as np


def bf16(x) -> np.ndarray:
    """Round float values to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    rounded = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return (rounded.astype(np.uint32)).view(np.float32).astype(np.float64)


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def forward(params, x, bf16_storage: bool = False):
    """params: list of (W [out, in], b [out]). Returns (y, cache) with cache = (h list, z list)."""
    h = bf16(x) if bf16_storage else np.asarray(x, dtype=np.float64)
    hs, zs = [h], []
    last = len(params) - 1
    for l, (W, b) in enumerate(params):
        Wl = bf16(W) if bf16_storage else W
        z = h @ Wl.T + b
        zs.append(z)
        if l < last:
            h = silu(z)
            if bf16_storage:
                h = bf16(h)
        else:
            h = z
        hs.append(h)
    return h, (hs, zs)


def mse(y, t) -> float:
    return float(np.mean((np.asarray(y) - np.asarray(t)) ** 2))


def backward(params, cache, y, t, bf16_storage: bool = False):
    """Gradients [(dW, db), ...] of the mean-squared error for one forward pass."""
    hs, zs = cache
    q = bf16 if bf16_storage else (lambda a: a)
    dz = q(2.0 * (y - t) / y.size)
    grads = [None] * len(params)
    for l in range(len(params) - 1, -1, -1):
        W, _ = params[l]
        Wl = bf16(W) if bf16_storage else W
        grads[l] = (dz.T @ hs[l], dz.sum(axis=0))
        if l > 0:
            dz = q((dz @ Wl) * silu_grad(zs[l - 1]))
    return grads


def adam_init(params):
    return [(np.zeros_like(W), np.zeros_like(b)) for W, b in params], \
           [(np.zeros_like(W), np.zeros_like(b)) for W, b in params]


def adam_step(params, grads, m, v, step: int, lr: float, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (step counts from 1). Returns new (params, m, v)."""
    out_p, out_m, out_v = [], [], []
    c1, c2 = 1.0 - b1 ** step, 1.0 - b2 ** step
    for (W, b), (gW, gb), (mW, mb), (vW, vb) in zip(params, grads, m, v):
        new = []
        for p, g, mm, vv in ((W, gW, mW, vW), (b, gb, mb, vb)):
            mm = b1 * mm + (1 - b1) * g
            vv = b2 * vv + (1 - b2) * g * g
            p = p - lr * (mm / c1) / (np.sqrt(vv / c2) + eps)
            new.append((p, mm, vv))
        out_p.append((new[0][0], new[1][0]))
        out_m.append((new[0][1], new[1][1]))
        out_v.append((new[0][2], new[1][2]))
    return out_p, out_m, out_v
