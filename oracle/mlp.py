"""FP64 numpy reference of the tile-proposal network -- TEST INFRASTRUCTURE ONLY.

The network (16 inputs -> 64 ReLU -> 1) is not from the paper; it is the
learned proposal of the exact tile cull.  This module restates, independently
of the CUDA code, (a) its inputs from their definition, (b) the forward pass
with the FP16 roundings the tensor-core kernel applies (inputs, weights and
hidden activations rounded to FP16; accumulation here in FP64), and (c) the
loss gradient of the training kernels (plain FP32/FP64 model, no rounding).
"""
from __future__ import annotations

import math

import numpy as np


def f16(x):
    return np.asarray(x, dtype=np.float64).astype(np.float16).astype(np.float64)


def tile_features(aabb, edge_counts, poses, r_foot):
    """[P, T, 16] inputs for poses [P, 3] and tile AABBs [T, 4] (xmin, ymin,
    xmax, ymax), following the definition in include/psdf.h."""
    ab = np.asarray(aabb, dtype=np.float64)
    ps = np.asarray(poses, dtype=np.float64)
    P, T = len(ps), len(ab)
    corners = np.stack([np.stack([ab[:, 0], ab[:, 1]], 1), np.stack([ab[:, 2], ab[:, 1]], 1),
                        np.stack([ab[:, 2], ab[:, 3]], 1), np.stack([ab[:, 0], ab[:, 3]], 1)],
                       axis=1)                                         # [T, 4, 2]
    out = np.zeros((P, T, 16))
    c = np.cos(ps[:, 2])[:, None, None]
    s = np.sin(ps[:, 2])[:, None, None]
    d = corners[None, :, :, :] - ps[:, None, None, 0:2]               # [P, T, 4, 2]
    lx = c * d[..., 0] + s * d[..., 1]
    ly = -s * d[..., 0] + c * d[..., 1]
    out[:, :, 0:8:2] = 0.1 * np.clip(lx, -20, 20)
    out[:, :, 1:8:2] = 0.1 * np.clip(ly, -20, 20)
    out[:, :, 8:12] = 0.1 * np.minimum(np.hypot(d[..., 0], d[..., 1]), 30)
    gx = np.maximum(np.maximum(ab[None, :, 0] - ps[:, None, 0], ps[:, None, 0] - ab[None, :, 2]), 0)
    gy = np.maximum(np.maximum(ab[None, :, 1] - ps[:, None, 1], ps[:, None, 1] - ab[None, :, 3]), 0)
    out[:, :, 12] = 0.1 * np.minimum(np.hypot(gx, gy), 30)
    out[:, :, 13] = r_foot
    out[:, :, 14] = np.asarray(edge_counts, dtype=np.float64)[None, :] / 256.0
    out[:, :, 15] = 1.0
    return out


def forward_f16(X, W1, w2, b2):
    """Scores with the tensor-core kernel's roundings: FP16 inputs, weights
    and ReLU activations; FP64 accumulation."""
    h = f16(X) @ f16(W1).T
    h = f16(np.maximum(h, 0.0))
    return h @ f16(w2) + float(b2)


def loss_and_grads(X, y, W1, w2, b2):
    """Mean squared error of s = w2 . relu(W1 x) + b2 and its gradients
    (dW1 [64, 16], dw2 [64], db2) -- the quantities the training kernels
    compute."""
    X = np.asarray(X, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    N = len(X)
    a = X @ W1.T                      # [N, 64]
    h = np.maximum(a, 0.0)
    s = h @ w2 + b2
    r = s - y
    loss = float(np.mean(r * r))
    ds = 2.0 * r / N
    dw2 = h.T @ ds
    db2 = float(ds.sum())
    dh = np.outer(ds, w2) * (a > 0)
    dW1 = dh.T @ X
    return loss, dW1, dw2, db2


def init_weights(seed: int):
    """He-normal hidden layer, small output layer (numpy reference init)."""
    g = np.random.default_rng(seed)
    W1 = g.normal(scale=math.sqrt(2.0 / 16), size=(64, 16))
    w2 = g.normal(scale=math.sqrt(1.0 / 64), size=64)
    return W1, w2, 0.0
