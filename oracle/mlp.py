"""FP64 reference of the learned priority scorer (test infrastructure only).

The network is 8 -> 64 (ReLU) -> 1.  Parameters, in order: W1[64][8]
(row-major), b1[64], w2[64], b2.  The GPU path rounds weights and inputs to
BF16 and accumulates in FP32; this reference takes the same BF16-rounded
weights and inputs and evaluates everything in FP64, so the two differ only
by FP32 accumulation.  With ``bf16=False`` it is the plain FP64 network, which
the finite-difference pins use.
"""
from __future__ import annotations

import numpy as np

N_IN, N_HID = 8, 64
N_PARAMS = N_HID * N_IN + N_HID + N_HID + 1


def bf16(x) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(params, round_bf16: bool = True):
    p = np.asarray(params, dtype=np.float64)
    if round_bf16:
        p = bf16(p)
    o = N_HID * N_IN
    W1 = p[:o].reshape(N_HID, N_IN)
    b1 = p[o:o + N_HID]
    w2 = p[o + N_HID:o + 2 * N_HID]
    b2 = p[o + 2 * N_HID]
    return W1, b1, w2, b2


def forward(params, X, bf16_inputs: bool = True):
    """y = w2 . relu(W1 x + b1) + b2 for every row x of X."""
    W1, b1, w2, b2 = unpack(params, bf16_inputs)
    X = np.asarray(X, dtype=np.float64).reshape(-1, N_IN)
    if bf16_inputs:
        X = bf16(X)
    H = np.maximum(X @ W1.T + b1, 0.0)
    return H @ w2 + b2


def mse_gradients(params, X, y, bf16_inputs: bool = True):
    """Gradient of L = mean_i (net(x_i) - y_i)^2 with respect to the parameters
    (chain rule by hand), and L."""
    W1, b1, w2, b2 = unpack(params, bf16_inputs)
    X = np.asarray(X, dtype=np.float64).reshape(-1, N_IN)
    if bf16_inputs:
        X = bf16(X)
    y = np.asarray(y, dtype=np.float64)
    n = X.shape[0]
    Z = X @ W1.T + b1
    H = np.maximum(Z, 0.0)
    out = H @ w2 + b2
    err = out - y
    dy = 2.0 * err / n                      # dL/d out
    g_w2 = H.T @ dy
    g_b2 = dy.sum()
    dH = np.outer(dy, w2) * (Z > 0)          # back through ReLU
    g_W1 = dH.T @ X
    g_b1 = dH.sum(axis=0)
    grad = np.concatenate([g_W1.ravel(), g_b1, g_w2, [g_b2]])
    return grad, float(np.mean(err ** 2))
