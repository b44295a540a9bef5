"""FP64 oracle of the learned preconditioning stage (test infrastructure).

The paper has no learned component; this stage is the build's addition,
used inside the flexible outer Krylov method (Sec. 4: FGMRES accepts a
preconditioner that changes from step to step).  The network is a plain
stack of 3x3 convolutions with zero padding and ReLU between layers:

    y_0 = x,  y_l = relu(conv(y_{l-1}; W_l, b_l))  (l < L),  y_L = conv(y_{L-1}; W_L, b_L)

Tensors are NHWC: x[b, i, j, c] with i the depth row and j the lateral
column of the node grid; weights W[co, dy, dx, ci] with the 3x3 taps
(dy, dx) in {0, 1, 2}^2 read at offset (dy-1, dx-1), i.e. a correlation:

    conv(x)[b, i, j, co] = bias[co] + sum_{dy, dx, ci} W[co, dy, dx, ci] x[b, i+dy-1, j+dx-1, ci]

(x = 0 outside the image).  ``backward`` writes the chain rule out layer by
layer.  Pinned by tests against scipy.signal.correlate2d and by central
finite differences.
"""
from __future__ import annotations

import numpy as np


def conv3x3(x: np.ndarray, W: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Direct summation over the nine taps (definition above)."""
    B, H, Wd, _ = x.shape
    Co = W.shape[0]
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0)))
    y = np.zeros((B, H, Wd, Co)) + b
    for dy in range(3):
        for dx in range(3):
            y += np.einsum("bhwc,oc->bhwo", xp[:, dy:dy + H, dx:dx + Wd, :], W[:, dy, dx, :])
    return y


def conv3x3_input_grad(gy: np.ndarray, W: np.ndarray) -> np.ndarray:
    """d(sum gy * conv(x)) / dx: each output (i, j) received x[i+dy-1, j+dx-1]
    with weight W[., dy, dx, .], so the gradient scatters gy back along the
    same taps."""
    B, H, Wd, _ = gy.shape
    Ci = W.shape[3]
    gx = np.zeros((B, H + 2, Wd + 2, Ci))
    for dy in range(3):
        for dx in range(3):
            gx[:, dy:dy + H, dx:dx + Wd, :] += np.einsum("bhwo,oc->bhwc", gy, W[:, dy, dx, :])
    return gx[:, 1:-1, 1:-1, :]


def conv3x3_weight_grad(x: np.ndarray, gy: np.ndarray):
    """(dW, db) of sum(gy * conv(x; W, b))."""
    B, H, Wd, Ci = x.shape
    Co = gy.shape[3]
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0)))
    dW = np.zeros((Co, 3, 3, Ci))
    for dy in range(3):
        for dx in range(3):
            dW[:, dy, dx, :] = np.einsum("bhwo,bhwc->oc", gy, xp[:, dy:dy + H, dx:dx + Wd, :])
    return dW, gy.sum(axis=(0, 1, 2))


def forward(x, params):
    """params: list of (W, b).  Returns the list of layer outputs y_0..y_L."""
    ys = [x]
    for l, (W, b) in enumerate(params):
        z = conv3x3(ys[-1], W, b)
        ys.append(np.maximum(z, 0.0) if l < len(params) - 1 else z)
    return ys


def backward(ys, params, gout):
    """Gradients of sum(gout * y_L) w.r.t. every (W, b) and the input."""
    grads = [None] * len(params)
    g = gout
    for l in range(len(params) - 1, -1, -1):
        if l < len(params) - 1:
            g = g * (ys[l + 1] > 0)      # ReLU of layer l
        grads[l] = conv3x3_weight_grad(ys[l], g)
        g = conv3x3_input_grad(g, params[l][0])
    return grads, g


def loss(pred: np.ndarray, target: np.ndarray) -> float:
    """Relative squared error per sample, averaged over the batch:
    mean_b ||pred_b - target_b||^2 / ||target_b||^2."""
    B = pred.shape[0]
    d = (pred - target).reshape(B, -1)
    t = target.reshape(B, -1)
    return float(np.mean(np.sum(d * d, axis=1) / np.sum(t * t, axis=1)))


def loss_grad(pred: np.ndarray, target: np.ndarray) -> np.ndarray:
    B = pred.shape[0]
    t2 = np.sum(target.reshape(B, -1) ** 2, axis=1).reshape(B, 1, 1, 1)
    return 2.0 * (pred - target) / t2 / B
