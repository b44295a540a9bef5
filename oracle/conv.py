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


# --------------------------------------------------------------------------
# residual loss of the corrected iterate
# --------------------------------------------------------------------------

def h2A_image(e: np.ndarray, coef: np.ndarray, adjoint: bool = False) -> np.ndarray:
    """K e on each image of a batch (B, H, W) complex, K = h^2 A of the
    Helmholtz operator (Sec. 2.1 Eq. helm in the library's sign) on the node
    grid in image order (pixel (i, j) = node i W + j): the 5-point stencil
    4 e - (the four neighbours, zero outside the grid) minus the mass term
    coef e, coef = h^2 omega^2 m (1 - i gamma).  adjoint: K^H, the same
    stencil with conj(coef)."""
    ep = np.pad(e, ((0, 0), (1, 1), (1, 1)))
    nb = ep[:, :-2, 1:-1] + ep[:, 2:, 1:-1] + ep[:, 1:-1, :-2] + ep[:, 1:-1, 2:]
    c = np.conj(coef) if adjoint else coef
    return 4.0 * e - nb - c * e


def residual_loss(pred: np.ndarray, r: np.ndarray, coef: np.ndarray) -> float:
    """mean_b ||r_b - K e_b||^2 / ||r_b||^2 with e_b = pred_b[..., 0] + i
    pred_b[..., 1] (pred: (B, H, W, C), C >= 2), r and coef complex (B, H, W):
    the residual left after adding the network's correction, relative to the
    residual before it (the learned stage's output is in units of h^2 rho,
    its input residual in units of rho)."""
    e = pred[..., 0] + 1j * pred[..., 1]
    q = r - h2A_image(e, coef)
    B = pred.shape[0]
    num = np.sum(np.abs(q.reshape(B, -1)) ** 2, axis=1)
    den = np.sum(np.abs(r.reshape(B, -1)) ** 2, axis=1)
    return float(np.mean(num / den))


def residual_loss_grad(pred: np.ndarray, r: np.ndarray, coef: np.ndarray) -> np.ndarray:
    """d residual_loss / d pred, channel by channel: for L_b = ||r - K e||^2
    and e = a + i b, dL/da = -2 Re(K^H q) and dL/db = -2 Im(K^H q), scaled
    by 1 / (B ||r_b||^2); zero in channels >= 2."""
    e = pred[..., 0] + 1j * pred[..., 1]
    q = r - h2A_image(e, coef)
    B = pred.shape[0]
    den = np.sum(np.abs(r.reshape(B, -1)) ** 2, axis=1).reshape(B, 1, 1)
    g = -2.0 * h2A_image(q, coef, adjoint=True) / (B * den)
    out = np.zeros_like(pred)
    out[..., 0] = g.real
    out[..., 1] = g.imag
    return out
