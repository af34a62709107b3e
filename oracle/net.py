"""FP64 oracle of the learned proposal net (plain numpy, direct convolution).

TEST INFRASTRUCTURE ONLY: the tests, the package smoke check and the CPU leg of the
benchmark may call it; the CUDA path never does. It shares no code with the library.

The net (a reading: the paper has no learned part; the network is fixed by the
workload specification): four 3x3 convolutions with zero padding of one pixel,
4 -> 32 -> 32 -> 32 -> 2 channels, ReLU after the first three. Input per pixel: observed
colour (R, G, B in [0, 1]) and depth D (metres). Output per pixel: the depth offset in
centimetres (delta = 0.01 * y[0] metres) and the opacity logit (y[1]).

    y_l[p, o] = b_l[o] + sum_{dy, dx in {-1, 0, 1}} sum_i W_l[dy + 1, dx + 1, i, o] * x_l[p + (dy, dx), i]

with x_l = 0 outside the image. Arrays are NHWC: x[n, y, x, c]; weights are
W[ky, kx, c_in, c_out].

Precision points of the GPU path (bf16 storage, wider accumulation) are modelled by
`bf16()`, round-to-nearest-even of float32 to bfloat16, applied where the path stores
bfloat16: the packed input, the weights, and the post-ReLU activations between layers.
The arithmetic itself is FP64.

Adjoint (hand-derived, checked against central differences in the tests):

    dx_l[p, i]       = sum_{dy, dx} sum_o W_l[dy + 1, dx + 1, i, o] * dy_l[p - (dy, dx), o]
    dW_l[ky, kx, i, o] = sum_p x_l[p + (ky - 1, kx - 1), i] * dy_l[p, o]
    db_l[o]          = sum_p dy_l[p, o]

and through a ReLU: dpre = dpost * [post > 0].
"""
from __future__ import annotations

import numpy as np

CHANNELS = (4, 32, 32, 32, 2)
DELTA_UNIT = 0.01          # metres per output unit of channel 0


def bf16(a) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), returned as float64 values."""
    f = np.ascontiguousarray(np.asarray(a, np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return (r.astype(np.uint32)).view(np.float32).astype(np.float64)


def conv3x3(x: np.ndarray, w: np.ndarray, b: np.ndarray) -> np.ndarray:
    """y = b + sum over taps and input channels (zero padding): x (N,H,W,Ci), w (3,3,Ci,Co)."""
    n, h, wd, ci = x.shape
    xp = np.zeros((n, h + 2, wd + 2, ci))
    xp[:, 1:-1, 1:-1] = x
    y = np.broadcast_to(np.asarray(b, np.float64), (n, h, wd, w.shape[3])).copy()
    for ky in range(3):
        for kx in range(3):
            y += np.einsum("nhwi,io->nhwo", xp[:, ky:ky + h, kx:kx + wd], w[ky, kx])
    return y


def conv3x3_backward(x: np.ndarray, w: np.ndarray, dy: np.ndarray):
    """(dx, dW, db) of conv3x3 for the output gradient dy (N,H,W,Co)."""
    n, h, wd, ci = x.shape
    xp = np.zeros((n, h + 2, wd + 2, ci))
    xp[:, 1:-1, 1:-1] = x
    dxp = np.zeros_like(xp)
    dw = np.zeros_like(w, dtype=np.float64)
    for ky in range(3):
        for kx in range(3):
            dw[ky, kx] = np.einsum("nhwi,nhwo->io", xp[:, ky:ky + h, kx:kx + wd], dy)
            dxp[:, ky:ky + h, kx:kx + wd] += np.einsum("nhwo,io->nhwi", dy, w[ky, kx])
    return dxp[:, 1:-1, 1:-1], dw, dy.sum(axis=(0, 1, 2))


def init_params(seed: int = 0):
    """He-normal weights, zero biases (float32 master copies)."""
    rng = np.random.default_rng(seed)
    ps = []
    for ci, co in zip(CHANNELS[:-1], CHANNELS[1:]):
        w = rng.normal(0.0, np.sqrt(2.0 / (9 * ci)), size=(3, 3, ci, co)).astype(np.float32)
        ps.append((w, np.zeros(co, np.float32)))
    return ps


def pack_input(rgb: np.ndarray, depth: np.ndarray) -> np.ndarray:
    """(N,3,H,W) colour and (N,H,W) depth -> (N,H,W,4) input, rounded to bfloat16."""
    x = np.concatenate([np.moveaxis(np.asarray(rgb, np.float64), 1, -1),
                        np.asarray(depth, np.float64)[..., None]], axis=-1)
    return bf16(x)


def forward(x0: np.ndarray, params, round_points: bool = True):
    """Activations [x0, x1, x2, x3, y4] of the net; x1..x3 are post-ReLU (rounded to
    bfloat16 when round_points), y4 is the raw output (N,H,W,2)."""
    acts = [x0]
    x = x0
    for l, (w, b) in enumerate(params):
        wq = bf16(w) if round_points else np.asarray(w, np.float64)
        y = conv3x3(x, wq, np.asarray(b, np.float64))
        if l < 3:
            y = np.maximum(y, 0.0)
            if round_points:
                y = bf16(y)
        acts.append(y)
        x = y
    return acts


def backward(acts, params, dy4: np.ndarray, round_points: bool = True):
    """Parameter gradients [(dW_l, db_l)] for the output gradient dy4 (N,H,W,2), and the
    pre-activation gradients of layers 1-3 (for per-layer checks)."""
    grads = [None] * 4
    dpre = [None] * 4
    d = np.asarray(dy4, np.float64)
    for l in range(3, -1, -1):
        w, _ = params[l]
        wq = bf16(w) if round_points else np.asarray(w, np.float64)
        dx, dw, db = conv3x3_backward(acts[l], wq, d)
        grads[l] = (dw, db)
        dpre[l] = d
        if l > 0:
            d = dx * (acts[l] > 0)
    return grads, dpre


def mse_loss(y4: np.ndarray, target_delta: np.ndarray, target_logit: np.ndarray, weight_logit: float = 1.0):
    """Training loss: mean over pixels of (y[0] - delta_t / 0.01)^2 + w (y[1] - logit_t)^2,
    and its gradient d loss / d y4."""
    t0 = np.asarray(target_delta, np.float64) / DELTA_UNIT
    t1 = np.asarray(target_logit, np.float64)
    e0 = y4[..., 0] - t0
    e1 = y4[..., 1] - t1
    npx = e0.size
    loss = (np.sum(e0 * e0) + weight_logit * np.sum(e1 * e1)) / npx
    d = np.stack([2.0 * e0 / npx, 2.0 * weight_logit * e1 / npx], axis=-1)
    return loss, d
