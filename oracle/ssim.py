"""FP64 oracle of the SSIM term of the mapping loss (Eq. 1, L_S), plain numpy.

TEST INFRASTRUCTURE ONLY: the tests and the CPU leg of the benchmark may call it; the
CUDA path never does. It shares no code with the library.

Reading (the paper names L_S "the SSIM loss between V_k and V'_k" and cites Wang et al.
2004 without window details): per colour channel, with an 11 x 11 Gaussian window of
standard deviation 1.5 (weights normalised to sum 1) and zero padding outside the image,

    mu_x = G * x,  mu_y = G * y,  s_xx = G * x^2 - mu_x^2,  s_yy = G * y^2 - mu_y^2,
    s_xy = G * (x y) - mu_x mu_y,
    SSIM = (2 mu_x mu_y + C1)(2 s_xy + C2) / ((mu_x^2 + mu_y^2 + C1)(s_xx + s_yy + C2)),

C1 = 0.01^2, C2 = 0.03^2 (dynamic range 1), and L_S = 1 - mean of SSIM over pixels and
channels. x is the rendered colour V', y the observed V.

Adjoint (hand-derived; checked against central differences in the tests): writing the
blurred moments m1 = G * x, m2 = G * x^2, m12 = G * (x y),

    dS/dm1  = S (2 mu_y / A1 - 2 mu_y / A2 - 2 m1 / B1 + 2 m1 / B2)
    dS/dm2  = -S / B2
    dS/dm12 = 2 S / A2

with A1 = 2 m1 mu_y + C1, A2 = 2 s_xy + C2, B1 = m1^2 + mu_y^2 + C1, B2 = s_xx + s_yy + C2,
and, G being symmetric and zero-padded, d L_S / d x = -(1/N) (G * dS/dm1 + 2 x (G * dS/dm2)
+ y (G * dS/dm12)), N = number of pixels times channels.
"""
from __future__ import annotations

import numpy as np

WINDOW = 11
SIGMA = 1.5
C1 = 0.01 ** 2
C2 = 0.03 ** 2


def window() -> np.ndarray:
    """The 11 x 11 Gaussian window (outer product of the normalised 1-D weights)."""
    i = np.arange(WINDOW) - WINDOW // 2
    g = np.exp(-(i * i) / (2.0 * SIGMA * SIGMA))
    g /= g.sum()
    return np.outer(g, g)


def blur(a: np.ndarray) -> np.ndarray:
    """Correlation of a (H, W) map with the window, zero padding, same size."""
    h, w = a.shape
    r = WINDOW // 2
    p = np.zeros((h + 2 * r, w + 2 * r))
    p[r:r + h, r:r + w] = a
    G = window()
    out = np.zeros((h, w))
    for dy in range(WINDOW):
        for dx in range(WINDOW):
            out += G[dy, dx] * p[dy:dy + h, dx:dx + w]
    return out


def ssim_map(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Per-pixel SSIM of (C, H, W) images."""
    out = np.empty(x.shape)
    for c in range(x.shape[0]):
        xc, yc = np.asarray(x[c], np.float64), np.asarray(y[c], np.float64)
        mx, my = blur(xc), blur(yc)
        sxx = blur(xc * xc) - mx * mx
        syy = blur(yc * yc) - my * my
        sxy = blur(xc * yc) - mx * my
        out[c] = (2 * mx * my + C1) * (2 * sxy + C2) / ((mx * mx + my * my + C1) * (sxx + syy + C2))
    return out


def ssim_loss_grad(x: np.ndarray, y: np.ndarray):
    """(L_S, d L_S / d x) for rendered x and observed y, both (C, H, W)."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    n = x.size
    S_all = ssim_map(x, y)
    grad = np.empty(x.shape)
    for c in range(x.shape[0]):
        xc, yc = x[c], y[c]
        m1, my = blur(xc), blur(yc)
        m2, m12, myy = blur(xc * xc), blur(xc * yc), blur(yc * yc)
        A1 = 2 * m1 * my + C1
        A2 = 2 * (m12 - m1 * my) + C2
        B1 = m1 * m1 + my * my + C1
        B2 = (m2 - m1 * m1) + (myy - my * my) + C2
        S = S_all[c]
        d1 = S * (2 * my / A1 - 2 * my / A2 - 2 * m1 / B1 + 2 * m1 / B2)
        d2 = -S / B2
        d12 = 2 * S / A2
        grad[c] = -(blur(d1) + 2 * xc * blur(d2) + yc * blur(d12)) / n
    return 1.0 - S_all.mean(), grad
