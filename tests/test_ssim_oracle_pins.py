"""Pins of the SSIM-term oracle (oracle/ssim.py): the blur against a library correlation,
the per-pixel SSIM against a brute-force evaluation of its definition, the closed forms
for identical and for constant images, and central differences of its adjoint."""
import numpy as np
import pytest

from oracle import ssim


def test_blur_equals_library_correlation():
    signal = pytest.importorskip("scipy.signal")
    rng = np.random.default_rng(0)
    a = rng.normal(size=(13, 17))
    ref = signal.correlate2d(a, ssim.window(), mode="same", boundary="fill")
    np.testing.assert_allclose(ssim.blur(a), ref, rtol=1e-12, atol=1e-12)
    assert abs(ssim.window().sum() - 1.0) < 1e-14


def test_ssim_map_matches_brute_force_definition():
    """Per pixel: window weights over the 11 x 11 neighbourhood (zero outside the image),
    weighted means, variances and covariance, then the SSIM formula."""
    rng = np.random.default_rng(1)
    x, y = rng.uniform(size=(2, 9, 8)), rng.uniform(size=(2, 9, 8))
    G = ssim.window()
    got = ssim.ssim_map(x, y)
    for c in range(2):
        for py in range(9):
            for px in range(8):
                sx = sy = sxx = syy = sxy = 0.0
                for dy in range(-5, 6):
                    for dx in range(-5, 6):
                        qy, qx = py + dy, px + dx
                        if 0 <= qy < 9 and 0 <= qx < 8:
                            wgt = G[dy + 5, dx + 5]
                            a, b = x[c, qy, qx], y[c, qy, qx]
                            sx += wgt * a
                            sy += wgt * b
                            sxx += wgt * a * a
                            syy += wgt * b * b
                            sxy += wgt * a * b
                vx, vy, cxy = sxx - sx * sx, syy - sy * sy, sxy - sx * sy
                ref = ((2 * sx * sy + ssim.C1) * (2 * cxy + ssim.C2)) / (
                    (sx * sx + sy * sy + ssim.C1) * (vx + vy + ssim.C2))
                assert abs(got[c, py, px] - ref) < 1e-12


def test_identical_images_give_zero_loss_and_gradient():
    rng = np.random.default_rng(2)
    x = rng.uniform(size=(3, 12, 14))
    loss, g = ssim.ssim_loss_grad(x, x.copy())
    assert abs(loss) < 1e-13
    assert np.abs(g).max() < 1e-13


def test_constant_images_interior_closed_form():
    """Away from the border (window inside the image) constants a, b give
    SSIM = (2ab + C1) / (a^2 + b^2 + C1)."""
    a, b = 0.3, 0.7
    x, y = np.full((1, 20, 20), a), np.full((1, 20, 20), b)
    s = ssim.ssim_map(x, y)[0, 5:15, 5:15]
    np.testing.assert_allclose(s, (2 * a * b + ssim.C1) / (a * a + b * b + ssim.C1), rtol=1e-10)


def test_adjoint_matches_central_differences():
    rng = np.random.default_rng(3)
    x, y = rng.uniform(size=(3, 9, 10)), rng.uniform(size=(3, 9, 10))
    loss, g = ssim.ssim_loss_grad(x, y)
    h = 1e-6
    for idx in [(0, 0, 0), (1, 4, 5), (2, 8, 9), (0, 3, 7), (2, 0, 9)]:
        xp, xm = x.copy(), x.copy()
        xp[idx] += h
        xm[idx] -= h
        fd = (ssim.ssim_loss_grad(xp, y)[0] - ssim.ssim_loss_grad(xm, y)[0]) / (2 * h)
        assert abs(fd - g[idx]) <= 1e-6 * abs(fd) + 1e-9, (idx, fd, g[idx])
