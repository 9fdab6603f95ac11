"""Pins of the FP64 D-SSIM reference (CPU): the window, SSIM of an image with
itself, the closed form for constant images, a brute-force evaluation of the
definition on a tiny image, and central finite differences of the gradient."""
import math

import numpy as np

from oracle import ssim as S


def test_window_is_normalised_separable_gaussian():
    w = S.window()
    assert w.shape == (11, 11) and abs(w.sum() - 1.0) < 1e-15
    g = np.exp(-((np.arange(11) - 5.0) ** 2) / (2 * 1.5 ** 2))
    g /= g.sum()
    np.testing.assert_allclose(w, np.outer(g, g), rtol=1e-14)
    assert w[5, 5] == w.max() and np.allclose(w, w.T) and np.allclose(w, w[::-1, ::-1])


def test_ssim_of_an_image_with_itself_is_one():
    rng = np.random.default_rng(0)
    x = rng.random((3, 20, 17))
    np.testing.assert_allclose(S.ssim_map(x, x), 1.0, atol=1e-12)
    assert abs(S.dssim(x, x)) < 1e-12
    np.testing.assert_allclose(S.dssim_grad(x, x), 0.0, atol=1e-12)


def test_constant_images_closed_form_inside():
    a, b = 0.3, 0.7
    x = np.full((1, 30, 30), a)
    y = np.full((1, 30, 30), b)
    m = S.ssim_map(x, y)[0]
    want = (2 * a * b + S.C1) / (a * a + b * b + S.C1)  # no variance once the window is inside
    np.testing.assert_allclose(m[5:25, 5:25], want, rtol=1e-12)
    # at a corner only a quarter-plus of the window sees the image: mean lower, not the interior value
    assert abs(m[0, 0] - want) > 1e-3


def test_brute_force_definition_tiny():
    rng = np.random.default_rng(1)
    x = rng.random((1, 9, 7))
    y = rng.random((1, 9, 7))
    w = S.window()
    H, W = 9, 7
    got = S.ssim_map(x, y)[0]
    for i in range(H):
        for j in range(W):
            sx = sy = sxx = syy = sxy = 0.0
            for di in range(-5, 6):
                for dj in range(-5, 6):
                    ii, jj = i + di, j + dj
                    if 0 <= ii < H and 0 <= jj < W:
                        g = w[di + 5, dj + 5]
                        xv, yv = x[0, ii, jj], y[0, ii, jj]
                        sx += g * xv; sy += g * yv
                        sxx += g * xv * xv; syy += g * yv * yv; sxy += g * xv * yv
            vx, vy, cxy = sxx - sx * sx, syy - sy * sy, sxy - sx * sy
            ref = (2 * sx * sy + S.C1) * (2 * cxy + S.C2) / ((sx * sx + sy * sy + S.C1) * (vx + vy + S.C2))
            assert math.isclose(got[i, j], ref, rel_tol=1e-12, abs_tol=1e-14)


def test_gradient_central_differences():
    rng = np.random.default_rng(2)
    x = rng.random((2, 13, 12))
    y = np.clip(x + 0.2 * rng.normal(size=x.shape), 0, 1)
    g = S.dssim_grad(x, y)
    h = 1e-6
    for (c, i, j) in [(0, 0, 0), (0, 6, 5), (1, 12, 11), (1, 3, 9), (0, 12, 0)]:
        xp, xm = x.copy(), x.copy()
        xp[c, i, j] += h
        xm[c, i, j] -= h
        fd = (S.dssim(xp, y) - S.dssim(xm, y)) / (2 * h)
        assert math.isclose(g[c, i, j], fd, rel_tol=1e-6, abs_tol=1e-11), (c, i, j, g[c, i, j], fd)
