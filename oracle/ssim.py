"""FP64 reference of the structural-similarity loss term (test infrastructure
only: imported by the tests, never by the CUDA package).

The paper's mapping loss (Sec. "Map Optimization") and tracking loss
(Eq. tracking_loss, Sec. "Camera Factor (Option 2)") carry a D-SSIM term and
defer its definition to 3D Gaussian Splatting (kerbl20233d), whose SSIM is the
one of Wang et al. (2004): per channel, local statistics under an 11 x 11
Gaussian window of standard deviation 1.5 (image borders padded with zeros),

    SSIM(p) = (2 mu_x mu_y + C1)(2 s_xy + C2) / ((mu_x^2 + mu_y^2 + C1)(s_x^2 + s_y^2 + C2)),
    mu_x = G * x,  s_x^2 = G * x^2 - mu_x^2,  s_xy = G * (x y) - mu_x mu_y,
    C1 = 0.01^2, C2 = 0.03^2 (dynamic range 1),

and D-SSIM = 1 - mean of SSIM over the channels and pixels of a view.  The
gradient with respect to x follows the chain rule through the three window
sums that contain x (written out below, no automatic differentiation).
"""
from __future__ import annotations

import numpy as np
from scipy.signal import correlate2d

WINDOW = 11
SIGMA = 1.5
C1 = 0.01 ** 2
C2 = 0.03 ** 2


def window() -> np.ndarray:
    """The 11 x 11 Gaussian window, normalised to sum 1."""
    r = np.arange(WINDOW, dtype=np.float64) - (WINDOW - 1) / 2
    xx, yy = np.meshgrid(r, r)
    w = np.exp(-(xx * xx + yy * yy) / (2.0 * SIGMA * SIGMA))
    return w / w.sum()


def _filt(img: np.ndarray) -> np.ndarray:
    """G * img over a [H][W] plane, zero padding, output the size of img."""
    return correlate2d(img, window(), mode="same", boundary="fill", fillvalue=0.0)


def _stats(x: np.ndarray, y: np.ndarray):
    mx, my = _filt(x), _filt(y)
    sxx = _filt(x * x) - mx * mx
    syy = _filt(y * y) - my * my
    sxy = _filt(x * y) - mx * my
    return mx, my, sxx, syy, sxy


def ssim_map(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """SSIM at every pixel of every channel; x, y: [C][H][W]."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    out = np.empty_like(x)
    for c in range(x.shape[0]):
        mx, my, sxx, syy, sxy = _stats(x[c], y[c])
        out[c] = ((2 * mx * my + C1) * (2 * sxy + C2)) / ((mx * mx + my * my + C1) * (sxx + syy + C2))
    return out


def dssim(x: np.ndarray, y: np.ndarray) -> float:
    """1 - mean SSIM of one view ([C][H][W])."""
    return float(1.0 - ssim_map(x, y).mean())


def dssim_grad(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """d(1 - mean SSIM)/dx for one view ([C][H][W]).

    SSIM(p) depends on x through m1 = G*x, m2 = G*x^2 and m3 = G*(x y):
      dS/dm1 = dS/dmu_x - 2 mu_x dS/ds_x^2 - mu_y dS/ds_xy,
      dS/dm2 = dS/ds_x^2,  dS/dm3 = dS/ds_xy,
    and dm1(p)/dx(q) = G(p - q), dm2(p)/dx(q) = 2 x(q) G(p - q),
    dm3(p)/dx(q) = y(q) G(p - q); the sum over p is a correlation with the
    mirrored window (the window is symmetric)."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    n = x.size
    g = np.empty_like(x)
    for c in range(x.shape[0]):
        mx, my, sxx, syy, sxy = _stats(x[c], y[c])
        a1 = 2 * mx * my + C1
        a2 = 2 * sxy + C2
        b1 = mx * mx + my * my + C1
        b2 = sxx + syy + C2
        s = a1 * a2 / (b1 * b2)
        ds_dmx = 2 * my * a2 / (b1 * b2) - s * 2 * mx / b1
        ds_dsxx = -s / b2
        ds_dsxy = 2 * a1 / (b1 * b2)
        d1 = ds_dmx - 2 * mx * ds_dsxx - my * ds_dsxy
        d2 = ds_dsxx
        d3 = ds_dsxy
        # loss = 1 - sum(S)/n
        g[c] = -(_filt(d1) + 2 * x[c] * _filt(d2) + y[c] * _filt(d3)) / n
    return g
