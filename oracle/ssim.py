"""Oracle of the SSIM loss the local-to-global bundle adjustment adds to the
RGB rendering (Sec. "Tracking and Local-to-Global Bundle Adjustment").
TEST INFRASTRUCTURE ONLY; numpy + scipy, FP64.

Readings (the paper names the loss, not its form): structural similarity of
Wang et al. with an 11x11 Gaussian window of standard deviation 1.5
(normalised), zero padding outside the image, C1 = 0.01^2, C2 = 0.03^2 (data
range 1), per colour channel; L_ssim = 1 - mean over views, channels and
pixels of SSIM(C, C_target).  The gradient is with respect to the rendered
image C.
"""
from __future__ import annotations

import numpy as np
from scipy.ndimage import correlate

C1 = 0.01 ** 2
C2 = 0.03 ** 2


def window(size: int = 11, sigma: float = 1.5) -> np.ndarray:
    r = np.arange(size) - size // 2
    g = np.exp(-(r * r) / (2 * sigma * sigma))
    g /= g.sum()
    return np.outer(g, g)


def _filt(img, w):
    return correlate(img, w, mode="constant", cval=0.0)


def ssim_loss(C, Ct, n_views: int, width: int, height: int):
    """C, Ct flat [views][3][H][W]; returns (L_ssim, dL/dC)."""
    w = window()
    x = np.asarray(C, np.float64).reshape(n_views * 3, height, width)
    y = np.asarray(Ct, np.float64).reshape(n_views * 3, height, width)
    M = x.size
    total = 0.0
    grad = np.zeros_like(x)
    for p in range(x.shape[0]):
        a, b = x[p], y[p]
        mx, my = _filt(a, w), _filt(b, w)
        sxx = _filt(a * a, w) - mx * mx
        syy = _filt(b * b, w) - my * my
        sxy = _filt(a * b, w) - mx * my
        a1, a2 = 2 * mx * my + C1, 2 * sxy + C2
        b1, b2 = mx * mx + my * my + C1, sxx + syy + C2
        S = a1 * a2 / (b1 * b2)
        total += S.sum()
        dS_dmx = 2 * my * a2 / (b1 * b2) - 2 * mx * S / b1
        dS_dsxx = -S / b2
        dS_dsxy = 2 * a1 / (b1 * b2)
        A = -(dS_dmx - 2 * mx * dS_dsxx - my * dS_dsxy) / M
        B = -dS_dsxx / M
        Cc = -dS_dsxy / M
        grad[p] = _filt(A, w) + 2 * a * _filt(B, w) + b * _filt(Cc, w)
    return 1.0 - total / M, grad.reshape(-1)
