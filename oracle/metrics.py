"""PSNR and SSIM in FP64 -- TEST INFRASTRUCTURE.

Section 6 (experimental results) defines, on luminances in [0, 1]:
  * PSNR(x~) = 20 log10( max x / sqrt(MSE(x, x~)) ), with max x the largest
    pixel value of the ORIGINAL image and MSE the mean squared difference;
  * SSIM as in Wang et al. (2004).  The paper prints the single-window
    formula with sample means, standard deviations and covariance and says
    the constants depend on the grey levels.  ``ssim`` is the standard
    Gaussian-window mean SSIM of Wang et al. (11x11 window, sigma 1.5,
    K1 = 0.01, K2 = 0.03, dynamic range R = 1 on luminances, statistics over
    the positions where the whole window fits); ``ssim_global`` is the
    printed single-window form (unbiased sample statistics).

Luminance of label k with L labels is k / (L - 1); an estimate in label
units (e.g. a posterior mean) is mapped the same way.
"""
from __future__ import annotations

import math

import numpy as np

K1, K2, WIN, WSIG = 0.01, 0.03, 11, 1.5


def luminance(labels, L: int) -> np.ndarray:
    return np.asarray(labels, dtype=np.float64) / float(L - 1)


def psnr(est_labels, clean_labels, L: int) -> float:
    x = luminance(clean_labels, L)
    y = luminance(est_labels, L)
    mse = float(np.mean((x - y) ** 2))
    mx = float(x.max())
    if mse == 0.0:
        return math.inf
    return 20.0 * math.log10(mx / math.sqrt(mse))


def gaussian_window(size: int = WIN, sigma: float = WSIG) -> np.ndarray:
    ax = np.arange(size, dtype=np.float64) - (size - 1) / 2.0
    g = np.exp(-(ax * ax) / (2.0 * sigma * sigma))
    w = np.outer(g, g)
    return w / w.sum()


def _filter_valid(img: np.ndarray, w: np.ndarray) -> np.ndarray:
    """Plain 2-D correlation over the positions where the window fits."""
    k = w.shape[0]
    H, W = img.shape
    out = np.zeros((H - k + 1, W - k + 1))
    for a in range(k):
        for b in range(k):
            out += w[a, b] * img[a:a + H - k + 1, b:b + W - k + 1]
    return out


def ssim(est_labels, clean_labels, L: int) -> float:
    x = luminance(clean_labels, L)
    y = luminance(est_labels, L)
    if x.shape[0] < WIN or x.shape[1] < WIN:
        return ssim_global(est_labels, clean_labels, L)
    c1 = (K1 * 1.0) ** 2
    c2 = (K2 * 1.0) ** 2
    w = gaussian_window()
    mx = _filter_valid(x, w)
    my = _filter_valid(y, w)
    sxx = _filter_valid(x * x, w) - mx * mx
    syy = _filter_valid(y * y, w) - my * my
    sxy = _filter_valid(x * y, w) - mx * my
    num = (2.0 * mx * my + c1) * (2.0 * sxy + c2)
    den = (mx * mx + my * my + c1) * (sxx + syy + c2)
    return float(np.mean(num / den))


def ssim_global(est_labels, clean_labels, L: int) -> float:
    x = luminance(clean_labels, L).reshape(-1)
    y = luminance(est_labels, L).reshape(-1)
    n = x.size
    c1 = (K1 * 1.0) ** 2
    c2 = (K2 * 1.0) ** 2
    mx, my = x.mean(), y.mean()
    vx = ((x - mx) ** 2).sum() / (n - 1)
    vy = ((y - my) ** 2).sum() / (n - 1)
    cxy = ((x - mx) * (y - my)).sum() / (n - 1)
    return float(((2 * mx * my + c1) * (2 * cxy + c2)) / ((mx * mx + my * my + c1) * (vx + vy + c2)))
