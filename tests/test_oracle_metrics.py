"""Pins for the oracle's PSNR / SSIM (Section 6) by hand-worked examples and
invariants.  CPU only."""
import math

import numpy as np
import pytest

from oracle import metrics
from pcad_inputs import random_lattice


def test_psnr_hand_worked_peak_one():
    # L = 5: luminances k/4.  clean [0, 1, .5, 1] (max 1), estimate differs by
    # 0.25 in one of 4 pixels: MSE = 0.0625/4, PSNR = 20 log10(1/0.125) = 20 log10 8.
    clean = np.array([[0, 4], [2, 4]])
    est = np.array([[0, 3], [2, 4]])
    assert abs(metrics.psnr(est, clean, 5) - 20 * math.log10(8.0)) < 1e-12


def test_psnr_uses_max_of_original_image():
    # clean luminances [0, .5, .25, .5] -> max x = 0.5; MSE = 0.015625
    clean = np.array([[0, 2], [1, 2]])
    est = np.array([[0, 2], [1, 1]])
    assert abs(metrics.psnr(est, clean, 5) - 20 * math.log10(0.5 / 0.125)) < 1e-12


def test_psnr_identical_is_infinite():
    x = random_lattice(1, 8, 8, 16)
    assert metrics.psnr(x, x, 16) == math.inf


def test_ssim_global_hand_worked():
    # x = [0,1,0,1], y = [0,1,1,1] (L = 2): mu_x = 1/2, mu_y = 3/4,
    # var_x = 1/3, var_y = 1/4, cov = 1/6 (unbiased), c1 = 1e-4, c2 = 9e-4.
    x = np.array([[0, 1], [0, 1]])
    y = np.array([[0, 1], [1, 1]])
    c1, c2 = 1e-4, 9e-4
    num = (2 * 0.5 * 0.75 + c1) * (2 * (1 / 6) + c2)
    den = (0.25 + 0.5625 + c1) * (1 / 3 + 0.25 + c2)
    assert abs(metrics.ssim_global(y, x, 2) - num / den) < 1e-14


def test_ssim_identity_and_symmetry():
    x = random_lattice(2, 40, 37, 256)
    y = random_lattice(3, 40, 37, 256)
    assert abs(metrics.ssim(x, x, 256) - 1.0) < 1e-12
    assert abs(metrics.ssim_global(x, x, 256) - 1.0) < 1e-12
    assert abs(metrics.ssim(x, y, 256) - metrics.ssim(y, x, 256)) < 1e-14
    assert metrics.ssim(x, y, 256) < 0.2


def test_ssim_constant_images_by_hand():
    # every window has zero variance: SSIM = (2ab + c1) / (a^2 + b^2 + c1)
    a_lab, b_lab, L = 3, 9, 16
    x = np.full((20, 24), a_lab)
    y = np.full((20, 24), b_lab)
    a, b, c1 = a_lab / 15, b_lab / 15, 1e-4
    assert abs(metrics.ssim(y, x, L) - (2 * a * b + c1) / (a * a + b * b + c1)) < 1e-12


def test_gaussian_window():
    w = metrics.gaussian_window()
    assert w.shape == (11, 11)
    assert abs(w.sum() - 1.0) < 1e-14
    assert np.allclose(w, w.T) and np.allclose(w, w[::-1, ::-1])
    # ratio of centre to a horizontal neighbour = exp(1/(2*1.5^2))
    assert abs(w[5, 5] / w[5, 6] - math.exp(1 / 4.5)) < 1e-12


def test_ssim_window_mean_over_valid_positions():
    """Brute-force one window position of the windowed SSIM by hand."""
    rng = np.random.default_rng(4)
    x = rng.integers(0, 16, size=(11, 11))
    y = rng.integers(0, 16, size=(11, 11))
    w = metrics.gaussian_window()
    xf, yf = x / 15.0, y / 15.0
    mx, my = (w * xf).sum(), (w * yf).sum()
    sxx = (w * xf * xf).sum() - mx * mx
    syy = (w * yf * yf).sum() - my * my
    sxy = (w * xf * yf).sum() - mx * my
    c1, c2 = 1e-4, 9e-4
    ref = ((2 * mx * my + c1) * (2 * sxy + c2)) / ((mx * mx + my * my + c1) * (sxx + syy + c2))
    assert metrics.ssim(y, x, 16) == pytest.approx(ref, rel=1e-12)
