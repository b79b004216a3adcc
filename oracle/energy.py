"""Posterior energy of a labelling -- TEST INFRASTRUCTURE.

    H(x) = sum over unordered neighbour pairs <ij> of V(x_i, x_j) + sum_i U(g_i, x_i),

the energy of the posterior Gibbs measure pi_post(x) ~ exp(-H(x)) (Section 4,
Eq. mrf_gauss_noise_posterior_distribution) with the per-edge pair weight of
the single-site conditional (Eq. gibbs_sampler_elementary_step): Potts
V(s, t) = -c_P 1{s = t}, truncated linear V(s, t) = c_T min(|s - t|, T);
Gaussian noise U(g, s) = (g - s)^2 / (2 sigma^2), flip noise U = -ln(1 - p)
when s = g and -ln p otherwise, no likelihood (prior only) U = 0.  A free
boundary: pairs leaving the image do not exist.

Every term is a model coefficient times an integer count, so H is computed
as (coefficient) x (integer sum): ``energy_terms`` returns the two integer
sums, ``posterior_energy`` their combination in FP64 with the model's
parameters rounded to FP32 (as the library receives them).
"""
from __future__ import annotations

import math

import numpy as np

from . import FLIP, GAUSS, POTTS, _f32


def _pairs(x: np.ndarray, nbhd: int):
    """(x_i, x_j) arrays of every unordered neighbour pair: right, down and,
    for the 8-neighbourhood, down-right and down-left."""
    out = [(x[:, :-1], x[:, 1:]), (x[:-1, :], x[1:, :])]
    if nbhd == 8:
        out += [(x[:-1, :-1], x[1:, 1:]), (x[:-1, 1:], x[1:, :-1])]
    return out


def energy_terms(m, g: np.ndarray, x: np.ndarray):
    """(pair_sum, data_sum): Potts -> number of pairs with equal labels,
    truncated linear -> sum of min(|x_i - x_j|, T); Gaussian -> sum of
    (g_i - x_i)^2, flip -> number of sites with x_i != g_i."""
    d = m.as_dict() if hasattr(m, "as_dict") else dict(m)
    X = np.asarray(x, dtype=np.int64)
    G = np.asarray(g, dtype=np.int64)
    pair = 0
    for a, b in _pairs(X, int(d.get("nbhd", 4))):
        if int(d.get("pair", 1)) == POTTS:
            pair += int(np.count_nonzero(a == b))
        else:
            pair += int(np.minimum(np.abs(a - b), int(d.get("pair_T", 1))).sum())
    noise = int(d.get("noise", GAUSS))
    if noise == GAUSS:
        data = int(((G - X) ** 2).sum())
    elif noise == FLIP:
        data = int(np.count_nonzero(G != X))
    else:   # no likelihood
        data = 0
    return pair, data


def combine(m, n_sites: int, pair: int, data: int) -> float:
    """H from the integer sums: (+/-) c * pair + data term."""
    d = m.as_dict() if hasattr(m, "as_dict") else dict(m)
    c = _f32(d.get("pair_coef", 0.0))
    pair_e = (-c if int(d.get("pair", 1)) == POTTS else c) * float(pair)
    noise = int(d.get("noise", GAUSS))
    if noise == GAUSS:
        s = _f32(d.get("sigma", 1.0))
        data_e = float(data) / (2.0 * s * s)
    elif noise != FLIP:
        data_e = 0.0
    else:
        p = _f32(d.get("flip_p", 0.1))
        data_e = -math.log1p(-p) * float(n_sites - data) - math.log(p) * float(data)
    return pair_e + data_e


def posterior_energy(m, g: np.ndarray, x: np.ndarray) -> float:
    pair, data = energy_terms(m, g, x)
    return combine(m, int(np.asarray(x).size), pair, data)
