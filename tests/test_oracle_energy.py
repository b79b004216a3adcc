"""Pins of the oracle's posterior energy H(x) (Section 4, Eq.
mrf_gauss_noise_posterior_distribution): against the exhaustive enumeration
of log pi_post (built edge by edge in oracle.exact) on every state of tiny
lattices, and closed forms on constant images."""
import numpy as np
import pytest

from oracle import energy, exact
from pcad_inputs import Model

POTTS, TL, GAUSS, FLIP = 0, 1, 0, 1

CASES = [
    ("gauss_tl_2x3_L3", np.array([[0, 2, 1], [1, 1, 0]], np.uint8),
     Model(L=3, pair=TL, pair_coef=0.7, pair_T=1, sigma=0.8)),
    ("gauss_tl_2x3_L4_T2", np.array([[3, 0, 2], [1, 3, 0]], np.uint8),
     Model(L=4, pair=TL, pair_coef=0.45, pair_T=2, sigma=1.3)),
    ("flip_potts_3x3_8nb", np.array([[0, 1, 1], [1, 0, 0], [1, 1, 0]], np.uint8),
     Model(L=2, nbhd=8, pair=POTTS, pair_coef=0.9, noise=FLIP, flip_p=0.2)),
    ("gauss_potts_2x2_L4", np.array([[0, 3], [2, 1]], np.uint8),
     Model(L=4, pair=POTTS, pair_coef=1.1, sigma=1.5)),
]


@pytest.mark.parametrize("name,g,m", CASES, ids=[c[0] for c in CASES])
def test_energy_is_minus_log_posterior(name, g, m):
    logw = exact.posterior_logweights(m, g)
    X = exact.states(g.size, m.L)
    for k in range(X.shape[0]):
        x = X[k].reshape(g.shape).astype(np.uint8)
        assert energy.posterior_energy(m, g, x) == pytest.approx(-logw[k], rel=1e-12, abs=1e-12)


def test_constant_images_closed_forms():
    H, W = 5, 7
    g = np.full((H, W), 3, np.uint8)
    x = g.copy()
    edges4 = H * (W - 1) + (H - 1) * W
    edges8 = edges4 + 2 * (H - 1) * (W - 1)
    for nb, ne in ((4, edges4), (8, edges8)):
        m = Model(L=5, nbhd=nb, pair=POTTS, pair_coef=0.5, sigma=2.0)
        assert energy.energy_terms(m, g, x) == (ne, 0)
        assert energy.posterior_energy(m, g, x) == pytest.approx(-0.5 * ne)
    # truncated linear with a vertical step of 4 and T = 3: every vertical pair
    # across the step costs min(4, 3) = 3
    x2 = x.copy()
    x2[2:, :] = 7
    m = Model(L=8, pair=TL, pair_coef=0.25, pair_T=3, sigma=2.0)
    pair, data = energy.energy_terms(m, g, x2)
    assert pair == 3 * W
    assert data == 16 * (H - 2) * W
    assert energy.posterior_energy(m, g, x2) == pytest.approx(0.25 * 3 * W + data / 8.0)


def test_flip_energy_counts_mismatches():
    g = np.zeros((4, 4), np.uint8)
    x = g.copy()
    x[1, 2] = 1
    m = Model(L=2, pair=POTTS, pair_coef=1.0, noise=FLIP, flip_p=0.25)
    pair, data = energy.energy_terms(m, g, x)
    assert data == 1
    # the flipped site breaks its 4 pairs out of 24
    assert pair == 24 - 4
    p = np.float32(0.25).item()
    expect = -1.0 * 20 - np.log1p(-p) * 15 - np.log(p) * 1
    assert energy.posterior_energy(m, g, x) == pytest.approx(expect, rel=1e-14)
