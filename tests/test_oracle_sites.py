"""Pin for the oracle's sampled-site draw (orc_pca_sites): at any list of
sites it must return exactly the labels and near-boundary flags of the full
lazy-PCA sweep (orc_pca_sweep, itself pinned by the transition matrix and
the chain-law tests), for the same state, uniforms and sweep index.  The
sampled-site parity tests at 512^2 and 8192^2 rely on it.  Sites include
every corner and edge, repeated sites, the 8-neighbourhood, L = 2 flip
noise, Potts and L = 256.  CPU only."""
import numpy as np
import pytest

import oracle
from pcad_inputs import Model, gaussian_noise, greyscale_scene, random_lattice

POTTS, TL, GAUSS, FLIP = 0, 1, 0, 1


def _scene(seed, H, W, L, sigma):
    clean = greyscale_scene(seed, H, W, L, n_shapes=6)
    return gaussian_noise(seed + 1, clean, sigma, L)


CASES = [
    ("tl_L256_4nb", lambda: _scene(41, 37, 53, 256, 20.0),
     Model(L=256, pair=TL, pair_coef=0.05, pair_T=30, sigma=20.0, inertia=2.0)),
    ("tl_L256_8nb", lambda: _scene(42, 29, 31, 256, 25.0),
     Model(L=256, nbhd=8, pair=TL, pair_coef=0.05, pair_T=30, sigma=25.0, inertia=2.0)),
    ("tl_L16_4nb", lambda: _scene(43, 40, 47, 16, 1.0),
     Model(L=16, pair=TL, pair_coef=0.05, pair_T=30, sigma=1.0, inertia=2.0)),
    ("potts_L5_8nb", lambda: _scene(44, 23, 26, 5, 1.0),
     Model(L=5, nbhd=8, pair=POTTS, pair_coef=0.9, sigma=1.0, inertia=0.7)),
    ("ising_flip", lambda: random_lattice(45, 19, 22, 2),
     Model(L=2, pair=POTTS, pair_coef=1.2, noise=FLIP, flip_p=0.1, inertia=1.0)),
]


def _site_list(rng, H, W, n):
    """Every corner, a stretch of each edge, random interior sites, repeats."""
    rows = [0, 0, H - 1, H - 1] + [0] * 5 + [H - 1] * 5 + list(rng.integers(0, H, 10)) * 2
    cols = [0, W - 1, 0, W - 1] + list(rng.integers(0, W, 10)) + [0] * 10 + [W - 1] * 10
    rows += list(rng.integers(0, H, n))
    cols += list(rng.integers(0, W, n))
    rows += rows[:7]
    cols += cols[:7]
    return np.array(rows, dtype=np.int32), np.array(cols, dtype=np.int32)


@pytest.mark.parametrize("name,make,m", CASES, ids=[c[0] for c in CASES])
def test_pca_sites_equals_pca_sweep(orc, name, make, m):
    g = make()
    H, W = g.shape
    rng = np.random.default_rng(7)
    # a state that is neither g nor constant: a few sweeps of the chain
    x = oracle.run_chain(m, g, 3, 0, seed=5, chain=2)[0]
    for seed, chain, t in ((5, 2, 3), (11, 0, 0), (2**40 + 3, 77, 1234)):
        full, near_full = oracle.pca_sweep(m, g, x, seed, chain, t)
        rows, cols = _site_list(rng, H, W, 200)
        part, near = oracle.pca_sites(m, g, x, rows, cols, seed, chain, t)
        assert np.array_equal(part, full[rows, cols])
        assert np.array_equal(near, near_full[rows, cols])
        # the draws depend on the sweep index and the site: a wrong counter
        # or a transposed index would change a good fraction of them
        other, _ = oracle.pca_sweep(m, g, x, seed, chain, t + 1)
        if m.L > 2:
            assert (other != full).mean() > 0.05


def test_pca_sites_single_pixel_and_full_list(orc):
    m = Model(L=7, pair=TL, pair_coef=0.3, pair_T=2, sigma=1.0, inertia=0.5)
    g = np.array([[3]], dtype=np.uint8)
    full, _ = oracle.pca_sweep(m, g, g, 1, 0, 4)
    part, _ = oracle.pca_sites(m, g, g, np.array([0]), np.array([0]), 1, 0, 4)
    assert part[0] == full[0, 0]
    g = _scene(46, 9, 11, 16, 1.0)
    mm = Model(L=16, nbhd=8, pair=TL, pair_coef=0.6, pair_T=3, sigma=1.0, inertia=1.0)
    rr, cc = np.meshgrid(np.arange(9), np.arange(11), indexing="ij")
    full, near_full = oracle.pca_sweep(mm, g, g, 3, 1, 2)
    part, near = oracle.pca_sites(mm, g, g, rr.ravel(), cc.ravel(), 3, 1, 2)
    assert np.array_equal(part.reshape(9, 11), full)
    assert np.array_equal(near.reshape(9, 11), near_full)
