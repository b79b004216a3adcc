"""Temporally blocked PCA sweeps (k sweeps per launch on TMA-loaded tiles
with recomputed halos) against unblocked single-sweep launches: labels and
posterior means must be bit-identical for every k, tile-ragged size, label
count and neighbourhood; one case is also checked against the oracle."""
import numpy as np
import pytest

import oracle
from pcad_inputs import Model, flip_noise, gaussian_noise, greyscale_scene, shapes_binary

pytestmark = pytest.mark.gpu

POTTS, TL, FLIP = 0, 1, 1


@pytest.fixture(scope="module")
def pc():
    import paper_2507_14869_gb300 as pc
    pc.lib()
    return pc


def _grey(seed, H, W, L, sigma):
    return gaussian_noise(seed + 1, greyscale_scene(seed, H, W, L, n_shapes=6), sigma, L)


CASES = [
    ("L16_100x129", lambda: (_grey(1, 100, 129, 16, 1.0),
                             Model(L=16, pair=TL, pair_coef=0.85, pair_T=2, sigma=1.0, inertia=2.0))),
    ("L256_37x70", lambda: (_grey(2, 37, 70, 256, 20.0),
                            Model(L=256, pair=TL, pair_coef=0.05, pair_T=30, sigma=20.0, inertia=2.0))),
    ("L2_flip_97x64", lambda: (flip_noise(3, shapes_binary(4, 97, 64), 0.1),
                               Model(L=2, pair=POTTS, pair_coef=1.2, noise=FLIP, flip_p=0.1,
                                     inertia=1.0))),
    ("L5_8nb_130x33", lambda: (_grey(5, 130, 33, 5, 1.0),
                               Model(L=5, nbhd=8, pair=POTTS, pair_coef=0.8, sigma=1.0, inertia=0.7))),
    ("L16_5x200", lambda: (_grey(6, 5, 200, 16, 1.2),
                           Model(L=16, pair=TL, pair_coef=0.6, pair_T=3, sigma=1.2, inertia=0.0))),
    ("L33_8nb_1x1", lambda: (np.array([[7]], np.uint8),
                             Model(L=33, nbhd=8, pair=TL, pair_coef=0.2, pair_T=5, sigma=3.0,
                                   inertia=0.4))),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_blocked_equals_unblocked(pc, name, make):
    g, m = make()
    n, burn = 45, 13            # 45 = 32 (one graph block) + 13, burn-in inside a block
    with pc.Chain(g, m, seed=3, chain_id=2, burn_in=burn) as ref:
        ref.run(n)
        x_ref, m_ref = ref.sample(), ref.mean()
    for k in (1, 2, 4, 8):
        with pc.Chain(g, m, seed=3, chain_id=2, burn_in=burn) as ch:
            ch.set_blocking(k)
            ch.run(20)
            ch.run(25)
            ch.sync()
            assert np.array_equal(ch.sample(), x_ref), k
            assert np.array_equal(ch.mean(), m_ref), k


def test_blocked_matches_oracle(pc):
    g = _grey(7, 61, 150, 16, 1.0)
    m = Model(L=16, pair=TL, pair_coef=0.85, pair_T=2, sigma=1.0, inertia=2.0)
    with pc.Chain(g, m, seed=9, chain_id=1, burn_in=3) as ch:
        ch.set_blocking(4)
        ch.run(16)
        xg, mg = ch.sample(), ch.mean()
    x, acc, nacc, _ = oracle.run_chain(m, g, 16, 3, seed=9, chain=1)
    assert np.array_equal(xg, x)
    np.testing.assert_allclose(mg, acc / nacc, rtol=1e-6, atol=0)


def test_blocking_rejects_bad_k_and_gibbs(pc):
    g = _grey(8, 20, 20, 16, 1.0)
    m = Model(L=16, pair=TL, pair_coef=0.6, pair_T=3, sigma=1.2, inertia=1.0)
    with pc.Chain(g, m, seed=1) as ch:
        for k in (3, 16, -1):
            with pytest.raises(pc.PcadError):
                ch.set_blocking(k)
    with pc.Chain(g, m, seed=1, sampler=1) as ch:
        with pytest.raises(pc.PcadError):
            ch.set_blocking(4)
