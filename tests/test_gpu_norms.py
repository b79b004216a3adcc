"""L1 / L2 inertia prices (lambda (|s - x_i| / (L - 1))^p, Section 3) on the
GPU against the oracle: free-running lazy-PCA chains must give identical
labels and posterior means; for L = 2 the price equals the L0 price; the
kernels that run the L0 price only refuse the norms."""
import numpy as np
import pytest

import oracle
from pcad_inputs import Model, gaussian_noise, greyscale_scene

pytestmark = pytest.mark.gpu

POTTS, TL = 0, 1


@pytest.fixture(scope="module")
def pc():
    import paper_2507_14869_gb300 as pc
    pc.lib()
    return pc


def _grey(seed, H, W, L, sigma):
    return gaussian_noise(seed + 1, greyscale_scene(seed, H, W, L, n_shapes=6), sigma, L)


CASES = [
    ("L5_potts8_l1", 5, dict(nbhd=8, pair=POTTS, pair_coef=0.8, sigma=0.9, inertia=1.5), 1),
    ("L5_potts8_l2", 5, dict(nbhd=8, pair=POTTS, pair_coef=0.8, sigma=0.9, inertia=3.0), 2),
    ("L16_tl_l1", 16, dict(pair=TL, pair_coef=0.6, pair_T=3, sigma=1.2, inertia=4.0), 1),
    ("L16_tl_l2", 16, dict(pair=TL, pair_coef=0.6, pair_T=3, sigma=1.2, inertia=8.0), 2),
    ("L33_tl8_l2", 33, dict(nbhd=8, pair=TL, pair_coef=0.2, pair_T=4, sigma=3.0, inertia=12.0), 2),
    ("L256_tl_l1", 256, dict(pair=TL, pair_coef=0.05, pair_T=30, sigma=20.0, inertia=6.0), 1),
    ("L256_tl_l2", 256, dict(pair=TL, pair_coef=0.05, pair_T=30, sigma=20.0, inertia=20.0), 2),
]


@pytest.mark.parametrize("name,L,kw,norm", CASES, ids=[c[0] for c in CASES])
def test_norm_chain_matches_oracle(pc, name, L, kw, norm):
    g = _grey(L, 27, 45, L, kw["sigma"])
    m = Model(L=L, inertia_norm=norm, **kw)
    with pc.Chain(g, m, seed=8, chain_id=5, burn_in=3) as ch:
        ch.run(20)
        ch.run(17)   # a graph block and a remainder
        xg, mg = ch.sample(), ch.mean()
    x, acc, nacc, _ = oracle.run_chain(m, g, 37, 3, seed=8, chain=5)
    assert np.array_equal(xg, x)
    np.testing.assert_allclose(mg, acc / nacc, rtol=1e-6, atol=0)


def test_binary_norm_equals_l0(pc):
    from pcad_inputs import flip_noise, shapes_binary
    g = flip_noise(3, shapes_binary(4, 40, 33), 0.1)
    base = dict(L=2, pair=POTTS, pair_coef=1.2, noise=1, flip_p=0.1, inertia=1.0)
    out = []
    for norm in (0, 1, 2):
        with pc.Chain(g, Model(**base, inertia_norm=norm), seed=2) as ch:
            ch.run(25)
            out.append(ch.sample())
    assert np.array_equal(out[0], out[1]) and np.array_equal(out[0], out[2])


def test_norms_refused_where_unsupported(pc):
    g = _grey(1, 20, 20, 256, 20.0)
    m = Model(L=256, pair=TL, pair_coef=0.05, pair_T=30, sigma=20.0, inertia=2.0, inertia_norm=1)
    with pc.Chain(g, m, seed=1) as ch:
        with pytest.raises(pc.PcadError):
            ch.set_blocking(2)
        with pytest.raises(pc.PcadError):
            ch.set_kernel(pc.PCAD_KERNEL_TENSOR)
        with pytest.raises(pc.PcadError):
            ch.set_model({**m.as_dict(), "inertia_norm": 2})
        ch.set_model({**m.as_dict(), "inertia": 3.0})
        ch.run(2)
    with pytest.raises(pc.PcadError):
        pc.pcad_batch_create([(g, m, 1, 0, 0)])
    with pytest.raises(pc.PcadError):
        pc.Chain(g, Model(L=16, pair=TL, pair_coef=0.5, pair_T=2, sigma=1.0, inertia_norm=3),
                 seed=1)
