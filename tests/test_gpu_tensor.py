"""Tensor-core PCA sweeps (windowed prior sums by tcgen05.mma, CDF on the
CUDA cores, many sweeps per wavefront launch) against the CUDA-core sweep
and the oracle: labels and posterior means must be bit-identical for
tile-ragged images, label counts that are not multiples of 8 or 32, both
neighbourhoods, Potts (T = 1), a negative (repulsive) prior coefficient
(no exponent offset, constant CUDA-core margin) and the widest supported
truncation, sharp
edges (neighbours outside a site's 64-label histogram window), images with
more tiles than the persistent grid, and per-sweep launches under energy
tracking; and the checkerboard Gibbs sweep on the same kernel."""
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


def _edges(seed, H, W):
    """8 x 8 blocks of levels 10 and 240 with mild noise: neighbourhoods across
    block edges span ~230 labels, beyond one site's histogram window."""
    rng = np.random.default_rng(seed)
    yy, xx = np.mgrid[0:H, 0:W]
    clean = np.where(((yy // 8) + (xx // 8)) % 2 == 0, 10, 240)
    return np.clip(np.rint(clean + rng.normal(0.0, 12.0, (H, W))), 0, 255).astype(np.uint8)


CASES = [
    ("L256_37x70", lambda: (_grey(2, 37, 70, 256, 20.0),
                            Model(L=256, pair=TL, pair_coef=0.05, pair_T=30, sigma=20.0,
                                  inertia=2.0))),
    ("L256_8nb_33x45", lambda: (_grey(3, 33, 45, 256, 25.0),
                                Model(L=256, nbhd=8, pair=TL, pair_coef=0.04, pair_T=30,
                                      sigma=25.0, inertia=1.5))),
    ("L64_T2_50x97", lambda: (_grey(4, 50, 97, 64, 4.0),
                              Model(L=64, pair=TL, pair_coef=0.5, pair_T=2, sigma=4.0,
                                    inertia=1.0))),
    ("L100_T10_41x66", lambda: (_grey(5, 41, 66, 100, 8.0),
                                Model(L=100, pair=TL, pair_coef=0.12, pair_T=10, sigma=8.0,
                                      inertia=0.5))),
    ("L192_8nb_T33_29x31", lambda: (_grey(6, 29, 31, 192, 15.0),
                                    Model(L=192, nbhd=8, pair=TL, pair_coef=0.03, pair_T=33,
                                          sigma=15.0, inertia=2.5))),
    ("L128_potts_30x40", lambda: (_grey(7, 30, 40, 128, 6.0),
                                  Model(L=128, pair=POTTS, pair_coef=1.1, sigma=6.0,
                                        inertia=1.0))),
    ("L128_T33_21x53", lambda: (_grey(8, 21, 53, 128, 15.0),
                                Model(L=128, pair=TL, pair_coef=0.02, pair_T=33, sigma=15.0,
                                      inertia=0.0))),
    ("L256_edges_64x96", lambda: (_edges(15, 64, 96),
                                  Model(L=256, pair=TL, pair_coef=0.05, pair_T=30, sigma=12.0,
                                        inertia=2.0))),
    ("L256_8nb_edges_40x70", lambda: (_edges(16, 40, 70),
                                      Model(L=256, nbhd=8, pair=TL, pair_coef=0.03, pair_T=25,
                                            sigma=12.0, inertia=1.0))),
    ("L256_repulsive_45x38", lambda: (_grey(17, 45, 38, 256, 20.0),
                                      Model(L=256, pair=TL, pair_coef=-0.02, pair_T=30,
                                            sigma=20.0, inertia=1.5))),
    ("L71_3x1", lambda: (_grey(9, 3, 1, 71, 5.0),
                         Model(L=71, pair=TL, pair_coef=0.3, pair_T=4, sigma=5.0, inertia=1.0))),
    ("L256_300x257", lambda: (_grey(10, 300, 257, 256, 20.0),
                              Model(L=256, pair=TL, pair_coef=0.05, pair_T=30, sigma=20.0,
                                    inertia=2.0))),
]


def _run(pc, g, m, kind, n=45, burn=13):
    with pc.Chain(g, m, seed=5, chain_id=4, burn_in=burn) as ch:
        ch.set_kernel(kind)
        ch.run(20)
        ch.run(n - 20)
        ch.sync()
        return ch.sample(), ch.mean(), ch.fp64_draws()


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_tensor_equals_cuda_core(pc, name, make):
    g, m = make()
    x_ref, m_ref, _ = _run(pc, g, m, pc.PCAD_KERNEL_CUDA_CORE)
    x_tc, m_tc, _ = _run(pc, g, m, pc.PCAD_KERNEL_TENSOR)
    assert np.array_equal(x_tc, x_ref)
    assert np.array_equal(m_tc, m_ref)


@pytest.mark.parametrize("nbhd", [4, 8])
def test_tensor_matches_oracle(pc, nbhd):
    g = _grey(11, 23, 45, 256, 20.0)
    m = Model(L=256, nbhd=nbhd, pair=TL, pair_coef=0.05, pair_T=30, sigma=20.0, inertia=2.0)
    with pc.Chain(g, m, seed=9, chain_id=1, burn_in=3) as ch:
        ch.set_kernel(pc.PCAD_KERNEL_TENSOR)
        ch.run(12)
        xg, mg = ch.sample(), ch.mean()
    x, acc, nacc, _ = oracle.run_chain(m, g, 12, 3, seed=9, chain=1)
    assert np.array_equal(xg, x)
    np.testing.assert_allclose(mg, acc / nacc, rtol=1e-6, atol=0)


def test_auto_equals_tensor_and_redraws_in_fp64(pc):
    g, m = CASES[0][1]()
    x_auto, m_auto, _ = _run(pc, g, m, pc.PCAD_KERNEL_AUTO)
    x_tc, m_tc, fp64 = _run(pc, g, m, pc.PCAD_KERNEL_TENSOR)
    assert np.array_equal(x_auto, x_tc) and np.array_equal(m_auto, m_tc)
    assert fp64 > 0   # some uniforms fall inside the certified margin


def test_set_kernel_rejects(pc):
    g = _grey(12, 20, 20, 16, 1.0)
    small = Model(L=16, pair=TL, pair_coef=0.6, pair_T=3, sigma=1.2, inertia=1.0)
    with pc.Chain(g, small, seed=1) as ch:
        with pytest.raises(pc.PcadError):
            ch.set_kernel(pc.PCAD_KERNEL_TENSOR)      # L < 64
        with pytest.raises(pc.PcadError):
            ch.set_kernel(99)                         # no such kind
        ch.set_kernel(pc.PCAD_KERNEL_CUDA_CORE)
    for T in (100, 34):   # T > 33: the tents of a 64-bin histogram leave the 128-label window
        wide = Model(L=256, pair=TL, pair_coef=0.01, pair_T=T, sigma=20.0, inertia=1.0)
        with pc.Chain(_grey(13, 20, 20, 256, 20.0), wide, seed=1) as ch:
            with pytest.raises(pc.PcadError):
                ch.set_kernel(pc.PCAD_KERNEL_TENSOR)
            ch.run(3)                                  # the CUDA-core kernel
    gibbs8 = Model(L=256, nbhd=8, pair=TL, pair_coef=0.05, pair_T=30, sigma=20.0, sampler=1)
    with pc.Chain(_grey(14, 20, 20, 256, 20.0), gibbs8, seed=1) as ch:
        with pytest.raises(pc.PcadError):   # the Gibbs form covers the 4-neighbourhood only
            ch.set_kernel(pc.PCAD_KERNEL_TENSOR)
        assert ch.kernel_in_use() == pc.PCAD_KERNEL_CUDA_CORE


def test_tensor_per_sweep_launches_under_energy_tracking(pc):
    """Energy tracking needs every sweep's state: the tensor-core path then
    launches one sweep at a time; energies and the minimum state must equal
    the CUDA-core chain's."""
    g, m = CASES[0][1]()
    out = []
    for kind in (pc.PCAD_KERNEL_CUDA_CORE, pc.PCAD_KERNEL_TENSOR):
        with pc.Chain(g, m, seed=3, chain_id=2, burn_in=4) as ch:
            ch.set_kernel(kind).track_energy(30)
            ch.run(23)
            out.append((ch.sample(), ch.energies(), ch.min_state()))
    assert np.array_equal(out[0][0], out[1][0])
    np.testing.assert_array_equal(out[0][1], out[1][1])
    assert np.array_equal(out[0][2][0], out[1][2][0]) and out[0][2][1:] == out[1][2][1:]


# Checkerboard Gibbs on the tensor-core kernel (4-neighbourhood): colour
# phases over 8 x 32 tiles, in place; must equal the CUDA-core colour phases
# and the oracle's colour-order Gibbs sweep bit for bit.
GIBBS_CASES = [
    ("L256_37x70", lambda: (_grey(2, 37, 70, 256, 20.0),
                            Model(L=256, pair=TL, pair_coef=0.05, pair_T=30, sigma=20.0,
                                  sampler=1))),
    ("L203_odd_41x67", lambda: (_grey(21, 41, 67, 203, 15.0),
                                Model(L=203, pair=TL, pair_coef=0.06, pair_T=25, sigma=15.0,
                                      sampler=1))),
    ("L64_T2_50x97", lambda: (_grey(4, 50, 97, 64, 4.0),
                              Model(L=64, pair=TL, pair_coef=0.5, pair_T=2, sigma=4.0,
                                    sampler=1))),
    ("L128_potts_30x40", lambda: (_grey(7, 30, 40, 128, 6.0),
                                  Model(L=128, pair=POTTS, pair_coef=1.1, sigma=6.0, sampler=1))),
    ("L256_edges_64x96", lambda: (_edges(15, 64, 96),
                                  Model(L=256, pair=TL, pair_coef=0.05, pair_T=30, sigma=12.0,
                                        sampler=1))),
    ("L256_1x33", lambda: (_grey(22, 1, 33, 256, 20.0),
                           Model(L=256, pair=TL, pair_coef=0.05, pair_T=30, sigma=20.0,
                                 sampler=1))),
    ("L256_300x257", lambda: (_grey(10, 300, 257, 256, 20.0),
                              Model(L=256, pair=TL, pair_coef=0.05, pair_T=30, sigma=20.0,
                                    sampler=1))),
]


@pytest.mark.parametrize("name,make", GIBBS_CASES, ids=[c[0] for c in GIBBS_CASES])
def test_tensor_gibbs_equals_cuda_core(pc, name, make):
    g, m = make()
    x_ref, m_ref, _ = _run(pc, g, m, pc.PCAD_KERNEL_CUDA_CORE)
    x_tc, m_tc, _ = _run(pc, g, m, pc.PCAD_KERNEL_TENSOR)
    assert np.array_equal(x_tc, x_ref)
    assert np.array_equal(m_tc, m_ref)


def test_tensor_gibbs_matches_oracle_and_auto(pc):
    g = _grey(23, 29, 51, 256, 20.0)
    m = Model(L=256, pair=TL, pair_coef=0.05, pair_T=30, sigma=20.0, sampler=1)
    with pc.Chain(g, m, seed=9, chain_id=2, burn_in=3) as ch:
        assert ch.kernel_in_use() == pc.PCAD_KERNEL_TENSOR   # AUTO: L >= 192
        ch.run(12)
        xg, mg = ch.sample(), ch.mean()
    x, acc, nacc, _ = oracle.run_chain(m, g, 12, 3, seed=9, chain=2, sampler=1,
                                       order=oracle.ORDER_COLOUR)
    assert np.array_equal(xg, x)
    np.testing.assert_allclose(mg, acc / nacc, rtol=1e-6, atol=0)


def test_tensor_gibbs_under_energy_tracking(pc):
    g, m = GIBBS_CASES[0][1]()
    out = []
    for kind in (pc.PCAD_KERNEL_CUDA_CORE, pc.PCAD_KERNEL_TENSOR):
        with pc.Chain(g, m, seed=3, chain_id=2, burn_in=4) as ch:
            ch.set_kernel(kind).track_energy(30)
            ch.run(17)
            out.append((ch.sample(), ch.energies(), ch.mean()))
    assert np.array_equal(out[0][0], out[1][0])
    np.testing.assert_array_equal(out[0][1], out[1][1])
    assert np.array_equal(out[0][2], out[1][2])
