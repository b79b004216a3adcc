"""Wavefront lazy-PCA launches (many sweeps per persistent launch, tiles
released by their 3 x 3 neighbourhood's progress) against one launch per
sweep: labels and posterior means must be bit-identical for every label
count, neighbourhood, tile-ragged and degenerate image shape, split runs and
graph blocks; one case also against the oracle."""
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
    ("L256_512x512", lambda: (_grey(2, 512, 512, 256, 20.0),
                              Model(L=256, pair=TL, pair_coef=0.05, pair_T=30, sigma=20.0,
                                    inertia=2.0))),
    ("L16_8nb_301x257", lambda: (_grey(3, 301, 257, 16, 1.0),
                                 Model(L=16, nbhd=8, pair=TL, pair_coef=0.85, pair_T=2, sigma=1.0,
                                       inertia=2.0))),
    ("L2_flip_97x64", lambda: (flip_noise(3, shapes_binary(4, 97, 64), 0.1),
                               Model(L=2, pair=POTTS, pair_coef=1.2, noise=FLIP, flip_p=0.1,
                                     inertia=1.0))),
    ("L5_potts8_3x700", lambda: (_grey(5, 3, 700, 5, 0.9),
                                 Model(L=5, nbhd=8, pair=POTTS, pair_coef=0.8, sigma=0.9,
                                       inertia=0.7))),
    ("L33_1x1", lambda: (np.array([[7]], np.uint8),
                         Model(L=33, nbhd=8, pair=TL, pair_coef=0.2, pair_T=5, sigma=3.0,
                               inertia=0.4))),
    ("L100_700x3", lambda: (_grey(6, 700, 3, 100, 8.0),
                            Model(L=100, pair=TL, pair_coef=0.12, pair_T=10, sigma=8.0,
                                  inertia=0.5))),
]


def _run(pc, g, m, kind, parts=(20, 45, 1), burn=13):
    with pc.Chain(g, m, seed=5, chain_id=4, burn_in=burn) as ch:
        ch.set_kernel(kind)
        for n in parts:
            ch.run(n)
        ch.sync()
        return ch.sample(), ch.mean()


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_wave_equals_per_sweep_launches(pc, name, make):
    g, m = make()
    x_ref, m_ref = _run(pc, g, m, pc.PCAD_KERNEL_CUDA_CORE)
    x_w, m_w = _run(pc, g, m, pc.PCAD_KERNEL_WAVE)
    assert np.array_equal(x_w, x_ref)
    assert np.array_equal(m_w, m_ref)


def test_wave_matches_oracle(pc):
    g = _grey(7, 61, 150, 16, 1.0)
    m = Model(L=16, pair=TL, pair_coef=0.85, pair_T=2, sigma=1.0, inertia=2.0)
    with pc.Chain(g, m, seed=9, chain_id=1, burn_in=3) as ch:
        ch.set_kernel(pc.PCAD_KERNEL_WAVE)
        ch.run(37)
        xg, mg = ch.sample(), ch.mean()
    x, acc, nacc, _ = oracle.run_chain(m, g, 37, 3, seed=9, chain=1)
    assert np.array_equal(xg, x)
    np.testing.assert_allclose(mg, acc / nacc, rtol=1e-6, atol=0)


def test_wave_refusals_and_fallbacks(pc):
    g = _grey(8, 30, 40, 16, 1.0)
    lp = Model(L=16, pair=TL, pair_coef=0.6, pair_T=3, sigma=1.2, inertia=2.0, inertia_norm=1)
    with pc.Chain(g, lp, seed=1) as ch:
        with pytest.raises(pc.PcadError):
            ch.set_kernel(pc.PCAD_KERNEL_WAVE)
    gibbs = Model(L=16, pair=TL, pair_coef=0.6, pair_T=3, sigma=1.2, sampler=1)
    with pc.Chain(g, gibbs, seed=1) as ch:
        with pytest.raises(pc.PcadError):
            ch.set_kernel(pc.PCAD_KERNEL_WAVE)
    m = Model(L=16, pair=TL, pair_coef=0.6, pair_T=3, sigma=1.2, inertia=2.0)
    # energy tracking needs every sweep's state: the chain falls back to one launch per sweep
    with pc.Chain(g, m, seed=2) as a, pc.Chain(g, m, seed=2) as b:
        a.set_kernel(pc.PCAD_KERNEL_WAVE).track_energy(40)
        b.track_energy(40)
        a.run(33)
        b.run(33)
        assert np.array_equal(a.sample(), b.sample())
        np.testing.assert_array_equal(a.energies(), b.energies())


def test_kernel_in_use_auto_rule(pc):
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    slots = 10 * sms
    m256 = Model(L=256, pair=TL, pair_coef=0.05, pair_T=30, sigma=20.0, inertia=2.0)
    # L >= 192 and eligible for the tensor-core sweep: that one on small
    # images, the windowed wavefront from 8 blocks of 4 x 32 sites per SM,
    # the per-sweep windowed sweep from 100
    for side in (128, 512, 2048):
        g = np.zeros((side, side), np.uint8)
        blocks = (side // 32) * (side // 4)
        big = blocks >= 8 * sms
        expect = (pc.PCAD_KERNEL_WINDOW if blocks >= 100 * sms else pc.PCAD_KERNEL_WINDOW_WAVE
                  if big else pc.PCAD_KERNEL_TENSOR)
        with pc.Chain(g, m256, seed=1) as ch:
            assert ch.kernel_in_use() == expect, side
            if big:
                ch.track_energy(4)   # every sweep's state: not the tensor-core wavefront
                assert ch.kernel_in_use() == pc.PCAD_KERNEL_CUDA_CORE
    # below L = 192 (or T > 33): the CUDA-core kernels by size
    m128 = Model(L=128, pair=TL, pair_coef=0.1, pair_T=15, sigma=10.0, inertia=2.0)
    wide = Model(L=256, pair=TL, pair_coef=0.05, pair_T=40, sigma=20.0, inertia=2.0)
    for side in (128, 512, 2048):
        tiles = (side // 32) * (side // 4)
        expect = pc.PCAD_KERNEL_WAVE if 2 * tiles >= slots and tiles <= 3 * slots \
            else pc.PCAD_KERNEL_CUDA_CORE
        g = np.zeros((side, side), np.uint8)
        for mm in (m128, wide):
            # T <= 33 on a large image: the windowed sweeps (64 <= L <= 256)
            e = expect
            if mm is m128 and tiles >= 8 * sms:
                e = pc.PCAD_KERNEL_WINDOW if tiles >= 100 * sms else pc.PCAD_KERNEL_WINDOW_WAVE
            with pc.Chain(g, mm, seed=1) as ch:
                assert ch.kernel_in_use() == e, (side, mm.L, mm.pair_T)
    g = np.zeros((512, 512), np.uint8)
    with pc.Chain(g, m256, seed=1) as ch:
        ch.set_blocking(2)
        assert ch.kernel_in_use() == -2
        ch.set_blocking(0)
        ch.track_energy(4)
        assert ch.kernel_in_use() == pc.PCAD_KERNEL_CUDA_CORE   # every sweep's state needed
        ch.track_energy(0)
        ch.set_kernel(pc.PCAD_KERNEL_WAVE)
        assert ch.kernel_in_use() == pc.PCAD_KERNEL_WAVE
        ch.set_kernel(pc.PCAD_KERNEL_TENSOR)
        assert ch.kernel_in_use() == pc.PCAD_KERNEL_TENSOR
    # two labels at 512^2 (2^18 sites): the two-label sweep
    binary = Model(L=2, pair=POTTS, pair_coef=1.2, noise=FLIP, flip_p=0.1, inertia=1.0)
    with pc.Chain(g, binary, seed=1) as ch:
        assert ch.kernel_in_use() == pc.PCAD_KERNEL_BINARY
