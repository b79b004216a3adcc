"""The small-label sweep (PCAD_KERNEL_SMALL: prior sums of all labels from a
table of neighbour pairs, chunk prefix sums in registers) against the
general CUDA-core kernel and the FP64 oracle: free-running chains are
label-for-label identical (both kernels decide every draw as the FP64
definition does), teacher-forced sweeps match the oracle at every site, and
AUTO takes the kernel exactly for the models it accepts."""
import numpy as np
import pytest

import oracle
from pcad_inputs import Model, gaussian_noise, greyscale_scene

pytestmark = pytest.mark.gpu

SMALL, CUDA_CORE = 4, 1


@pytest.fixture(scope="module")
def pc():
    import paper_2507_14869_gb300 as pc
    pc.lib()
    return pc


def _grey(seed, H, W, L, sigma):
    return gaussian_noise(seed + 1, greyscale_scene(seed, H, W, L, n_shapes=6), sigma, L)


CASES = [
    ("L16_T30", lambda: _grey(81, 130, 257, 16, 1.0),
     Model(L=16, pair=1, pair_coef=0.05, pair_T=30, sigma=1.0, inertia=2.0)),
    ("L16_8nb", lambda: _grey(82, 67, 95, 16, 4.0),
     Model(L=16, nbhd=8, pair=1, pair_coef=0.6, pair_T=4, sigma=4.0, inertia=0.5)),
    ("L13_masked", lambda: _grey(83, 50, 70, 13, 0.7),
     Model(L=13, pair=1, pair_coef=2.4, pair_T=3, sigma=0.7, inertia=4.0)),
    ("L5_potts8", lambda: _grey(84, 41, 40, 5, 1.0),
     Model(L=5, nbhd=8, pair=0, pair_coef=0.833, sigma=1.0, inertia=0.7)),
    ("L8_naive", lambda: _grey(85, 33, 100, 8, 1.5),
     Model(L=8, pair=1, pair_coef=0.9, pair_T=2, sigma=1.5, inertia=0.0)),
    ("L3_prior_only", lambda: _grey(86, 29, 31, 3, 1.0),
     Model(L=3, pair=0, pair_coef=1.0, noise=2, sigma=1.0, inertia=1.0)),
    ("one_col", lambda: _grey(87, 77, 1, 16, 1.0),
     Model(L=16, nbhd=8, pair=1, pair_coef=0.8, pair_T=2, sigma=1.0, inertia=1.0)),
    ("one_row", lambda: _grey(90, 1, 300, 16, 1.0),
     Model(L=16, pair=1, pair_coef=0.05, pair_T=30, sigma=1.0, inertia=2.0)),
    ("two_rows_8nb", lambda: _grey(91, 2, 33, 12, 1.0),
     Model(L=12, nbhd=8, pair=1, pair_coef=0.4, pair_T=5, sigma=1.0, inertia=1.0)),
    ("w32_h97_8nb", lambda: _grey(92, 97, 32, 16, 2.0),
     Model(L=16, nbhd=8, pair=1, pair_coef=0.3, pair_T=6, sigma=2.0, inertia=1.5)),
    ("w64_h65", lambda: _grey(93, 65, 64, 16, 1.0),
     Model(L=16, pair=1, pair_coef=0.05, pair_T=30, sigma=1.0, inertia=2.0)),
]


@pytest.mark.parametrize("name,make,m", CASES, ids=[c[0] for c in CASES])
def test_small_kernel_equals_general_kernel_and_oracle(pc, name, make, m):
    g = make()
    outs = {}
    for kind in (SMALL, CUDA_CORE):
        with pc.Chain(g, m, seed=13, chain_id=6, burn_in=9) as ch:
            ch.set_kernel(kind)
            assert ch.kernel_in_use() == kind
            ch.run(45)
            outs[kind] = (ch.sample(), ch.mean())
    assert np.array_equal(outs[SMALL][0], outs[CUDA_CORE][0])
    assert np.array_equal(outs[SMALL][1], outs[CUDA_CORE][1])
    xo, acc, nacc, _ = oracle.run_chain(m, g, 45, 9, seed=13, chain=6)
    assert np.array_equal(outs[SMALL][0], xo)
    np.testing.assert_allclose(outs[SMALL][1], acc / nacc, rtol=1e-6, atol=0)


def test_auto_takes_the_small_kernel_where_it_applies(pc):
    g = _grey(88, 20, 40, 16, 1.0)
    takes = [Model(L=16, pair=1, pair_coef=0.05, pair_T=30, sigma=1.0, inertia=2.0),
             Model(L=3, pair=0, pair_coef=0.5, sigma=1.0, inertia=0.0)]
    not_small = [Model(L=16, pair=1, pair_coef=-0.05, pair_T=30, sigma=1.0, inertia=2.0),
                 Model(L=16, pair=1, pair_coef=0.05, pair_T=3, sigma=1.0, inertia=2.0,
                       inertia_norm=1),
                 Model(L=17, pair=1, pair_coef=0.05, pair_T=3, sigma=1.0, inertia=2.0)]
    for m in takes:
        with pc.Chain(np.minimum(g, m.L - 1), m, seed=1) as ch:
            assert ch.kernel_in_use() == SMALL
    for m in not_small:
        with pc.Chain(np.minimum(g, m.L - 1), m, seed=1) as ch:
            assert ch.kernel_in_use() != SMALL
            with pytest.raises(pc.PcadError) as e:
                ch.set_kernel(SMALL)
            assert e.value.status == 1
    gm = Model(L=16, pair=1, pair_coef=0.05, pair_T=30, sigma=1.0, sampler=1)
    with pc.Chain(g, gm, seed=1) as ch:
        with pytest.raises(pc.PcadError):
            ch.set_kernel(SMALL)


def test_small_kernel_with_energy_tracking_and_blocking(pc):
    """Energy tracking runs it one sweep at a time (as before); temporal
    blocking takes over from it; results stay those of the general kernel."""
    g = _grey(89, 60, 70, 16, 2.0)
    m = Model(L=16, pair=1, pair_coef=0.6, pair_T=4, sigma=2.0, inertia=0.8)
    res = []
    for kind, k, track in ((SMALL, 0, True), (CUDA_CORE, 0, False), (0, 4, False)):
        with pc.Chain(g, m, seed=2, chain_id=1, burn_in=3) as ch:
            ch.set_kernel(kind)
            if track:
                ch.track_energy(64)
            ch.set_blocking(k)
            ch.run(24)
            res.append((ch.sample(), ch.mean()))
    for x, mu in res[1:]:
        assert np.array_equal(x, res[0][0]) and np.array_equal(mu, res[0][1])


TILE_CASES = [
    # 4 neighbours, W % 4 != 0 (scalar accumulator updates), ragged tiles
    ("L16_5801x5790", lambda: np.ascontiguousarray(_big16()[:5801, :5790]),
     Model(L=16, pair=1, pair_coef=0.05, pair_T=30, sigma=1.0, inertia=2.0)),
    # 8 neighbours, masked labels, W % 4 == 0 (float4 accumulator updates)
    ("L12_8nb_2901x2900", lambda: _grey(94, 2901, 2900, 12, 1.5),
     Model(L=12, nbhd=8, pair=1, pair_coef=0.3, pair_T=4, sigma=1.5, inertia=1.0)),
]


def _big16():
    from pcad_inputs import large_image
    return large_image(L=16)[1]


@pytest.mark.parametrize("name,make,m", TILE_CASES, ids=[c[0] for c in TILE_CASES])
def test_tile_form_for_large_images_equals_general_kernel(pc, name, make, m):
    """From 2^23 sites a small-label chain sweeps on TMA-loaded tiles
    (persistent, double-buffered); it stays the small-label kernel for AUTO
    and SMALL, and its labels and means equal the general kernel's."""
    g = make()
    assert g.size >= 1 << 23
    outs = {}
    for kind in (0, SMALL, CUDA_CORE):
        with pc.Chain(g, m, seed=5, chain_id=3, burn_in=1) as ch:
            ch.set_kernel(kind)
            assert ch.kernel_in_use() == (CUDA_CORE if kind == CUDA_CORE else SMALL)
            ch.run(3)
            ch.sync()
            outs[kind] = (ch.sample(), ch.mean())
    for kind in (0, SMALL):
        assert np.array_equal(outs[kind][0], outs[CUDA_CORE][0])
        assert np.array_equal(outs[kind][1], outs[CUDA_CORE][1])
