"""The CUDA-core windowed sweeps (PCAD_KERNEL_WINDOW: the tensor-core sweep's
weights, tent sums of each site's hull of labels from a byte table, the
other chunks from the outside table; lazy PCA and checkerboard Gibbs colour
phases) against the FP64 oracle and the other kernels: free-running chains
are label for label the oracle's, on ragged sizes, both neighbourhoods,
Potts and truncated-linear priors, L not a multiple of 8, one row, one
column and one pixel."""
import numpy as np
import pytest

import oracle
from pcad_inputs import Model, gaussian_noise, greyscale_scene

pytestmark = pytest.mark.gpu

WINDOW, TENSOR, CUDA_CORE = 6, 2, 1
POTTS, TL = 0, 1


@pytest.fixture(scope="module")
def pc():
    import paper_2507_14869_gb300 as pc
    pc.lib()
    return pc


def _grey(seed, H, W, L, sigma):
    return gaussian_noise(seed + 1, greyscale_scene(seed, H, W, L, n_shapes=6), sigma, L)


CASES = [
    ("L256_T30", lambda: _grey(91, 70, 131, 256, 25.0),
     Model(L=256, pair=TL, pair_coef=0.05, pair_T=30, sigma=25.0, inertia=2.0)),
    ("L256_noise_only_far_neighbours", lambda: np.random.default_rng(5).integers(
        0, 256, (40, 50)).astype(np.uint8),
     Model(L=256, pair=TL, pair_coef=0.3, pair_T=33, sigma=40.0, inertia=0.5)),
    ("L201_8nb_T25", lambda: _grey(92, 45, 61, 201, 18.0),
     Model(L=201, nbhd=8, pair=TL, pair_coef=0.05, pair_T=25, sigma=18.0, inertia=1.5)),
    ("L200_potts", lambda: _grey(93, 33, 40, 200, 15.0),
     Model(L=200, pair=POTTS, pair_coef=2.0, sigma=15.0, inertia=1.5)),
    ("L64_T2", lambda: _grey(94, 37, 70, 64, 4.0),
     Model(L=64, pair=TL, pair_coef=0.6, pair_T=2, sigma=4.0, inertia=0.0)),
    ("L100_8nb_T31", lambda: _grey(95, 29, 33, 100, 8.0),
     Model(L=100, nbhd=8, pair=TL, pair_coef=0.1, pair_T=31, sigma=8.0, inertia=1.0)),
    ("one_row", lambda: _grey(96, 1, 97, 256, 20.0),
     Model(L=256, pair=TL, pair_coef=0.05, pair_T=30, sigma=20.0, inertia=2.0)),
    ("one_col_8nb", lambda: _grey(97, 83, 1, 128, 10.0),
     Model(L=128, nbhd=8, pair=TL, pair_coef=0.1, pair_T=20, sigma=10.0, inertia=1.0)),
    ("one_pixel", lambda: np.array([[200]], dtype=np.uint8),
     Model(L=256, pair=TL, pair_coef=0.05, pair_T=30, sigma=20.0, inertia=2.0)),
    # fewer labels: the windowed kernels take 9 <= L <= 256
    ("L33_potts8", lambda: _grey(100, 40, 70, 33, 3.0),
     Model(L=33, nbhd=8, pair=POTTS, pair_coef=0.833, sigma=3.0, inertia=0.39)),
    ("L17_T2", lambda: _grey(101, 37, 45, 17, 1.5),
     Model(L=17, pair=TL, pair_coef=0.7, pair_T=2, sigma=1.5, inertia=1.0)),
    ("L9_8nb_T31", lambda: _grey(102, 30, 33, 9, 1.0),
     Model(L=9, nbhd=8, pair=TL, pair_coef=0.15, pair_T=31, sigma=1.0, inertia=0.5)),
]


@pytest.mark.parametrize("name,make,m", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("sampler", [0, 1], ids=["pca", "gibbs"])
def test_window_kernel_matches_oracle_and_other_kernels(pc, name, make, m, sampler):
    g = make()
    sweeps, burn = 14, 5
    kinds = [WINDOW, CUDA_CORE]
    if m.L >= 64 and (sampler == 0 or m.nbhd == 4):
        kinds.append(TENSOR)
    outs = {}
    for kind in kinds:
        with pc.Chain(g, m, seed=17, chain_id=3, burn_in=burn, sampler=sampler) as ch:
            ch.set_kernel(kind)
            assert ch.kernel_in_use() == kind
            ch.run(9)
            ch.run(sweeps - 9)
            outs[kind] = (ch.sample(), ch.mean())
    kw = {} if sampler == 0 else {"order": oracle.ORDER_COLOUR}
    xo, acc, nacc, _ = oracle.run_chain(m, g, sweeps, burn, seed=17, chain=3, sampler=sampler,
                                        **kw)
    for kind in outs:
        assert np.array_equal(outs[kind][0], xo), kind
        np.testing.assert_allclose(outs[kind][1], acc / nacc, rtol=1e-6, atol=0)


def test_window_kernel_long_chain_and_model_change(pc):
    """40 sweeps (a captured block and single sweeps) with an annealing
    schedule: the outside table follows set_model."""
    g = _grey(98, 64, 96, 256, 20.0)
    stages = [Model(L=256, pair=TL, pair_coef=c, pair_T=30, sigma=20.0, inertia=2.0)
              for c in (0.02, 0.05, 0.09)]
    res = {}
    for kind in (WINDOW, CUDA_CORE):
        with pc.Chain(g, stages[0], seed=4, chain_id=1, burn_in=3) as ch:
            ch.set_kernel(kind)
            ch.run_schedule(stages, [33, 4, 3])
            res[kind] = (ch.sample(), ch.mean())
    assert np.array_equal(res[WINDOW][0], res[CUDA_CORE][0])
    assert np.array_equal(res[WINDOW][1], res[CUDA_CORE][1])


def test_window_kernel_is_validated(pc):
    g = _grey(99, 20, 30, 16, 1.0)
    for m, sampler in ((Model(L=8, pair=TL, pair_coef=0.1, pair_T=3, sigma=1.0), 0),
                       (Model(L=256, pair=TL, pair_coef=0.05, pair_T=40, sigma=20.0), 1),
                       (Model(L=256, nbhd=8, pair=TL, pair_coef=0.05, pair_T=33, sigma=20.0), 0)):
        with pc.Chain(np.minimum(g * 16, m.L - 1).astype(np.uint8), m, seed=1,
                      sampler=sampler) as ch:
            with pytest.raises(pc.PcadError) as e:
                ch.set_kernel(WINDOW)
            assert e.value.status == 1


def test_auto_rule_for_windowed_gibbs(pc):
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    for side in (256, 1024, 2048):
        blocks = (side // 32) * (side // 4)
        g = np.zeros((side, side), np.uint8)
        for nbhd in (4, 8):
            m = Model(L=256, nbhd=nbhd, pair=TL, pair_coef=0.05, pair_T=30, sigma=20.0,
                      sampler=1)
            if nbhd == 8:
                expect = pc.PCAD_KERNEL_WINDOW_WAVE if blocks >= 3 * sms else CUDA_CORE
            elif blocks >= 100 * sms:
                expect = WINDOW
            else:
                expect = pc.PCAD_KERNEL_WINDOW_WAVE if blocks >= 8 * sms else TENSOR
            with pc.Chain(g, m, seed=1, sampler=1) as ch:
                assert ch.kernel_in_use() == expect, (side, nbhd)


@pytest.mark.parametrize("name,make,m", CASES[:6], ids=[c[0] for c in CASES[:6]])
@pytest.mark.parametrize("sampler", [0, 1], ids=["pca", "gibbs"])
def test_window_wavefront_matches_per_sweep_and_oracle(pc, name, make, m, sampler):
    """PCAD_KERNEL_WINDOW_WAVE: the windowed draw as one persistent wavefront
    launch per block of sweeps (of colour phases for Gibbs; a captured
    32-sweep block, then odd and single sweeps): the per-sweep windowed
    kernel's labels, means and FP64 re-draw counts, and the oracle's
    labels."""
    g = make()
    outs = {}
    for kind in (pc.PCAD_KERNEL_WINDOW_WAVE, WINDOW):
        with pc.Chain(g, m, seed=11, chain_id=2, burn_in=4, sampler=sampler) as ch:
            ch.set_kernel(kind)
            assert ch.kernel_in_use() == kind
            for n in (32, 3, 1):
                ch.run(n)
            outs[kind] = (ch.sample(), ch.mean(), ch.fp64_draws())
            ch.sync()
    a, b = outs[pc.PCAD_KERNEL_WINDOW_WAVE], outs[WINDOW]
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and a[2] == b[2]
    kw = {} if sampler == 0 else {"order": oracle.ORDER_COLOUR}
    xo, _, _, _ = oracle.run_chain(m, g, 36, 4, seed=11, chain=2, sampler=sampler, **kw)
    assert np.array_equal(a[0], xo)
