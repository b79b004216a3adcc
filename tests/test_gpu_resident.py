"""The resident two-label kernel (PCAD_KERNEL_RESIDENT: every sweep of a run
in one launch of one CTA holding the state in shared memory, each draw a
comparison of the uniform with a threshold of the site's configuration)
against the per-sweep CUDA-core kernel and the FP64 oracle.

Free-running chains must be label-for-label identical to the per-sweep
kernel and to the oracle, for both samplers and both neighbourhoods, on
images whose width is not a multiple of 4, one row or column, tall and
narrow, with 1, 2 and 4 quads of 4 sites per thread, and at the largest
accepted sizes; the FP64 re-draw counts must agree too.  Runs are split so that a captured block of
sweeps, an odd number of PCA sweeps (the state ends in the other plane) and
single sweeps follow one another."""
import numpy as np
import pytest

import oracle
from pcad_inputs import Model, binary_64, random_lattice

pytestmark = pytest.mark.gpu

RESIDENT, CUDA_CORE = 5, 1
POTTS = 0


@pytest.fixture(scope="module")
def pc():
    import paper_2507_14869_gb300 as pc
    pc.lib()
    return pc


def _ising(seed, H, W, nbhd=4, flip=True):
    g = random_lattice(seed, H, W, 2)
    if flip:
        m = Model(L=2, nbhd=nbhd, pair=POTTS, pair_coef=0.9, noise=1, flip_p=0.2, inertia=0.6)
    else:
        m = Model(L=2, nbhd=nbhd, pair=POTTS, pair_coef=0.7, sigma=0.6, inertia=0.4)
    return g, m


CASES = [
    ("ising64", lambda: binary_64()[1:]),
    ("ragged_33x65", lambda: _ising(1, 33, 65)),
    ("ragged_8nb_45x77", lambda: _ising(2, 45, 77, nbhd=8, flip=False)),
    ("short_5x13", lambda: _ising(3, 5, 13)),
    ("short_8nb_3x9", lambda: _ising(4, 3, 9, nbhd=8)),
    ("one_row", lambda: _ising(5, 1, 97, flip=False)),
    ("one_col_8nb", lambda: _ising(6, 83, 1, nbhd=8)),
    ("one_pixel", lambda: _ising(7, 1, 1)),
    ("tall_1000x3", lambda: _ising(13, 1000, 3)),
    ("two_quads_8nb_64x100", lambda: _ising(14, 64, 100, nbhd=8)),
    ("max_128x128", lambda: _ising(8, 128, 128, nbhd=8)),
    ("max_120x136", lambda: _ising(9, 120, 136, flip=False)),
]

SPLIT = (7, 32, 1, 5)   # 45 sweeps: odd start, a captured block, single sweeps


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("sampler", [0, 1], ids=["pca", "gibbs"])
def test_resident_equals_per_sweep_kernel_and_oracle(pc, name, make, sampler):
    g, m = make()
    outs = {}
    for kind in (RESIDENT, CUDA_CORE):
        with pc.Chain(g, m, seed=21, chain_id=5, burn_in=11, sampler=sampler) as ch:
            ch.set_kernel(kind)
            assert ch.kernel_in_use() == kind
            for n in SPLIT:
                ch.run(n)
            outs[kind] = (ch.sample(), ch.mean(), ch.fp64_draws())
    assert np.array_equal(outs[RESIDENT][0], outs[CUDA_CORE][0])
    assert np.array_equal(outs[RESIDENT][1], outs[CUDA_CORE][1])
    assert outs[RESIDENT][2] == outs[CUDA_CORE][2]
    kw = {} if sampler == 0 else {"order": oracle.ORDER_COLOUR}
    xo, acc, nacc, _ = oracle.run_chain(m, g, sum(SPLIT), 11, seed=21, chain=5, sampler=sampler,
                                        **kw)
    assert np.array_equal(outs[RESIDENT][0], xo)
    np.testing.assert_allclose(outs[RESIDENT][1], acc / nacc, rtol=1e-6, atol=0)


def test_resident_binary_64_500_sweeps_matches_oracle(pc):
    """The two-label image workload: 64 x 64, 500 sweeps, burn-in 100, in
    one call (15 captured blocks of 32 sweeps and a 20-sweep launch)."""
    clean, noisy, m = binary_64()
    for sampler in (0, 1):
        with pc.Chain(noisy, m, seed=1, chain_id=0, burn_in=100, sampler=sampler) as ch:
            assert ch.kernel_in_use() == RESIDENT
            ch.run(500)
            xg, mg = ch.sample(), ch.mean()
        kw = {} if sampler == 0 else {"order": oracle.ORDER_COLOUR}
        xo, acc, nacc, _ = oracle.run_chain(m, noisy, 500, 100, seed=1, chain=0,
                                            sampler=sampler, **kw)
        assert np.array_equal(xg, xo)
        np.testing.assert_allclose(mg, acc / nacc, rtol=1e-6, atol=0)


def test_auto_takes_the_resident_kernel_where_it_applies(pc):
    g, m = _ising(10, 64, 64)
    for sampler in (0, 1):
        with pc.Chain(g, m, seed=1, sampler=sampler) as ch:
            assert ch.kernel_in_use() == RESIDENT
            ch.track_energy(8)
            assert ch.kernel_in_use() != RESIDENT   # every sweep's state is needed
    # 132 rows of 33 quads exceed 4096 quads
    g2, _ = _ising(11, 132, 132)
    with pc.Chain(g2, m, seed=1) as ch:
        assert ch.kernel_in_use() != RESIDENT
        with pytest.raises(pc.PcadError) as e:
            ch.set_kernel(RESIDENT)
        assert e.value.status == 1
    # more than two labels
    mo = Model(L=3, pair=POTTS, pair_coef=0.5, sigma=1.0, inertia=0.3)
    with pc.Chain(np.minimum(g, 2), mo, seed=1) as ch:
        assert ch.kernel_in_use() != RESIDENT
        with pytest.raises(pc.PcadError):
            ch.set_kernel(RESIDENT)
    # with two labels (|s - x_i| / (L - 1))^p is 1{s != x_i}: every price is the L0 one
    mo = Model(L=2, pair=POTTS, pair_coef=0.5, sigma=1.0, inertia=0.3, inertia_norm=2)
    with pc.Chain(g, mo, seed=1) as ch:
        assert ch.kernel_in_use() == RESIDENT


def test_resident_blocked_mode_and_export_continue_identically(pc):
    """Temporal blocking takes over from the resident kernel and back; an
    exported chain continues on the resident kernel as it would have."""
    g, m = _ising(12, 48, 52)
    with pc.Chain(g, m, seed=3, chain_id=2, burn_in=4) as ref:
        ref.set_kernel(CUDA_CORE)
        ref.run(40)
        x_ref, m_ref = ref.sample(), ref.mean()
    with pc.Chain(g, m, seed=3, chain_id=2, burn_in=4) as ch:
        ch.run(9)
        blob = ch.export()
        ch.set_blocking(4)
        ch.run(12)
        ch.set_blocking(0)
        assert ch.kernel_in_use() == RESIDENT
        ch.run(19)
        assert np.array_equal(ch.sample(), x_ref)
        assert np.array_equal(ch.mean(), m_ref)
    with pc.Chain.from_blob(blob) as ch2:
        assert ch2.kernel_in_use() == RESIDENT
        ch2.run(31)
        assert np.array_equal(ch2.sample(), x_ref)
        assert np.array_equal(ch2.mean(), m_ref)


def test_resident_follows_model_changes(pc):
    """An annealing schedule (set_model between stages) rebuilds the
    threshold table in stream order: the same labels as the per-sweep
    kernel, whose draws read the coefficients directly."""
    g, m = _ising(15, 40, 44, nbhd=8)
    stages = [Model(L=2, nbhd=8, pair=POTTS, pair_coef=c, noise=1, flip_p=0.2, inertia=0.6)
              for c in (0.4, 0.9, 1.6)]
    outs = {}
    for kind in (RESIDENT, CUDA_CORE):
        with pc.Chain(g, m, seed=8, chain_id=1, burn_in=6) as ch:
            ch.set_kernel(kind)
            ch.run_schedule(stages, [5, 11, 7])
            outs[kind] = (ch.sample(), ch.mean(), ch.fp64_draws())
    assert np.array_equal(outs[RESIDENT][0], outs[CUDA_CORE][0])
    assert np.array_equal(outs[RESIDENT][1], outs[CUDA_CORE][1])
    assert outs[RESIDENT][2] == outs[CUDA_CORE][2]


def test_batched_resident_chains_equal_single_chains(pc):
    """Small two-label chains in a batch run one CTA each in one launch per
    neighbourhood, next to a two-label chain too large for it and a
    16-label chain; runs end inside slices and one chain's coefficients
    change between runs.  Every chain's sample, mean and the batch's FP64
    re-draw count equal the chains run alone."""
    shapes = [(64, 64, 4), (33, 65, 4), (45, 77, 8), (1, 1, 4), (7, 3, 8), (128, 128, 4),
              (130, 130, 4)]
    jobs = []
    for k, (H, W, nb) in enumerate(shapes):
        g, m = _ising(40 + k, H, W, nbhd=nb, flip=k % 2 == 0)
        jobs.append((g, m, 50 + k, k, 6))
    from pcad_inputs import gaussian_noise, greyscale_scene
    g16 = gaussian_noise(61, greyscale_scene(60, 40, 50, 16, n_shapes=4), 1.0, 16)
    jobs.append((g16, Model(L=16, pair=1, pair_coef=0.6, pair_T=3, sigma=1.0, inertia=1.0),
                 70, 9, 5))
    m_new = Model(L=2, nbhd=8, pair=POTTS, pair_coef=1.4, noise=1, flip_p=0.15, inertia=0.2)
    b = pc.pcad_batch_create(jobs, autotune=False)
    try:
        pc.pcad_batch_run(b, 21)
        pc.pcad_batch_set_model(b, 2, m_new)
        pc.pcad_batch_run(b, 30)
        pc.pcad_batch_sync(b)
        fp64 = 0
        for i, (g, m, seed, chain, burn) in enumerate(jobs):
            with pc.Chain(g, m, seed=seed, chain_id=chain, burn_in=burn) as ch:
                if m.L == 16:   # the batch's general kernel: the same re-draw count
                    ch.set_kernel(CUDA_CORE)
                ch.run(21)
                if i == 2:
                    ch.set_model(m_new)
                ch.run(30)
                xs, ms = ch.sample(), ch.mean()
                fp64 += ch.fp64_draws()
            assert np.array_equal(pc.pcad_batch_read_sample(b, i, *g.shape), xs), i
            assert np.array_equal(pc.pcad_batch_read_mean(b, i, *g.shape), ms), i
        assert pc.pcad_batch_info(b)["fp64_draws"] == fp64
    finally:
        pc.pcad_batch_destroy(b)
