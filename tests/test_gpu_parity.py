"""GPU parity: the CUDA sweeps against the FP64 oracle, label for label.

Teacher forcing: at every sweep t the oracle starts from the GPU's state
x^(t) and draws x^(t+1) with the same Philox uniforms; every site is
compared.  A mismatch is allowed only at a draw the oracle flags as lying
within 1e-6 of an FP64 CDF boundary, and the mismatch fraction must stay
below 1e-6 (the kernels re-evaluate uncertain draws in FP64, so none is
expected).  All calls go through the C ABI."""
import numpy as np
import pytest

import oracle
from oracle import metrics as om
from pcad_inputs import (Model, binary_64, gaussian_noise, greyscale_512, greyscale_scene,
                         random_lattice)

pytestmark = pytest.mark.gpu

POTTS, TL, GAUSS, FLIP = 0, 1, 0, 1
MAX_MISMATCH_FRACTION = 1e-6


@pytest.fixture(scope="module")
def pc():
    import paper_2507_14869_gb300 as pc
    pc.lib()
    return pc


def _scene(seed, H, W, L, sigma):
    clean = greyscale_scene(seed, H, W, L, n_shapes=6)
    return clean, gaussian_noise(seed + 1, clean, sigma, L)


def teacher_forced(pc, m, g, sweeps, seed=7, chain=3, sampler=0):
    ch = pc.Chain(g, m, seed=seed, chain_id=chain, burn_in=0, sampler=sampler)
    x = np.array(g, copy=True)
    mism = unflagged = total = 0
    try:
        for t in range(sweeps):
            ch.run(1)
            xg = ch.sample()
            if sampler == 0:
                xo, near = oracle.pca_sweep(m, g, x, seed, chain, t)
            else:
                xo, near = oracle.gibbs_sweep(m, g, x, seed, chain, t, order=oracle.ORDER_COLOUR)
            d = xg != xo
            mism += int(d.sum())
            unflagged += int((d & (near == 0)).sum())
            total += d.size
            x = xg
        fp64 = ch.fp64_draws()
    finally:
        ch.close()
    return mism, unflagged, total, fp64


CASES = [
    ("ising_flip_64", lambda: binary_64()[1:]),
    ("tl_L16_ragged", lambda: (_scene(1, 45, 77, 16, 1.0)[1],
                               Model(L=16, pair=TL, pair_coef=0.85, pair_T=2, sigma=1.0,
                                     inertia=2.0))),
    ("tl_L256_ragged", lambda: (_scene(2, 37, 70, 256, 20.0)[1],
                                Model(L=256, pair=TL, pair_coef=0.05, pair_T=30, sigma=20.0,
                                      inertia=2.0))),
    ("potts8_L5", lambda: (_scene(3, 40, 41, 5, 1.0)[1],
                           Model(L=5, nbhd=8, pair=POTTS, pair_coef=0.833, sigma=1.0,
                                 inertia=0.7))),
    ("potts8_L33", lambda: (_scene(4, 33, 29, 33, 3.2)[1],
                            Model(L=33, nbhd=8, pair=POTTS, pair_coef=0.833, sigma=3.2,
                                  inertia=0.39))),
    ("tl8_L9", lambda: (_scene(5, 31, 36, 9, 1.6)[1],
                        Model(L=9, nbhd=8, pair=TL, pair_coef=0.5, pair_T=2, sigma=1.6,
                              inertia=0.26))),
    ("naive_q0_L16", lambda: (_scene(6, 20, 50, 16, 1.2)[1],
                              Model(L=16, pair=TL, pair_coef=0.7, pair_T=3, sigma=1.2,
                                    inertia=0.0))),
    ("gauss_L2", lambda: (random_lattice(7, 33, 65, 2),
                          Model(L=2, pair=POTTS, pair_coef=0.9, sigma=0.6, inertia=0.5))),
    ("L50_masked_8nb", lambda: (_scene(8, 19, 23, 50, 4.0)[1],
                                Model(L=50, nbhd=8, pair=TL, pair_coef=0.2, pair_T=6,
                                      sigma=4.0, inertia=1.0))),
    ("L200_potts", lambda: (_scene(9, 17, 40, 200, 15.0)[1],
                            Model(L=200, pair=POTTS, pair_coef=2.0, sigma=15.0,
                                  inertia=1.5))),
    ("one_row", lambda: (_scene(10, 1, 97, 16, 1.0)[1],
                         Model(L=16, pair=TL, pair_coef=0.8, pair_T=2, sigma=1.0,
                               inertia=1.0))),
    ("one_col_8nb", lambda: (_scene(11, 83, 1, 16, 1.0)[1],
                             Model(L=16, nbhd=8, pair=TL, pair_coef=0.8, pair_T=2,
                                   sigma=1.0, inertia=1.0))),
    ("one_pixel", lambda: (np.array([[3]], dtype=np.uint8),
                           Model(L=7, pair=TL, pair_coef=0.3, pair_T=2, sigma=1.0,
                                 inertia=0.5))),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("sampler", [0, 1], ids=["pca", "gibbs"])
def test_teacher_forced_parity(pc, name, make, sampler):
    g, m = make()
    sweeps = 6 if m.L >= 200 else 12
    mism, unflagged, total, fp64 = teacher_forced(pc, m, g, sweeps, sampler=sampler)
    assert unflagged == 0, f"{unflagged} mismatches at draws not near a CDF boundary"
    assert mism / total < MAX_MISMATCH_FRACTION or mism == 0, (mism, total)
    assert fp64 <= max(10, 0.05 * total), (fp64, total)


def test_binary_64_free_running_matches_oracle(pc):
    """Binary 64x64, 500 sweeps, burn-in 100: the whole chain and its
    posterior mean equal the oracle's; PSNR within 0.05 dB (identical)."""
    clean, noisy, m = binary_64()
    for sampler, order in ((0, None), (1, oracle.ORDER_COLOUR)):
        with pc.Chain(noisy, m, seed=1, chain_id=0, burn_in=100, sampler=sampler) as ch:
            ch.run(500)
            xg = ch.sample()
            mg = ch.mean()
            p_gpu, s_gpu = ch.metrics(clean, 0)
        kw = {} if order is None else {"order": order}
        xo, acc, nacc, _ = oracle.run_chain(m, noisy, 500, 100, seed=1, chain=0,
                                            sampler=sampler, **kw)
        assert nacc == 400
        assert np.array_equal(xg, xo)
        np.testing.assert_allclose(mg, acc / nacc, rtol=1e-6, atol=0)
        p_orc = om.psnr(acc / nacc, clean, 2)
        assert abs(p_gpu - p_orc) < 0.05
        assert abs(s_gpu - om.ssim(acc / nacc, clean, 2)) < 1e-6


def test_greyscale_512_sampled_parity(pc):
    """Greyscale 512^2, L=256: full-size launch; 20000 sampled sites per sweep
    recomputed by the oracle from the GPU's previous state."""
    clean, noisy, m = greyscale_512()
    rng = np.random.default_rng(0)
    H, W = noisy.shape
    with pc.Chain(noisy, m, seed=2, chain_id=0, burn_in=0) as ch:
        x = noisy.copy()
        for t in range(3):
            ch.run(1)
            xg = ch.sample()
            rows = rng.integers(0, H, 20000)
            cols = rng.integers(0, W, 20000)
            xo, near = oracle.pca_sites(m, noisy, x, rows, cols, 2, 0, t)
            d = xg[rows, cols] != xo
            assert int((d & (near == 0)).sum()) == 0
            assert int(d.sum()) == 0
            x = xg
        fp64 = ch.fp64_draws()
    assert fp64 < 0.01 * 3 * H * W


@pytest.mark.parametrize("L", [16, 256])
def test_large_8192_sampled_parity(pc, L):
    """8192^2 single image (L=16, sigma 1 / L=256, sigma 25): two full sweeps,
    sampled sites checked against the oracle."""
    from pcad_inputs import large_image
    clean, noisy, m = large_image(L=L)
    rng = np.random.default_rng(1)
    H, W = noisy.shape
    with pc.Chain(noisy, m, seed=3, chain_id=1, burn_in=0) as ch:
        x = noisy
        for t in range(2):
            ch.run(1)
            xg = ch.sample()
            rows = rng.integers(0, H, 20000)
            cols = rng.integers(0, W, 20000)
            xo, near = oracle.pca_sites(m, noisy, x, rows, cols, 3, 1, t)
            d = xg[rows, cols] != xo
            assert int((d & (near == 0)).sum()) == 0
            x = xg


@pytest.mark.parametrize("sampler", [0, 1])
def test_split_runs_and_graph_blocks_are_bit_identical(pc, sampler):
    _, g = _scene(12, 50, 61, 16, 1.3)
    m = Model(L=16, pair=TL, pair_coef=0.6, pair_T=3, sigma=1.3, inertia=1.2)
    outs = []
    for splits in ((500,), (300, 200), (33, 467), (1,) * 40 + (460,)):
        with pc.Chain(g, m, seed=5, chain_id=9, burn_in=120, sampler=sampler) as ch:
            for s in splits:
                ch.run(s)
            outs.append((ch.sample(), ch.mean(), ch.sweeps()))
    for x, mu, sw in outs[1:]:
        assert np.array_equal(x, outs[0][0])
        assert np.array_equal(mu, outs[0][1])
        assert sw == outs[0][2] == (500, 380)


def test_export_import_continues_identically(pc):
    _, g = _scene(13, 40, 44, 32, 2.0)
    m = Model(L=32, nbhd=8, pair=TL, pair_coef=0.3, pair_T=4, sigma=2.0, inertia=0.8)
    with pc.Chain(g, m, seed=8, chain_id=4, burn_in=20) as a:
        a.run(100)
        blob = a.export()
        b = pc.Chain.from_blob(blob)
        try:
            a.run(77)
            b.run(77)
            assert np.array_equal(a.sample(), b.sample())
            assert np.array_equal(a.mean(), b.mean())
            assert a.sweeps() == b.sweeps()
        finally:
            b.close()


def test_metrics_match_oracle(pc):
    rng = np.random.default_rng(3)
    for (H, W, L) in ((64, 80, 256), (7, 30, 16), (12, 11, 2)):
        clean = rng.integers(0, L, size=(H, W)).astype(np.uint8)
        est = np.clip(clean + rng.normal(0, L / 10, size=(H, W)), 0, L - 1).astype(np.float32)
        p, s = pc.pcad_metrics(est, clean, L)
        assert abs(p - om.psnr(est, clean, L)) < 1e-9
        ref = om.ssim(est, clean, L)
        assert abs(s - ref) < 1e-9 * max(1.0, abs(ref))


def test_invalid_arguments_are_rejected(pc):
    g = np.zeros((8, 8), dtype=np.uint8)
    bad = [Model(L=1), Model(L=257), Model(L=16, noise=FLIP, flip_p=0.1),
           Model(L=16, pair=TL, pair_coef=1.0, pair_T=30), Model(L=16, sigma=0.0),
           Model(L=16, inertia=-1.0), Model(L=16, nbhd=6)]
    for m in bad:
        with pytest.raises(pc.PcadError) as e:
            pc.Chain(g, m, seed=1)
        assert e.value.status == 1
    with pytest.raises(pc.PcadError):
        pc.Chain(np.full((4, 4), 20, np.uint8), Model(L=16), seed=1)
    with pc.Chain(g, Model(L=4, pair=TL, pair_coef=0.1, pair_T=1), seed=1) as ch:
        with pytest.raises(pc.PcadError):
            ch.set_sample(np.full((8, 8), 4, np.uint8))
        with pytest.raises(pc.PcadError) as e:
            ch.mean()
        assert e.value.status == 5
