"""Full-size GPU parity: the launches the benchmark times, against the FP64
oracle.

* The 512^2, L = 256 chain (truncated-linear prior, sigma 20, lambda 2) with
  the default kernel -- the windowed wavefront, 32 sweeps per launch --
  free-running for 64 sweeps: every label and the posterior mean equal the
  oracle's chain.
* Teacher-forced, every site, at least 4.2e6 draws per case (512^2 L = 256
  PCA on the windowed wavefront and checkerboard Gibbs on the tensor-core
  kernel, 1024^2 L = 16 PCA on the small-label kernel, 1024^2 L = 256 PCA
  and Gibbs on the windowed CUDA-core kernels): the mismatch count (zero
  expected), the fraction of draws
  the oracle flags as lying within 1e-6 of an FP64 CDF boundary, and the
  FP64 re-draws are printed.  With no mismatch in n >= 4.2e6 draws the
  one-sided 95 % bound on the mismatch rate is 3/n < 1e-6.
* The whole 512^2 workload -- 2000 sweeps, burn-in 500 -- against the
  oracle's OpenMP chain: identical labels, posterior mean and PSNR.
* 8192^2, L = 256 and L = 16, 32 sweeps in one captured graph (the headline
  L = 256 chain on the windowed sweep),
  checked at sampled sites through the sweeps' light cone: the oracle
  recomputes, sweep by sweep, only the sites within 31 - t of a sample, so
  the comparison after 32 sweeps is exact without running the whole image.
"""
import numpy as np
import pytest

import oracle
from oracle import metrics as om
from pcad_inputs import Model, gaussian_noise, greyscale_512, greyscale_scene, large_image

pytestmark = pytest.mark.gpu

MAX_MISMATCH_FRACTION = 1e-6


@pytest.fixture(scope="module")
def pc():
    import paper_2507_14869_gb300 as pc
    pc.lib()
    return pc


def test_512_default_kernel_multisweep_free_running(pc):
    clean, noisy, m = greyscale_512()
    with pc.Chain(noisy, m, seed=2, chain_id=0, burn_in=16) as ch:
        assert ch.kernel_in_use() == pc.PCAD_KERNEL_WINDOW_WAVE
        ch.run(32).run(32)          # two 32-sweep wavefront launches
        xg = ch.sample()
        mg = ch.mean()
        p_gpu, _ = ch.metrics(clean, 0)
    xo, acc, nacc, _ = oracle.run_chain(m, noisy, 64, 16, seed=2, chain=0)
    assert nacc == 48
    assert int((xg != xo).sum()) == 0
    np.testing.assert_allclose(mg, acc / nacc, rtol=1e-6, atol=0)
    assert abs(p_gpu - om.psnr(acc / nacc, clean, 256)) < 0.05


def _teacher_forced(pc, m, g, sweeps, sampler, seed, chain):
    ch = pc.Chain(g, m, seed=seed, chain_id=chain, burn_in=0, sampler=sampler)
    x = np.array(g, copy=True)
    mism = unflagged = near_total = total = 0
    try:
        kind = ch.kernel_in_use()
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
            near_total += int((near != 0).sum())
            total += d.size
            x = xg
        fp64 = ch.fp64_draws()
    finally:
        ch.close()
    return kind, mism, unflagged, near_total, total, fp64


def _l16_1024():
    clean = greyscale_scene(51, 1024, 1024, 16, n_shapes=20)
    noisy = gaussian_noise(52, clean, 1.0, 16)
    return noisy, Model(L=16, pair=1, pair_coef=0.05, pair_T=30, sigma=1.0, inertia=2.0)


def _l256_1024():
    """The roofline scene and prior at 1024^2: AUTO runs the windowed sweep."""
    _, noisy, m = large_image(seed=3, side=1024, L=256)
    return noisy, m


MANY = {
    "pca_512_L256": (lambda: greyscale_512()[1:], 0, 16),
    "gibbs_512_L256": (lambda: greyscale_512()[1:], 1, 16),
    "pca_1024_L16": (_l16_1024, 0, 4),
    "pca_1024_L256_windowed": (_l256_1024, 0, 4),
    "gibbs_1024_L256_windowed": (_l256_1024, 1, 4),
}


@pytest.mark.parametrize("name", list(MANY))
def test_teacher_forced_many_draws(pc, name):
    make, sampler, sweeps = MANY[name]
    g, m = make()
    kind, mism, unflagged, near, total, fp64 = _teacher_forced(pc, m, g, sweeps, sampler, 2, 0)
    if name.endswith("windowed"):
        assert kind in (pc.PCAD_KERNEL_WINDOW, pc.PCAD_KERNEL_WINDOW_WAVE)
    print(f"\n[parity] {name}: kernel {kind}, {total} draws, {mism} mismatches, "
          f"{near} near-boundary ({near / total:.3e}), {fp64} FP64 re-draws "
          f"({fp64 / total:.3e}); 95% bound on the mismatch rate {3.0 / total:.2e}")
    assert total >= 4_194_304
    assert unflagged == 0
    assert mism / total < MAX_MISMATCH_FRACTION
    assert mism == 0


@pytest.mark.slow
def test_512_whole_workload_matches_oracle(pc):
    """2000 sweeps, burn-in 500, as the benchmark runs it (about a minute of
    oracle time on 16 cores)."""
    clean, noisy, m = greyscale_512()
    with pc.Chain(noisy, m, seed=2, chain_id=0, burn_in=500) as ch:
        ch.run(2000)
        xg = ch.sample()
        mg = ch.mean()
        p_gpu, s_gpu = ch.metrics(clean, 0)
    xo, acc, nacc, _ = oracle.run_chain(m, noisy, 2000, 500, seed=2, chain=0)
    assert nacc == 1500
    assert int((xg != xo).sum()) == 0
    np.testing.assert_allclose(mg, acc / nacc, rtol=1e-6, atol=0)
    p_orc = om.psnr(acc / nacc, clean, 256)
    print(f"\n[parity] 512^2 L=256 2000 sweeps: PSNR GPU {p_gpu:.4f} dB, oracle {p_orc:.4f} dB")
    assert abs(p_gpu - p_orc) < 0.05
    assert abs(s_gpu - om.ssim(acc / nacc, clean, 256)) < 1e-6


def _boxes(sr, sc, r, H, W):
    """Row and column indices of the union of the squares of radius r around
    the samples (clipped to the image), each site once."""
    idx = []
    for a, b in zip(sr, sc):
        rr = np.arange(max(0, a - r), min(H, a + r + 1), dtype=np.int64)
        cc = np.arange(max(0, b - r), min(W, b + r + 1), dtype=np.int64)
        idx.append((rr[:, None] * W + cc[None, :]).ravel())
    u = np.unique(np.concatenate(idx))
    return (u // W).astype(np.int32), (u % W).astype(np.int32)


def _cone_check(m, g, xg, seed, chain, nsweeps, samples, r_end=2):
    """Oracle state after nsweeps at the sites within r_end of each sample,
    computing at sweep t only the sites within r_end + nsweeps - 1 - t (the
    sites whose later values reach the samples)."""
    H, W = g.shape
    x = np.array(g, copy=True)
    sr = [s[0] for s in samples]
    sc = [s[1] for s in samples]
    for t in range(nsweeps):
        rows, cols = _boxes(sr, sc, r_end + nsweeps - 1 - t, H, W)
        xo, _ = oracle.pca_sites(m, g, x, rows, cols, seed, chain, t)
        x[rows, cols] = xo          # every read of this sweep happened inside the call
    rows, cols = _boxes(sr, sc, r_end, H, W)
    return int((xg[rows, cols] != x[rows, cols]).sum()), int(rows.size)


@pytest.mark.parametrize("L", [256, 16])
def test_8192_one_32_sweep_launch_light_cone(pc, L):
    clean, noisy, m = large_image(L=L)
    H, W = noisy.shape
    rng = np.random.default_rng(5)
    samples = [(0, 0), (0, W - 1), (H - 1, 0), (H - 1, W - 1), (0, W // 2), (H // 2, 0),
               (H - 1, 4097), (3001, W - 1), (4095, 4096)]
    samples += [(int(a), int(b)) for a, b in zip(rng.integers(0, H, 31), rng.integers(0, W, 31))]
    with pc.Chain(noisy, m, seed=3, chain_id=1, burn_in=0) as ch:
        ch.run(32)                   # one captured 32-sweep block
        xg = ch.sample()
    bad, n = _cone_check(m, noisy, xg, 3, 1, 32, samples)
    print(f"\n[parity] 8192^2 L={L}, 32 sweeps in one graph: {n} sites compared, {bad} differ")
    assert bad == 0
