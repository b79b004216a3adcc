"""The allocation-free entry point (pcad_pca_run_noalloc) against the chain
API.  It exists for callers that must not allocate device memory -- their
framework already owns the GPU's memory, or their loop cannot afford
cudaMalloc/cudaFree, which may synchronise the device -- so it keeps its
extra label plane, tables and counters in a fixed array inside the library.
Three calls in a row (different sizes and models; the last one with a row
pitch wider than the image and the 8-neighbourhood) must each reproduce the
chain API's sample and posterior mean; the later calls also show that the
shared array is re-initialised, and the padding bytes of the pitched output
stay untouched.  This file is collected last."""
import numpy as np
import pytest

from pcad_inputs import Model, gaussian_noise, greyscale_scene

pytestmark = pytest.mark.gpu


def _case(seed, H, W, L, sigma):
    clean = greyscale_scene(seed, H, W, L, n_shapes=6)
    return gaussian_noise(seed + 1, clean, sigma, L)


CALLS = [
    (_case(21, 70, 97, 16, 1.2), Model(L=16, pair=1, pair_coef=0.6, pair_T=3, sigma=1.2,
                                       inertia=1.5), 11, 2, 53, 20),
    (_case(22, 45, 64, 256, 20.0), Model(L=256, pair=1, pair_coef=0.05, pair_T=30, sigma=20.0,
                                         inertia=2.0), 12, 5, 40, 10),
    (_case(23, 37, 51, 16, 1.0), Model(L=16, nbhd=8, pair=1, pair_coef=0.3, pair_T=4,
                                       sigma=1.0, inertia=1.0), 13, 6, 25, 5),
]
PITCH_PAD = (0, 0, 29)   # extra bytes per row of the third call's pitched planes


def test_noalloc_matches_chain_api_twice_in_a_row():
    torch = pytest.importorskip("torch")
    import paper_2507_14869_gb300 as pc
    assert torch.cuda.is_available()
    stream = torch.cuda.current_stream()
    for (g, m, seed, chain, n, burn), pad in zip(CALLS, PITCH_PAD):
        H, W = g.shape
        P = W + pad
        with pc.Chain(g, m, seed=seed, chain_id=chain, burn_in=burn) as ch:
            ch.run(n)
            x_ref = ch.sample()
            mean_ref = ch.mean()
        g_pad = np.full((H, P), 7, dtype=np.uint8)
        g_pad[:, :W] = g
        g_dev = torch.from_numpy(g_pad).cuda()
        sample = torch.full((H, P), 0xAB, dtype=torch.uint8, device="cuda")
        mean = torch.full((H, W), -1.0, dtype=torch.float32, device="cuda")
        pc.pcad_pca_run_noalloc(g_dev.data_ptr(), H, W, P, m, seed, chain, n, burn,
                                sample.data_ptr(), mean.data_ptr(), stream)
        torch.cuda.synchronize()
        out = sample.cpu().numpy()
        assert np.array_equal(out[:, :W], x_ref)
        assert (out[:, W:] == 0xAB).all()
        np.testing.assert_allclose(mean.cpu().numpy(), mean_ref, rtol=1e-6, atol=0.0)


def test_noalloc_rejects_oversize_and_gibbs():
    torch = pytest.importorskip("torch")
    import paper_2507_14869_gb300 as pc
    m = Model(L=16, pair=1, pair_coef=0.6, pair_T=3, sigma=1.2, inertia=1.5)
    g = torch.zeros((4, 4), dtype=torch.uint8, device="cuda")
    out = torch.zeros((4, 4), dtype=torch.uint8, device="cuda")
    mean = torch.zeros((4, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(pc.PcadError) as e:
        pc.pcad_pca_run_noalloc(g.data_ptr(), 4096, 4096, 4096, m, 1, 0, 1, 0,
                                out.data_ptr(), mean.data_ptr(), None)
    assert e.value.status == 1
    for off in (0, 3, -3):                   # the sample plane over the observation
        with pytest.raises(pc.PcadError) as e:
            pc.pcad_pca_run_noalloc(out.data_ptr(), 4, 4, 4, m, 1, 0, 1, 0,
                                    out.data_ptr() + off, mean.data_ptr(), None)
        assert e.value.status == 1
    with pytest.raises(pc.PcadError) as e:   # the mean buffer over the sample plane
        pc.pcad_pca_run_noalloc(g.data_ptr(), 4, 4, 4, m, 1, 0, 1, 0,
                                out.data_ptr(), out.data_ptr() + 8, None)
    assert e.value.status == 1
    nm = Model(L=16, pair=1, pair_coef=0.6, pair_T=3, sigma=1.2, inertia=1.5, inertia_norm=1)
    with pytest.raises(pc.PcadError) as e:
        pc.pcad_pca_run_noalloc(g.data_ptr(), 4, 4, 4, nm, 1, 0, 1, 0,
                                out.data_ptr(), mean.data_ptr(), None)
    assert e.value.status == 1
    gm = Model(L=16, pair=1, pair_coef=0.6, pair_T=3, sigma=1.2, inertia=1.5, sampler=1)
    with pytest.raises(pc.PcadError) as e:
        pc.pcad_pca_run_noalloc(g.data_ptr(), 4, 4, 4, gm, 1, 0, 1, 0,
                                out.data_ptr(), mean.data_ptr(), None)
    assert e.value.status == 1
