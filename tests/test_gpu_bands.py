"""Row bands of one image on one GPU: 1, 2 and 3 band chains exchanging
their halo rows after every block of `halo` sweeps (pcad_bands_*) equal the
whole-image chain bit for bit -- sample and posterior mean -- on the
tensor-core sweep (L = 256) and the CUDA-core kernels (L = 16, 4- and
8-neighbourhood), for run lengths that end inside a block and burn-ins that
end inside one.  The pieces of the one-band-per-rank runner (a chain's row
offset and device-to-device row writes) are checked the same way with the
exchange done in one process."""
import numpy as np
import pytest

from pcad_inputs import Model, gaussian_noise, greyscale_scene

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pc():
    import paper_2507_14869_gb300 as pc
    pc.lib()
    return pc


def _grey(seed, H, W, L, sigma):
    return gaussian_noise(seed + 1, greyscale_scene(seed, H, W, L, n_shapes=6), sigma, L)


CASES = {
    "tc_L256": (lambda: _grey(71, 150, 96, 256, 20.0),
                Model(L=256, pair=1, pair_coef=0.05, pair_T=30, sigma=20.0, inertia=2.0),
                (1, 2, 3), 32, 70, 20),
    "L16_4nb": (lambda: _grey(72, 97, 130, 16, 2.0),
                Model(L=16, pair=1, pair_coef=0.6, pair_T=4, sigma=2.0, inertia=0.8),
                (2, 3), 5, 41, 7),
    "L16_8nb": (lambda: _grey(73, 64, 77, 16, 2.0),
                Model(L=16, nbhd=8, pair=1, pair_coef=0.4, pair_T=4, sigma=2.0, inertia=0.8),
                (3,), 8, 33, 40),
}


def _whole(pc, g, m, n, burn, seed=12, chain=5):
    with pc.Chain(g, m, seed=seed, chain_id=chain, burn_in=burn) as ch:
        ch.run(n)
        return ch.sample(), (ch.mean() if n > burn else None)


@pytest.mark.parametrize("name", list(CASES))
def test_bands_equal_the_whole_image(pc, name):
    make, m, counts, halo, n, burn = CASES[name]
    g = make()
    H, W = g.shape
    x_ref, mean_ref = _whole(pc, g, m, n, burn)
    for nb in counts:
        b = pc.pcad_bands_create(g, m, seed=12, chain_id=5, burn_in=burn, nbands=nb, halo=halo)
        try:
            pc.pcad_bands_run(b, 23)            # two runs, the first ending inside a block
            pc.pcad_bands_run(b, n - 23)
            pc.pcad_bands_sync(b)
            info = [pc.pcad_bands_info(b, i) for i in range(nb)]
            assert info[0]["own0"] == 0 and info[-1]["own1"] == H and info[0]["t"] == n
            x = pc.pcad_bands_read_sample(b, H, W)
            assert np.array_equal(x, x_ref), (nb, int((x != x_ref).sum()))
            if mean_ref is not None:
                assert np.array_equal(pc.pcad_bands_read_mean(b, H, W), mean_ref), nb
        finally:
            pc.pcad_bands_destroy(b)


def test_bands_refuse_gibbs_and_oversized_halos(pc):
    g = _grey(74, 40, 40, 16, 1.0)
    m = Model(L=16, pair=1, pair_coef=0.6, pair_T=4, sigma=1.0, inertia=0.8)
    for kw in (dict(nbands=2, halo=21), dict(nbands=0, halo=4), dict(nbands=2, halo=0),
               dict(nbands=65, halo=1), dict(nbands=2, halo=65)):
        with pytest.raises(pc.PcadError) as e:
            pc.pcad_bands_create(g, m, seed=1, **kw)
        assert e.value.status == 1, kw
    gm = Model(L=16, pair=1, pair_coef=0.6, pair_T=4, sigma=1.0, sampler=1)
    with pytest.raises(pc.PcadError):
        pc.pcad_bands_create(g, gm, seed=1, nbands=2, halo=4)
    with pc.Chain(g, gm, seed=1) as ch:
        with pytest.raises(pc.PcadError):
            ch.set_row_offset(8)


def test_rank_runner_pieces_in_one_process(pc):
    """The one-band-per-rank runner's steps -- a chain per band with its row
    offset, the current state read to device memory, the halo rows written
    back from the neighbours' -- with the exchange done in one process by
    the same halo plan: the owned rows equal the whole-image chain."""
    torch = pytest.importorskip("torch")
    from paper_2507_14869_gb300 import bands as bd
    g = _grey(75, 90, 70, 16, 2.0)
    m = Model(L=16, pair=1, pair_coef=0.6, pair_T=4, sigma=2.0, inertia=0.8)
    n, halo, world = 29, 6, 3
    x_ref, mean_ref = _whole(pc, g, m, n, 4)
    lay = bd.layout(g.shape[0], world, halo)
    chains = []
    try:
        for me in lay:
            ch = pc.Chain(g[me.buf0:me.buf1], m, seed=12, chain_id=5, burn_in=4)
            ch.set_row_offset(me.buf0)
            chains.append(ch)
        W = g.shape[1]
        bufs = [torch.empty((me.buf1 - me.buf0, W), dtype=torch.uint8, device="cuda")
                for me in lay]
        for done in range(0, n, halo):
            for ch, x in zip(chains, bufs):
                ch.run(min(halo, n - done))
                pc.pcad_chain_read_sample_dev(ch.h, x.data_ptr(), W)
                ch.sync()
            for r, (ch, me) in enumerate(zip(chains, lay)):
                for nb, r0, r1 in bd.halo_plan(lay, r):
                    src = bufs[nb][r0 - lay[nb].buf0:r1 - lay[nb].buf0].contiguous()
                    ch.write_rows_dev(r0 - me.buf0, r1 - r0, src.data_ptr(), W)
                    ch.sync()
        got = np.concatenate([ch.sample()[me.own0 - me.buf0:me.own1 - me.buf0]
                              for ch, me in zip(chains, lay)])
        mean = np.concatenate([ch.mean()[me.own0 - me.buf0:me.own1 - me.buf0]
                               for ch, me in zip(chains, lay)])
        assert np.array_equal(got, x_ref)
        assert np.array_equal(mean, mean_ref)
    finally:
        for ch in chains:
            ch.close()
