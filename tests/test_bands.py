"""Host logic of the row-band decomposition, on the CPU.

* The band layout: owned rows partition the image, each buffer is the owned
  rows plus `halo` rows on each inner side, clipped at the image edges.
* The exchange schedule over a gloo process group (2 and 3 ranks): each rank
  runs the FP64 oracle's lazy-PCA draws on its band's buffer only (global
  rows, so the draws are the whole image's), exchanges halos after every
  block of `halo` sweeps through bands.exchange, and the owned rows gathered
  at the end equal the oracle's whole-image chain label for label.  A
  schedule that exchanged too late, sent the wrong rows or skipped a
  neighbour would leave wrong labels near the band edges."""
import os
import socket

import numpy as np
import pytest

from paper_2507_14869_gb300 import bands as bd


def test_layout_partitions_rows_and_clips_halos():
    for H, n, halo in ((37, 3, 4), (64, 2, 32), (100, 7, 5), (9, 1, 64), (12, 4, 3)):
        lay = bd.layout(H, n, halo)
        assert lay[0].own0 == 0 and lay[-1].own1 == H
        for a, b in zip(lay, lay[1:]):
            assert a.own1 == b.own0
        for b in lay:
            assert b.own1 - b.own0 >= (halo if n > 1 else 1)
            assert b.buf0 == max(0, b.own0 - halo) and b.buf1 == min(H, b.own1 + halo)
        for i in range(n):
            for nb, r0, r1 in bd.halo_plan(lay, i):
                assert abs(nb - i) == 1
                assert lay[nb].own0 <= r0 < r1 <= lay[nb].own1       # the neighbour owns them
                assert lay[i].buf0 <= r0 and r1 <= lay[i].buf1       # this band holds them
    with pytest.raises(ValueError):
        bd.layout(10, 3, 4)        # bands of 3 rows cannot carry a 4-row halo
    with pytest.raises(ValueError):
        bd.layout(10, 0, 1)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _case(name):
    """Weak data term, strong prior: a wrong halo row changes labels several
    rows in within the test's sweeps (checked: skipping the exchange leaves
    dozens of wrong labels in each case)."""
    from pcad_inputs import Model, gaussian_noise, greyscale_scene
    if name == "L16_8nb":
        g = gaussian_noise(62, greyscale_scene(61, 37, 23, 16, n_shapes=5), 4.0, 16)
        m = Model(L=16, nbhd=8, pair=1, pair_coef=0.6, pair_T=4, sigma=4.0, inertia=0.5)
    else:
        g = gaussian_noise(66, greyscale_scene(65, 31, 29, 16, n_shapes=5), 4.0, 16)
        m = Model(L=16, nbhd=4, pair=1, pair_coef=0.9, pair_T=4, sigma=4.0, inertia=0.5)
    return g, m


SWEEPS, SEED, CHAIN = 40, 9, 4


def _band_rank(rank, world, port, q, name, halo):
    import torch
    import torch.distributed as dist

    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        g, m = _case(name)
        H, W = g.shape
        lay = bd.layout(H, world, halo)
        me = lay[rank]
        x = np.array(g, copy=True)     # only this band's buffer rows are kept up to date
        rr, cc = np.meshgrid(np.arange(me.buf0, me.buf1), np.arange(W), indexing="ij")
        rows, cols = rr.ravel().astype(np.int32), cc.ravel().astype(np.int32)
        for start in range(0, SWEEPS, halo):
            for t in range(start, min(SWEEPS, start + halo)):
                xo, _ = oracle.pca_sites(m, g, x, rows, cols, SEED, CHAIN, t)
                x[rows, cols] = xo
            buf = torch.from_numpy(np.ascontiguousarray(x[me.buf0:me.buf1]))
            bd.exchange(buf, lay, rank, dist)
            x[me.buf0:me.buf1] = buf.numpy()
        q.put((rank, me.own0, x[me.own0:me.own1].copy()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("name,world,halo", [("L16_8nb", 3, 4), ("L16_8nb", 2, 5),
                                             ("L16_4nb", 2, 3)])
def test_exchange_schedule_over_gloo_matches_the_whole_image(orc, name, world, halo):
    import multiprocessing as mpl
    ctx = mpl.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_band_rank, args=(r, world, port, q, name, halo))
             for r in range(world)]
    for p in procs:
        p.start()
    parts = {}
    try:
        for _ in range(world):
            rank, own0, rows = q.get(timeout=180)
            parts[rank] = (own0, rows)
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert all(p.exitcode == 0 for p in procs)
    g, m = _case(name)
    x_whole, _, _, _ = orc.run_chain(m, g, SWEEPS, 0, seed=SEED, chain=CHAIN)
    got = np.concatenate([parts[r][1] for r in range(world)], axis=0)
    assert got.shape == g.shape
    assert np.array_equal(got, x_whole)
