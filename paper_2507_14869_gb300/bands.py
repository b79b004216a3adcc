"""Row bands of one image over several processes (one band per rank).

The lazy PCA draws every site from the previous configuration only (Section
3, Eq. general_pca_definition), so after k sweeps a label depends only on
the sites within k rows of it.  Band b owns rows [floor(b H / n),
floor((b + 1) H / n)) and holds `halo` extra rows on each inner side; after
every block of `halo` sweeps the bands exchange those rows with their
neighbours (one send and one receive per neighbour: the single exchange
step of a block).  The same rule drives ``pcad_bands_*`` inside one process
(include/pcaden.h); here the exchange goes through ``torch.distributed``
point-to-point calls (NCCL between GPUs, gloo on CPU tensors), and each rank
runs its band with a chain whose row offset keys the draws by global row.
"""
from __future__ import annotations

from dataclasses import dataclass


@dataclass(frozen=True)
class Band:
    own0: int   # first owned row (global)
    own1: int   # one past the last owned row
    buf0: int   # first row of the band's buffer (owned rows plus halos)
    buf1: int


def layout(H: int, nbands: int, halo: int) -> list:
    """Owned and buffered rows of every band (the rule pcad_bands_create uses)."""
    if nbands < 1 or halo < 1:
        raise ValueError("nbands and halo must be >= 1")
    if nbands > 1 and H // nbands < halo:
        raise ValueError("every band must own at least `halo` rows")
    out = []
    for b in range(nbands):
        o0, o1 = b * H // nbands, (b + 1) * H // nbands
        out.append(Band(o0, o1, max(0, o0 - halo), min(H, o1 + halo)))
    return out


def halo_plan(bands: list, b: int) -> list:
    """The copies band b receives after a block: (neighbour, global row range),
    each range owned by that neighbour and mirrored by b's halo."""
    me = bands[b]
    plan = []
    if b > 0 and me.buf0 < me.own0:
        plan.append((b - 1, me.buf0, me.own0))
    if b + 1 < len(bands) and me.own1 < me.buf1:
        plan.append((b + 1, me.own1, me.buf1))
    return plan


def exchange(x, bands: list, rank: int, dist, group=None) -> None:
    """One exchange step for this rank's band: x is its buffer (buf1 - buf0
    rows, a torch tensor on the transport's device).  Sends the owned rows
    each neighbour mirrors and receives this band's halo rows in place."""
    me = bands[rank]
    ops, recv = [], []
    for nb, r0, r1 in halo_plan(bands, rank):
        buf = x.new_empty((r1 - r0,) + tuple(x.shape[1:]))
        ops.append(dist.P2POp(dist.irecv, buf, nb, group))
        recv.append((buf, r0 - me.buf0, r1 - me.buf0))
    for nb in (rank - 1, rank + 1):
        if 0 <= nb < len(bands):
            for who, r0, r1 in halo_plan(bands, nb):
                if who == rank:      # rows of mine that neighbour nb mirrors
                    ops.append(dist.P2POp(dist.isend, x[r0 - me.buf0:r1 - me.buf0].contiguous(),
                                          nb, group))
    if ops:
        for req in dist.batch_isend_irecv(ops):
            req.wait()
    for buf, a, b in recv:
        x[a:b] = buf


def run_rank(pc, torch, dist, g, model, seed: int, chain_id: int, burn_in: int, nsweeps: int,
             halo: int, rank: int, world: int, stream=None):
    """This rank's band of the chain on its current GPU, exchanging halos over
    `dist` (NCCL) after every block of `halo` sweeps.  Returns the band's
    owned rows of the final sample and of the posterior mean (numpy)."""
    bands = layout(g.shape[0], world, halo)
    me = bands[rank]
    H_b, W = me.buf1 - me.buf0, g.shape[1]
    ch = pc.Chain(g[me.buf0:me.buf1], model, seed=seed, chain_id=chain_id, burn_in=burn_in,
                  stream=stream)
    try:
        ch.set_row_offset(me.buf0)
        x = torch.empty((H_b, W), dtype=torch.uint8, device="cuda")
        for done in range(0, nsweeps, halo):
            ch.run(min(halo, nsweeps - done))
            pc.pcad_chain_read_sample_dev(ch.h, x.data_ptr(), W)
            ch.sync()
            exchange(x, bands, rank, dist)
            torch.cuda.synchronize()   # received rows in x before the chain's stream reads them
            for _, r0, r1 in halo_plan(bands, rank):
                ch.write_rows_dev(r0 - me.buf0, r1 - r0, x[r0 - me.buf0].data_ptr(), W)
        a, b = me.own0 - me.buf0, me.own1 - me.buf0
        return ch.sample()[a:b], ch.mean()[a:b]
    finally:
        ch.close()
