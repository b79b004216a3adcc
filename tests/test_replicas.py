"""Host logic of the multi-rank path, on the CPU: the work assignment (every
item to exactly one rank, LPT balance), distinct chain ids, and -- in a
world_size-2 gloo process group -- the max-over-ranks time, the aggregate
rate and the gathered results that bench.py reports through."""
import os
import socket

import pytest

from paper_2507_14869_gb300 import replicas as rp


def test_shard_covers_disjointly_and_balances():
    costs = [5, 1, 8, 3, 3, 9, 2, 7, 4, 6, 1, 1]
    for world in (1, 2, 3, 5):
        parts = rp.shard(costs, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(costs)))
        loads = [sum(costs[i] for i in p) for p in parts]
        # LPT: the heaviest rank exceeds the mean by at most the largest item
        assert max(loads) <= sum(costs) / world + max(costs)
        assert parts == rp.shard(costs, world)   # deterministic
    assert rp.shard([], 3) == [[], [], []]
    with pytest.raises(ValueError):
        rp.shard([1], 0)


def test_chain_ids_are_distinct():
    ids = {rp.chain_id(r, k, 4) for r in range(8) for k in range(4)}
    assert len(ids) == 32
    with pytest.raises(ValueError):
        rp.chain_id(0, 4, 4)


def test_single_process_reductions_are_identities():
    assert rp.max_time(1.5) == 1.5
    assert rp.gather({3: "a"}) == {3: "a"}
    assert rp.aggregate_rate(10.0, 2.0, 1) == 5.0


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


COSTS = [5, 1, 8, 3, 3, 9, 2, 7, 4, 6]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = rp.shard(COSTS, world)[rank]
        results = rp.gather({i: 2 * COSTS[i] for i in mine})
        t = rp.max_time(1.0 + rank)
        rate = rp.aggregate_rate(100.0, 1.0 + rank, world)
        dist.barrier()
        q.put((rank, mine, results, t, rate))
    finally:
        dist.destroy_process_group()


def test_two_ranks_over_gloo():
    import multiprocessing as mpl
    ctx = mpl.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = {}
    try:
        for _ in range(2):
            rank, mine, results, t, rate = q.get(timeout=180)
            out[rank] = (mine, results, t, rate)
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert all(p.exitcode == 0 for p in procs)
    assert sorted(out[0][0] + out[1][0]) == list(range(len(COSTS)))
    expect = {i: 2 * c for i, c in enumerate(COSTS)}
    for r in (0, 1):
        mine, results, t, rate = out[r]
        assert results == expect           # every rank sees every item once
        assert t == 2.0                    # the slower rank's time
        assert rate == pytest.approx(2 * 100.0 / 2.0)
