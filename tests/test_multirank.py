"""The N>1 host path on CPU with the gloo backend (world_size 2): each rank
computes its shard of the 96-grid batch independently, the shards are
disjoint and cover the batch, loads are balanced, and the timing reduction
returns the maximum over ranks."""
import os
import socket

import pytest

import synth
from paper_2303_08365_gb300 import shard


def test_shard_covers_and_balances():
    items = synth.batch_items(synth.SEED_BATCH)
    for world in (1, 2, 3, 8):
        parts = shard.shard_items(items, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(items)))
        loads = [sum(shard.item_cost(items[i]) for i in p) for p in parts]
        biggest = max(shard.item_cost(it) for it in items)
        assert max(loads) - min(loads) <= biggest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        items = synth.batch_items(synth.SEED_BATCH)
        mine = shard.rank_items(items, rank, world)
        import torch
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)
        t_max = shard.max_over_ranks(1.5 + rank)
        n_all = shard.sum_over_ranks(len(mine))
        q.put((rank, gathered, t_max, n_all))
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_gloo_ranks_partition_the_batch():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=100) for _ in range(2)]
    for p in procs:
        p.join(timeout=30)
        assert p.exitcode == 0
    items = synth.batch_items(synth.SEED_BATCH)
    for rank, gathered, t_max, n_all in res:
        assert t_max == 2.5
        assert n_all == len(items)
        a, b = gathered
        assert not set(a) & set(b)
        assert sorted(a + b) == list(range(len(items)))
