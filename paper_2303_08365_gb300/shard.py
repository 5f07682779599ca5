"""Host-side work split across ranks (one process per GPU).

The single-grid sweeps run as independent replicas, one per rank.  The
batched form is a set of independent grids, so it is partitioned: each rank
advances a disjoint subset, chosen by greedy longest-processing-time packing
on the cost cells x T, and no data moves between ranks.  The only collective
is the timing reduction (barrier, then the maximum over ranks).
"""


def item_cost(item):
    ny, nx, _alpha, T = item
    return int(ny) * int(nx) * int(T)


def shard_items(items, world):
    """Index lists, one per rank: every item exactly once, loads balanced by
    assigning items in decreasing cost to the least-loaded rank (ties: the
    lowest rank; equal costs keep their input order)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(items)), key=lambda i: (-item_cost(items[i]), i))
    loads = [0] * world
    parts = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (loads[k], k))
        parts[r].append(i)
        loads[r] += item_cost(items[i])
    for p in parts:
        p.sort()
    return parts


def rank_items(items, rank, world):
    return shard_items(items, world)[rank]


def max_over_ranks(value, group=None):
    """Barrier, then the maximum of a host float over all ranks (gloo or nccl)."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized():
        return float(value)
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.barrier(group)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def sum_over_ranks(value, group=None):
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized():
        return float(value)
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return float(t.item())
