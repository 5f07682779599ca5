"""Slab decomposition with one halo exchange per Tb-step block (paper Sec. 5.3),
on CPU: the exchange schedule and, with the oracle as each slab's local step,
the gathered result equals the oracle run over the whole grid bit for bit --
in one process (every slab's halo copied locally) and across world_size 2 and
3 gloo ranks (isend/irecv of host buffers)."""
import os
import socket

import numpy as np
import pytest

import oracle
import synth
from paper_2303_08365_gb300 import slabs

DIRICHLET, PERIODIC = 0, 1


def weights(ndim, radius, seed):
    v = synth.uniform(seed, (2 * radius + 1,) * ndim)
    return v / v.sum()


def test_bounds_and_halos():
    assert slabs.slab_bounds(10, 3) == [(0, 4), (4, 7), (7, 10)]
    L = slabs.SlabLayout((10, 5), 3, 1, 2, periodic=False)
    assert L.H == 2 and L.halo == [(0, 2), (2, 2), (2, 0)]
    assert [L.local_shape(k) for k in range(3)] == [(6, 5), (7, 5), (5, 5)]
    # slab 1 gets slab 0's last two owned planes below and slab 2's first two above
    assert (0, slice(2, 4), 1, slice(0, 2)) in L.messages()
    assert (2, slice(2, 4), 1, slice(5, 7)) in L.messages()
    P = slabs.SlabLayout((10, 5), 3, 2, 1, periodic=True)
    assert P.halo == [(2, 2)] * 3
    assert (2, slice(3, 5), 0, slice(0, 2)) in P.messages()  # the wrap: last slab feeds the first
    assert slabs.SlabLayout((9,), 1, 1, 4, periodic=True).halo == [(0, 0)]
    assert slabs.message_bytes(L) == 4 * 2 * 5 * 8
    with pytest.raises(ValueError):
        slabs.SlabLayout((5, 3), 3, 1, 2, periodic=False)  # slabs thinner than the halo


def oracle_step(w, radius, boundary):
    def step(k, a, steps):
        a[...] = oracle.run(np.asarray(a), w, radius, boundary, steps)
    return step


CASES = [
    # shape, radius, boundary, Tb, nslabs, T
    ((37, 23), 1, DIRICHLET, 3, 4, 10),
    ((37, 23), 1, PERIODIC, 3, 4, 10),
    ((17, 6, 5), 1, PERIODIC, 2, 3, 7),
    ((17, 6, 5), 1, DIRICHLET, 4, 2, 9),
    ((30, 11), 2, PERIODIC, 2, 3, 9),
    ((50,), 2, DIRICHLET, 4, 5, 13),
    ((12, 9), 1, PERIODIC, 5, 1, 11),
    ((8, 4, 4), 1, PERIODIC, 4, 2, 8),     # each slab exactly one halo deep; two neighbours are one slab
]


@pytest.mark.parametrize("shape,radius,boundary,Tb,nslabs,T", CASES)
def test_local_slabs_equal_the_whole_grid_bitwise(shape, radius, boundary, Tb, nslabs, T):
    w = weights(len(shape), radius, 40 + len(shape))
    u0 = synth.normal(41, shape)
    L = slabs.SlabLayout(shape, nslabs, radius, Tb, boundary == PERIODIC)
    arrays = []
    for k, (z0, z1) in enumerate(L.bounds):
        a = np.zeros(L.local_shape(k))
        a[L.owned_slice(k)] = u0[z0:z1]
        arrays.append(a)
    S = slabs.LocalSlabs(L, arrays, oracle_step(w, radius, boundary))
    S.run(T)
    got = S.gather(np.empty(shape))
    assert np.array_equal(got, oracle.run(u0, w, radius, boundary, T))
    assert S.exchanges == -(-T // Tb)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q, case):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        shape, radius, boundary, Tb, T = case
        w = weights(len(shape), radius, 50)
        u0 = synth.normal(51, shape)
        L = slabs.SlabLayout(shape, world, radius, Tb, boundary == PERIODIC)
        z0, z1 = L.bounds[rank]
        a = torch.zeros(L.local_shape(rank), dtype=torch.float64)
        a[L.owned_slice(rank)] = torch.from_numpy(u0[z0:z1])

        def step(k, arr, steps):
            arr.copy_(torch.from_numpy(oracle.run(arr.numpy(), w, radius, boundary, steps)))

        S = slabs.DistSlab(L, a, step)
        S.run(T)
        q.put((rank, z0, z1, S.owned().numpy().copy(), S.exchanges))
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(180)
@pytest.mark.parametrize("world,case", [
    (2, ((21, 13), 1, PERIODIC, 3, 8)),
    (2, ((10, 6, 7), 1, DIRICHLET, 2, 5)),
    (3, ((24, 9), 2, PERIODIC, 2, 7)),
])
def test_gloo_ranks_exchange_halos_and_equal_the_whole_grid(world, case):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q, case)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=150) for _ in range(world)]
    for p in procs:
        p.join(timeout=30)
        assert p.exitcode == 0
    shape, radius, boundary, Tb, T = case
    w = weights(len(shape), radius, 50)
    u0 = synth.normal(51, shape)
    ref = oracle.run(u0, w, radius, boundary, T)
    got = np.empty(shape)
    for rank, z0, z1, owned, nex in res:
        got[z0:z1] = owned
        assert nex == -(-T // Tb)
    assert np.array_equal(got, ref)
