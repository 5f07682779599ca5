"""Slab decomposition on one GPU (the multi-GPU path emulated with k slabs on
one device, halos exchanged by device-local copies once per Tb-step block):
the gathered grid is bitwise equal to the single-grid sweep, whatever kernel
each slab's plan runs, and within 1e-12 of the oracle."""
import numpy as np
import pytest

import oracle
import synth
from conftest import normwise_rel
from paper_2303_08365_gb300 import slabs

pytestmark = pytest.mark.gpu
TOL = 1e-12
DIRICHLET, PERIODIC = 0, 1


@pytest.fixture(scope="module")
def st():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2303_08365_gb300 import build
    build.build()
    import paper_2303_08365_gb300 as st
    return st


def weights(ndim, radius, seed, star=False):
    v = synth.uniform(seed, (2 * radius + 1,) * ndim)
    if star:
        c = (radius,) * ndim
        m = np.zeros_like(v, dtype=bool)
        for d in range(ndim):
            idx = list(c)
            for o in range(2 * radius + 1):
                idx[d] = o
                m[tuple(idx)] = True
            idx[d] = radius
        v = np.where(m, v, 0.0)
    return v / v.sum()


CASES = [
    # shape, radius, boundary, star, Tb, nslabs, T, local tuning (Tb, variant name) or None
    ((40, 64, 128), 1, PERIODIC, True, 4, 3, 9, None),
    ((40, 64, 128), 1, PERIODIC, True, 4, 3, 9, (4, "exchange")),
    ((30, 40, 64), 1, DIRICHLET, False, 2, 4, 7, None),
    ((30, 40, 64), 1, DIRICHLET, False, 8, 2, 17, (8, "exchange")),
    ((300, 257), 1, DIRICHLET, True, 8, 2, 19, None),
    ((120, 96), 2, PERIODIC, False, 3, 4, 10, None),
    ((5000,), 2, DIRICHLET, True, 8, 3, 21, None),
]


@pytest.mark.parametrize("shape,radius,boundary,star,Tb,nslabs,T,tuning", CASES)
def test_slabs_on_one_device_equal_the_single_grid(st, shape, radius, boundary, star, Tb, nslabs, T, tuning):
    import torch
    w = weights(len(shape), radius, 60 + len(shape), star=star)
    u0 = synth.normal(61, shape)
    g = torch.from_numpy(u0.copy()).cuda()
    L = slabs.SlabLayout(shape, nslabs, radius, Tb, boundary == PERIODIC)
    tun = None if tuning is None else (tuning[0], {"exchange": st.VARIANT_EXCHANGE}[tuning[1]])
    step, plans = slabs.make_gpu_steps(L, radius, w, boundary, tuning=tun)
    S = slabs.LocalSlabs.scatter(L, g, step)
    S.run(T)
    got = S.gather(torch.empty_like(g)).cpu().numpy()
    for p in plans:
        assert p.status() == 0
        p.close()
    single = st.Plan(shape, radius, w, boundary)
    single.run(g, T)
    ref_gpu = g.cpu().numpy()
    single.close()
    assert np.array_equal(got, ref_gpu)
    assert normwise_rel(got, oracle.run(u0, w, radius, boundary, T, nthreads=0)) <= TOL
    assert S.exchanges == -(-T // Tb)
