"""Grids of more than 2^31 cells: the sweeps address cells with 64-bit
offsets, so results past the 2^31-th cell must still match the oracle.

Each input is a seeded block of prime side lengths tiled over the grid (the
tile period is co-prime with every power of two, so a wrong 32-bit offset
lands on a different value).  The oracle evaluates windows past the 2^31-th
cell from their light cones: a sub-grid that extends r*T cells beyond the
window (clipped at the grid's faces, where its own Dirichlet ghosts are the
true ones) gives exact values on the window after T steps.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from conftest import normwise_rel

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
TOL = 1e-12
DIRICHLET = 0


@pytest.fixture(scope="module")
def st():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2303_08365_gb300 import build
    build.build()
    import paper_2303_08365_gb300 as st
    return st


def star_weights(ndim, radius, seed):
    v = synth.uniform(seed, (2 * radius * ndim + 1,))
    v = v / v.sum()
    w = np.zeros((2 * radius + 1,) * ndim)
    c = (radius,) * ndim
    w[c] = v[0]
    k = 1
    for d in range(ndim):
        for o in range(-radius, radius + 1):
            if o:
                idx = list(c)
                idx[d] += o
                w[tuple(idx)] = v[k]
                k += 1
    return w


def tiled_on_device(block, shape):
    """The grid u0[x] = block[x mod block.shape], built slab by slab on the device."""
    import torch
    bd = torch.from_numpy(block).cuda()
    g = torch.empty(shape, dtype=torch.float64, device="cuda")
    reps = [1] + [math.ceil(n / b) for n, b in zip(shape[1:], block.shape[1:])]
    for s0 in range(0, shape[0], block.shape[0]):
        h = min(block.shape[0], shape[0] - s0)
        slab = bd[:h].repeat(*reps)
        g[s0:s0 + h] = slab[(slice(None),) + tuple(slice(0, n) for n in shape[1:])]
        del slab
    return g


def tiled_on_host(block, lo, hi):
    idx = [np.arange(a, b) % n for a, b, n in zip(lo, hi, block.shape)]
    return block[np.ix_(*idx)]


def window_by_light_cone(block, shape, w, radius, T, lo, hi):
    m = radius * T
    slo = [max(0, a - m) for a in lo]
    shi = [min(n, b + m) for b, n in zip(hi, shape)]
    sub = tiled_on_host(block, slo, shi)
    out = oracle.run(sub, w, radius, DIRICHLET, T)
    return out[tuple(slice(a - s, b - s) for a, b, s in zip(lo, hi, slo))]


CASES = [
    # shape, radius, block, T, windows (lo corners; 9 or 5 cells a side)
    ((33100, 65000), 1, (997, 1009), 2,
     [(0, 0), (33050, 0), (33050, 32500), (33091, 64991)]),
    ((1300, 1300, 1300), 1, (97, 101, 103), 2,
     [(0, 0, 0), (1280, 650, 640), (1295, 1295, 1295), (1299, 0, 1295)]),
    ((1300, 1300, 1300), 2, (97, 101, 103), 2,
     [(1280, 3, 1201), (1295, 1295, 1295)]),
]


@pytest.mark.parametrize("shape,radius,bshape,T,windows", CASES)
def test_grid_past_2_31_cells_matches_oracle(st, shape, radius, bshape, T, windows):
    import torch
    cells = math.prod(shape)
    assert cells > 2 ** 31
    need = 2.3 * cells * 8  # grid + the plan's partner buffer + one fill slab
    if torch.cuda.mem_get_info()[0] < need:
        pytest.skip(f"needs {need / 2**30:.0f} GiB of free device memory")
    ndim = len(shape)
    block = synth.uniform(synth.SEED_HEAT3D + 40 + ndim + radius, bshape)
    w = star_weights(ndim, radius, synth.SEED_HEAT3D + 50 + ndim + radius)
    g = tiled_on_device(block, shape)
    p = st.Plan(shape, radius, w, DIRICHLET)
    p.run(g, T)
    torch.cuda.synchronize()
    side = 9 if ndim == 2 else 5
    assert max(int(np.ravel_multi_index(lo, shape)) for lo in windows) > 2 ** 31
    for lo in windows:
        hi = tuple(min(a + side, n) for a, n in zip(lo, shape))
        ref = window_by_light_cone(block, shape, w, radius, T, lo, hi)
        got = g[tuple(slice(a, b) for a, b in zip(lo, hi))].cpu().numpy()
        assert normwise_rel(got, ref) <= TOL, lo
    p.close()
    del g
    torch.cuda.empty_cache()
