"""GPU parity of the batched persistent sweep: every item equals the same
grid advanced alone by stencil_run, bitwise (same tap order and FMA chain),
and the oracle within 1e-12; uneven sizes, ragged tiles and T = 0 items."""
import numpy as np
import pytest

import oracle
import synth
from conftest import normwise_rel

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


def single(st, u0, alpha, T, boundary):
    import torch
    g = torch.from_numpy(u0.copy()).cuda()
    p = st.Plan(u0.shape, 1, synth.heat_weights(2, alpha), boundary)
    p.run(g, T)
    out = g.cpu().numpy()
    p.close()
    return out


@pytest.mark.parametrize("boundary", [DIRICHLET, PERIODIC])
def test_small_batch_matches_single_and_oracle(st, boundary):
    import torch
    items = [(37, 91, 0.11, 13), (128, 64, 0.2, 6), (5, 3, 0.05, 9), (200, 130, 0.24, 0),
             (1, 1, 0.1, 4), (70, 250, 0.15, 21)]
    grids = [synth.uniform(50 + i, (ny, nx)) for i, (ny, nx, _, _) in enumerate(items)]
    dev = [torch.from_numpy(g.copy()).cuda() for g in grids]
    b = st.Batch(dev, [a for _, _, a, _ in items], [T for *_, T in items], boundary)
    b.run()
    assert b.status() == 0
    for g0, d, (ny, nx, a, T) in zip(grids, dev, items):
        got = d.cpu().numpy()
        assert np.array_equal(got, single(st, g0, a, T, boundary))
        ref = oracle.run(g0, synth.heat_weights(2, a), 1, boundary, T)
        assert normwise_rel(got, ref) <= TOL
    b.close()


def test_replay_advances_again(st):
    import torch
    g0 = synth.uniform(9, (64, 80))
    d = torch.from_numpy(g0.copy()).cuda()
    b = st.Batch([d], [0.1], [7])
    b.run()
    b.run()
    assert b.status() == 0
    assert np.array_equal(d.cpu().numpy(), single(st, g0, 0.1, 14, DIRICHLET))
    b.close()


@pytest.mark.slow
def test_full_96_item_batch(st):
    """The 96-grid workload: items bitwise equal to their single-grid runs,
    the smallest against the whole-grid oracle and the two largest on oracle
    windows at their full T."""
    import torch
    items = synth.batch_items(synth.SEED_BATCH)
    grids = [synth.uniform(synth.SEED_BATCH + 1000 + i, (ny, nx)) for i, (ny, nx, _, _) in enumerate(items)]
    dev = [torch.from_numpy(g).cuda() for g in grids]
    b = st.Batch(dev, [a for _, _, a, _ in items], [T for *_, T in items])
    b.run()
    assert b.status() == 0
    order = sorted(range(len(items)), key=lambda i: items[i][0] * items[i][1])
    for i in order[:4] + order[-2:]:
        ny, nx, a, T = items[i]
        assert np.array_equal(dev[i].cpu().numpy(), single(st, grids[i], a, T, DIRICHLET)), i
    for i in order[:3]:
        ny, nx, a, T = items[i]
        ref = oracle.run(grids[i], synth.heat_weights(2, a), 1, DIRICHLET, T, nthreads=0)
        assert normwise_rel(dev[i].cpu().numpy(), ref) <= TOL
    # the two largest items at their full T: windows from the oracle's light
    # cone at a corner (ghost cells on two sides), on an edge and inside
    for i in order[-2:]:
        ny, nx, a, T = items[i]
        got = dev[i].cpu().numpy()
        w = synth.heat_weights(2, a)
        for lo in ((0, 0), (0, nx // 2), (ny // 3, nx // 5), (ny - 6, nx - 10)):
            hi = (min(ny, lo[0] + 6), min(nx, lo[1] + 10))
            ref = oracle.run_window(grids[i], w, 1, DIRICHLET, T, lo, hi)
            assert normwise_rel(got[lo[0]:hi[0], lo[1]:hi[1]], ref) <= TOL, (i, lo)
    b.close()


def test_bounded_wait_reports_timeout_and_context_survives(st):
    """Failure detection without a GPU fault: a device-wide barrier that can
    never complete gives up after its 20 ms wall-time limit, the kernel
    reports STENCIL_ERR_TIMEOUT, and the next sweep runs normally."""
    import torch
    assert st.stencil_selftest_barrier_timeout(20.0) == st.ERR_TIMEOUT
    g0 = synth.uniform(31, (40, 70))
    d = torch.from_numpy(g0.copy()).cuda()
    b = st.Batch([d], [0.1], [5])
    b.run()
    assert b.status() == 0
    ref = oracle.run(g0, synth.heat_weights(2, 0.1), 1, DIRICHLET, 5)
    assert normwise_rel(d.cpu().numpy(), ref) <= TOL
    b.close()


def test_one_call_entry_matches_batch_object(st):
    """stencil_run_batched (create, run once, wait, destroy) gives the same
    bits as a Batch object, periodic boundary included."""
    import torch
    items = [(45, 64, 0.2, 11), (17, 29, 0.07, 3), (64, 33, 0.24, 8)]
    grids = [synth.uniform(70 + i, (ny, nx)) for i, (ny, nx, _, _) in enumerate(items)]
    for boundary in (DIRICHLET, PERIODIC):
        a = [torch.from_numpy(g.copy()).cuda() for g in grids]
        b = [torch.from_numpy(g.copy()).cuda() for g in grids]
        st.stencil_run_batched(a, [x[2] for x in items], [x[3] for x in items], boundary)
        batch = st.Batch(b, [x[2] for x in items], [x[3] for x in items], boundary)
        batch.run()
        assert batch.status() == 0
        batch.close()
        for x, y, g0, (_, _, al, T) in zip(a, b, grids, items):
            assert np.array_equal(x.cpu().numpy(), y.cpu().numpy())
            ref = oracle.run(g0, synth.heat_weights(2, al), 1, boundary, T)
            assert normwise_rel(x.cpu().numpy(), ref) <= TOL


def test_autotuner_leaves_grids_alone_and_every_configuration_agrees(st):
    """The batch autotuner probes on scratch copies (the caller's grids are not
    modified), keeps a valid configuration, and every (cells per thread,
    blocks per SM) gives the same bits as single-grid runs."""
    import torch
    items = [(37, 91, 0.11, 13), (128, 64, 0.2, 6), (5, 3, 0.05, 9), (300, 257, 0.15, 21), (1, 1, 0.1, 4)]
    grids = [synth.uniform(90 + i, (ny, nx)) for i, (ny, nx, _, _) in enumerate(items)]
    refs = [single(st, g0, a, T, DIRICHLET) for g0, (_, _, a, T) in zip(grids, items)]
    dev = [torch.from_numpy(g.copy()).cuda() for g in grids]
    b = st.Batch(dev, [x[2] for x in items], [x[3] for x in items])
    rate = b.autotune(probe_steps=4)
    assert rate > 0
    for g0, d in zip(grids, dev):
        assert np.array_equal(d.cpu().numpy(), g0)      # untouched by the probes
    tb, cpt, per_sm = b.get_tuning()
    assert tb in (1, 2, 4, 8) and per_sm >= 1 and (cpt in (1, 2, 4) if tb == 1 else cpt == 0)
    b.run()
    assert b.status() == 0
    for d, r in zip(dev, refs):
        assert np.array_equal(d.cpu().numpy(), r)
    configs = [(1, cpt, per_sm) for cpt in (1, 2, 4) for per_sm in (1, 3)] + [(2, 0, 0), (4, 0, 0), (8, 0, 0)]
    for tb, cpt, per_sm in configs:
        for g0, d in zip(grids, dev):
            d.copy_(torch.from_numpy(g0))
        b.set_tuning(tb, cpt, per_sm)
        assert b.get_tuning()[0] == tb
        b.run()
        assert b.status() == 0
        for d, r in zip(dev, refs):
            assert np.array_equal(d.cpu().numpy(), r), (tb, cpt, per_sm)
    with pytest.raises(st.StencilError):
        b.set_tuning(1, 3, 0)
    with pytest.raises(st.StencilError):
        b.set_tuning(3, 0, 0)
    b.close()


@pytest.mark.parametrize("boundary", [DIRICHLET, PERIODIC])
@pytest.mark.parametrize("Tb", [2, 4, 8])
def test_batched_temporal_blocking_matches_single_grids(st, boundary, Tb):
    """Tb steps per exchange over many grids at once (each grid its own alpha
    and T, odd block counts, T = 0, a single cell, grids smaller than the
    halo): bitwise equal to single-grid runs and within 1e-12 of the oracle."""
    import torch
    items = [(37, 91, 0.11, 13), (128, 64, 0.2, 6), (5, 3, 0.05, 9), (200, 130, 0.24, 0), (1, 1, 0.1, 4),
             (70, 250, 0.15, 21), (16, 32, 0.19, 8), (33, 2, 0.07, 17)]
    grids = [synth.uniform(110 + i, (ny, nx)) for i, (ny, nx, _, _) in enumerate(items)]
    dev = [torch.from_numpy(g.copy()).cuda() for g in grids]
    b = st.Batch(dev, [x[2] for x in items], [x[3] for x in items], boundary)
    b.set_tuning(Tb)
    b.run()
    assert b.status() == 0
    for g0, d, (ny, nx, a, T) in zip(grids, dev, items):
        got = d.cpu().numpy()
        assert np.array_equal(got, single(st, g0, a, T, boundary)), (ny, nx, T)
        assert normwise_rel(got, oracle.run(g0, synth.heat_weights(2, a), 1, boundary, T)) <= TOL
    b.run()                                  # replay: T more steps each
    assert b.status() == 0
    for g0, d, (ny, nx, a, T) in zip(grids, dev, items):
        assert np.array_equal(d.cpu().numpy(), single(st, g0, a, 2 * T, boundary)), (ny, nx, T)
    b.close()


def test_tile_flag_wait_reports_timeout_and_context_survives(st):
    """Failure detection without a GPU fault, for the tile-flag waits: a flag
    that nothing sets makes the neighbouring tiles give up after their 20 ms
    limit with STENCIL_ERR_TIMEOUT, and the next batch runs normally."""
    import torch
    assert st.stencil_selftest_flag_timeout(20.0) == st.ERR_TIMEOUT
    g0 = synth.uniform(32, (40, 70))
    d = torch.from_numpy(g0.copy()).cuda()
    b = st.Batch([d], [0.1], [9])
    b.set_tuning(4)
    b.run()
    assert b.status() == 0
    ref = oracle.run(g0, synth.heat_weights(2, 0.1), 1, DIRICHLET, 9)
    assert normwise_rel(d.cpu().numpy(), ref) <= TOL
    b.close()
