"""Guard bands around every caller-owned buffer: no kernel writes outside the
cells it owns.

Each grid (and every output of the adjoint) is a contiguous view into the
middle of a larger allocation whose head and tail are filled with a canary
value; after the run the canaries must be bit-for-bit unchanged.  With T >= 2
every sweep writes the caller's buffer on even steps and the plan's partner
buffer on odd ones, so the same index arithmetic is checked in both
directions.  The results are also compared with the oracle.
"""
import numpy as np
import pytest

import oracle
import synth
from conftest import normwise_rel

pytestmark = pytest.mark.gpu
TOL = 1e-12
PERIODIC, DIRICHLET = 1, 0
GUARD = 4096           # doubles on each side (32 KiB: keeps 16-byte alignment)
CANARY = -7.0e300      # a value no sweep of these inputs can produce


@pytest.fixture(scope="module")
def st():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2303_08365_gb300 import build
    build.build()
    import paper_2303_08365_gb300 as st
    return st


class Guarded:
    """A device array of `shape` with canary bands on both sides."""

    def __init__(self, values):
        import torch
        values = np.ascontiguousarray(values, dtype=np.float64)
        self.n = values.size
        self.buf = torch.full((self.n + 2 * GUARD,), CANARY, dtype=torch.float64, device="cuda")
        self.view = self.buf[GUARD:GUARD + self.n].view(values.shape)
        self.view.copy_(torch.from_numpy(values))

    def intact(self):
        import torch
        torch.cuda.synchronize()
        head = self.buf[:GUARD]
        tail = self.buf[GUARD + self.n:]
        return bool((head == CANARY).all()) and bool((tail == CANARY).all())

    def numpy(self):
        return self.view.cpu().numpy()


def star(ndim, radius, seed):
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


def box(ndim, radius, seed):
    v = synth.uniform(seed, (2 * radius + 1,) * ndim)
    return v / v.sum()


CASES = [
    # shape, radius, kind, boundary, Tb, variant name, T
    ((37, 70), 1, "star", DIRICHLET, 1, "direct", 3),
    ((37, 70), 1, "box", PERIODIC, 1, "direct", 2),
    ((33, 130), 1, "star", DIRICHLET, 1, "stream", 3),
    ((48, 128), 1, "box", PERIODIC, 1, "stream", 2),
    ((29, 66), 2, "box", DIRICHLET, 1, "stream", 3),
    ((13, 37, 70), 1, "star", DIRICHLET, 1, "stream", 3),
    ((8, 32, 128), 1, "box", PERIODIC, 1, "stream", 2),
    ((13, 37, 70), 1, "box", DIRICHLET, 2, "temporal", 5),
    ((11, 37, 70), 1, "star", DIRICHLET, 2, "temporal", 5),     # 3D star, stage by stage
    ((9, 37, 70), 1, "star", PERIODIC, 8, "temporal", 17),
    ((7, 20, 33), 1, "box", DIRICHLET, 4, "temporal", 9),
    ((50, 300), 1, "star", PERIODIC, 8, "temporal", 19),
    ((5001,), 2, "star", DIRICHLET, 8, "temporal", 17),
    ((37, 53), 1, "star", DIRICHLET, 1, "persistent", 5),
    ((37, 53), 1, "star", PERIODIC, 4, "persistent", 9),
    ((300, 257), 1, "box", DIRICHLET, 2, "persistent", 7),
    ((9, 10, 11), 2, "box", PERIODIC, 1, "direct", 2),
    ((13, 37, 128), 1, "star", DIRICHLET, 4, "exchange", 9),
    ((6, 40, 192), 1, "box", PERIODIC, 8, "exchange", 17),
]


@pytest.mark.parametrize("shape,radius,kind,boundary,Tb,variant,T", CASES)
def test_sweep_writes_stay_inside_the_grid(st, shape, radius, kind, boundary, Tb, variant, T):
    ndim = len(shape)
    w = (star if kind == "star" else box)(ndim, radius, 900 + ndim + radius)
    u0 = synth.uniform(77, shape)
    g = Guarded(u0)
    p = st.Plan(shape, radius, w, boundary)
    p.set_tuning(Tb, {"direct": st.VARIANT_DIRECT, "stream": st.VARIANT_STREAM,
                      "temporal": st.VARIANT_TEMPORAL, "persistent": st.VARIANT_PERSISTENT,
                      "exchange": st.VARIANT_EXCHANGE}[variant])
    p.run(g.view, T)
    assert g.intact()
    assert normwise_rel(g.numpy(), oracle.run(u0, w, radius, boundary, T, nthreads=0)) <= TOL
    p.close()


@pytest.mark.parametrize("Tb", [1, 4])
def test_batched_writes_stay_inside_each_grid(st, Tb):
    items = [(37, 91, 0.11, 13), (128, 64, 0.2, 6), (5, 3, 0.05, 9), (1, 1, 0.1, 4), (70, 250, 0.15, 21)]
    grids = [synth.uniform(60 + i, (ny, nx)) for i, (ny, nx, _, _) in enumerate(items)]
    gs = [Guarded(x) for x in grids]
    b = st.Batch([g.view for g in gs], [a for _, _, a, _ in items], [T for *_, T in items])
    b.set_tuning(Tb)
    b.run()
    assert b.status() == 0
    for x, g, (_, _, a, T) in zip(grids, gs, items):
        assert g.intact()
        assert normwise_rel(g.numpy(), oracle.run(x, synth.heat_weights(2, a), 1, DIRICHLET, T)) <= TOL
    b.close()


def test_static_entry_writes_stay_inside_the_grid(st):
    u0 = synth.uniform(81, (45, 77))
    w = synth.heat_weights(2, 0.2)
    g = Guarded(u0)
    st.stencil_run_2d_static(g.view, w, DIRICHLET, 11)
    assert g.intact()
    assert normwise_rel(g.numpy(), oracle.run(u0, w, 1, DIRICHLET, 11)) <= TOL


@pytest.mark.parametrize("boundary", [PERIODIC, DIRICHLET])
def test_adjoint_writes_stay_inside_its_outputs(st, boundary):
    shape = (9, 14, 19)
    u0 = synth.uniform(91, shape)
    kappa = synth.lognormal(92, shape, 0.5)
    target = synth.normal(93, shape)
    dt = 0.1 / float(kappa.max())
    T = 11
    gu, gk = Guarded(np.zeros(shape)), Guarded(np.zeros(shape))
    ins = [Guarded(u0), Guarded(kappa), Guarded(target)]
    p = st.Plan.varcoef(shape, boundary)
    loss = st.stencil_adjoint(p.handle, ins[0].view, ins[1].view, dt, ins[2].view, T, 4, gu.view, gk.view)
    assert all(g.intact() for g in [gu, gk] + ins)
    rl, rgu, rgk = oracle.varcoef_adjoint(u0, kappa, dt, target, boundary, T, ckpt_every=4)
    assert abs(loss - rl) <= 1e-12 * abs(rl)
    assert normwise_rel(gu.numpy(), rgu) <= TOL and normwise_rel(gk.numpy(), rgk) <= TOL
    fwd = Guarded(u0)
    p.run(fwd.view, T, ins[1].view, dt)
    assert fwd.intact()
    p.close()
