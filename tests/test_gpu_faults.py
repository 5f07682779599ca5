"""Host-side fault injection: device allocations that fail.

stencil_debug_fail_allocations(k) lets k more allocations succeed and fails
the rest, without touching the driver.  For every entry point, each k up to
the first success must give STENCIL_ERR_OOM with a message; turning the
injection off must leave a plan (or a new batch) that runs and matches the
oracle.  No GPU is faulted or hung.
"""
import numpy as np
import pytest

import oracle
import synth
from conftest import normwise_rel

pytestmark = pytest.mark.gpu
TOL = 1e-12
PERIODIC, DIRICHLET = 1, 0


@pytest.fixture(scope="module")
def st():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2303_08365_gb300 import build
    build.build()
    import paper_2303_08365_gb300 as st
    yield st
    st.stencil_debug_fail_allocations(-1)


def first_success(st, fn, limit=24):
    """Calls fn() with k = 0, 1, ... allocations allowed; every failure must be
    an OOM.  Returns the k that first succeeded."""
    for k in range(limit):
        st.stencil_debug_fail_allocations(k)
        try:
            fn()
            return k
        except st.StencilError as e:
            assert e.code == st.ERR_OOM, str(e)
            assert "alloc" in str(e), str(e)
        finally:
            st.stencil_debug_fail_allocations(-1)
    raise AssertionError("never succeeded")


@pytest.mark.parametrize("shape,radius,w_kind,boundary,T", [
    ((37, 53), 1, "heat", DIRICHLET, 9),          # persistent temporal (flags)
    ((700, 700), 1, "heat", DIRICHLET, 5),        # persistent one-step (batch inside the plan)
    ((8, 32, 128), 1, "heat", PERIODIC, 4),       # 3D streaming
    ((5001,), 2, "star", DIRICHLET, 17),          # 1D temporal
])
def test_constant_weight_run_reports_oom_and_recovers(st, shape, radius, w_kind, boundary, T):
    import torch
    ndim = len(shape)
    if w_kind == "heat":
        w = synth.heat_weights(ndim, 0.1)
    else:
        v = synth.uniform(5, (5,))
        w = v / v.sum()
    u0 = synth.uniform(31, shape)
    p = st.Plan(shape, radius, w, boundary)
    g = torch.from_numpy(u0.copy()).cuda()
    k = first_success(st, lambda: p.run(torch.from_numpy(u0.copy()).cuda(), T))
    assert k >= 1
    p.run(g, T)
    assert normwise_rel(g.cpu().numpy(), oracle.run(u0, w, radius, boundary, T, nthreads=0)) <= TOL
    p.close()
    # a fresh plan whose first run fails part-way still runs correctly afterwards
    p2 = st.Plan(shape, radius, w, boundary)
    st.stencil_debug_fail_allocations(k - 1)
    with pytest.raises(st.StencilError):
        p2.run(torch.from_numpy(u0.copy()).cuda(), T)
    st.stencil_debug_fail_allocations(-1)
    g2 = torch.from_numpy(u0.copy()).cuda()
    p2.run(g2, T)
    assert np.array_equal(g2.cpu().numpy(), g.cpu().numpy())
    p2.close()


def test_batch_retuning_reports_oom_and_recovers(st):
    """Switching a batch to Tb = 4 rebuilds its work list; allocation failures
    there are reported, and a later successful switch runs correctly."""
    import torch
    grids = [synth.uniform(42, (40, 70)), synth.uniform(43, (33, 20))]
    alphas, Ts = [0.1, 0.2], [9, 4]
    dev = [torch.from_numpy(x.copy()).cuda() for x in grids]
    b = st.Batch(dev, alphas, Ts)
    # a rebuild that fails part-way leaves no work list: running it is refused
    st.stencil_debug_fail_allocations(1)
    with pytest.raises(st.StencilError):
        b.set_tuning(2)
    st.stencil_debug_fail_allocations(-1)
    with pytest.raises(st.StencilError):
        b.run()
    first_success(st, lambda: b.set_tuning(4))
    assert b.get_tuning()[0] == 4
    b.run()
    assert b.status() == 0
    for x, d, a, T in zip(grids, dev, alphas, Ts):
        assert normwise_rel(d.cpu().numpy(), oracle.run(x, synth.heat_weights(2, a), 1, DIRICHLET, T)) <= TOL
    b.close()


def test_batch_create_reports_oom_and_a_new_batch_runs(st):
    import torch
    grids = [synth.uniform(40, (40, 70)), synth.uniform(41, (33, 20))]
    alphas, Ts = [0.1, 0.2], [9, 4]
    first_success(st, lambda: st.Batch([torch.from_numpy(x.copy()).cuda() for x in grids], alphas, Ts).close())
    dev = [torch.from_numpy(x.copy()).cuda() for x in grids]
    b = st.Batch(dev, alphas, Ts)
    b.run()
    assert b.status() == 0
    for x, d, a, T in zip(grids, dev, alphas, Ts):
        assert normwise_rel(d.cpu().numpy(), oracle.run(x, synth.heat_weights(2, a), 1, DIRICHLET, T)) <= TOL
    b.close()


def test_adjoint_and_host_entry_report_oom_and_recover(st):
    import torch
    shape = (10, 12, 14)
    u = synth.uniform(21, shape)
    kap = synth.lognormal(22, shape, 0.5)
    tg = synth.normal(23, shape)
    dt = 0.1 / float(kap.max())
    p = st.Plan.varcoef(shape, PERIODIC)
    cu, ck, ct = (torch.from_numpy(x).cuda() for x in (u, kap, tg))
    first_success(st, lambda: p.adjoint(cu, ck, dt, ct, 15, ckpt_every=4))
    loss, gu, gk = p.adjoint(cu, ck, dt, ct, 15, ckpt_every=4)
    rl, rgu, rgk = oracle.varcoef_adjoint(u, kap, dt, tg, PERIODIC, 15, ckpt_every=4)
    assert abs(loss - rl) <= 1e-12 * abs(rl)
    assert normwise_rel(gu.cpu().numpy(), rgu) <= TOL and normwise_rel(gk.cpu().numpy(), rgk) <= TOL
    p.close()
    # the host-buffer entry of a constant-weight plan
    w = synth.heat_weights(2, 0.1)
    u2 = synth.uniform(24, (64, 96))
    q = st.Plan(u2.shape, 1, w, DIRICHLET)
    first_success(st, lambda: q.run_host(torch.from_numpy(u2.copy()), 6))
    h = torch.from_numpy(u2.copy())
    q.run_host(h, 6)
    assert normwise_rel(h.numpy(), oracle.run(u2, w, 1, DIRICHLET, 6)) <= TOL
    q.close()
