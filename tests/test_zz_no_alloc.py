"""The allocation-free entry point stencil_run_2d_static, called through the
C ABI.

It exists for callers that cannot allocate device memory when they want a
sweep: code whose HBM is owned by another allocator's pool (a cudaMalloc
behind the pool's back fails or steals its reserve), and loops that must not
take the device-wide synchronisation of cudaMalloc/cudaFree.  Its scratch is
one array reserved when the library's device code is loaded and shared by
every call, so the tests make calls in a row with different shapes and step
counts and check each against the oracle and the regular entry point
(stencil_run), that no device memory is allocated or freed around a call, and
that a bounded wait that gives up is reported by stencil_static_status.  This
file runs last on purpose.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synth
from conftest import normwise_rel

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module")
def st():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2303_08365_gb300 import build
    build.build()
    import paper_2303_08365_gb300 as st
    return st


def static_run(st, grid, weights, boundary, T):
    import torch
    w = np.ascontiguousarray(weights, dtype=np.float64).reshape(-1)
    rc = st.lib().stencil_run_2d_static(grid.shape[0], grid.shape[1],
                                        w.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), boundary,
                                        ctypes.c_void_p(grid.data_ptr()), T,
                                        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc


def static_status(st):
    import torch
    return st.lib().stencil_static_status(ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def regular_run(st, u0, weights, boundary, T):
    import torch
    g = torch.from_numpy(u0.copy()).cuda()
    p = st.Plan(u0.shape, 1, weights, boundary)
    p.run(g, T)
    out = g.cpu().numpy()
    p.close()
    return out


# (shape, weights, boundary, T, seed): calls in a row, each a different shape;
# 1024 x 1024 is exactly the 2^20-cell limit (every tile of the static list in
# use) with odd T, so the result is copied back from the static partner grid
CASES = [((300, 257), synth.heat_weights(2, 0.1), 0, 37, 61),
         ((64, 128), synth.heat_weights(2, 0.2), 1, 20, 62),
         ((1024, 1024), synth.heat_weights(2, 0.15), 0, 7, 63),
         ((1, 1), synth.heat_weights(2, 0.1), 0, 5, 64),
         ((1, 1), synth.heat_weights(2, 0.1), 1, 3, 65),
         ((33, 1), synth.heat_weights(2, 0.24), 1, 9, 66)]


def test_calls_in_a_row_match_the_oracle_and_stencil_run(st):
    import torch
    for shape, w, boundary, T, seed in CASES:
        u0 = synth.uniform(seed, shape)
        g = torch.from_numpy(u0.copy()).cuda()
        assert static_run(st, g, w, boundary, T) == 0, st.last_error()
        assert static_status(st) == 0, st.last_error()
        got = g.cpu().numpy()
        ref = oracle.run(u0, w, 1, boundary, T, nthreads=0)
        assert normwise_rel(got, ref) <= TOL, shape
        assert normwise_rel(got, regular_run(st, u0, w, boundary, T)) <= TOL, shape


def test_zero_steps_leave_the_grid_unchanged(st):
    import torch
    u0 = synth.uniform(67, (40, 50))
    g = torch.from_numpy(u0.copy()).cuda()
    assert static_run(st, g, synth.heat_weights(2, 0.1), 0, 0) == 0
    assert np.array_equal(g.cpu().numpy(), u0)


def test_no_device_memory_is_allocated_or_freed(st):
    """After a first call (the device code and its array are loaded by then),
    a call with the library's allocation hook set to fail every allocation
    still succeeds, and the device's free memory is the same before and after
    (nothing was allocated or freed behind the caller's back)."""
    import torch
    w = synth.heat_weights(2, 0.1)
    u0 = synth.uniform(68, (512, 512))
    g = torch.from_numpy(u0.copy()).cuda()
    assert static_run(st, g, w, 0, 3) == 0
    torch.cuda.synchronize()
    g.copy_(torch.from_numpy(u0))
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    st.stencil_debug_fail_allocations(0)
    try:
        rc = static_run(st, g, w, 0, 11)
        assert rc == 0, st.last_error()
        assert static_status(st) == 0
    finally:
        st.stencil_debug_fail_allocations(-1)
    free1, _ = torch.cuda.mem_get_info()
    assert free0 == free1
    ref = oracle.run(u0, w, 1, 0, 11, nthreads=0)
    assert normwise_rel(g.cpu().numpy(), ref) <= TOL


def test_bounded_wait_timeout_is_reported_and_next_call_runs(st):
    """Failure detection without a GPU fault: the entry's kernel launched with
    a barrier that counts one block more than the launch has gives up after
    its 20 ms limit, stencil_static_status reports STENCIL_ERR_TIMEOUT once,
    and the next call runs normally."""
    import torch
    assert st.stencil_selftest_static_timeout(20.0) == st.ERR_TIMEOUT
    assert static_status(st) == 0  # the word was cleared when it was read
    u0 = synth.uniform(69, (48, 72))
    g = torch.from_numpy(u0.copy()).cuda()
    w = synth.heat_weights(2, 0.2)
    assert static_run(st, g, w, 1, 13) == 0
    assert static_status(st) == 0
    assert normwise_rel(g.cpu().numpy(), oracle.run(u0, w, 1, 1, 13)) <= TOL


def test_rejects_grids_beyond_the_limit(st):
    import torch
    for shape in ((1025, 1024), (1, (1 << 20) + 1)):
        g = torch.zeros(shape, dtype=torch.float64, device="cuda")
        rc = static_run(st, g, synth.heat_weights(2, 0.1), 0, 1)
        assert rc == st.ERR_UNSUPPORTED
        assert "exceeds the static scratch limit" in st.last_error()
