"""The allocation-free entry point stencil_run_2d_static, called through the
C ABI, gives the same grids as the regular entry point stencil_run.

It exists for callers that cannot allocate device memory when they want a
sweep (a caller whose HBM is owned by another allocator's pool, or a loop
that must not take the device-wide synchronisation of cudaMalloc/cudaFree).
Its scratch is one array reserved at load time and shared by every call, so
the test makes two calls in a row, with different shapes and step counts,
and checks each against stencil_run.  This file runs last on purpose.
"""
import ctypes

import numpy as np
import pytest

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


def regular_run(st, u0, weights, boundary, T):
    import torch
    g = torch.from_numpy(u0.copy()).cuda()
    p = st.Plan(u0.shape, 1, weights, boundary)
    p.run(g, T)
    out = g.cpu().numpy()
    p.close()
    return out


def test_two_calls_in_a_row_match_stencil_run(st):
    import torch
    cases = [((300, 257), synth.heat_weights(2, 0.1), st.DIRICHLET_ZERO, 37, 61),
             ((64, 128), synth.heat_weights(2, 0.2), st.PERIODIC, 20, 62)]
    for shape, w, boundary, T, seed in cases:
        u0 = synth.uniform(seed, shape)
        g = torch.from_numpy(u0.copy()).cuda()
        assert static_run(st, g, w, boundary, T) == 0, st.last_error()
        torch.cuda.synchronize()
        ref = regular_run(st, u0, w, boundary, T)
        assert normwise_rel(g.cpu().numpy(), ref) <= TOL


def test_rejects_grids_beyond_the_limit(st):
    import torch
    g = torch.zeros((1025, 1024), dtype=torch.float64, device="cuda")
    rc = static_run(st, g, synth.heat_weights(2, 0.1), st.DIRICHLET_ZERO, 1)
    assert rc == st.ERR_UNSUPPORTED
    assert "exceeds the static scratch limit" in st.last_error()
