"""Python binding of the GB300 FP64 iterative-stencil library (C ABI in
include/stencil.h).

Argument marshalling only: every step of the sweep runs in the CUDA kernels of
libstencil_gb300.so.  There is no CPU fallback: if the library has not been
built, importing the binding's functions raises.  Device buffers are torch
tensors (CUDA, float64, contiguous); PyTorch supplies memory and streams.

The update (paper Sec. 2.1, Listing 1, Eq. 3): u^{t+1}(x) = sum_o w_o u^t(x+o),
weights a dense (2r+1)^ndim array, correlation convention, Dirichlet-zero or
periodic boundaries.
"""
import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libstencil_gb300.so")

DIRICHLET_ZERO = 0
PERIODIC = 1

OK = 0
ERR_ARG = -1
ERR_UNSUPPORTED = -2
ERR_OOM = -3
ERR_CUDA = -4
ERR_TIMEOUT = -5

VARIANT_AUTO = 0
VARIANT_DIRECT = 1
VARIANT_STREAM = 2
VARIANT_TEMPORAL = 3
VARIANT_PERSISTENT = 4
VARIANT_EXCHANGE = 5

# (name, restype, argtypes) of every entry point of include/stencil.h
_VP = ctypes.c_void_p
_I64P = ctypes.POINTER(ctypes.c_int64)
_DP = ctypes.POINTER(ctypes.c_double)
_IP = ctypes.POINTER(ctypes.c_int)


class BatchItem(ctypes.Structure):
    """stencil_batch_item: one 2D heat grid of a batch."""
    _fields_ = [("ny", ctypes.c_int64), ("nx", ctypes.c_int64), ("alpha", ctypes.c_double),
                ("T", ctypes.c_int64), ("d_grid", ctypes.c_void_p)]


SIGNATURES = [
    ("stencil_create", ctypes.c_int, [ctypes.c_int, _I64P, ctypes.c_int, _DP, ctypes.c_int, ctypes.POINTER(_VP)]),
    ("stencil_create_varcoef", ctypes.c_int, [ctypes.c_int, _I64P, ctypes.c_int, ctypes.POINTER(_VP)]),
    ("stencil_destroy", None, [_VP]),
    ("stencil_run", ctypes.c_int, [_VP, _VP, ctypes.c_int64, _VP, ctypes.c_double, _VP]),
    ("stencil_run_host", ctypes.c_int, [_VP, _VP, ctypes.c_int64, _VP, ctypes.c_double, _VP]),
    ("stencil_run_f32", ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int64, _VP]),
    ("stencil_adjoint", ctypes.c_int, [_VP, _VP, _VP, ctypes.c_double, _VP, ctypes.c_int64, ctypes.c_int,
                                       _VP, _VP, _DP, _VP]),
    ("stencil_adjoint_vjp", ctypes.c_int, [_VP, _VP, _VP, ctypes.c_double, ctypes.c_int64, ctypes.c_int,
                                           _VP, _VP, _VP, _VP]),
    ("stencil_batch_create", ctypes.c_int, [ctypes.POINTER(BatchItem), ctypes.c_int, ctypes.c_int,
                                            ctypes.POINTER(_VP)]),
    ("stencil_batch_run", ctypes.c_int, [_VP, _VP]),
    ("stencil_batch_status", ctypes.c_int, [_VP]),
    ("stencil_batch_destroy", None, [_VP]),
    ("stencil_run_batched", ctypes.c_int, [ctypes.POINTER(BatchItem), ctypes.c_int, ctypes.c_int, _VP]),
    ("stencil_batch_set_tuning", ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    ("stencil_batch_get_tuning", ctypes.c_int, [_VP, _IP, _IP, _IP]),
    ("stencil_batch_autotune", ctypes.c_int, [_VP, ctypes.c_int64, _VP, _DP]),
    ("stencil_plan_status", ctypes.c_int, [_VP, _VP]),
    ("stencil_set_tuning", ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int]),
    ("stencil_get_tuning", ctypes.c_int, [_VP, _IP, _IP]),
    ("stencil_set_tile", ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int]),
    ("stencil_get_tile", ctypes.c_int, [_VP, _IP, _IP]),
    ("stencil_exchange_layout", ctypes.c_int, [_VP, ctypes.c_int, _IP, ctypes.POINTER(ctypes.c_int64)]),
    ("stencil_autotune", ctypes.c_int, [_VP, _VP, ctypes.c_int64, _VP, _DP]),
    ("stencil_variant_name", ctypes.c_char_p, [ctypes.c_int]),
    ("stencil_last_error", ctypes.c_char_p, []),
    ("stencil_launch_count", ctypes.c_int64, []),
    ("stencil_fp64_peak", ctypes.c_int, [ctypes.c_double, _DP, _VP]),
    ("stencil_selftest_barrier_timeout", ctypes.c_int, [ctypes.c_double, _VP]),
    ("stencil_debug_fail_allocations", None, [ctypes.c_int]),
    ("stencil_selftest_flag_timeout", ctypes.c_int, [ctypes.c_double, _VP]),
    ("stencil_selftest_tma_timeout", ctypes.c_int, [ctypes.c_double, _VP]),
    ("stencil_run_2d_static", ctypes.c_int, [ctypes.c_int64, ctypes.c_int64, _DP, ctypes.c_int, _VP,
                                             ctypes.c_int64, _VP]),
    ("stencil_static_status", ctypes.c_int, [_VP]),
    ("stencil_selftest_static_timeout", ctypes.c_int, [ctypes.c_double, _VP]),
]

_lib = None


class StencilError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"stencil status {code}: {msg}")
        self.code = code


def lib():
    """The loaded CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                "libstencil_gb300.so is missing: build it with "
                "`python -c 'import __graft_entry__ as g; g.build()'` "
                "(there is no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def last_error():
    return lib().stencil_last_error().decode()


def _check(rc):
    if rc != OK:
        raise StencilError(rc, last_error())


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _dev_ptr(t, name, shape=None):
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch tensor")
    if t.device.type != "cuda" or t.dtype != torch.float64 or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous float64 CUDA tensor")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return t.data_ptr()


def _host_ptr(a, name, shape=None):
    try:
        import torch
        if isinstance(a, torch.Tensor):
            if a.device.type != "cpu" or a.dtype != torch.float64 or not a.is_contiguous():
                raise TypeError(f"{name} must be a contiguous float64 CPU tensor")
            if shape is not None and tuple(a.shape) != tuple(shape):
                raise ValueError(f"{name} has shape {tuple(a.shape)}, expected {tuple(shape)}")
            return a.data_ptr()
    except ImportError:
        pass
    if not isinstance(a, np.ndarray) or a.dtype != np.float64 or not a.flags.c_contiguous:
        raise TypeError(f"{name} must be a C-contiguous float64 array")
    if shape is not None and tuple(a.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {a.shape}, expected {tuple(shape)}")
    return a.ctypes.data


def _dims(dims):
    return (ctypes.c_int64 * len(dims))(*[int(d) for d in dims])


# ----------------------------------------------------------------- C names

def stencil_create(dims, radius, weights, boundary):
    """Plan for the constant-weight stencil; returns an opaque handle."""
    w = np.ascontiguousarray(weights, dtype=np.float64)
    if w.size != (2 * radius + 1) ** len(dims):
        raise ValueError("weights must have (2r+1)^ndim entries")
    h = _VP()
    _check(lib().stencil_create(len(dims), _dims(dims), int(radius),
                                w.ctypes.data_as(_DP), int(boundary), ctypes.byref(h)))
    return h


def stencil_create_varcoef(dims, boundary):
    h = _VP()
    _check(lib().stencil_create_varcoef(len(dims), _dims(dims), int(boundary), ctypes.byref(h)))
    return h


def stencil_destroy(h):
    lib().stencil_destroy(h)


def stencil_run(h, grid, T, kappa=None, dt=0.0, stream=None):
    gp = _dev_ptr(grid, "grid")
    kp = _dev_ptr(kappa, "kappa", grid.shape) if kappa is not None else None
    _check(lib().stencil_run(h, gp, int(T), kp, float(dt), _stream(stream)))


def stencil_run_f32(h, grid, work, T, stream=None):
    """FP32 twin of stencil_run (accuracy studies only): grid and work are
    contiguous float32 CUDA tensors of the plan's shape."""
    import torch
    for t, name in ((grid, "grid"), (work, "work")):
        if t.device.type != "cuda" or t.dtype != torch.float32 or not t.is_contiguous():
            raise TypeError(f"{name} must be a contiguous float32 CUDA tensor")
    _check(lib().stencil_run_f32(h, grid.data_ptr(), work.data_ptr(), int(T), _stream(stream)))


def stencil_run_host(h, grid, T, kappa=None, dt=0.0, stream=None):
    gp = _host_ptr(grid, "grid")
    kp = _host_ptr(kappa, "kappa", grid.shape) if kappa is not None else None
    _check(lib().stencil_run_host(h, gp, int(T), kp, float(dt), _stream(stream)))


def stencil_adjoint(h, u0, kappa, dt, target, T, ckpt_every, grad_u0, grad_kappa, stream=None):
    """Loss 0.5||u^T - target||^2; fills grad_u0 and grad_kappa; returns the loss."""
    shape = u0.shape
    loss = ctypes.c_double(0.0)
    _check(lib().stencil_adjoint(h, _dev_ptr(u0, "u0"), _dev_ptr(kappa, "kappa", shape), float(dt),
                                 _dev_ptr(target, "target", shape), int(T), int(ckpt_every),
                                 _dev_ptr(grad_u0, "grad_u0", shape),
                                 _dev_ptr(grad_kappa, "grad_kappa", shape), ctypes.byref(loss),
                                 _stream(stream)))
    return loss.value


def stencil_adjoint_vjp(h, u0, kappa, dt, T, ckpt_every, lambda_T, grad_u0, grad_kappa, stream=None):
    """dL/du0 and dL/dkappa for a given dL/du^T (lambda_T); asynchronous."""
    shape = u0.shape
    _check(lib().stencil_adjoint_vjp(h, _dev_ptr(u0, "u0"), _dev_ptr(kappa, "kappa", shape), float(dt),
                                     int(T), int(ckpt_every), _dev_ptr(lambda_T, "lambda_T", shape),
                                     _dev_ptr(grad_u0, "grad_u0", shape),
                                     _dev_ptr(grad_kappa, "grad_kappa", shape), _stream(stream)))


def _batch_items(grids, alphas, steps):
    n = len(grids)
    arr = (BatchItem * n)()
    for i, (g, a, T) in enumerate(zip(grids, alphas, steps)):
        if g.dim() != 2:
            raise ValueError("batched grids are 2D")
        arr[i] = BatchItem(g.shape[0], g.shape[1], float(a), int(T), _dev_ptr(g, f"grid {i}"))
    return arr


def stencil_batch_create(grids, alphas, steps, boundary=DIRICHLET_ZERO):
    arr = _batch_items(grids, alphas, steps)
    h = _VP()
    _check(lib().stencil_batch_create(arr, len(arr), int(boundary), ctypes.byref(h)))
    return h


def stencil_batch_run(h, stream=None):
    _check(lib().stencil_batch_run(h, _stream(stream)))


def stencil_batch_status(h):
    return lib().stencil_batch_status(h)


def stencil_batch_destroy(h):
    lib().stencil_batch_destroy(h)


def stencil_run_batched(grids, alphas, steps, boundary=DIRICHLET_ZERO, stream=None):
    arr = _batch_items(grids, alphas, steps)
    _check(lib().stencil_run_batched(arr, len(arr), int(boundary), _stream(stream)))


def stencil_plan_status(h, stream=None):
    """Waits for the stream; returns the plan's device status (0 = OK)."""
    return lib().stencil_plan_status(h, _stream(stream))


def stencil_set_tuning(h, Tb, variant=0):
    _check(lib().stencil_set_tuning(h, int(Tb), int(variant)))


def stencil_get_tuning(h):
    tb, v = ctypes.c_int(0), ctypes.c_int(0)
    _check(lib().stencil_get_tuning(h, ctypes.byref(tb), ctypes.byref(v)))
    return tb.value, v.value


def stencil_autotune(h, scratch_grid, probe_steps, stream=None):
    best = ctypes.c_double(0.0)
    _check(lib().stencil_autotune(h, _dev_ptr(scratch_grid, "scratch_grid"), int(probe_steps),
                                  _stream(stream), ctypes.byref(best)))
    return best.value


def stencil_variant_name(v):
    return lib().stencil_variant_name(int(v)).decode()


def stencil_run_2d_static(grid, weights, boundary, T, stream=None):
    """Allocation-free 2D 5-point sweep of a small grid (see include/stencil.h)."""
    w = np.ascontiguousarray(weights, dtype=np.float64).reshape(-1)
    if w.size != 9:
        raise ValueError("weights must be a dense 3x3 array")
    _check(lib().stencil_run_2d_static(int(grid.shape[0]), int(grid.shape[1]), w.ctypes.data_as(_DP),
                                       int(boundary), _dev_ptr(grid, "grid"), int(T), _stream(stream)))


def stencil_static_status(stream=None):
    """Waits for the stream; the status word of the last allocation-free sweep."""
    return lib().stencil_static_status(_stream(stream))


def stencil_selftest_static_timeout(limit_ms=20.0, stream=None):
    """Runs the allocation-free entry's bounded-wait failure path; returns the
    status code (ERR_TIMEOUT when it behaved)."""
    return lib().stencil_selftest_static_timeout(float(limit_ms), _stream(stream))


def stencil_selftest_flag_timeout(limit_ms=20.0, stream=None):
    """Runs the tile-flag wait's failure path on the GPU; returns the status
    code (ERR_TIMEOUT when it behaved)."""
    return lib().stencil_selftest_flag_timeout(float(limit_ms), _stream(stream))


def stencil_selftest_tma_timeout(limit_ms=20.0, stream=None):
    """Runs the streaming kernel's starved-mbarrier failure path; returns the
    status code (ERR_TIMEOUT when it behaved)."""
    return lib().stencil_selftest_tma_timeout(float(limit_ms), _stream(stream))


def stencil_debug_fail_allocations(after):
    """Test hook: the allocation after `after` more successful ones fails (< 0: off)."""
    lib().stencil_debug_fail_allocations(int(after))


def stencil_selftest_barrier_timeout(limit_ms=20.0, stream=None):
    """Runs the bounded-wait failure path on the GPU; returns the status code
    (ERR_TIMEOUT when it behaved)."""
    return lib().stencil_selftest_barrier_timeout(float(limit_ms), _stream(stream))


def stencil_exchange_layout(h, Tb):
    nb, rows = ctypes.c_int(0), ctypes.c_int64(0)
    _check(lib().stencil_exchange_layout(h, int(Tb), ctypes.byref(nb), ctypes.byref(rows)))
    return nb.value, rows.value


def stencil_launch_count():
    return int(lib().stencil_launch_count())


def stencil_fp64_peak(millis=200.0, stream=None):
    """DFMA instructions per second measured on the current device."""
    r = ctypes.c_double(0.0)
    _check(lib().stencil_fp64_peak(float(millis), ctypes.byref(r), _stream(stream)))
    return r.value


# --------------------------------------------------------- convenience class

class Plan:
    """Owns a stencil plan.  Plan(dims, radius, weights, boundary) for constant
    weights; Plan.varcoef(dims, boundary) for the variable-coefficient form."""

    def __init__(self, dims, radius=None, weights=None, boundary=DIRICHLET_ZERO, _handle=None):
        self.dims = tuple(int(d) for d in dims)
        self.handle = _handle if _handle is not None else stencil_create(self.dims, radius, weights,
                                                                          boundary)

    @classmethod
    def varcoef(cls, dims, boundary=PERIODIC):
        return cls(dims, _handle=stencil_create_varcoef(tuple(dims), boundary))

    def run(self, grid, T, kappa=None, dt=0.0, stream=None):
        stencil_run(self.handle, grid, T, kappa, dt, stream)
        return grid

    def run_host(self, grid, T, kappa=None, dt=0.0, stream=None):
        stencil_run_host(self.handle, grid, T, kappa, dt, stream)
        return grid

    def adjoint(self, u0, kappa, dt, target, T, ckpt_every=0, stream=None):
        import torch
        gu = torch.empty_like(u0)
        gk = torch.empty_like(u0)
        loss = stencil_adjoint(self.handle, u0, kappa, dt, target, T, ckpt_every, gu, gk, stream)
        return loss, gu, gk

    def set_tuning(self, Tb, variant=0):
        stencil_set_tuning(self.handle, Tb, variant)

    def status(self, stream=None):
        return stencil_plan_status(self.handle, stream)

    def set_tile(self, tile_x=0, tile_y=0):
        """Tile of the 3D streaming kernel (64 x 8/16/32; 0 = default)."""
        _check(lib().stencil_set_tile(self.handle, int(tile_x), int(tile_y)))

    def get_tile(self):
        tx, ty = ctypes.c_int(0), ctypes.c_int(0)
        _check(lib().stencil_get_tile(self.handle, ctypes.byref(tx), ctypes.byref(ty)))
        return tx.value, ty.value

    def get_tuning(self):
        return stencil_get_tuning(self.handle)

    def exchange_layout(self, Tb):
        """(bands, rows computed) of the exchange kernel for Tb on this device."""
        return stencil_exchange_layout(self.handle, Tb)

    def autotune(self, scratch_grid, probe_steps=4, stream=None):
        return stencil_autotune(self.handle, scratch_grid, probe_steps, stream)

    def close(self):
        if self.handle:
            stencil_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Owns a batch plan of 2D heat grids (advanced in place by run())."""

    def __init__(self, grids, alphas, steps, boundary=DIRICHLET_ZERO):
        self.grids = list(grids)  # keep the tensors alive
        self.handle = stencil_batch_create(self.grids, alphas, steps, boundary)

    def run(self, stream=None):
        stencil_batch_run(self.handle, stream)

    def set_tuning(self, Tb=1, cells_per_thread=0, blocks_per_sm=0):
        _check(lib().stencil_batch_set_tuning(self.handle, int(Tb), int(cells_per_thread), int(blocks_per_sm)))

    def get_tuning(self):
        """(Tb, cells per thread, blocks per SM) of the batch's kernel."""
        t, c, b = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
        _check(lib().stencil_batch_get_tuning(self.handle, ctypes.byref(t), ctypes.byref(c), ctypes.byref(b)))
        return t.value, c.value, b.value

    def autotune(self, probe_steps=8, stream=None):
        """Times the kernel configurations on scratch copies of the items and
        keeps the fastest; returns its rate (GStencil/s)."""
        r = ctypes.c_double(0.0)
        _check(lib().stencil_batch_autotune(self.handle, int(probe_steps), _stream(stream), ctypes.byref(r)))
        return r.value

    def status(self):
        return stencil_batch_status(self.handle)

    def close(self):
        if self.handle:
            stencil_batch_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
