"""Plain CPU FP64 oracle for the iterative stencil sweep (ctypes wrapper).

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
benchmark's cpu_baseline / reference leg may import this package.  It shares
no code with the CUDA library: the arithmetic lives in oracle.c, written from
the paper's definition (Sec. 2.1, Listing 1, Eq. 3) and, for the
variable-coefficient adjoint, from the chain rule applied to that update.

Parity pins (tests/test_oracle_*.py): brute-force dense matrices on tiny grids,
the sine-mode eigenvalue closed forms, the Fourier symbol of general weights,
shift stencils, invariants (constant field, conserved sum, maximum principle),
the adjoint dot-product identity and central finite differences.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        i64p = ctypes.POINTER(ctypes.c_int64)
        dp = ctypes.POINTER(ctypes.c_double)
        L.oracle_run.argtypes = [ctypes.c_int, i64p, ctypes.c_int, dp, ctypes.c_int, dp,
                                 ctypes.c_int64, ctypes.c_int]
        L.oracle_run_window.argtypes = [ctypes.c_int, i64p, ctypes.c_int, dp, ctypes.c_int, dp,
                                        ctypes.c_int64, i64p, i64p, dp]
        L.oracle_varcoef_run.argtypes = [ctypes.c_int, i64p, ctypes.c_int, dp, dp,
                                         ctypes.c_double, ctypes.c_int64, ctypes.c_int]
        L.oracle_varcoef_adjoint.argtypes = [ctypes.c_int, i64p, ctypes.c_int, dp, dp,
                                             ctypes.c_double, dp, ctypes.c_int64, ctypes.c_int,
                                             dp, dp, dp, ctypes.c_int]
        L.oracle_varcoef_transpose_step.argtypes = [ctypes.c_int, i64p, ctypes.c_int, dp,
                                                    ctypes.c_double, dp, dp]
        for f in (L.oracle_run, L.oracle_run_window, L.oracle_varcoef_run,
                  L.oracle_varcoef_adjoint, L.oracle_varcoef_transpose_step):
            f.restype = ctypes.c_int
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _i64(seq):
    arr = (ctypes.c_int64 * len(seq))(*[int(v) for v in seq])
    return arr


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _check(rc, name):
    if rc != 0:
        raise ValueError(f"{name}: bad argument (status {rc})")


def run(u0, weights, radius, boundary, T, nthreads=1):
    """u after T steps of u'(x) = sum_o w_o u(x+o); u0 is not modified.

    weights: dense (2r+1)^ndim array; boundary 0 = Dirichlet zero, 1 = periodic.
    """
    u = _f64(u0).copy()
    w = _f64(weights)
    assert w.size == (2 * radius + 1) ** u.ndim, "weights must be (2r+1)^ndim"
    rc = lib().oracle_run(u.ndim, _i64(u.shape), radius, _dp(w), boundary, _dp(u), int(T),
                          int(nthreads))
    _check(rc, "oracle_run")
    return u


def run_window(u0, weights, radius, boundary, T, lo, hi):
    """Values on the box [lo, hi) after T steps, from the light cone of the box only."""
    u = _f64(u0)
    w = _f64(weights)
    shape = tuple(int(h) - int(l) for l, h in zip(lo, hi))
    out = np.empty(shape, dtype=np.float64)
    rc = lib().oracle_run_window(u.ndim, _i64(u.shape), radius, _dp(w), boundary, _dp(u),
                                 int(T), _i64(lo), _i64(hi), _dp(out))
    _check(rc, "oracle_run_window")
    return out


def varcoef_run(u0, kappa, dt, boundary, T, nthreads=1):
    """u after T steps of u'_i = u_i + dt sum_faces 0.5(k_i+k_n)(u_n-u_i)."""
    u = _f64(u0).copy()
    k = _f64(kappa)
    assert k.shape == u.shape
    rc = lib().oracle_varcoef_run(u.ndim, _i64(u.shape), boundary, _dp(u), _dp(k), float(dt),
                                  int(T), int(nthreads))
    _check(rc, "oracle_varcoef_run")
    return u


def varcoef_adjoint(u0, kappa, dt, target, boundary, T, ckpt_every=0, nthreads=1):
    """(loss, dL/du0, dL/dkappa) for L = 0.5 ||u^T - target||^2, dt held fixed."""
    u = _f64(u0)
    k = _f64(kappa)
    tg = _f64(target)
    gu = np.empty_like(u)
    gk = np.empty_like(u)
    loss = np.zeros(1, dtype=np.float64)
    rc = lib().oracle_varcoef_adjoint(u.ndim, _i64(u.shape), boundary, _dp(u), _dp(k),
                                      float(dt), _dp(tg), int(T), int(ckpt_every), _dp(gu),
                                      _dp(gk), _dp(loss), int(nthreads))
    _check(rc, "oracle_varcoef_adjoint")
    return float(loss[0]), gu, gk


def varcoef_transpose_step(lam, kappa, dt, boundary):
    """A(kappa)^T lam for one variable-coefficient step (scatter of A's rows)."""
    lm = _f64(lam)
    k = _f64(kappa)
    out = np.empty_like(lm)
    rc = lib().oracle_varcoef_transpose_step(lm.ndim, _i64(lm.shape), boundary, _dp(k),
                                             float(dt), _dp(lm), _dp(out))
    _check(rc, "oracle_varcoef_transpose_step")
    return out

