"""Pins of the oracle's variable-coefficient sweep and its adjoint.

The forward update is the explicit step of du/dt = div(kappa grad u) with the
arithmetic mean kappa on each face: u'_i = u_i + dt sum_faces
0.5(kappa_i+kappa_n)(u_n - u_i); with a constant kappa it is the heat stencil
of Eq. 3 with mu = dt*kappa.  The loss is 0.5 ||u^T - target||^2.  Pins:
a dense A(kappa) built entry by entry, the constant-kappa reduction to Eq. 3,
the dot-product identity <A^T v, w> = <v, A w>, gradients from dense matrix
products (A is affine in kappa, so dA/dkappa_m = A(e_m) - A(0) exactly),
central finite differences, and checkpoint-interval independence.
"""
import itertools

import numpy as np
import pytest

import oracle
import synth
from conftest import normwise_rel

PERIODIC, DIRICHLET = 1, 0


def dense_varcoef(shape, kappa, dt, boundary):
    n = int(np.prod(shape))
    A = np.eye(n)
    k = kappa.reshape(-1)
    for i, x in enumerate(itertools.product(*[range(s) for s in shape])):
        for d in range(len(shape)):
            for step in (-1, 1):
                y = list(x)
                y[d] += step
                if boundary == PERIODIC:
                    y[d] %= shape[d]
                elif y[d] < 0 or y[d] >= shape[d]:
                    A[i, i] -= dt * k[i]          # ghost face: kf = kappa_i, u_n = 0
                    continue
                j = np.ravel_multi_index(y, shape)
                kf = 0.5 * (k[i] + k[j])
                A[i, j] += dt * kf
                A[i, i] -= dt * kf
    return A


def dense_gradients(shape, u0, kappa, dt, target, boundary, T):
    A = dense_varcoef(shape, kappa, dt, boundary)
    us = [u0.reshape(-1)]
    for _ in range(T):
        us.append(A @ us[-1])
    r = us[-1] - target.reshape(-1)
    loss = 0.5 * float(r @ r)
    lams = [None] * (T + 1)
    lams[T] = r
    for t in range(T - 1, -1, -1):
        lams[t] = A.T @ lams[t + 1]
    A0 = dense_varcoef(shape, np.zeros_like(kappa), dt, boundary)
    gk = np.zeros(kappa.size)
    for m in range(kappa.size):
        e = np.zeros(kappa.size)
        e[m] = 1.0
        B = dense_varcoef(shape, e.reshape(shape), dt, boundary) - A0
        gk[m] = sum(float(lams[t + 1] @ (B @ us[t])) for t in range(T))
    return loss, lams[0].reshape(shape), gk.reshape(shape)


def inputs(shape, seed):
    u0 = synth.uniform(seed, shape)
    kappa = synth.lognormal(seed + 1, shape, 0.5)
    target = synth.normal(seed + 2, shape)
    dt = 0.1 / float(kappa.max())
    return u0, kappa, target, dt


@pytest.mark.parametrize("shape,boundary", [((4, 5, 3), PERIODIC), ((4, 5, 3), DIRICHLET),
                                            ((6, 7), PERIODIC), ((2, 3, 4), PERIODIC)])
def test_forward_matches_dense_matrix(shape, boundary):
    u0, kappa, _, dt = inputs(shape, 31)
    A = dense_varcoef(shape, kappa, dt, boundary)
    ref = u0.reshape(-1)
    for _ in range(9):
        ref = A @ ref
    got = oracle.varcoef_run(u0, kappa, dt, boundary, 9)
    assert normwise_rel(got, ref.reshape(shape)) <= 1e-14


def test_constant_kappa_reduces_to_heat_stencil():
    shape = (7, 8, 9)
    u0 = synth.uniform(2, shape)
    k = 0.8
    dt = 0.1 / k
    got = oracle.varcoef_run(u0, np.full(shape, k), dt, PERIODIC, 15)
    ref = oracle.run(u0, synth.heat_weights(3, dt * k), 1, PERIODIC, 15)
    assert normwise_rel(got, ref) <= 1e-14


@pytest.mark.parametrize("boundary", [PERIODIC, DIRICHLET])
def test_transpose_dot_product_identity(boundary):
    shape = (5, 6, 4)
    _, kappa, _, dt = inputs(shape, 41)
    v = synth.normal(50, shape)
    w = synth.normal(51, shape)
    Atv = oracle.varcoef_transpose_step(v, kappa, dt, boundary)
    Aw = oracle.varcoef_run(w, kappa, dt, boundary, 1)
    lhs = float(np.sum(Atv * w))
    rhs = float(np.sum(v * Aw))
    assert abs(lhs - rhs) <= 1e-13 * max(abs(lhs), 1.0)
    A = dense_varcoef(shape, kappa, dt, boundary)
    assert normwise_rel(Atv.reshape(-1), A.T @ v.reshape(-1)) <= 1e-14


@pytest.mark.parametrize("shape,boundary,T", [((3, 4, 5), PERIODIC, 7), ((3, 4, 5), DIRICHLET, 6),
                                              ((5, 6), PERIODIC, 9), ((2, 2, 3), PERIODIC, 4)])
def test_gradients_match_dense_chain_rule(shape, boundary, T):
    u0, kappa, target, dt = inputs(shape, 61)
    loss, gu, gk = oracle.varcoef_adjoint(u0, kappa, dt, target, boundary, T)
    rloss, rgu, rgk = dense_gradients(shape, u0, kappa, dt, target, boundary, T)
    assert abs(loss - rloss) <= 1e-13 * abs(rloss)
    assert normwise_rel(gu, rgu) <= 1e-12
    assert normwise_rel(gk, rgk) <= 1e-12


def test_central_finite_differences():
    shape = (6, 5, 7)
    boundary = PERIODIC
    T = 20
    u0, kappa, target, dt = inputs(shape, 71)
    loss, gu, gk = oracle.varcoef_adjoint(u0, kappa, dt, target, boundary, T)

    def L(u, k):
        uT = oracle.varcoef_run(u, k, dt, boundary, T)
        return 0.5 * float(np.sum((uT - target) ** 2))

    assert abs(L(u0, kappa) - loss) <= 1e-13 * loss
    du = synth.normal(80, shape)
    dk = synth.normal(81, shape) * kappa
    h = 1e-4
    fd_u = (L(u0 + h * du, kappa) - L(u0 - h * du, kappa)) / (2 * h)
    assert abs(fd_u - float(np.sum(gu * du))) <= 1e-8 * abs(fd_u)
    h = 1e-5
    fd_k = (L(u0, kappa + h * dk) - L(u0, kappa - h * dk)) / (2 * h)
    assert abs(fd_k - float(np.sum(gk * dk))) <= 1e-7 * abs(fd_k)


def test_checkpoint_interval_does_not_change_results():
    shape = (4, 6, 5)
    T = 23
    u0, kappa, target, dt = inputs(shape, 91)
    ref = oracle.varcoef_adjoint(u0, kappa, dt, target, PERIODIC, T, ckpt_every=0)
    for c in (1, 3, 7, 23, 30):
        got = oracle.varcoef_adjoint(u0, kappa, dt, target, PERIODIC, T, ckpt_every=c)
        assert got[0] == ref[0]
        assert np.array_equal(got[1], ref[1]) and np.array_equal(got[2], ref[2])


def test_zero_steps():
    shape = (3, 3, 3)
    u0, kappa, target, dt = inputs(shape, 5)
    loss, gu, gk = oracle.varcoef_adjoint(u0, kappa, dt, target, PERIODIC, 0)
    assert np.array_equal(gu, u0 - target)
    assert not gk.any()
    assert abs(loss - 0.5 * float(np.sum((u0 - target) ** 2))) <= 1e-14 * loss
