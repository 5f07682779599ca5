"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Each test checks the oracle against mathematics the paper's definition fixes
(Sec. 2.1 and Listing 1: a point's new value is a weighted sum of itself and
its neighbours at the previous step; Eq. 3: the heat weights 1-4mu and mu):
dense matrices built entry by entry on tiny grids, exact shifts and impulse
responses, eigenvector closed forms, Fourier symbols, invariants, and the
light-cone window evaluation against the whole-grid run.  A dropped tap, a
flipped offset sign (convolution instead of correlation), transposed axes, a
wrong boundary reading or a ping-pong slip each fails at least one of them.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
import synth
from conftest import normwise_rel

PERIODIC, DIRICHLET = 1, 0


def dense_matrix(shape, weights, radius, boundary):
    """A with (A u)_i = sum_o w_o u~(x_i + o), built cell by cell."""
    n = int(np.prod(shape))
    A = np.zeros((n, n))
    offs = list(itertools.product(range(-radius, radius + 1), repeat=len(shape)))
    wflat = np.asarray(weights).reshape(-1)
    for i, x in enumerate(itertools.product(*[range(s) for s in shape])):
        for o, w in zip(offs, wflat):
            if w == 0.0:
                continue
            y = [a + b for a, b in zip(x, o)]
            if boundary == PERIODIC:
                y = [v % s for v, s in zip(y, shape)]
            elif any(v < 0 or v >= s for v, s in zip(y, shape)):
                continue
            A[i, np.ravel_multi_index(y, shape)] += w
    return A


def matrix_power_apply(A, u0, T):
    v = u0.reshape(-1).copy()
    for _ in range(T):
        v = A @ v
    return v


CASES = [
    # (shape, radius, boundary, weight kind)
    ((11,), 1, PERIODIC, "random"),
    ((13,), 2, DIRICHLET, "random"),
    ((5, 7), 1, DIRICHLET, "heat"),
    ((5, 7), 1, PERIODIC, "random"),
    ((6, 5), 2, PERIODIC, "random"),
    ((7, 6), 2, DIRICHLET, "random"),
    ((2, 3), 1, PERIODIC, "random"),   # axis of 2: both neighbours are the same cell
    ((1, 5), 1, PERIODIC, "random"),   # axis of 1: every neighbour is the cell itself
    ((3, 4, 5), 1, DIRICHLET, "random"),
    ((3, 4, 5), 1, PERIODIC, "heat"),
    ((4, 3, 5), 1, PERIODIC, "random"),
    ((2, 3, 2), 1, DIRICHLET, "random"),
]


@pytest.mark.parametrize("shape,radius,boundary,kind", CASES)
def test_brute_force_dense_matrix(shape, radius, boundary, kind):
    ndim = len(shape)
    if kind == "heat":
        w = synth.heat_weights(ndim, 0.1)
    else:
        w = synth.uniform(17 + ndim + radius, (2 * radius + 1,) * ndim) - 0.3
    u0 = synth.uniform(5, shape) - 0.5
    T = 6
    A = dense_matrix(shape, w, radius, boundary)
    ref = matrix_power_apply(A, u0, T).reshape(shape)
    got = oracle.run(u0, w, radius, boundary, T)
    assert normwise_rel(got, ref) <= 1e-14


def test_shift_stencil_is_exact_roll_and_shift():
    """A single unit weight at offset o gives u'(x) = u(x+o): the correlation
    convention, axis order and both boundary rules, exactly."""
    u = synth.uniform(3, (4, 5, 6))
    for axis in range(3):
        for sign in (-1, 1):
            w = np.zeros((3, 3, 3))
            idx = [1, 1, 1]
            idx[axis] = 1 + sign
            w[tuple(idx)] = 1.0
            got = oracle.run(u, w, 1, PERIODIC, 1)
            assert np.array_equal(got, np.roll(u, -sign, axis=axis))
            got = oracle.run(u, w, 1, DIRICHLET, 1)
            exp = np.zeros_like(u)
            src = [slice(None)] * 3
            dst = [slice(None)] * 3
            if sign > 0:
                src[axis], dst[axis] = slice(1, None), slice(0, -1)
            else:
                src[axis], dst[axis] = slice(0, -1), slice(1, None)
            exp[tuple(dst)] = u[tuple(src)]
            assert np.array_equal(got, exp)


@pytest.mark.parametrize("ndim,radius", [(1, 2), (2, 1), (2, 2), (3, 1)])
def test_impulse_response_is_reflected_weights(ndim, radius):
    """One step on a unit impulse at c gives u'(c - o) = w_o."""
    side = 2 * radius + 1
    w = synth.uniform(40 + ndim, (side,) * ndim)
    shape = (side + 4,) * ndim
    u = np.zeros(shape)
    c = tuple(s // 2 for s in shape)
    u[c] = 1.0
    got = oracle.run(u, w, radius, DIRICHLET, 1)
    win = tuple(slice(ci - radius, ci + radius + 1) for ci in c)
    assert np.array_equal(got[win], np.flip(w))
    rest = got.copy()
    rest[win] = 0.0
    assert not rest.any()


def test_table1_point_counts():
    """Star and box shapes of radius r have the point counts of Table 1."""
    rows = [ln.split() for ln in open(__file__.replace("test_oracle_pins.py",
                                                       "golden/paper_table1_benchmarks.txt"))
            if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 8
    for name, ndim, radius, kind, pts, _ in rows:
        ndim, radius, pts = int(ndim), int(radius), int(pts)
        side = 2 * radius + 1
        if kind == "box":
            w = np.ones((side,) * ndim)
        else:
            w = np.zeros((side,) * ndim)
            for d in range(ndim):
                idx = [radius] * ndim
                for k in range(side):
                    idx[d] = k
                    w[tuple(idx)] = 1.0
        shape = (side + 2,) * ndim
        u = np.zeros(shape)
        u[tuple(s // 2 for s in shape)] = 1.0
        got = oracle.run(u, w, radius, DIRICHLET, 1)
        assert int(np.count_nonzero(got)) == pts, name


def dirichlet_heat_eigenvalue(shape, k, alpha):
    return 1.0 - 4.0 * alpha * sum(math.sin(math.pi * kd / (2.0 * (n + 1))) ** 2
                                   for n, kd in zip(shape, k))


def periodic_heat_eigenvalue(shape, k, alpha):
    return 1.0 - 4.0 * alpha * sum(math.sin(math.pi * kd / n) ** 2 for n, kd in zip(shape, k))


@pytest.mark.parametrize("shape,k,T", [((40, 56), (2, 3), 100), ((256, 256), (1, 1), 100),
                                       ((9, 12, 10), (1, 2, 3), 40)])
def test_dirichlet_sine_mode_decays_by_lambda_power(shape, k, T):
    """sin(pi k (x+1)/(N+1)) per axis is an eigenvector of the zero-Dirichlet
    heat stencil (Eq. 3) with eigenvalue 1 - 4 alpha sum sin^2(pi k/(2(N+1))).
    A frozen-boundary-ring reading of Listing 1 would fail this."""
    alpha = 0.1
    m = synth.dirichlet_sine_mode(shape, k)
    lam = dirichlet_heat_eigenvalue(shape, k, alpha)
    got = oracle.run(m, synth.heat_weights(len(shape), alpha), 1, DIRICHLET, T)
    # rounding error is measured against the initial amplitude max|m| = O(1)
    assert np.max(np.abs(got - lam ** T * m)) <= 1e-13 * np.max(np.abs(m))
    if shape == (256, 256):
        assert abs(lam ** T - 0.997016) < 1e-6


@pytest.mark.parametrize("shape,k,T", [((12, 16, 20), (1, 2, 3), 50), ((64, 48), (3, 5), 200)])
def test_periodic_sine_mode_decays_by_lambda_power(shape, k, T):
    """prod sin(2 pi k x / N) is an eigenvector of the periodic heat stencil
    with eigenvalue 1 - 4 alpha sum sin^2(pi k / N); by linearity the same
    holds on top of a random field."""
    alpha = 0.1
    w = synth.heat_weights(len(shape), alpha)
    m = synth.sine_mode(shape, k)
    lam = periodic_heat_eigenvalue(shape, k, alpha)
    got = oracle.run(m, w, 1, PERIODIC, T)
    assert np.max(np.abs(got - lam ** T * m)) <= 1e-13 * np.max(np.abs(m))
    r = synth.uniform(9, shape)
    diff = oracle.run(r + m, w, 1, PERIODIC, T) - oracle.run(r, w, 1, PERIODIC, T)
    assert np.max(np.abs(diff - lam ** T * m)) <= 1e-12


def test_config_eigenvalue_512_cube():
    """Closed-form decay for the 512^3, k=(3,5,7), alpha=0.1 configuration."""
    lam = periodic_heat_eigenvalue((512, 512, 512), (3, 5, 7), 0.1)
    assert abs(lam - 0.99875062) < 1e-8
    assert abs(lam ** 1000 - 0.28646) < 1e-5


@pytest.mark.parametrize("shape,radius,k,T", [((8, 12, 10), 1, (1, 2, 3), 12),
                                              ((16, 20), 2, (3, 1), 15),
                                              ((30,), 2, (4,), 25)])
def test_fourier_symbol_general_weights(shape, radius, k, T):
    """Under periodic wrap, e^{i theta.x} is an eigenvector of any constant
    stencil with eigenvalue S = sum_o w_o e^{i theta.o}; so cos(theta.x) maps
    to Re(e^{i theta.x} S^T).  Asymmetric weights: convolution in place of
    correlation (S -> conj S) fails this."""
    ndim = len(shape)
    v = synth.uniform(71 + ndim, (2 * radius + 1,) * ndim)
    w = v / v.sum()
    theta = [2.0 * math.pi * kd / n for kd, n in zip(k, shape)]
    grids = np.meshgrid(*[np.arange(n, dtype=np.float64) for n in shape], indexing="ij")
    phase = sum(t * g for t, g in zip(theta, grids))
    S = 0j
    for o in itertools.product(range(-radius, radius + 1), repeat=ndim):
        wo = w[tuple(oi + radius for oi in o)]
        S += wo * np.exp(1j * sum(t * oi for t, oi in zip(theta, o)))
    exp = np.real(np.exp(1j * phase) * S ** T)
    got = oracle.run(np.cos(phase), w, radius, PERIODIC, T)
    assert np.max(np.abs(got - exp)) <= 1e-13
    assert abs(S.imag) > 1e-3  # the test really exercises the asymmetric part


def test_invariants_constant_sum_maximum():
    shape = (10, 9, 11)
    v = synth.uniform(123, (3, 3, 3))
    w = v / v.sum()
    const = np.full(shape, 0.7)
    got = oracle.run(const, w, 1, PERIODIC, 20)
    assert np.max(np.abs(got - 0.7)) <= 1e-15
    u = synth.uniform(4, shape)
    got = oracle.run(u, w, 1, PERIODIC, 30)
    s0 = math.fsum(u.ravel())
    s1 = math.fsum(got.ravel())
    assert abs(s1 - s0) / abs(s0) <= 1e-13
    assert got.min() >= u.min() - 1e-15 and got.max() <= u.max() + 1e-15
    gd = oracle.run(u, w, 1, DIRICHLET, 30)
    assert gd.min() >= 0.0 and gd.max() <= u.max() + 1e-15
    assert math.fsum(gd.ravel()) < s0


def test_composition_and_zero_steps():
    u = synth.uniform(8, (7, 9))
    w = synth.heat_weights(2, 0.2)
    assert np.array_equal(oracle.run(u, w, 1, DIRICHLET, 0), u)
    a = oracle.run(oracle.run(u, w, 1, DIRICHLET, 3), w, 1, DIRICHLET, 4)
    b = oracle.run(u, w, 1, DIRICHLET, 7)
    assert np.array_equal(a, b)
    one = oracle.run(np.array([[2.5]]), w, 1, PERIODIC, 5)
    assert abs(one[0, 0] - 2.5) <= 1e-15  # weights sum to 1, every neighbour is itself


WINDOW_CASES = [
    ((40, 50), 1, DIRICHLET, 7, (0, 0), (5, 9)),
    ((40, 50), 1, DIRICHLET, 7, (35, 44), (40, 50)),
    ((40, 50), 1, PERIODIC, 7, (0, 45), (4, 50)),
    ((40, 50), 2, PERIODIC, 6, (18, 20), (23, 29)),
    ((40, 50), 2, DIRICHLET, 30, (18, 20), (23, 29)),   # cone covers the whole grid
    ((20, 18, 22), 1, PERIODIC, 5, (0, 3, 19), (3, 8, 22)),
    ((20, 18, 22), 1, DIRICHLET, 5, (17, 0, 0), (20, 4, 6)),
    ((20, 18, 22), 1, PERIODIC, 12, (5, 5, 5), (8, 9, 7)),  # wraps on some axes
]


@pytest.mark.parametrize("shape,radius,boundary,T,lo,hi", WINDOW_CASES)
def test_window_matches_whole_grid_run(shape, radius, boundary, T, lo, hi):
    ndim = len(shape)
    v = synth.uniform(90 + radius, (2 * radius + 1,) * ndim) - 0.2
    u = synth.normal(6, shape)
    full = oracle.run(u, v, radius, boundary, T)
    win = oracle.run_window(u, v, radius, boundary, T, lo, hi)
    sl = tuple(slice(a, b) for a, b in zip(lo, hi))
    assert np.array_equal(win, full[sl])


def test_bad_arguments_are_rejected():
    u = np.zeros((4, 4))
    with pytest.raises(ValueError):
        oracle.run(u, np.ones((3, 3)), 1, 2, 1)
    with pytest.raises(ValueError):
        oracle.run_window(u, np.ones((3, 3)), 1, 0, 1, (0, 0), (5, 1))


@pytest.mark.parametrize("shape,radius,boundary,T", [((7, 9), 1, 0, 3), ((5, 6, 7), 1, 1, 2), ((11,), 2, 0, 4),
                                                     ((6, 8), 2, 1, 3)])
def test_transpose_is_the_reflected_stencil(shape, radius, boundary, T):
    """<S_refl^T v, z> = <v, S^T z> (S^T: T steps; S_refl: the weights w_{-o}),
    for both boundary rules: the adjoint of the sweep is the sweep with
    reflected weights.  Also checked entry by entry against the transposed
    dense matrix."""
    ndim = len(shape)
    side = 2 * radius + 1
    w = synth.uniform(800 + ndim, (side,) * ndim)
    wr = np.ascontiguousarray(w[(slice(None, None, -1),) * ndim])
    v = synth.normal(801, shape)
    z = synth.normal(802, shape)
    lhs = float(np.sum(oracle.run(v, wr, radius, boundary, T) * z))
    rhs = float(np.sum(v * oracle.run(z, w, radius, boundary, T)))
    assert abs(lhs - rhs) <= 1e-13 * max(abs(lhs), abs(rhs))
    n = int(np.prod(shape))
    A = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        A[:, j] = oracle.run(e.reshape(shape), w, radius, boundary, 1).reshape(-1)
    AT = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        AT[:, j] = oracle.run(e.reshape(shape), wr, radius, boundary, 1).reshape(-1)
    assert np.allclose(AT, A.T, rtol=0, atol=1e-15)
