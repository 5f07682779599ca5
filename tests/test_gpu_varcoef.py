"""GPU parity of the variable-coefficient sweep and its adjoint.

Forward: element-wise against the oracle (normwise relative <= 1e-12).
Adjoint: loss and both gradients against the oracle's adjoint (which stores
every state on small grids, or checkpoints like the library on larger ones),
the checkpoint interval leaves the GPU result bitwise unchanged, and central
finite differences of the GPU's own forward sweep agree with the GPU
gradient along random directions at the full 256^3 size.
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
    return st


def inputs(shape, seed):
    u0 = synth.uniform(seed, shape)
    kappa = synth.lognormal(seed + 1, shape, 0.5)
    target = synth.normal(seed + 2, shape)
    dt = 0.1 / float(kappa.max())
    return u0, kappa, target, dt


def cuda(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("shape,boundary,T", [((24, 20, 28), PERIODIC, 30), ((24, 20, 28), DIRICHLET, 25),
                                              ((33, 47), PERIODIC, 40), ((31, 29), DIRICHLET, 40),
                                              ((1, 5, 2), PERIODIC, 6)])
def test_forward_parity(st, shape, boundary, T):
    u0, kappa, _, dt = inputs(shape, 11)
    ref = oracle.varcoef_run(u0, kappa, dt, boundary, T, nthreads=0)
    p = st.Plan.varcoef(shape, boundary)
    g = cuda(u0)
    p.run(g, T, cuda(kappa), dt)
    assert normwise_rel(g.cpu().numpy(), ref) <= TOL
    p.close()


@pytest.mark.parametrize("shape,boundary,T,ck", [((16, 16, 16), PERIODIC, 20, 0), ((12, 14, 10), DIRICHLET, 21, 4),
                                                 ((32, 32, 32), PERIODIC, 64, 8), ((20, 24), DIRICHLET, 30, 0),
                                                 # odd rows: the kernels pair cells along y
                                                 ((9, 13, 11), PERIODIC, 17, 5), ((15, 21), DIRICHLET, 19, 3),
                                                 ((7, 1, 9), DIRICHLET, 6, 2)])
def test_adjoint_parity(st, shape, boundary, T, ck):
    u0, kappa, target, dt = inputs(shape, 21)
    rl, rgu, rgk = oracle.varcoef_adjoint(u0, kappa, dt, target, boundary, T, ckpt_every=ck, nthreads=0)
    p = st.Plan.varcoef(shape, boundary)
    loss, gu, gk = p.adjoint(cuda(u0), cuda(kappa), dt, cuda(target), T, ckpt_every=ck)
    assert abs(loss - rl) <= TOL * abs(rl)
    assert normwise_rel(gu.cpu().numpy(), rgu) <= TOL
    assert normwise_rel(gk.cpu().numpy(), rgk) <= TOL
    p.close()


def test_checkpoint_interval_is_bitwise_neutral(st):
    shape = (20, 18, 22)
    u0, kappa, target, dt = inputs(shape, 31)
    p = st.Plan.varcoef(shape, PERIODIC)
    # T = 37 leaves a last segment of 1..c steps; T = 36 with c = 6 or 12 a full one
    # (the forward sweep keeps the last segment's states, the others are recomputed)
    for T, cs in ((37, (0, 2, 5, 36, 37, 50)), (36, (6, 12, 35))):
        ref = p.adjoint(cuda(u0), cuda(kappa), dt, cuda(target), T, ckpt_every=1)
        for c in cs:
            got = p.adjoint(cuda(u0), cuda(kappa), dt, cuda(target), T, ckpt_every=c)
            assert got[0] == ref[0]
            assert bool((got[1] == ref[1]).all()) and bool((got[2] == ref[2]).all())
    p.close()


@pytest.mark.slow
def test_forward_parity_at_config_size(st):
    """The 256^3 periodic var-coef workload, in the launch configuration the
    benchmark times: three steps of the GPU sweep against the oracle element by
    element over all 16.8 million cells."""
    shape = (256, 256, 256)
    u0, kappa, _, dt = inputs(shape, synth.SEED_ADJOINT)
    T = 3
    ref = oracle.varcoef_run(u0, kappa, dt, PERIODIC, T, nthreads=0)
    p = st.Plan.varcoef(shape, PERIODIC)
    g = cuda(u0)
    p.run(g, T, cuda(kappa), dt)
    assert normwise_rel(g.cpu().numpy(), ref) <= TOL
    p.close()


@pytest.mark.slow
def test_adjoint_parity_at_config_size(st):
    """The 256^3 periodic adjoint workload (checkpoint interval 32 as in the
    benchmark; T = 2 keeps the oracle's reverse sweep to seconds): loss and
    both gradients against the oracle's adjoint over every cell."""
    shape = (256, 256, 256)
    u0, kappa, target, dt = inputs(shape, synth.SEED_ADJOINT)
    T = 2
    rl, rgu, rgk = oracle.varcoef_adjoint(u0, kappa, dt, target, PERIODIC, T, nthreads=0)
    p = st.Plan.varcoef(shape, PERIODIC)
    loss, gu, gk = p.adjoint(cuda(u0), cuda(kappa), dt, cuda(target), T, ckpt_every=32)
    assert abs(loss - rl) <= TOL * abs(rl)
    assert normwise_rel(gu.cpu().numpy(), rgu) <= TOL
    assert normwise_rel(gk.cpu().numpy(), rgk) <= TOL
    p.close()


@pytest.mark.slow
def test_full_size_finite_differences(st):
    """256^3, T=1000, checkpoints every 32: directional derivatives of the
    loss along random directions match the adjoint gradient."""
    import torch
    shape = (256, 256, 256)
    seed = synth.SEED_ADJOINT
    u0, kappa, target, dt = inputs(shape, seed)
    T = 1000
    p = st.Plan.varcoef(shape, PERIODIC)
    U0, K, TG = cuda(u0), cuda(kappa), cuda(target)
    loss, gu, gk = p.adjoint(U0, K, dt, TG, T, ckpt_every=32)

    def final(u, k):
        x = u.clone()
        p.run(x, T, k, dt)
        return x

    def dL(up, um):
        # L(+) - L(-) summed element by element as (u+ - u-)(u+ + u- - 2 target)/2,
        # so the difference is not lost in the rounding of two ~1e7 sums
        return 0.5 * float(((up - um) * (up + um - 2.0 * TG)).sum())

    base = final(U0, K)
    assert abs(0.5 * float(((base - TG) ** 2).sum()) - loss) <= 1e-12 * loss
    du = cuda(synth.normal(seed + 10, shape))
    dk = cuda(synth.normal(seed + 11, shape)) * K
    h = 1e-3
    fd_u = dL(final(U0 + h * du, K), final(U0 - h * du, K)) / (2 * h)
    an_u = float((gu * du).sum())
    assert abs(fd_u - an_u) <= 1e-8 * abs(an_u)
    h = 1e-5
    fd_k = dL(final(U0, K + h * dk), final(U0, K - h * dk)) / (2 * h)
    an_k = float((gk * dk).sum())
    assert abs(fd_k - an_k) <= 1e-6 * abs(an_k)
    p.close()
    torch.cuda.synchronize()


def test_autograd_function_matches_adjoint_and_oracle(st):
    """StencilAdjointFn: backward of 0.5||u^T - target||^2 through torch
    autograd equals the loss-form adjoint bitwise, and a linear functional
    sum(w * u^T) gives the oracle's gradients."""
    import torch
    from paper_2303_08365_gb300.autograd import diffuse
    shape = (12, 10, 14)
    u0, kappa, target, dt = inputs(shape, 41)
    T, ck = 23, 5
    p = st.Plan.varcoef(shape, PERIODIC)
    U = cuda(u0).requires_grad_(True)
    K = cuda(kappa).requires_grad_(True)
    TG = cuda(target)
    uT = diffuse(U, K, p, dt, T, ck)
    loss = 0.5 * ((uT - TG) ** 2).sum()
    loss.backward()
    ref_loss, gu, gk = p.adjoint(cuda(u0), cuda(kappa), dt, TG, T, ckpt_every=ck)
    assert abs(float(loss.detach()) - ref_loss) <= 1e-12 * ref_loss
    assert bool((U.grad == gu).all()) and bool((K.grad == gk).all())
    # linear functional L = sum(w u^T): lambda^T = w; the oracle sees target = u^T - w
    w = synth.normal(77, shape)
    U.grad = None
    K.grad = None
    (diffuse(U, K, p, dt, T, ck) * cuda(w)).sum().backward()
    uT_o = oracle.varcoef_run(u0, kappa, dt, PERIODIC, T)
    _, rgu, rgk = oracle.varcoef_adjoint(u0, kappa, dt, uT_o - w, PERIODIC, T)
    assert normwise_rel(U.grad.cpu().numpy(), rgu) <= TOL
    assert normwise_rel(K.grad.cpu().numpy(), rgk) <= TOL
    p.close()


@pytest.mark.parametrize("shape,radius,boundary,T", [((23, 31), 1, DIRICHLET, 9), ((9, 10, 11), 1, PERIODIC, 7),
                                                     ((29, 33), 2, DIRICHLET, 5), ((400,), 2, PERIODIC, 12)])
def test_constant_weight_autograd_is_the_reflected_stencil(st, shape, radius, boundary, T):
    """d<v, S^T u0>/du0 = (S^T)^T v: the transposed stencil (reflected weights)
    swept T steps over v.  Checked against the oracle with reflected weights and
    by the dot-product identity <(S^T)^T v, w> = <v, S^T w> with the oracle's S."""
    import torch
    from paper_2303_08365_gb300 import autograd as ag
    ndim = len(shape)
    side = 2 * radius + 1
    w = synth.uniform(500 + ndim + radius, (side,) * ndim)
    w /= w.sum()
    u0 = synth.uniform(501, shape)
    v = synth.normal(502, shape)
    x = torch.from_numpy(u0.copy()).cuda().requires_grad_(True)
    uT = ag.sweep(x, shape, radius, w, boundary, T)
    loss = (uT * torch.from_numpy(v).cuda()).sum()
    loss.backward()
    g = x.grad.cpu().numpy()
    assert normwise_rel(uT.detach().cpu().numpy(), oracle.run(u0, w, radius, boundary, T, nthreads=0)) <= TOL
    assert normwise_rel(g, oracle.run(v, ag.reflected(w), radius, boundary, T, nthreads=0)) <= TOL
    z = synth.normal(503, shape)
    lhs = float(np.sum(g * z))
    rhs = float(np.sum(v * oracle.run(z, w, radius, boundary, T, nthreads=0)))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), abs(rhs), 1.0)
