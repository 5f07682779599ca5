"""GPU parity of the constant-weight sweep against the CPU oracle.

Bar: normwise relative error max|g - o| / max|o| <= 1e-12 after T steps (the
GPU fuses multiply-adds and orders the taps differently; every workload is a
non-expansive map, so rounding does not grow beyond ~T ulp).  Small and
ragged grids are compared element by element over the whole grid; the
full-size workloads are compared on sampled windows computed from their
light cones, and through closed forms at the full step count.
"""
import math

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


def gpu_run(st, u0, w, radius, boundary, T, Tb=0, variant=0):
    import torch
    g = torch.from_numpy(np.ascontiguousarray(u0)).cuda()
    p = st.Plan(u0.shape, radius, w, boundary)
    if Tb:
        p.set_tuning(Tb, variant)
    p.run(g, T)
    torch.cuda.synchronize()
    out = g.cpu().numpy()
    p.close()
    return out


def weights_for(kind, ndim, radius, seed):
    side = 2 * radius + 1
    if kind == "heat":
        return synth.heat_weights(ndim, 0.1)
    if kind == "box_eq":
        return synth.box_weights(ndim, 1.0 / side ** ndim)
    if kind == "box_rand":
        v = synth.uniform(seed, (side,) * ndim)
        return v / v.sum()
    if kind == "star_rand":
        w = np.zeros((side,) * ndim)
        v = synth.uniform(seed, (2 * ndim * radius + 1,))
        v /= v.sum()
        c = (radius,) * ndim
        w[c] = v[0]
        k = 1
        for d in range(ndim):
            for o in range(-radius, radius + 1):
                if o == 0:
                    continue
                idx = list(c)
                idx[d] += o
                w[tuple(idx)] = v[k]
                k += 1
        return w
    raise ValueError(kind)


SMALL = [
    # shape, radius, boundary, kind, T
    ((256, 256), 1, DIRICHLET, "heat", 100),      # the 256^2 heat workload, full size
    ((37, 53), 1, DIRICHLET, "heat", 17),
    ((37, 53), 1, PERIODIC, "box_eq", 9),
    ((61, 45), 1, PERIODIC, "box_rand", 12),
    ((29, 33), 2, DIRICHLET, "box_rand", 7),
    ((29, 33), 2, PERIODIC, "star_rand", 8),
    ((13, 17, 19), 1, PERIODIC, "heat", 11),
    ((13, 17, 19), 1, DIRICHLET, "box_rand", 10),
    ((9, 40, 70), 1, DIRICHLET, "star_rand", 6),
    ((11, 12, 13), 2, PERIODIC, "star_rand", 5),
    ((7, 9, 11), 2, DIRICHLET, "box_rand", 4),
    ((1000,), 1, PERIODIC, "star_rand", 25),
    ((777,), 2, DIRICHLET, "star_rand", 13),
    ((1, 1), 1, PERIODIC, "heat", 3),
    ((1, 7), 1, DIRICHLET, "heat", 4),
    ((3, 2), 2, PERIODIC, "box_rand", 5),   # axes shorter than the radius
    ((2, 1, 3), 1, PERIODIC, "box_rand", 4),
]


@pytest.mark.parametrize("shape,radius,boundary,kind,T", SMALL)
def test_parity_whole_grid(st, shape, radius, boundary, kind, T):
    ndim = len(shape)
    w = weights_for(kind, ndim, radius, 100 + len(shape) + radius)
    u0 = synth.uniform(7, shape) if kind != "box_rand" else synth.normal(7, shape)
    ref = oracle.run(u0, w, radius, boundary, T, nthreads=0)
    got = gpu_run(st, u0, w, radius, boundary, T)
    assert normwise_rel(got, ref) <= TOL


def test_zero_steps_is_identity(st):
    u0 = synth.uniform(3, (20, 30))
    got = gpu_run(st, u0, synth.heat_weights(2, 0.1), 1, DIRICHLET, 0)
    assert np.array_equal(got, u0)


def test_odd_and_even_step_counts_compose(st):
    import torch
    u0 = synth.uniform(4, (33, 65))
    w = synth.heat_weights(2, 0.2)
    g = torch.from_numpy(u0.copy()).cuda()
    p = st.Plan(u0.shape, 1, w, DIRICHLET)
    p.run(g, 3)
    p.run(g, 4)
    a = g.cpu().numpy()
    g2 = torch.from_numpy(u0.copy()).cuda()
    p.run(g2, 7)
    assert np.array_equal(a, g2.cpu().numpy())


def test_host_entry_matches_device_entry(st):
    u0 = synth.uniform(5, (48, 40, 36))
    w = synth.heat_weights(3, 0.1)
    dev = gpu_run(st, u0, w, 1, PERIODIC, 9)
    h = u0.copy()
    p = st.Plan(u0.shape, 1, w, PERIODIC)
    p.run_host(h, 9)
    p.close()
    assert np.array_equal(h, dev)


# Full-size workloads: sampled windows from the light cone at a short step
# count, in the launch configuration the benchmark times.
FULL = [
    ((512, 512, 512), 1, PERIODIC, "heat", 3, synth.SEED_HEAT3D),
    ((16384, 16384), 1, PERIODIC, "box_eq", 3, synth.SEED_BOX2D),
    ((384, 384, 384), 1, DIRICHLET, "box_rand", 3, synth.SEED_BOX3D),
    # the widened workloads, in the launch configuration the benchmark times
    ((8192, 8192), 2, PERIODIC, "star_rand", 3, synth.SEED_BOX2D + 11),
    ((8192, 8192), 2, PERIODIC, "box_rand", 3, synth.SEED_BOX2D + 11),
    ((9600, 9600), 1, DIRICHLET, "heat", 4, synth.SEED_HEAT2D + 30),
    ((10_000_000,), 1, DIRICHLET, "heat", 16, synth.SEED_HEAT2D + 20),
    ((10_000_000,), 2, PERIODIC, "star_rand", 17, synth.SEED_HEAT2D + 21),
]


def window_boxes(shape):
    """Corner, edge and interior windows (ragged sizes)."""
    boxes = []
    for pos in ("lo", "mid", "hi"):
        lo, hi = [], []
        for n in shape:
            w = 5 if len(shape) == 3 else 9
            a = {"lo": 0, "mid": n // 2 - 3, "hi": n - w}[pos]
            lo.append(a)
            hi.append(a + w)
        boxes.append((tuple(lo), tuple(hi)))
    return boxes


@pytest.mark.slow
@pytest.mark.parametrize("shape,radius,boundary,kind,T,seed", FULL)
def test_parity_full_size_windows(st, shape, radius, boundary, kind, T, seed):
    import torch
    ndim = len(shape)
    w = weights_for(kind, ndim, radius, seed)
    u0 = synth.normal(seed, shape) if kind == "box_rand" else synth.uniform(seed, shape)
    g = torch.from_numpy(u0).cuda()
    p = st.Plan(shape, radius, w, boundary)
    p.run(g, T)
    torch.cuda.synchronize()
    for lo, hi in window_boxes(shape):
        ref = oracle.run_window(u0, w, radius, boundary, T, lo, hi)
        sl = tuple(slice(a, b) for a, b in zip(lo, hi))
        got = g[sl].cpu().numpy()
        assert normwise_rel(got, ref) <= TOL, (lo, hi)
    p.close()


# The temporal kernel at the full sizes, for every Tb the plan autotuner
# offers: windows against the oracle after two Tb-blocks and a remainder step.
FULL_TEMPORAL = [
    ((512, 512, 512), PERIODIC, "heat", synth.SEED_HEAT3D),
    ((384, 384, 384), DIRICHLET, "box_rand", synth.SEED_BOX3D),
    ((16384, 16384), PERIODIC, "box_eq", synth.SEED_BOX2D),
]


@pytest.mark.slow
@pytest.mark.parametrize("shape,boundary,kind,seed", FULL_TEMPORAL)
def test_temporal_full_size_windows(st, shape, boundary, kind, seed):
    import torch
    w = weights_for(kind, len(shape), 1, seed)
    u0 = synth.normal(seed, shape) if kind == "box_rand" else synth.uniform(seed, shape)
    g = torch.empty(shape, dtype=torch.float64, device="cuda")
    p = st.Plan(shape, 1, w, boundary)
    for Tb in (2, 4, 8):
        T = 2 * Tb + 1
        p.set_tuning(Tb, st.VARIANT_TEMPORAL)
        g.copy_(torch.from_numpy(u0))
        p.run(g, T)
        torch.cuda.synchronize()
        for lo, hi in window_boxes(shape):
            ref = oracle.run_window(u0, w, 1, boundary, T, lo, hi)
            sl = tuple(slice(a, b) for a, b in zip(lo, hi))
            assert normwise_rel(g[sl].cpu().numpy(), ref) <= TOL, (Tb, lo, hi)
    p.close()


@pytest.mark.slow
def test_full_size_512_cube_sine_mode_closed_form(st):
    """512^3 periodic heat, T=1000: by linearity run(r + m) - run(r) = lam^T m
    for the sine mode k=(3,5,7); the mean is conserved."""
    import torch
    shape = (512, 512, 512)
    w = synth.heat_weights(3, 0.1)
    T = 1000
    lam = 1.0 - 0.4 * sum(math.sin(math.pi * k / 512) ** 2 for k in (3, 5, 7))
    r = torch.from_numpy(synth.uniform(synth.SEED_HEAT3D, shape)).cuda()
    m = torch.from_numpy(synth.sine_mode(shape, (3, 5, 7))).cuda()
    a = r + m
    b = r.clone()
    p = st.Plan(shape, 1, w, PERIODIC)
    mean0 = float(r.mean())
    p.run(a, T)
    p.run(b, T)
    torch.cuda.synchronize()
    d = (a - b) - (lam ** T) * m
    assert float(d.abs().max()) <= TOL * float(a.abs().max())
    assert abs(float(b.mean()) - mean0) <= 1e-12
    assert float(b.min()) >= float(r.min()) - 1e-12 and float(b.max()) <= float(r.max()) + 1e-12
    p.close()


def test_launch_count_advances(st):
    import torch
    before = st.stencil_launch_count()
    u0 = synth.uniform(1, (16, 16))
    gpu_run(st, u0, synth.heat_weights(2, 0.1), 1, DIRICHLET, 5, Tb=1, variant=st.VARIANT_DIRECT)
    assert st.stencil_launch_count() >= before + 5
    mid = st.stencil_launch_count()
    gpu_run(st, u0, synth.heat_weights(2, 0.1), 1, DIRICHLET, 5, Tb=1, variant=st.VARIANT_PERSISTENT)
    assert st.stencil_launch_count() == mid + 1   # one persistent launch for all 5 steps
    torch.cuda.synchronize()


def test_fp64_peak_is_plausible(st):
    r = st.stencil_fp64_peak(50.0)
    assert 1e11 < r < 1e13


STREAM_CASES = [
    # shape, boundary, kind
    ((40, 64, 128), PERIODIC, "heat"),
    ((40, 48, 128), PERIODIC, "box_rand"),
    ((13, 37, 70), DIRICHLET, "heat"),
    ((13, 37, 70), DIRICHLET, "box_rand"),
    ((5, 20, 130), DIRICHLET, "star_rand"),
    ((1, 16, 64), PERIODIC, "box_rand"),
    ((3, 1, 2), DIRICHLET, "box_rand"),
]


@pytest.mark.parametrize("shape,boundary,kind", STREAM_CASES)
def test_stream_kernel_matches_direct_bitwise_and_oracle(st, shape, boundary, kind):
    """The TMA streaming kernel applies the taps in the direct kernel's order:
    the two agree bit for bit; both match the oracle."""
    w = weights_for(kind, 3, 1, 300)
    u0 = synth.normal(8, shape)
    T = 6
    a = gpu_run(st, u0, w, 1, boundary, T, Tb=1, variant=st.VARIANT_STREAM)
    b = gpu_run(st, u0, w, 1, boundary, T, Tb=1, variant=st.VARIANT_DIRECT)
    assert np.array_equal(a, b)
    ref = oracle.run(u0, w, 1, boundary, T, nthreads=0)
    assert normwise_rel(a, ref) <= TOL


def test_stream_kernel_rejects_ineligible_shapes(st):
    import torch
    u0 = synth.uniform(2, (8, 20, 70))   # periodic needs nx % 64 == 0 and ny % 16 == 0
    p = st.Plan(u0.shape, 1, synth.heat_weights(3, 0.1), PERIODIC)
    p.set_tuning(1, st.VARIANT_STREAM)
    g = torch.from_numpy(u0).cuda()
    with pytest.raises(st.StencilError) as ei:
        p.run(g, 2)
    assert ei.value.code == st.ERR_UNSUPPORTED
    p.set_tuning(0, 0)          # automatic choice falls back to the direct kernel
    p.run(g, 2)
    assert p.status() == 0
    p.close()


STREAM2D_CASES = [
    ((32, 128), PERIODIC, "star_rand"),
    ((32, 128), PERIODIC, "box_rand"),
    ((37, 70), DIRICHLET, "heat"),
    ((37, 70), DIRICHLET, "box_rand"),
    ((130, 64), DIRICHLET, "star_rand"),
    ((1, 2), DIRICHLET, "box_rand"),
]


@pytest.mark.parametrize("shape,boundary,kind", STREAM2D_CASES)
def test_stream2d_matches_direct_bitwise_and_oracle(st, shape, boundary, kind):
    w = weights_for(kind, 2, 1, 400)
    u0 = synth.normal(9, shape)
    T = 7
    a = gpu_run(st, u0, w, 1, boundary, T, Tb=1, variant=st.VARIANT_STREAM)
    b = gpu_run(st, u0, w, 1, boundary, T, Tb=1, variant=st.VARIANT_DIRECT)
    assert np.array_equal(a, b)
    assert normwise_rel(a, oracle.run(u0, w, 1, boundary, T, nthreads=0)) <= TOL


@pytest.mark.parametrize("shape,boundary,T", [((64, 256), PERIODIC, 40), ((45, 94), DIRICHLET, 33),
                                              ((16, 64), PERIODIC, 1)])
def test_equal_weight_box_shared_sums(st, shape, boundary, T):
    """Equal box weights take the shared partial-sum form (a different
    rounding order): checked against the oracle only."""
    w = synth.box_weights(2, 1.0 / 9.0)
    u0 = synth.uniform(10, shape)
    got = gpu_run(st, u0, w, 1, boundary, T, Tb=1, variant=st.VARIANT_STREAM)
    assert normwise_rel(got, oracle.run(u0, w, 1, boundary, T, nthreads=0)) <= TOL


@pytest.mark.parametrize("shape,boundary,T", [((256, 256), DIRICHLET, 100), ((37, 53), DIRICHLET, 17),
                                              ((48, 64), PERIODIC, 9), ((1, 1), PERIODIC, 2)])
def test_persistent_single_grid_matches_direct_bitwise(st, shape, boundary, T):
    w = weights_for("star_rand", 2, 1, 500)
    u0 = synth.uniform(11, shape)
    a = gpu_run(st, u0, w, 1, boundary, T, Tb=1, variant=st.VARIANT_PERSISTENT)
    b = gpu_run(st, u0, w, 1, boundary, T, Tb=1, variant=st.VARIANT_DIRECT)
    assert np.array_equal(a, b)
    assert normwise_rel(a, oracle.run(u0, w, 1, boundary, T, nthreads=0)) <= TOL


TEMPORAL_CASES = [
    # shape, boundary, kind, Tb, T
    ((20, 40, 128), PERIODIC, "heat", 2, 7),
    ((20, 40, 128), PERIODIC, "box_rand", 4, 9),
    ((17, 37, 70), DIRICHLET, "heat", 4, 8),
    ((17, 37, 70), DIRICHLET, "box_rand", 2, 5),
    ((5, 3, 9), PERIODIC, "box_rand", 4, 6),      # axes shorter than the halo
    ((50, 300), PERIODIC, "heat", 8, 19),
    ((50, 300), DIRICHLET, "box_rand", 4, 12),
    ((33, 61), DIRICHLET, "star_rand", 2, 3),
    ((7, 5), PERIODIC, "box_eq", 8, 16),
    ((11, 37, 70), PERIODIC, "heat", 8, 19),       # 3D Tb = 8: 16 x 16 tiles, ragged edges
    ((9, 20, 33), DIRICHLET, "box_rand", 8, 11),
    ((4, 3, 5), PERIODIC, "heat", 8, 9),           # every axis shorter than the halo
    ((6, 70, 100), DIRICHLET, "heat", 4, 4),       # several 32 x 32 tiles, ragged in y and x
    ((40, 530), DIRICHLET, "star_rand", 8, 8),     # 2D: three 256-cell tiles, ragged
]


@pytest.mark.parametrize("shape,boundary,kind,Tb,T", TEMPORAL_CASES)
def test_temporal_blocking_matches_single_steps_bitwise(st, shape, boundary, kind, Tb, T):
    """Tb fused steps per launch (overlapped tiles, Sec. 4.1's temporal tiling)
    apply the same per-cell FMA chain as single steps: bitwise equal to the
    direct kernel, remainder steps included, and within 1e-12 of the oracle."""
    ndim = len(shape)
    w = weights_for(kind, ndim, 1, 600 + Tb)
    if kind == "box_eq":
        w = synth.box_weights(ndim, 1.0 / 3 ** ndim)
    u0 = synth.normal(12, shape)
    a = gpu_run(st, u0, w, 1, boundary, T, Tb=Tb, variant=st.VARIANT_TEMPORAL)
    b = gpu_run(st, u0, w, 1, boundary, T, Tb=1, variant=st.VARIANT_DIRECT)
    if kind != "box_eq":  # the equal-weight 2D box shares partial sums: another summation order
        assert np.array_equal(a, b)
    assert normwise_rel(a, oracle.run(u0, w, 1, boundary, T, nthreads=0)) <= TOL


EXCHANGE_CASES = [
    # shape, boundary, kind, Tb, T
    ((13, 45, 64), PERIODIC, "heat", 2, 5),
    ((13, 45, 64), PERIODIC, "heat", 4, 9),
    ((13, 45, 64), PERIODIC, "heat", 8, 17),
    ((9, 30, 128), DIRICHLET, "box_rand", 4, 9),
    ((9, 30, 128), PERIODIC, "box_rand", 8, 19),
    ((2, 5, 64), PERIODIC, "box_rand", 8, 16),      # fewer planes than the stage skew
    ((1, 1, 64), DIRICHLET, "heat", 2, 4),          # one row of one plane
    ((20, 33, 192), DIRICHLET, "star_rand", 8, 8),  # one-row tiles, three tile columns
    ((7, 150, 64), PERIODIC, "heat", 4, 4),         # 150 one-row tiles in one column
    ((6, 400, 128), DIRICHLET, "box_rand", 2, 7),   # tiles of 5 and 6 rows
    ((31, 64, 256), PERIODIC, "star_rand", 4, 12),
    # planes taller than 152 co-resident tiles of 32 rows cover: bands of rows,
    # one launch each, with Tb - 1 margin rows toward each neighbouring band
    ((6, 300, 2432), PERIODIC, "heat", 2, 5),        # 38 tile columns: 3 bands, margins wrap
    ((5, 150, 4864), DIRICHLET, "box_rand", 8, 17),  # 76 tile columns: 3 bands of 57-64 rows
    ((4, 40, 9728), PERIODIC, "box_rand", 8, 16),    # one tile row per band, margins of 7 rows
    ((9, 100, 9728), DIRICHLET, "heat", 4, 9),       # 4 bands
    ((12, 70, 4864), PERIODIC, "star_rand", 4, 12),  # 2 bands, each the other's neighbour twice
    ((7, 130, 4864), PERIODIC, "box_rand", 4, 9),    # 3 bands, box halo across the margins
    ((5, 300, 2432), DIRICHLET, "heat", 2, 6),       # 3 bands, one margin row each side
    # nx not a multiple of 64 (Dirichlet): the last tile column is ragged
    ((9, 70, 1000), DIRICHLET, "box_rand", 4, 9),
    ((6, 33, 130), DIRICHLET, "star_rand", 2, 5),    # a last column of two cells
    ((5, 300, 2400), DIRICHLET, "heat", 8, 17),      # ragged and cut into bands
    ((3, 20, 2), DIRICHLET, "box_rand", 2, 4),       # one cell pair wide
]


@pytest.mark.parametrize("shape,boundary,kind,Tb,T", EXCHANGE_CASES)
def test_exchange_kernel_matches_single_steps_bitwise(st, shape, boundary, kind, Tb, T):
    """Tb fused steps with no recomputed halo (tiles hand their intermediate
    levels to each other through L2): the same per-cell FMA chain as single
    steps, so bitwise equal to the direct kernel, remainder steps included,
    and within 1e-12 of the oracle."""
    w = weights_for(kind, 3, 1, 700 + Tb)
    u0 = synth.normal(13, shape)
    a = gpu_run(st, u0, w, 1, boundary, T, Tb=Tb, variant=st.VARIANT_EXCHANGE)
    b = gpu_run(st, u0, w, 1, boundary, T, Tb=1, variant=st.VARIANT_DIRECT)
    assert np.array_equal(a, b)
    assert normwise_rel(a, oracle.run(u0, w, 1, boundary, T, nthreads=0)) <= TOL


def test_exchange_kernel_rejects_shapes_it_cannot_take(st):
    import torch
    for shape, radius, bnd in (((9, 30, 100), 1, PERIODIC), ((40, 128), 1, PERIODIC), ((9, 30, 64), 2, PERIODIC),
                               ((3, 4, 64 * 160), 1, PERIODIC), ((9, 30, 99), 1, DIRICHLET)):
        w = np.zeros((2 * radius + 1,) * len(shape))
        w[(radius,) * len(shape)] = 1.0
        p = st.Plan(shape, radius, w, bnd)
        p.set_tuning(4, st.VARIANT_EXCHANGE)
        g = torch.zeros(shape, dtype=torch.float64, device="cuda")
        with pytest.raises(st.StencilError) as e:
            p.run(g, 4)
        assert e.value.code == st.ERR_UNSUPPORTED
        p.close()


def _random_exchange_cases(n, seed):
    """Seeded shapes for the exchange kernel: nx a multiple of 64 up to 76
    tile columns (so planes of a few hundred rows are cut into bands), any
    ny and nz, either boundary, star or box weights, every Tb."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        nx = 64 * int(rng.choice([1, 3, 8, 19, 38, 76]))
        ny = int(rng.integers(1, 420))
        nz = int(rng.integers(1, 14))
        Tb = int(rng.choice([2, 4, 8]))
        T = int(rng.integers(Tb, 3 * Tb + 2))
        bnd = int(rng.integers(0, 2))
        if bnd == DIRICHLET and rng.integers(0, 2):
            nx -= 2 * int(rng.integers(1, 32))  # a ragged last tile column
        out.append(((nz, ny, nx), bnd, str(rng.choice(["star_rand", "box_rand"])), Tb, T))
    return out


@pytest.mark.parametrize("shape,boundary,kind,Tb,T", _random_exchange_cases(20, 2303))
def test_exchange_kernel_random_shapes_bitwise(st, shape, boundary, kind, Tb, T):
    """Random shapes (bands included where the plane is taller than the
    co-resident tiles cover): bitwise equal to single direct steps."""
    w = weights_for(kind, 3, 1, 800 + Tb)
    u0 = synth.normal(29, shape)
    a = gpu_run(st, u0, w, 1, boundary, T, Tb=Tb, variant=st.VARIANT_EXCHANGE)
    b = gpu_run(st, u0, w, 1, boundary, T, Tb=1, variant=st.VARIANT_DIRECT)
    assert np.array_equal(a, b)


@pytest.mark.slow
@pytest.mark.parametrize("boundary", [PERIODIC, DIRICHLET])
def test_exchange_bands_at_the_1024_plane(st, boundary):
    """Table 1's 3D plane (1024 x 1024) on fewer planes: four bands per
    Tb-block.  Bitwise equal to single direct steps over the whole grid, and
    oracle windows at band edges (rows 253-259 straddle the first interior
    edge at Tb = 4) and at the grid's corners."""
    import torch
    shape = (24, 1024, 1024)
    w = weights_for("star_rand", 3, 1, 41)
    u0 = synth.normal(41, shape)
    g = torch.empty(shape, dtype=torch.float64, device="cuda")
    ref = torch.empty_like(g)
    p = st.Plan(shape, 1, w, boundary)
    q = st.Plan(shape, 1, w, boundary)
    q.set_tuning(1, st.VARIANT_DIRECT)
    for Tb in (4, 8):
        T = 2 * Tb + 1
        p.set_tuning(Tb, st.VARIANT_EXCHANGE)
        g.copy_(torch.from_numpy(u0))
        nbands, rows = p.exchange_layout(Tb)
        assert nbands == 4 and rows > 1024                   # four bands, margins computed twice
        l0 = st.stencil_launch_count()
        p.run(g, T)
        assert p.status() == 0
        assert st.stencil_launch_count() - l0 == 2 * nbands + 1  # two blocks of four bands, one single step
        ref.copy_(torch.from_numpy(u0))
        q.run(ref, T)
        assert torch.equal(g, ref), Tb
        for lo, hi in [((0, 248, 0), (3, 264, 70)), ((10, 500, 960), (14, 520, 1024)),
                       ((21, 1016, 0), (24, 1024, 8)), ((0, 0, 1000), (2, 6, 1024))]:
            want = oracle.run_window(u0, w, 1, boundary, T, lo, hi)
            sl = tuple(slice(a, b) for a, b in zip(lo, hi))
            assert normwise_rel(g[sl].cpu().numpy(), want) <= TOL, (Tb, lo, hi)
    p.close()
    q.close()


@pytest.mark.slow
@pytest.mark.parametrize("shape,boundary,kind,seed", FULL_TEMPORAL[:2])
def test_exchange_full_size_windows(st, shape, boundary, kind, seed):
    """The exchange kernel at the benchmark's sizes and launch configuration,
    for Tb = 2, 4, 8: windows against the oracle after two Tb-blocks and a
    remainder step."""
    import torch
    w = weights_for(kind, len(shape), 1, seed)
    u0 = synth.normal(seed, shape) if kind == "box_rand" else synth.uniform(seed, shape)
    g = torch.empty(shape, dtype=torch.float64, device="cuda")
    p = st.Plan(shape, 1, w, boundary)
    for Tb in (2, 4, 8):
        T = 2 * Tb + 1
        p.set_tuning(Tb, st.VARIANT_EXCHANGE)
        g.copy_(torch.from_numpy(u0))
        p.run(g, T)
        assert p.status() == 0
        for lo, hi in window_boxes(shape):
            ref = oracle.run_window(u0, w, 1, boundary, T, lo, hi)
            sl = tuple(slice(a, b) for a, b in zip(lo, hi))
            assert normwise_rel(g[sl].cpu().numpy(), ref) <= TOL, (Tb, lo, hi)
    p.close()


@pytest.mark.parametrize("shape,boundary,Tb,T", [((64, 256), PERIODIC, 2, 9), ((45, 94), DIRICHLET, 4, 13),
                                                ((33, 600), DIRICHLET, 8, 17), ((7, 5), PERIODIC, 8, 16),
                                                ((1, 300), PERIODIC, 4, 8)])
def test_temporal_equal_weight_box_shares_partial_sums(st, shape, boundary, Tb, T):
    """The 2D 9-point box with equal weights in the temporal kernel: column
    sums shared by each pair of cells (12 FP64 instructions per pair instead
    of 18), within 1e-12 of the oracle, ragged segments and remainder steps
    included."""
    w = synth.box_weights(2, 1.0 / 9.0)
    u0 = synth.uniform(15, shape)
    a = gpu_run(st, u0, w, 1, boundary, T, Tb=Tb, variant=st.VARIANT_TEMPORAL)
    assert normwise_rel(a, oracle.run(u0, w, 1, boundary, T, nthreads=0)) <= TOL


def test_temporal_unsupported_tb_is_rejected(st):
    import torch
    w = np.zeros((5, 5, 5))
    w[2, 2, 2] = 1.0
    p = st.Plan((8, 8, 8), 2, w, PERIODIC)
    p.set_tuning(4, st.VARIANT_TEMPORAL)   # 2D/3D temporal blocking covers radius 1
    g = torch.from_numpy(synth.uniform(1, (8, 8, 8))).cuda()
    with pytest.raises(st.StencilError) as ei:
        p.run(g, 8)
    assert ei.value.code == st.ERR_UNSUPPORTED
    p.close()


FIXED_TB_CASES = [
    # shape, radius, boundary, kind, Tb, T, the kernel the library picks
    ((24, 64, 128), 1, PERIODIC, "heat", 4, 9, "exchange"),
    ((10, 20, 70), 1, DIRICHLET, "box_rand", 2, 5, "exchange"),     # a ragged last tile column
    ((10, 20, 70), 1, PERIODIC, "box_rand", 2, 5, "temporal"),      # periodic: nx off the 64-column tiles
    ((96, 96), 1, DIRICHLET, "heat", 8, 19, "persistent"),
    ((600, 520), 1, PERIODIC, "star_rand", 4, 10, "temporal"),
    ((5000,), 2, PERIODIC, "star_rand", 2, 7, "temporal"),
    ((5000,), 1, DIRICHLET, "heat", 1, 3, "direct"),
]


@pytest.mark.parametrize("shape,radius,boundary,kind,Tb,T,want", FIXED_TB_CASES)
def test_fixed_tb_without_variant_runs_a_fused_kernel(st, shape, radius, boundary, kind, Tb, T, want):
    """set_tuning(Tb, 0): the library keeps the Tb and picks the kernel;
    bitwise equal to single direct steps (the same per-cell FMA chain) and
    within the bar of the oracle."""
    import torch
    w = weights_for(kind, len(shape), radius, 900 + Tb)
    u0 = synth.normal(17, shape)
    g = torch.from_numpy(u0.copy()).cuda()
    p = st.Plan(shape, radius, w, boundary)
    p.set_tuning(Tb, 0)
    assert p.get_tuning() == (Tb, {"exchange": st.VARIANT_EXCHANGE, "temporal": st.VARIANT_TEMPORAL,
                                   "persistent": st.VARIANT_PERSISTENT, "direct": st.VARIANT_DIRECT}[want])
    l0 = st.stencil_launch_count()
    p.run(g, T)
    torch.cuda.synchronize()
    assert p.status() == 0
    if Tb > 1 and want != "persistent":
        assert st.stencil_launch_count() - l0 < T     # Tb steps per launch
    a = g.cpu().numpy()
    p.close()
    b = gpu_run(st, u0, w, radius, boundary, T, Tb=1, variant=st.VARIANT_DIRECT)
    assert np.array_equal(a, b)
    assert normwise_rel(a, oracle.run(u0, w, radius, boundary, T, nthreads=0)) <= TOL


def test_fixed_tb_without_a_fused_kernel_is_refused(st):
    """A 2D radius-2 plan has no fused kernel: set_tuning(4, 0) makes the run
    report STENCIL_ERR_UNSUPPORTED instead of dropping the Tb; the automatic
    choice runs again after set_tuning(0, 0)."""
    import torch
    w = weights_for("star_rand", 2, 2, 5)
    u0 = synth.uniform(3, (64, 64))
    g = torch.from_numpy(u0.copy()).cuda()
    p = st.Plan(u0.shape, 2, w, PERIODIC)
    p.set_tuning(4, 0)
    with pytest.raises(st.StencilError) as ei:
        p.run(g, 8)
    assert ei.value.code == st.ERR_UNSUPPORTED
    assert np.array_equal(g.cpu().numpy(), u0)      # nothing ran
    p.set_tuning(0, 0)
    p.run(g, 8)
    assert p.status() == 0
    assert normwise_rel(g.cpu().numpy(), oracle.run(u0, w, 2, PERIODIC, 8, nthreads=0)) <= TOL
    p.close()


def test_autotune_picks_a_candidate_and_keeps_results(st):
    import torch
    shape = (24, 48, 128)
    w = synth.heat_weights(3, 0.1)
    p = st.Plan(shape, 1, w, PERIODIC)
    scratch = torch.from_numpy(synth.uniform(3, shape)).cuda()
    rate = p.autotune(scratch, 4)
    assert rate > 0
    tb, v = p.get_tuning()
    assert (tb, v) in [(1, st.VARIANT_DIRECT), (1, st.VARIANT_STREAM), (2, st.VARIANT_TEMPORAL),
                       (4, st.VARIANT_TEMPORAL), (8, st.VARIANT_TEMPORAL), (2, st.VARIANT_EXCHANGE),
                       (4, st.VARIANT_EXCHANGE), (8, st.VARIANT_EXCHANGE)]
    u0 = synth.uniform(4, shape)
    g = torch.from_numpy(u0.copy()).cuda()
    p.run(g, 10)
    assert normwise_rel(g.cpu().numpy(), oracle.run(u0, w, 1, PERIODIC, 10, nthreads=0)) <= TOL
    p.close()


@pytest.mark.parametrize("shape,boundary,kind,Tb,T", [((256, 256), DIRICHLET, "heat", 8, 100),
                                                      ((256, 256), PERIODIC, "heat", 4, 37),
                                                      ((37, 53), DIRICHLET, "star_rand", 4, 17),
                                                      ((48, 64), PERIODIC, "box_rand", 8, 21),
                                                      ((5, 3), PERIODIC, "heat", 8, 9),
                                                      ((300, 257), DIRICHLET, "box_eq", 2, 7),
                                                      ((1024, 1024), DIRICHLET, "star_rand", 4, 13),
                                                      ((1030, 998), PERIODIC, "box_rand", 2, 9),
                                                      ((1, 700), PERIODIC, "star_rand", 8, 24),
                                                      ((700, 2), DIRICHLET, "box_rand", 4, 11),
                                                      ((2, 2), DIRICHLET, "heat", 2, 5)])
def test_persistent_temporal_matches_single_steps_bitwise(st, shape, boundary, kind, Tb, T):
    """Tb steps in shared memory per exchange, tiles synchronised by per-tile
    flags: bitwise equal to single steps (same per-cell chain), remainder
    blocks, odd block counts (result copied back), several tiles per CTA and
    halos that reach past the nearest tile included."""
    w = weights_for(kind, 2, 1, 700 + Tb) if kind != "box_eq" else synth.box_weights(2, 1.0 / 9.0)
    u0 = synth.uniform(13, shape)
    a = gpu_run(st, u0, w, 1, boundary, T, Tb=Tb, variant=st.VARIANT_PERSISTENT)
    b = gpu_run(st, u0, w, 1, boundary, T, Tb=1, variant=st.VARIANT_DIRECT)
    assert np.array_equal(a, b)
    assert normwise_rel(a, oracle.run(u0, w, 1, boundary, T, nthreads=0)) <= TOL


@pytest.mark.parametrize("shape,boundary,kind", [((32, 128), PERIODIC, "star_rand"), ((32, 128), PERIODIC, "box_rand"),
                                                 ((37, 70), DIRICHLET, "star_rand"), ((37, 70), DIRICHLET, "box_rand"),
                                                 ((130, 64), DIRICHLET, "box_rand"), ((3, 4), DIRICHLET, "star_rand")])
def test_stream2d_radius2_matches_direct_bitwise_and_oracle(st, shape, boundary, kind):
    """Table 1's Star-2D9P and Box-2D25P shapes (radius 2) in the streaming
    kernel: bitwise equal to the direct kernel, within 1e-12 of the oracle."""
    w = weights_for(kind, 2, 2, 800)
    u0 = synth.normal(14, shape)
    T = 6
    a = gpu_run(st, u0, w, 2, boundary, T, Tb=1, variant=st.VARIANT_STREAM)
    b = gpu_run(st, u0, w, 2, boundary, T, Tb=1, variant=st.VARIANT_DIRECT)
    assert np.array_equal(a, b)
    assert normwise_rel(a, oracle.run(u0, w, 2, boundary, T, nthreads=0)) <= TOL


@pytest.mark.parametrize("n,radius,boundary,Tb,T", [(10000, 1, PERIODIC, 8, 29), (10000, 2, DIRICHLET, 8, 21),
                                                    (4097, 1, DIRICHLET, 4, 10), (5, 2, PERIODIC, 8, 17),
                                                    (2048, 2, PERIODIC, 2, 5)])
def test_temporal_1d_matches_direct_bitwise_and_oracle(st, n, radius, boundary, Tb, T):
    """Table 1's Heat-1D / Star-1D5P shapes: Tb steps per launch in shared
    memory, bitwise equal to single steps, within 1e-12 of the oracle."""
    w = synth.uniform(900 + radius, (2 * radius + 1,))
    w = w / w.sum()
    u0 = synth.normal(15, (n,))
    a = gpu_run(st, u0, w, radius, boundary, T, Tb=Tb, variant=st.VARIANT_TEMPORAL)
    b = gpu_run(st, u0, w, radius, boundary, T, Tb=1, variant=st.VARIANT_DIRECT)
    assert np.array_equal(a, b)
    assert normwise_rel(a, oracle.run(u0, w, radius, boundary, T, nthreads=0)) <= TOL


def test_fp32_twin_is_single_precision_and_close(st):
    """The FP32 twin (accuracy studies only) follows the same stencil: within
    float rounding of the oracle, and measurably less exact than FP64."""
    import torch
    shape = (96, 128)
    w = synth.heat_weights(2, 0.23)
    u0 = synth.gaussian_plate(shape, 100.0, 12.0)
    ref = oracle.run(u0, w, 1, DIRICHLET, 50, nthreads=0)
    p = st.Plan(shape, 1, w, DIRICHLET)
    g32 = torch.from_numpy(u0.astype(np.float32)).cuda()
    st.stencil_run_f32(p.handle, g32, torch.empty_like(g32), 50)
    got = g32.cpu().numpy().astype(np.float64)
    err = normwise_rel(got, ref)
    assert 1e-9 < err <= 1e-5
    p.close()


def test_tuning_record_is_shared_by_plans_with_the_same_key(st):
    import torch
    shape = (24, 64, 128)
    w = synth.heat_weights(3, 0.1)
    a = st.Plan(shape, 1, w, PERIODIC)
    a.autotune(torch.from_numpy(synth.uniform(3, shape)).cuda(), 3)
    b = st.Plan(shape, 1, w, PERIODIC)
    assert b.get_tuning() == a.get_tuning()
    a.close()
    b.close()


def test_tma_mbarrier_wait_reports_timeout_and_context_survives(st):
    """Failure detection without a GPU fault, for the TMA-fed streaming kernel:
    its producer posts no copy for one plane, so the consumers' mbarrier waits
    give up after their 20 ms limit with STENCIL_ERR_TIMEOUT, and the next
    sweep on the same kernel matches the oracle."""
    import time
    import torch
    t0 = time.perf_counter()
    assert st.stencil_selftest_tma_timeout(20.0) == st.ERR_TIMEOUT
    assert time.perf_counter() - t0 < 5.0
    shape = (8, 32, 128)
    u0 = synth.uniform(33, shape)
    w = synth.heat_weights(3, 0.1)
    g = torch.from_numpy(u0.copy()).cuda()
    p = st.Plan(shape, 1, w, PERIODIC)
    p.set_tuning(1, st.VARIANT_STREAM)
    p.run(g, 5)
    assert p.status() == 0
    assert normwise_rel(g.cpu().numpy(), oracle.run(u0, w, 1, PERIODIC, 5)) <= TOL
    p.close()


@pytest.mark.parametrize("shape,boundary,kind", [((10, 64, 128), PERIODIC, "heat"), ((9, 64, 192), PERIODIC, "box_rand"),
                                                 ((7, 37, 70), DIRICHLET, "heat"), ((7, 37, 70), DIRICHLET, "box_rand")])
def test_every_stream_tile_height_matches_direct_bitwise(st, shape, boundary, kind):
    """The 3D streaming kernel's tile heights (the tuning dimension the
    autotuner searches): each is bitwise equal to the direct kernel and
    within 1e-12 of the oracle."""
    import torch
    w = weights_for(kind, 3, 1, 800)
    u0 = synth.normal(14, shape)
    ref = gpu_run(st, u0, w, 1, boundary, 5, Tb=1, variant=st.VARIANT_DIRECT)
    assert normwise_rel(ref, oracle.run(u0, w, 1, boundary, 5, nthreads=0)) <= TOL
    for ty in (8, 16, 32):
        g = torch.from_numpy(u0.copy()).cuda()
        p = st.Plan(shape, 1, w, boundary)
        p.set_tuning(1, st.VARIANT_STREAM)
        p.set_tile(64, ty)
        assert p.get_tile() == (64, ty)
        p.run(g, 5)
        assert p.status() == 0
        assert np.array_equal(g.cpu().numpy(), ref), ty
        p.close()


def test_autotune_records_the_tile(st, tmp_path):
    import torch
    shape = (12, 64, 128)
    w = weights_for("box_rand", 3, 1, 801)
    p = st.Plan(shape, 1, w, PERIODIC)
    scratch = torch.from_numpy(synth.uniform(5, shape)).cuda()
    p.autotune(scratch, 2)
    tb, v = p.get_tuning()
    tx, ty = p.get_tile()
    if v == st.VARIANT_STREAM:
        assert tx == 64 and ty in (8, 16, 32)
    else:
        assert (tx, ty) == (0, 0)
    u0 = synth.uniform(6, shape)
    g = torch.from_numpy(u0.copy()).cuda()
    p.run(g, 6)
    assert normwise_rel(g.cpu().numpy(), oracle.run(u0, w, 1, PERIODIC, 6, nthreads=0)) <= TOL
    p.close()
