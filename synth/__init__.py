"""Seeded synthetic inputs shared by the oracle side and the CUDA side.

This module holds no stencil arithmetic: it only draws random numbers and
lays out workload descriptions, so that the oracle and the CUDA library are
fed the very same bytes.  Nothing here imports the oracle or the library.

Generator: SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014), used counter-style: value i of stream s is
mix(s + (i+1) * 0x9E3779B97F4A7C15), mix being the published finaliser.  A
double in [0,1) takes the top 53 bits.  Normals use Box-Muller on two
consecutive uniforms (1-u1 keeps the log finite).
"""
import math

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
M1 = np.uint64(0xBF58476D1CE4E5B9)
M2 = np.uint64(0x94D049BB133111EB)
_CHUNK = 1 << 22


class _Stream:
    """Counter-based SplitMix64 evaluated chunk by chunk in reusable buffers."""

    def __init__(self, seed):
        self.seed = np.uint64(seed)
        self.z = np.empty(_CHUNK, dtype=np.uint64)
        self.t = np.empty(_CHUNK, dtype=np.uint64)

    def raw(self, start, count):
        z, t = self.z[:count], self.t[:count]
        with np.errstate(over="ignore"):
            z[:] = np.arange(start + 1, start + count + 1, dtype=np.uint64)
            np.multiply(z, GOLDEN, out=z)
            np.add(z, self.seed, out=z)
            np.right_shift(z, np.uint64(30), out=t)
            np.bitwise_xor(z, t, out=z)
            np.multiply(z, M1, out=z)
            np.right_shift(z, np.uint64(27), out=t)
            np.bitwise_xor(z, t, out=z)
            np.multiply(z, M2, out=z)
            np.right_shift(z, np.uint64(31), out=t)
            np.bitwise_xor(z, t, out=z)
        return z

    def unit(self, start, count, out):
        """Doubles in [0,1): the top 53 bits of each raw output."""
        z = self.raw(start, count)
        np.right_shift(z, np.uint64(11), out=z)
        np.multiply(z.view(np.int64), 1, out=out, casting="unsafe")
        np.multiply(out, 1.0 / 9007199254740992.0, out=out)
        return out


def splitmix64(seed, start, count):
    """Raw 64-bit outputs start .. start+count-1 of stream `seed`."""
    out = np.empty(count, dtype=np.uint64)
    st = _Stream(seed)
    for s in range(0, count, _CHUNK):
        c = min(_CHUNK, count - s)
        out[s:s + c] = st.raw(start + s, c)
    return out


def uniform(seed, shape, lo=0.0, hi=1.0):
    """Doubles uniform in [lo, hi) (53-bit resolution), C order."""
    n = int(np.prod(shape))
    out = np.empty(n, dtype=np.float64)
    st = _Stream(seed)
    for s in range(0, n, _CHUNK):
        c = min(_CHUNK, n - s)
        st.unit(s, c, out[s:s + c])
    if lo != 0.0 or hi != 1.0:
        out *= (hi - lo)
        out += lo
    return out.reshape(shape)


def normal(seed, shape):
    """Standard normal doubles, Box-Muller on uniform pairs (2i, 2i+1)."""
    n = int(np.prod(shape))
    out = np.empty(n, dtype=np.float64)
    st = _Stream(seed)
    buf = np.empty(_CHUNK, dtype=np.float64)
    for s in range(0, n, _CHUNK // 2):
        c = min(_CHUNK // 2, n - s)
        u = st.unit(2 * s, 2 * c, buf[:2 * c])
        u1, u2 = u[0::2], u[1::2]
        o = out[s:s + c]
        np.negative(u1, out=o)
        np.log1p(o, out=o)
        o *= -2.0
        np.sqrt(o, out=o)
        o *= np.cos(2.0 * math.pi * u2)
    return out.reshape(shape)


def lognormal(seed, shape, sigma=0.5):
    """exp(sigma * N(0,1))."""
    return np.exp(sigma * normal(seed, shape))


def heat_weights(ndim, alpha):
    """Dense 3^ndim weights of the radius-1 heat stencil (paper Eq. 3):
    1 - 2*ndim*alpha at the centre and alpha at each face neighbour."""
    w = np.zeros((3,) * ndim, dtype=np.float64)
    c = (1,) * ndim
    w[c] = 1.0 - 2 * ndim * alpha
    for d in range(ndim):
        for s in (0, 2):
            idx = list(c)
            idx[d] = s
            w[tuple(idx)] = alpha
    return w


def box_weights(ndim, value=None, seed=None):
    """Dense 3^ndim box weights: all equal to `value` (e.g. 1/9), or drawn
    uniform [0,1) from `seed` and divided by their sum."""
    if seed is None:
        return np.full((3,) * ndim, value, dtype=np.float64)
    v = uniform(seed, (3,) * ndim)
    return v / v.sum()


def sine_mode(shape, k):
    """prod_d sin(2 pi k_d x_d / N_d) on a periodic grid (amplitude 1)."""
    m = np.ones(shape, dtype=np.float64)
    for d, (n, kd) in enumerate(zip(shape, k)):
        x = np.arange(n, dtype=np.float64)
        s = np.sin(2.0 * math.pi * kd * x / n)
        view = [1] * len(shape)
        view[d] = n
        m = m * s.reshape(view)
    return m


def dirichlet_sine_mode(shape, k):
    """prod_d sin(pi k_d (x_d+1) / (N_d+1)): eigenvector of the zero-Dirichlet
    Laplacian stencil on a grid of N_d cells per axis."""
    m = np.ones(shape, dtype=np.float64)
    for d, (n, kd) in enumerate(zip(shape, k)):
        x = np.arange(n, dtype=np.float64)
        s = np.sin(math.pi * kd * (x + 1.0) / (n + 1.0))
        view = [1] * len(shape)
        view[d] = n
        m = m * s.reshape(view)
    return m


def gaussian_plate(shape, peak=100.0, sigma=None):
    """Gaussian temperature field peaked at the plate centre (the initial state
    of the paper's copper-plate case study).  sigma in cells; by default 1376
    cells scaled to the grid: the width for which the free-space solution of
    the heat equation, sigma_T^2 = sigma_0^2 + 2 mu T, brings the centre from
    100 to 52.0 degrees after 3.8e6 steps at mu = 0.23 on a 9600^2 grid."""
    ny, nx = shape
    if sigma is None:
        sigma = 1376.0 * nx / 9600.0
    y = (np.arange(ny, dtype=np.float64) - (ny - 1) / 2.0).reshape(-1, 1)
    x = (np.arange(nx, dtype=np.float64) - (nx - 1) / 2.0).reshape(1, -1)
    return peak * np.exp(-(y * y + x * x) / (2.0 * sigma * sigma))


def batch_items(seed, count=96, side_lo=128, side_hi=4096, alpha_lo=0.05, alpha_hi=0.24,
                t_lo=50, t_hi=500):
    """Descriptors of `count` independent 2D grids: (ny, nx, alpha, T).

    Sides are log-uniform in [side_lo, side_hi] per axis, drawn independently
    (non-square allowed); alpha uniform in [alpha_lo, alpha_hi); T uniform in
    the integers t_lo .. t_hi.
    """
    u = uniform(seed, (count, 4))
    lo, hi = math.log(side_lo), math.log(side_hi)
    items = []
    for i in range(count):
        ny = int(round(math.exp(lo + (hi - lo) * u[i, 0])))
        nx = int(round(math.exp(lo + (hi - lo) * u[i, 1])))
        a = alpha_lo + (alpha_hi - alpha_lo) * u[i, 2]
        T = t_lo + min(int(u[i, 3] * (t_hi - t_lo + 1)), t_hi - t_lo)
        items.append((ny, nx, float(a), int(T)))
    return items


# Seeds: base 2303 plus the workload index.
SEED_HEAT2D = 2303
SEED_HEAT3D = 2304
SEED_BOX2D = 2305
SEED_BOX3D = 2306
SEED_BATCH = 2307
SEED_ADJOINT = 2308
