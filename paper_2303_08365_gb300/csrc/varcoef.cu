// varcoef.cu -- variable-coefficient diffusion sweep and its adjoint.
//
// Forward step (explicit step of du/dt = div(kappa grad u), the heat equation
// of the paper's Eq. 1 with a per-cell diffusivity; arithmetic-mean face
// diffusivity):
//   u'_i = u_i + dt * sum_{faces n} kf_in * (u_n - u_i),  kf_in = (kappa_i + kappa_n)/2
// rewritten with coefficients prepared once per run (kappa and dt are fixed
// for a whole sweep):
//   u'_i = c0_i * u_i + sum_{faces n} c_in * u_n,  c_in = dt * kf_in,
//   c0_i = 1 - dt * sum_{faces n} kf_in
// which costs one multiply and 2*ndim FMAs per cell.  Dirichlet zero: a ghost
// neighbour has u_n = 0 and kf = kappa_i (it only enters c0_i).
//
// Adjoint: A(kappa) is symmetric (c_in = c_ni), so lambda^t = A^T lambda^{t+1}
// is the same gather as the forward step.  The kappa-gradient is accumulated
// per face, each face once: for a face f = (i, n)
//   G_f += (u_n - u_i) * (lambda_i - lambda_n)     (u = u^t, lambda = lambda^{t+1})
// and at the end dL/dkappa_i = (dt/2) * sum_{faces f of i} G_f + dt * Gg_i,
// Gg_i collecting -u_i * lambda_i once per ghost face of cell i.
#include "internal.h"
#include "taps.cuh"

namespace gbst {
namespace {

struct Nbr {
  int64_t idx;  // linear index of the neighbour (valid when in == true)
  bool in;      // false: ghost cell outside the grid (Dirichlet)
};

__device__ __forceinline__ Nbr nbr(int c, int n, int step, bool periodic, int64_t base,
                                   int64_t stride) {
  int m = c + step;
  Nbr r;
  if (periodic) {
    m = m < 0 ? m + n : (m >= n ? m - n : m);
    r.in = true;
  } else {
    r.in = (unsigned)m < (unsigned)n;
  }
  r.idx = base + (int64_t)(m - c) * stride;
  return r;
}

// One thread per cell; (x, y) from the block, z from blockIdx.z.
#define CELL_COORDS                                           \
  const int x = blockIdx.x * blockDim.x + threadIdx.x;        \
  const int y = blockIdx.y * blockDim.y + threadIdx.y;        \
  const int z = blockIdx.z;                                   \
  if (x >= nx || y >= ny) return;                             \
  const int64_t sy = nx, sz = (int64_t)nx * ny;               \
  const int64_t i = (int64_t)z * sz + (int64_t)y * sy + x;

template <int NDIM>
__global__ void __launch_bounds__(256) k_prepare(const double* __restrict__ kappa, double dt,
                                                 bool periodic, int nz, int ny, int nx,
                                                 double* __restrict__ c0, double* __restrict__ cx,
                                                 double* __restrict__ cy,
                                                 double* __restrict__ cz) {
  CELL_COORDS
  const double ki = kappa[i];
  double sum = 0.0;  // sum of the face diffusivities of cell i
  double face_plus[3] = {0.0, 0.0, 0.0};
  const int cs[3] = {x, y, z};
  const int ns[3] = {nx, ny, nz};
  const int64_t st[3] = {1, sy, sz};
#pragma unroll
  for (int d = 0; d < NDIM; ++d) {
#pragma unroll
    for (int s = -1; s <= 1; s += 2) {
      Nbr q = nbr(cs[d], ns[d], s, periodic, i, st[d]);
      double kf = q.in ? 0.5 * (ki + kappa[q.idx]) : ki;
      sum += kf;
      if (s > 0) face_plus[d] = q.in ? dt * kf : 0.0;
    }
  }
  c0[i] = 1.0 - dt * sum;
  cx[i] = face_plus[0];
  if (NDIM >= 2) cy[i] = face_plus[1];
  if (NDIM >= 3) cz[i] = face_plus[2];
}

// u'_i = c0_i u_i + sum over faces of c_f u_n (the -face of cell i is the
// +face of its lower neighbour, whose coefficient array entry is read).
template <int NDIM>
__device__ __forceinline__ double apply_a(const double* __restrict__ u, const double* __restrict__ c0,
                                          const double* __restrict__ cx, const double* __restrict__ cy,
                                          const double* __restrict__ cz, bool periodic, int x, int y,
                                          int z, int nx, int ny, int nz, int64_t i, int64_t sy,
                                          int64_t sz, double zero) {
  double acc = fma(__ldg(c0 + i), __ldg(u + i), zero);
  const int cs[3] = {x, y, z};
  const int ns[3] = {nx, ny, nz};
  const int64_t st[3] = {1, sy, sz};
  const double* cf[3] = {cx, cy, cz};
#pragma unroll
  for (int d = 0; d < NDIM; ++d) {
    Nbr lo = nbr(cs[d], ns[d], -1, periodic, i, st[d]);
    Nbr hi = nbr(cs[d], ns[d], +1, periodic, i, st[d]);
    if (lo.in) acc = fma(__ldg(cf[d] + lo.idx), __ldg(u + lo.idx), acc);
    if (hi.in) acc = fma(__ldg(cf[d] + i), __ldg(u + hi.idx), acc);
  }
  return acc;
}

// Two cells per thread, (x, y0) and (x, y0 + 1): the pair shares the two
// centre values and the coefficient of the face between them, and a thread
// carries two independent FMA chains.  Each cell's chain is the same as in
// apply_a (centre, then -/+ x, -/+ y, -/+ z), so results are bitwise equal.
#define PAIR_COORDS                                                     \
  const int x = blockIdx.x * blockDim.x + threadIdx.x;                  \
  const int y = 2 * (blockIdx.y * blockDim.y + threadIdx.y);            \
  const int z = blockIdx.z;                                             \
  if (x >= nx || y >= ny) return;                                       \
  const bool has1 = y + 1 < ny;                                         \
  const int64_t sy = nx, sz = (int64_t)nx * ny;                         \
  const int64_t i = (int64_t)z * sz + (int64_t)y * sy + x;              \
  const int64_t i1 = i + sy;

template <int NDIM>
__device__ __forceinline__ void apply_a_pair(const double* __restrict__ u, const double* __restrict__ c0,
                                             const double* __restrict__ cx, const double* __restrict__ cy,
                                             const double* __restrict__ cz, bool periodic, int x, int y,
                                             int z, int nx, int ny, int nz, int64_t i, int64_t i1,
                                             int64_t sy, int64_t sz, bool has1, double zero, double u0,
                                             double u1, double& a0, double& a1) {
  a0 = fma(__ldg(c0 + i), u0, zero);
  if (has1) a1 = fma(__ldg(c0 + i1), u1, zero);
  {  // x
    Nbr lo = nbr(x, nx, -1, periodic, i, 1);
    Nbr hi = nbr(x, nx, +1, periodic, i, 1);
    if (lo.in) a0 = fma(__ldg(cx + lo.idx), __ldg(u + lo.idx), a0);
    if (hi.in) a0 = fma(__ldg(cx + i), __ldg(u + hi.idx), a0);
    if (has1) {
      if (lo.in) a1 = fma(__ldg(cx + lo.idx + sy), __ldg(u + lo.idx + sy), a1);
      if (hi.in) a1 = fma(__ldg(cx + i1), __ldg(u + hi.idx + sy), a1);
    }
  }
  if (NDIM >= 2) {  // y: the face between the two cells is cy[i]
    Nbr lo = nbr(y, ny, -1, periodic, i, sy);
    if (lo.in) a0 = fma(__ldg(cy + lo.idx), __ldg(u + lo.idx), a0);
    const double cyi = __ldg(cy + i);
    if (has1) {
      a0 = fma(cyi, u1, a0);
      a1 = fma(cyi, u0, a1);
      Nbr hi1 = nbr(y + 1, ny, +1, periodic, i1, sy);
      if (hi1.in) a1 = fma(__ldg(cy + i1), __ldg(u + hi1.idx), a1);
    } else {
      Nbr hi = nbr(y, ny, +1, periodic, i, sy);
      if (hi.in) a0 = fma(cyi, __ldg(u + hi.idx), a0);
    }
  }
  if (NDIM >= 3) {  // z
    Nbr lo = nbr(z, nz, -1, periodic, i, sz);
    Nbr hi = nbr(z, nz, +1, periodic, i, sz);
    if (lo.in) a0 = fma(__ldg(cz + lo.idx), __ldg(u + lo.idx), a0);
    if (hi.in) a0 = fma(__ldg(cz + i), __ldg(u + hi.idx), a0);
    if (has1) {
      if (lo.in) a1 = fma(__ldg(cz + lo.idx + sy), __ldg(u + lo.idx + sy), a1);
      if (hi.in) a1 = fma(__ldg(cz + i1), __ldg(u + hi.idx + sy), a1);
    }
  }
}

template <int NDIM>
__global__ void __launch_bounds__(256) k_step(const double* __restrict__ src, double* __restrict__ dst,
                                              const double* __restrict__ c0, const double* __restrict__ cx,
                                              const double* __restrict__ cy, const double* __restrict__ cz,
                                              bool periodic, int nz, int ny, int nx,
                                              const double* __restrict__ zp) {
  PAIR_COORDS
  const double u0 = __ldg(src + i), u1 = has1 ? __ldg(src + i1) : 0.0;
  double a0, a1 = 0.0;
  apply_a_pair<NDIM>(src, c0, cx, cy, cz, periodic, x, y, z, nx, ny, nz, i, i1, sy, sz, has1, __ldg(zp), u0,
                     u1, a0, a1);
  dst[i] = a0;
  if (has1) dst[i1] = a1;
}

template <int NDIM>
__global__ void __launch_bounds__(256) k_adjoint(const double* __restrict__ lam,
                                                 const double* __restrict__ u,
                                                 double* __restrict__ lam_out,
                                                 const double* __restrict__ c0,
                                                 const double* __restrict__ cx,
                                                 const double* __restrict__ cy,
                                                 const double* __restrict__ cz, double* __restrict__ gx,
                                                 double* __restrict__ gy, double* __restrict__ gz,
                                                 double* __restrict__ gg, bool periodic, int nz,
                                                 int ny, int nx, const double* __restrict__ zp) {
  PAIR_COORDS
  const double l0 = __ldg(lam + i), l1 = has1 ? __ldg(lam + i1) : 0.0;
  double a0, a1 = 0.0;
  apply_a_pair<NDIM>(lam, c0, cx, cy, cz, periodic, x, y, z, nx, ny, nz, i, i1, sy, sz, has1, __ldg(zp), l0,
                     l1, a0, a1);
  lam_out[i] = a0;
  if (has1) lam_out[i1] = a1;
  // differences as fma(a, 1, -b): the rounding of a - b at the FMA's full rate
  const double one = __ldg(zp + kZeroSlots);
  const double u0 = __ldg(u + i), u1 = has1 ? __ldg(u + i1) : 0.0;
  double* g[3] = {gx, gy, gz};
  const int ns[3] = {nx, ny, nz};
  const int64_t st[3] = {1, sy, sz};
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    if (c == 1 && !has1) break;
    const int64_t ic = c ? i1 : i;
    const double ui = c ? u1 : u0, li = c ? l1 : l0;
    const int cs[3] = {x, y + c, z};
    int ghosts = 0;
#pragma unroll
    for (int d = 0; d < NDIM; ++d) {
      double un, ln;
      bool in;
      if (d == 1 && c == 0 && has1) {  // the face between the pair: both centres at hand
        un = u1;
        ln = l1;
        in = true;
      } else {
        Nbr hi = nbr(cs[d], ns[d], +1, periodic, ic, st[d]);
        in = hi.in;
        un = in ? __ldg(u + hi.idx) : 0.0;
        ln = in ? __ldg(lam + hi.idx) : 0.0;
      }
      if (in) {
        const double du = fma(un, one, -ui);
        const double dl = fma(li, one, -ln);
        g[d][ic] = fma(du, dl, g[d][ic]);
      } else {
        ++ghosts;
      }
      if (!periodic && cs[d] == 0) ++ghosts;
    }
    if (ghosts) gg[ic] = fma(-(double)ghosts * ui, li, gg[ic]);
  }
}

template <int NDIM>
__global__ void __launch_bounds__(256) k_finalize(const double* __restrict__ gx,
                                                  const double* __restrict__ gy,
                                                  const double* __restrict__ gz,
                                                  const double* __restrict__ gg, double half_dt,
                                                  double dt, bool periodic, int nz, int ny, int nx,
                                                  double* __restrict__ grad) {
  CELL_COORDS
  const int cs[3] = {x, y, z};
  const int ns[3] = {nx, ny, nz};
  const int64_t st[3] = {1, sy, sz};
  const double* g[3] = {gx, gy, gz};
  double s = 0.0;
#pragma unroll
  for (int d = 0; d < NDIM; ++d) {
    Nbr lo = nbr(cs[d], ns[d], -1, periodic, i, st[d]);
    Nbr hi = nbr(cs[d], ns[d], +1, periodic, i, st[d]);
    if (hi.in) s += g[d][i];
    if (lo.in) s += g[d][lo.idx];
  }
  double r = half_dt * s;
  if (!periodic) r = fma(dt, gg[i], r);
  grad[i] = r;
}

constexpr int kLossThreads = 256;

// lam = u - target; block b reduces 0.5*r^2 over a fixed strided subset in a
// fixed tree order (deterministic for a given launch shape).
__global__ void __launch_bounds__(kLossThreads) k_residual(int64_t n, const double* __restrict__ u,
                                                           const double* __restrict__ target,
                                                           double* __restrict__ lam,
                                                           double* __restrict__ partials) {
  __shared__ double red[kLossThreads];
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * kLossThreads + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * kLossThreads) {
    const double r = u[i] - target[i];
    lam[i] = r;
    s = fma(0.5 * r, r, s);
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = kLossThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[blockIdx.x] = red[0];
}

__global__ void __launch_bounds__(kLossThreads) k_sum_partials(const double* __restrict__ partials,
                                                               int n, double* __restrict__ out) {
  __shared__ double red[kLossThreads];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += kLossThreads) s += partials[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = kLossThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

void cell_launch_shape(const Geom& g, dim3& grid, dim3& block) {
  block = dim3(32, 8, 1);
  grid = dim3((g.nx + 31) / 32, (g.ny + 7) / 8, g.nz);
}

// Launch shape of the two-cells-per-thread kernels (k_step, k_adjoint).
void pair_launch_shape(const Geom& g, dim3& grid, dim3& block) {
  block = dim3(32, 8, 1);
  grid = dim3((g.nx + 31) / 32, (g.ny + 15) / 16, g.nz);
}

}  // namespace

cudaError_t launch_varcoef_prepare(int ndim, int boundary, const Geom& g, const double* kappa,
                                   double dt, VarcoefBufs b, cudaStream_t stream) {
  dim3 grid, block;
  cell_launch_shape(g, grid, block);
  bool per = boundary == kPeriodic;
  if (ndim == 3)
    k_prepare<3><<<grid, block, 0, stream>>>(kappa, dt, per, g.nz, g.ny, g.nx, b.c0, b.cx, b.cy, b.cz);
  else if (ndim == 2)
    k_prepare<2><<<grid, block, 0, stream>>>(kappa, dt, per, g.nz, g.ny, g.nx, b.c0, b.cx, b.cy, b.cz);
  else
    k_prepare<1><<<grid, block, 0, stream>>>(kappa, dt, per, g.nz, g.ny, g.nx, b.c0, b.cx, b.cy, b.cz);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

cudaError_t launch_varcoef_step(int ndim, int boundary, const Geom& g, VarcoefBufs b,
                                const double* src, double* dst, const double* zero,
                                cudaStream_t stream) {
  dim3 grid, block;
  pair_launch_shape(g, grid, block);
  bool per = boundary == kPeriodic;
  if (ndim == 3)
    k_step<3><<<grid, block, 0, stream>>>(src, dst, b.c0, b.cx, b.cy, b.cz, per, g.nz, g.ny, g.nx, zero);
  else if (ndim == 2)
    k_step<2><<<grid, block, 0, stream>>>(src, dst, b.c0, b.cx, b.cy, b.cz, per, g.nz, g.ny, g.nx, zero);
  else
    k_step<1><<<grid, block, 0, stream>>>(src, dst, b.c0, b.cx, b.cy, b.cz, per, g.nz, g.ny, g.nx, zero);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

cudaError_t launch_adjoint_step(int ndim, int boundary, const Geom& g, VarcoefBufs b,
                                const double* lam_in, const double* u, double* lam_out,
                                double* gx, double* gy, double* gz, double* gg, const double* zero,
                                cudaStream_t stream) {
  dim3 grid, block;
  pair_launch_shape(g, grid, block);
  bool per = boundary == kPeriodic;
  if (ndim == 3)
    k_adjoint<3><<<grid, block, 0, stream>>>(lam_in, u, lam_out, b.c0, b.cx, b.cy, b.cz, gx, gy, gz,
                                             gg, per, g.nz, g.ny, g.nx, zero);
  else if (ndim == 2)
    k_adjoint<2><<<grid, block, 0, stream>>>(lam_in, u, lam_out, b.c0, b.cx, b.cy, b.cz, gx, gy, gz,
                                             gg, per, g.nz, g.ny, g.nx, zero);
  else
    k_adjoint<1><<<grid, block, 0, stream>>>(lam_in, u, lam_out, b.c0, b.cx, b.cy, b.cz, gx, gy, gz,
                                             gg, per, g.nz, g.ny, g.nx, zero);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

cudaError_t launch_adjoint_finalize(int ndim, int boundary, const Geom& g, double dt,
                                    const double* gx, const double* gy, const double* gz,
                                    const double* gg, double* grad_kappa, cudaStream_t stream) {
  dim3 grid, block;
  cell_launch_shape(g, grid, block);
  bool per = boundary == kPeriodic;
  if (ndim == 3)
    k_finalize<3><<<grid, block, 0, stream>>>(gx, gy, gz, gg, 0.5 * dt, dt, per, g.nz, g.ny, g.nx,
                                              grad_kappa);
  else if (ndim == 2)
    k_finalize<2><<<grid, block, 0, stream>>>(gx, gy, gz, gg, 0.5 * dt, dt, per, g.nz, g.ny, g.nx,
                                              grad_kappa);
  else
    k_finalize<1><<<grid, block, 0, stream>>>(gx, gy, gz, gg, 0.5 * dt, dt, per, g.nz, g.ny, g.nx,
                                              grad_kappa);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

cudaError_t launch_loss_residual(int64_t n, const double* u, const double* target, double* lam,
                                 double* partials, int nblocks, double* loss_out,
                                 cudaStream_t stream) {
  k_residual<<<nblocks, kLossThreads, 0, stream>>>(n, u, target, lam, partials);
  k_sum_partials<<<1, kLossThreads, 0, stream>>>(partials, nblocks, loss_out);
  g_launches.fetch_add(2, std::memory_order_relaxed);
  return cudaGetLastError();
}

}  // namespace gbst
