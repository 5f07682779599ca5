// direct.cu -- the plain one-step sweep: every thread owns one (y, x) column
// of a tile and walks a chunk of planes along z, summing its taps straight
// from global memory (the L1 cache serves the neighbour reuse).  It handles
// every shape, radius and boundary and is the reference point that the
// streaming and temporal-blocking kernels are measured against.
//
// Operation: one step of u'(x) = sum_o w_o u~(x+o) (paper Sec. 2.1, Listing 1).
#include "internal.h"
#include "taps.cuh"

namespace gbst {
namespace {

// Index of a neighbour along one axis under each boundary mode.
//   MODE 0: Dirichlet zero -- returns false when outside [0, n)
//   MODE 1: periodic, |offset| <= n -- one conditional add or subtract
//   MODE 2: periodic, any offset -- true modulo (axes shorter than the radius)
template <int MODE>
__device__ __forceinline__ bool axis_index(int c, int n, int& out) {
  if (MODE == 0) {
    out = c;
    return (unsigned)c < (unsigned)n;
  } else if (MODE == 1) {
    out = c < 0 ? c + n : (c >= n ? c - n : c);
    return true;
  } else {
    int m = c % n;
    out = m < 0 ? m + n : m;
    return true;
  }
}

template <int NT, int MODE>
__global__ void __launch_bounds__(256) k_direct(const double* __restrict__ src,
                                                double* __restrict__ dst, int nz, int ny, int nx,
                                                int zper, const __grid_constant__ TapList<NT> tp,
                                                const double* __restrict__ wdev) {
  // up to 27 taps the weights live in registers (full FP64 rate); the
  // 125-tap radius-2 box keeps them in the constant bank instead of spilling
  constexpr bool kRegs = NT <= 27;
  RegWeights<kRegs ? NT : 1> W;
  if (kRegs) W.load(wdev);
  const double zero = kRegs ? W.z[0] : 0.0;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= nx || y >= ny) return;
  const int z0 = blockIdx.z * zper;
  const int z1 = min(nz, z0 + zper);
  for (int z = z0; z < z1; ++z) {
    double acc = 0.0;
#pragma unroll
    for (int k = 0; k < NT; ++k) {
      int zz, yy, xx;
      bool in = axis_index<MODE>(z + tp.dz[k], nz, zz);
      in &= axis_index<MODE>(y + tp.dy[k], ny, yy);
      in &= axis_index<MODE>(x + tp.dx[k], nx, xx);
      double v = 0.0;
      if (in) v = __ldg(src + ((int64_t)zz * ny + yy) * nx + xx);
      if constexpr (kRegs)
        W.tap(acc, k, v, 0);
      else
        acc = fma(tp.w[k], v, k == 0 ? zero : acc);
    }
    dst[((int64_t)z * ny + y) * nx + x] = acc;
  }
}

// FP32 twin of the direct sweep, for accuracy studies only (the paper's
// Table 4 compares an FP32 run of its thermal case with FP64): the same tap
// order with the weights rounded to float and float FMAs.
template <int NT, int MODE>
__global__ void __launch_bounds__(256) k_direct_f32(const float* __restrict__ src, float* __restrict__ dst,
                                                    int nz, int ny, int nx, int zper,
                                                    const __grid_constant__ TapList<NT> tp) {
  float w[NT];
#pragma unroll
  for (int k = 0; k < NT; ++k) w[k] = (float)tp.w[k];
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= nx || y >= ny) return;
  const int z0 = blockIdx.z * zper;
  const int z1 = min(nz, z0 + zper);
  for (int z = z0; z < z1; ++z) {
    float acc = 0.0f;
#pragma unroll
    for (int k = 0; k < NT; ++k) {
      int zz, yy, xx;
      bool in = axis_index<MODE>(z + tp.dz[k], nz, zz);
      in &= axis_index<MODE>(y + tp.dy[k], ny, yy);
      in &= axis_index<MODE>(x + tp.dx[k], nx, xx);
      float v = 0.0f;
      if (in) v = __ldg(src + ((int64_t)zz * ny + yy) * nx + xx);
      acc = (k == 0) ? w[0] * v : fmaf(w[k], v, acc);
    }
    dst[((int64_t)z * ny + y) * nx + x] = acc;
  }
}

void direct_shape(const Geom& g, dim3& grid, dim3& block, int& zper) {
  zper = 1;
  if (g.ny == 1 && g.nz == 1) {
    block = dim3(256, 1, 1);
    grid = dim3((g.nx + 255) / 256, 1, 1);
  } else {
    block = dim3(32, 8, 1);
    unsigned gx = (g.nx + 31) / 32, gy = (g.ny + 7) / 8;
    int64_t tiles = (int64_t)gx * gy;
    int64_t want = 152 * 16;
    int64_t zchunks = (want + tiles - 1) / tiles;
    if (zchunks > g.nz) zchunks = g.nz;
    if (zchunks < 1) zchunks = 1;
    zper = (int)((g.nz + zchunks - 1) / zchunks);
    zchunks = (g.nz + zper - 1) / zper;
    grid = dim3(gx, gy, (unsigned)zchunks);
  }
}

template <int NT>
cudaError_t launch_nt_f32(int mode, const Geom& g, const HostTaps& ht, const float* src, float* dst,
                          cudaStream_t stream) {
  TapList<NT> tp;
  for (int k = 0; k < NT; ++k) {
    tp.w[k] = ht.w[k];
    tp.dz[k] = ht.dz[k];
    tp.dy[k] = ht.dy[k];
    tp.dx[k] = ht.dx[k];
  }
  dim3 block, grid;
  int zper;
  direct_shape(g, grid, block, zper);
  switch (mode) {
    case 0: k_direct_f32<NT, 0><<<grid, block, 0, stream>>>(src, dst, g.nz, g.ny, g.nx, zper, tp); break;
    case 1: k_direct_f32<NT, 1><<<grid, block, 0, stream>>>(src, dst, g.nz, g.ny, g.nx, zper, tp); break;
    default: k_direct_f32<NT, 2><<<grid, block, 0, stream>>>(src, dst, g.nz, g.ny, g.nx, zper, tp); break;
  }
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

template <int NT>
cudaError_t launch_nt(int mode, const Geom& g, const HostTaps& ht, const double* wdev,
                      const double* src, double* dst, cudaStream_t stream) {
  TapList<NT> tp;
  for (int k = 0; k < NT; ++k) {
    tp.w[k] = ht.w[k];
    tp.dz[k] = ht.dz[k];
    tp.dy[k] = ht.dy[k];
    tp.dx[k] = ht.dx[k];
  }
  dim3 block, grid;
  int zper = 1;
  if (g.ny == 1 && g.nz == 1) {
    block = dim3(256, 1, 1);
    grid = dim3((g.nx + 255) / 256, 1, 1);
  } else {
    block = dim3(32, 8, 1);
    unsigned gx = (g.nx + 31) / 32, gy = (g.ny + 7) / 8;
    // enough blocks for every SM several times over; the rest of z is walked
    int64_t tiles = (int64_t)gx * gy;
    int64_t want = 152 * 16;
    int64_t zchunks = (want + tiles - 1) / tiles;
    if (zchunks > g.nz) zchunks = g.nz;
    if (zchunks < 1) zchunks = 1;
    zper = (int)((g.nz + zchunks - 1) / zchunks);
    zchunks = (g.nz + zper - 1) / zper;
    grid = dim3(gx, gy, (unsigned)zchunks);
  }
  switch (mode) {
    case 0: k_direct<NT, 0><<<grid, block, 0, stream>>>(src, dst, g.nz, g.ny, g.nx, zper, tp, wdev); break;
    case 1: k_direct<NT, 1><<<grid, block, 0, stream>>>(src, dst, g.nz, g.ny, g.nx, zper, tp, wdev); break;
    default: k_direct<NT, 2><<<grid, block, 0, stream>>>(src, dst, g.nz, g.ny, g.nx, zper, tp, wdev); break;
  }
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_direct(int ndim, int radius, Shape shape, int boundary, const Geom& g,
                          const HostTaps& taps, const double* wdev, const double* src, double* dst,
                          cudaStream_t stream) {
  int mode = 0;
  if (boundary == kPeriodic) {
    bool small = g.nx < radius || (ndim >= 2 && g.ny < radius) || (ndim >= 3 && g.nz < radius);
    mode = small ? 2 : 1;
  }
  switch (taps.n) {
    case 3: return launch_nt<3>(mode, g, taps, wdev, src, dst, stream);
    case 5: return launch_nt<5>(mode, g, taps, wdev, src, dst, stream);
    case 7: return launch_nt<7>(mode, g, taps, wdev, src, dst, stream);
    case 9: return launch_nt<9>(mode, g, taps, wdev, src, dst, stream);
    case 13: return launch_nt<13>(mode, g, taps, wdev, src, dst, stream);
    case 25: return launch_nt<25>(mode, g, taps, wdev, src, dst, stream);
    case 27: return launch_nt<27>(mode, g, taps, wdev, src, dst, stream);
    case 125: return launch_nt<125>(mode, g, taps, wdev, src, dst, stream);
    default: return cudaErrorInvalidValue;
  }
  (void)shape;
}

cudaError_t launch_direct_f32(int ndim, int radius, int boundary, const Geom& g, const HostTaps& taps,
                              const float* src, float* dst, cudaStream_t stream) {
  int mode = 0;
  if (boundary == kPeriodic) {
    bool small = g.nx < radius || (ndim >= 2 && g.ny < radius) || (ndim >= 3 && g.nz < radius);
    mode = small ? 2 : 1;
  }
  switch (taps.n) {
    case 3: return launch_nt_f32<3>(mode, g, taps, src, dst, stream);
    case 5: return launch_nt_f32<5>(mode, g, taps, src, dst, stream);
    case 7: return launch_nt_f32<7>(mode, g, taps, src, dst, stream);
    case 9: return launch_nt_f32<9>(mode, g, taps, src, dst, stream);
    case 13: return launch_nt_f32<13>(mode, g, taps, src, dst, stream);
    case 25: return launch_nt_f32<25>(mode, g, taps, src, dst, stream);
    case 27: return launch_nt_f32<27>(mode, g, taps, src, dst, stream);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace gbst
