// temporal.cu -- temporal blocking: Tb time steps per HBM round trip.
//
// The paper stretches its spatial tiles along the time dimension so that a
// tile is read once and updated Tb times before it is written back (Sec. 4.1,
// "Temporal Tiling"; triangles in 2D become tetrahedra in space-time).  This
// kernel does the same with overlapped tiles, streamed along the slowest axis:
//
//   - a CTA owns an output tile of the "plane" orthogonal to the streaming
//     axis (3D: 64 x 16 cells of an (y, x) plane, streamed along z; 2D: 256
//     cells of a row, streamed along y) and loads it with a halo of Tb cells;
//   - stage s = 1 .. Tb holds the tile at time t+s on a region that shrinks by
//     one cell per side per stage (the halo cells are recomputed by the
//     neighbouring tiles: the overlapped-tile redundancy);
//   - along the streaming axis nothing is recomputed: stage s produces plane
//     i - s when input plane i arrives, from its own ring of 3 planes of stage
//     s-1 output, so each input plane is read once from HBM and each output
//     plane written once;
//   - input planes arrive by cp.async (8-byte copies with zero fill for
//     Dirichlet ghosts and wrapped addresses for periodic grids; a periodic
//     halo of width Tb does not fit the TMA box model at the grid edges);
//   - each cell applies its taps in the direct kernel's lexicographic order
//     with register-resident weights, so a Tb-fused sweep is bitwise equal to
//     Tb single steps.
// Dirichlet ghost cells (outside the grid, at every time level) stay zero.
#include "internal.h"
#include "taps.cuh"

namespace gbst {
namespace {

constexpr int kThreads = 256;

// Threads of the 2D/3D temporal kernel: deep blocks (Tb >= 4) take a CTA per
// SM and need 16 warps to keep the FP64 pipe busy (measured: 3D 7-point Tb 4
// 58.6 vs 56.1 GStencil/s, 2D 9-point Tb 8 59.0 vs 54.4); Tb = 2 runs two
// CTAs of 8 warps (77.0 vs 73.7).
template <int TB>
constexpr int temporal_threads() { return TB >= 4 ? 512 : 256; }

template <int NDIM>
struct Geo {
  static constexpr int TX = NDIM == 3 ? 64 : 256;  // output tile width (x)
  static constexpr int TY = NDIM == 3 ? 16 : 1;    // output tile height (y); 2D: the plane is a row
};

template <int NDIM, int TB>
struct PlaneDims {
  static constexpr int PX = Geo<NDIM>::TX + 2 * TB;
  static constexpr int PY = NDIM == 3 ? Geo<NDIM>::TY + 2 * TB : 1;
  static constexpr int P = PX * PY;  // doubles per plane
  static constexpr int kIn = 4;      // input ring slots
  static constexpr int kStageRing = 3;
  static constexpr int planes = kIn + kStageRing * (TB - 1);
  static constexpr size_t bytes = (size_t)planes * P * sizeof(double);
};

struct TParams {
  const double* src;
  double* dst;
  int nw, ny, nx;       // streaming-axis extent (nz in 3D, ny in 2D), grid ny, nx
  int tiles_x, tiles_y;
  long long work;       // tiles * nw
  const double* wdev;
};

__device__ __forceinline__ int wrapn(int c, int n) {
  int m = c % n;
  return m < 0 ? m + n : m;
}

__device__ __forceinline__ void cp_async8(double* dst, const double* src, bool valid) {
  const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
  const int sz = valid ? 8 : 0;  // 0: nothing is read, the 8 bytes are zero-filled
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(src), "r"(sz) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Issues the copies of input plane w (global streaming coordinate) of the tile
// whose output origin is (y0, x0) into `slot`.
template <int NDIM, int TB, bool PERIODIC>
__device__ __forceinline__ void load_plane(double* slot, const TParams& P, int w, int y0, int x0) {
  using D = PlaneDims<NDIM, TB>;
  bool win = true;
  int ww = w;
  if (PERIODIC) ww = wrapn(w, P.nw);
  else win = (unsigned)w < (unsigned)P.nw;
  for (int c = threadIdx.x; c < D::P; c += temporal_threads<TB>()) {
    const int px = c % D::PX, py = c / D::PX;
    int x = x0 - TB + px;
    int y = NDIM == 3 ? y0 - TB + py : 0;
    bool in = win;
    if (PERIODIC) {
      x = wrapn(x, P.nx);
      if (NDIM == 3) y = wrapn(y, P.ny);
    } else {
      in = in && (unsigned)x < (unsigned)P.nx && (NDIM == 2 || (unsigned)y < (unsigned)P.ny);
    }
    int64_t gi;
    if (NDIM == 3) gi = ((int64_t)(in ? ww : 0) * P.ny + (in ? y : 0)) * P.nx + (in ? x : 0);
    else gi = (int64_t)(in ? ww : 0) * P.nx + (in ? x : 0);
    cp_async8(slot + c, P.src + gi, in);
  }
}

// Tap index of (dw, dv, du) in the lexicographic tap list (dw = streaming
// axis offset; 3D: (dz, dy, dx); 2D: (dy, -, dx) with dv = 0).
template <int NDIM, bool BOX>
__device__ __forceinline__ constexpr int tidx(int dw, int dv, int du) {
  if (NDIM == 3) {
    if (BOX) return ((dw + 1) * 3 + (dv + 1)) * 3 + (du + 1);
    return dw < 0 ? 0 : dw > 0 ? 6 : dv < 0 ? 1 : dv > 0 ? 5 : 3 + du;
  }
  if (BOX) return (dw + 1) * 3 + (du + 1);
  return dw < 0 ? 0 : dw > 0 ? 4 : 2 + du;
}

// One cell of a stage: taps over planes (pm, p0, pp) of the previous stage at
// in-plane position (py, px).
template <int NDIM, int NT, bool BOX, int PX>
__device__ __forceinline__ double cell_update(const RegWeights<NT>& W, const double* pm,
                                              const double* p0, const double* pp, int py, int px) {
  const double* pl[3] = {pm, p0, pp};
  double acc = 0.0;
#pragma unroll
  for (int dw = -1; dw <= 1; ++dw) {
#pragma unroll
    for (int dv = -1; dv <= 1; ++dv) {
      if (NDIM == 2 && dv != 0) continue;
#pragma unroll
      for (int du = -1; du <= 1; ++du) {
        const int nz_axes = (dw != 0) + (dv != 0) + (du != 0);
        if (!BOX && nz_axes > 1) continue;
        const double v = pl[dw + 1][(py + dv) * PX + px + du];
        W.tap(acc, tidx<NDIM, BOX>(dw, dv, du), v, 0);
      }
    }
  }
  return acc;
}

template <int NDIM, int NT, bool BOX, bool PERIODIC, int TB>
__global__ void __launch_bounds__(temporal_threads<TB>(), 1) k_temporal(const TParams P) {
  using D = PlaneDims<NDIM, TB>;
  constexpr int PX = D::PX, PY = D::PY;
  constexpr int TX = Geo<NDIM>::TX, TY = Geo<NDIM>::TY;
  extern __shared__ __align__(16) double sm[];
  double* in_ring = sm;                       // kIn planes
  double* st_ring = sm + D::kIn * D::P;       // (TB-1) stages x 3 planes
  RegWeights<NT> W;
  W.load(P.wdev);

  const long long G = gridDim.x;
  const long long f_begin = P.work * blockIdx.x / G;
  const long long f_end = P.work * (blockIdx.x + 1) / G;
  for (long long f = f_begin; f < f_end;) {
    const int tile = (int)(f / P.nw);
    const int wa = (int)(f % P.nw);
    const long long rem = f_end - f;
    const int wb = (long long)P.nw < wa + rem ? P.nw : (int)(wa + rem);
    f += wb - wa;
    const int x0 = (tile % P.tiles_x) * TX;
    const int y0 = (tile / P.tiles_x) * TY;
    const int nin = (wb - wa) + 2 * TB;  // input planes wa-TB .. wb+TB-1
    // prologue: planes 0 and 1 in flight
    load_plane<NDIM, TB, PERIODIC>(in_ring + 0 * D::P, P, wa - TB, y0, x0);
    cp_async_commit();
    load_plane<NDIM, TB, PERIODIC>(in_ring + 1 * D::P, P, wa - TB + 1, y0, x0);
    cp_async_commit();
    for (int k = 0; k < nin; ++k) {
      cp_async_wait<1>();  // plane k has landed (plane k+1 may still be in flight)
      __syncthreads();
#pragma unroll
      for (int s = 1; s <= TB; ++s) {
        const int i = k - s;  // plane index this stage produces now
        if (i < s || i >= nin - s) continue;
        const double *pm, *p0, *pp;
        if (s == 1) {
          pm = in_ring + ((i - 1) & 3) * D::P;
          p0 = in_ring + (i & 3) * D::P;
          pp = in_ring + ((i + 1) & 3) * D::P;
        } else {
          const double* r = st_ring + (s - 2) * 3 * D::P;
          pm = r + ((i - 1) % 3) * D::P;
          p0 = r + (i % 3) * D::P;
          pp = r + ((i + 1) % 3) * D::P;
        }
        const int w = wa - TB + i;  // streaming coordinate of the produced plane
        const bool wghost = !PERIODIC && (unsigned)w >= (unsigned)P.nw;
        const int sy = NDIM == 3 ? s : 0;
        const int cw = PX - 2 * s, ch = PY - 2 * sy;
        if (s < TB) {
          double* out = st_ring + (s - 1) * 3 * D::P + (i % 3) * D::P;
          for (int c = threadIdx.x; c < cw * ch; c += temporal_threads<TB>()) {
            const int px = s + c % cw, py = sy + c / cw;
            const int x = x0 - TB + px, y = NDIM == 3 ? y0 - TB + py : 0;
            const bool ghost = !PERIODIC && (wghost || (unsigned)x >= (unsigned)P.nx ||
                                             (NDIM == 3 && (unsigned)y >= (unsigned)P.ny));
            out[py * PX + px] = ghost ? 0.0 : cell_update<NDIM, NT, BOX, PX>(W, pm, p0, pp, py, px);
          }
        } else {
          // last stage: the tile itself, straight to global memory
          for (int c = threadIdx.x; c < cw * ch; c += temporal_threads<TB>()) {
            const int px = s + c % cw, py = sy + c / cw;
            const int x = x0 - TB + px, y = NDIM == 3 ? y0 - TB + py : 0;
            if (x >= P.nx || (NDIM == 3 && y >= P.ny)) continue;
            const double v = cell_update<NDIM, NT, BOX, PX>(W, pm, p0, pp, py, px);
            if (NDIM == 3) P.dst[((int64_t)w * P.ny + y) * P.nx + x] = v;
            else P.dst[(int64_t)w * P.nx + x] = v;
          }
        }
        __syncthreads();
      }
      // input plane k+2 goes into the slot of plane k-2 (no stage reads it any more)
      if (k + 2 < nin) load_plane<NDIM, TB, PERIODIC>(in_ring + ((k + 2) & 3) * D::P, P, wa - TB + k + 2, y0, x0);
      cp_async_commit();
    }
    cp_async_wait<0>();
    __syncthreads();
  }
  (void)TY;
}

template <int NDIM, int NT, bool BOX, bool PERIODIC, int TB>
cudaError_t launch_tb(const Geom& g, const double* wdev, const double* src, double* dst, int sms,
                      cudaStream_t stream) {
  using D = PlaneDims<NDIM, TB>;
  auto kern = k_temporal<NDIM, NT, BOX, PERIODIC, TB>;
  static std::atomic<int> cache[kMaxDeviceOrdinals];
  const int occ = cached_per_device(cache, [kern] {
    int n = 0;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)D::bytes) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, temporal_threads<TB>(), D::bytes) != cudaSuccess)
      n = 0;
    return n;
  });
  if (occ < 1) return cudaErrorInvalidConfiguration;
  TParams P;
  P.src = src;
  P.dst = dst;
  P.nw = NDIM == 3 ? g.nz : g.ny;
  P.ny = g.ny;
  P.nx = g.nx;
  P.tiles_x = (g.nx + Geo<NDIM>::TX - 1) / Geo<NDIM>::TX;
  P.tiles_y = NDIM == 3 ? (g.ny + Geo<NDIM>::TY - 1) / Geo<NDIM>::TY : 1;
  P.work = (long long)P.tiles_x * P.tiles_y * P.nw;
  P.wdev = wdev;
  long long grid = (long long)sms * occ;
  if (grid > P.work) grid = P.work;
  kern<<<(unsigned)grid, temporal_threads<TB>(), D::bytes, stream>>>(P);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

template <int NDIM, int NT, bool BOX, bool PERIODIC>
cudaError_t by_tb(int Tb, const Geom& g, const double* wdev, const double* src, double* dst, int sms,
                  cudaStream_t stream) {
  switch (Tb) {
    case 2: return launch_tb<NDIM, NT, BOX, PERIODIC, 2>(g, wdev, src, dst, sms, stream);
    case 4: return launch_tb<NDIM, NT, BOX, PERIODIC, 4>(g, wdev, src, dst, sms, stream);
    case 8:
      if (NDIM == 2) return launch_tb<NDIM, NT, BOX, PERIODIC, (NDIM == 2 ? 8 : 4)>(g, wdev, src, dst, sms, stream);
      return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
  }
}

// ---------------------------------------------------------------------------
// 1D: a CTA owns 2048 consecutive cells, loads them with a halo of R*Tb cells
// per side into shared memory, advances them Tb steps there (the region
// shrinks by R per side per step) and writes the 2048 cells back: one launch
// per Tb steps, (2048 + R*Tb)/2048 of the single-step FP64 work.  Taps in
// lexicographic order with register weights, as in every other sweep.
constexpr int k1W = 2048;

template <int R, bool PERIODIC, int TB>
__global__ void __launch_bounds__(kThreads) k_temporal1d(const double* __restrict__ src,
                                                         double* __restrict__ dst, int n,
                                                         const double* __restrict__ wdev) {
  constexpr int NT = 2 * R + 1;
  constexpr int H = R * TB;
  constexpr int L = k1W + 2 * H;
  __shared__ double buf[2][L];
  RegWeights<NT> W;
  W.load(wdev);
  const long long x0 = (long long)blockIdx.x * k1W;
  for (int i = threadIdx.x; i < L; i += kThreads) {
    long long x = x0 - H + i;
    double v = 0.0;
    if (PERIODIC) {
      x %= n;
      if (x < 0) x += n;
      v = __ldg(src + x);
    } else if (x >= 0 && x < n) {
      v = __ldg(src + x);
    }
    buf[0][i] = v;
  }
  __syncthreads();
  int cur = 0;
#pragma unroll 1
  for (int s = 1; s <= TB; ++s) {
    const double* in = buf[cur];
    double* out = buf[cur ^ 1];
    for (int i = R * s + threadIdx.x; i < L - R * s; i += kThreads) {
      const long long x = x0 - H + i;
      double acc = 0.0;
      if (PERIODIC || (x >= 0 && x < n)) {
#pragma unroll
        for (int k = 0; k < NT; ++k) W.tap(acc, k, in[i + k - R], 0);
      }
      out[i] = acc;
    }
    __syncthreads();
    cur ^= 1;
  }
  for (int i = threadIdx.x; i < k1W; i += kThreads) {
    const long long x = x0 + i;
    if (x < n) dst[x] = buf[cur][H + i];
  }
}

template <int R, bool PERIODIC>
cudaError_t launch_1d(int Tb, const Geom& g, const double* wdev, const double* src, double* dst,
                      cudaStream_t stream) {
  const unsigned blocks = (unsigned)((g.nx + k1W - 1) / k1W);
  switch (Tb) {
    case 2: k_temporal1d<R, PERIODIC, 2><<<blocks, kThreads, 0, stream>>>(src, dst, g.nx, wdev); break;
    case 4: k_temporal1d<R, PERIODIC, 4><<<blocks, kThreads, 0, stream>>>(src, dst, g.nx, wdev); break;
    case 8: k_temporal1d<R, PERIODIC, 8><<<blocks, kThreads, 0, stream>>>(src, dst, g.nx, wdev); break;
    default: return cudaErrorInvalidValue;
  }
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

}  // namespace

bool temporal_supported(int ndim, int radius, int Tb) {
  if (ndim == 1) return (radius == 1 || radius == 2) && (Tb == 2 || Tb == 4 || Tb == 8);
  if (radius != 1) return false;
  if (ndim == 3) return Tb == 2 || Tb == 4;
  if (ndim == 2) return Tb == 2 || Tb == 4 || Tb == 8;
  return false;
}

cudaError_t launch_temporal(int ndim, int radius, Shape shape, int boundary, int Tb, const Geom& g,
                            const double* wdev, const double* src, double* dst, int sms,
                            cudaStream_t stream) {
  const bool per = boundary == kPeriodic;
  const bool box = shape == Shape::kBox;
  if (ndim == 1) {
    // the radius is implied by the tap count (3 or 5)
    (void)box;
    if (radius == 2)
      return per ? launch_1d<2, true>(Tb, g, wdev, src, dst, stream)
                 : launch_1d<2, false>(Tb, g, wdev, src, dst, stream);
    return per ? launch_1d<1, true>(Tb, g, wdev, src, dst, stream)
               : launch_1d<1, false>(Tb, g, wdev, src, dst, stream);
  }
  if (ndim == 3) {
    if (box) return per ? by_tb<3, 27, true, true>(Tb, g, wdev, src, dst, sms, stream)
                        : by_tb<3, 27, true, false>(Tb, g, wdev, src, dst, sms, stream);
    return per ? by_tb<3, 7, false, true>(Tb, g, wdev, src, dst, sms, stream)
               : by_tb<3, 7, false, false>(Tb, g, wdev, src, dst, sms, stream);
  }
  if (box) return per ? by_tb<2, 9, true, true>(Tb, g, wdev, src, dst, sms, stream)
                      : by_tb<2, 9, true, false>(Tb, g, wdev, src, dst, sms, stream);
  return per ? by_tb<2, 5, false, true>(Tb, g, wdev, src, dst, sms, stream)
             : by_tb<2, 5, false, false>(Tb, g, wdev, src, dst, sms, stream);
}

}  // namespace gbst
