// temporal.cu -- temporal blocking: Tb time steps per HBM round trip.
//
// The paper stretches its spatial tiles along the time dimension so that a
// tile is read once and updated Tb times before it is written back (Sec. 4.1,
// "Temporal Tiling"; triangles in 2D become tetrahedra in space-time).  This
// kernel does the same with overlapped tiles, streamed along the slowest axis:
//
//   - a CTA owns an output tile of the "plane" orthogonal to the streaming
//     axis (3D: a square of the (y, x) plane, streamed along z; 2D: 256 cells
//     of a row, streamed along y) and loads it with a halo of Tb cells;
//   - stage s = 1 .. Tb holds the tile at time t+s on a region that shrinks by
//     one cell per side per stage (the halo cells are recomputed by the
//     neighbouring tiles: the overlapped-tile redundancy);
//   - along the streaming axis nothing is recomputed: each stage keeps a ring
//     of planes of its own output, so each input plane is read once from HBM
//     and each output plane written once;
//   - the stages are skewed by two planes (stage s produces plane k - 2s while
//     input plane k lands), so that within one iteration no stage reads what
//     another writes: one barrier per input plane covers all Tb stages, and
//     the iteration's cells of every stage form one flat list of jobs (pairs
//     of x-neighbours) spread over all warps, with no partial warp per stage;
//   - input planes arrive by cp.async (8-byte copies with zero fill for
//     Dirichlet ghosts and wrapped addresses for periodic grids; a periodic
//     halo of width Tb does not fit the TMA box model at the grid edges);
//   - each cell applies its taps in the direct kernel's lexicographic order
//     with register-resident weights, so a Tb-fused sweep is bitwise equal to
//     Tb single steps; the last stage stores its pairs as 16-byte stores.
// Dirichlet ghost cells (outside the grid, at every time level) stay zero.
#include "internal.h"
#include "taps.cuh"

namespace gbst {
namespace {

constexpr int kThreads = 256;  // 1D kernel

// Output tile (y, x) of the 2D/3D kernel.  3D: Tb = 2: 16 x 64 (1.08x the
// single-step work in halo recompute; the 27-point box: 32 x 64, 1.05x);
// Tb = 4: 32 x 32 (1.20x), the tile with the shortest perimeter per cell
// whose stage rings fit in shared memory; Tb = 8: 16 x 16 (2.15x).  2D: a row segment of about 256 cells, cut so that
// one iteration's jobs (Tb stages of pairs) fill just under Tb whole rounds of
// 8 warps (Tb = 2: 254 cells, 255 pairs; 4: 252, 510; 8: 248, 1020): a round
// with a few pairs left over would cost a whole warp instruction per FP64
// operation for them.
template <int NDIM, int TB, bool BOX>
struct Geo {
  static constexpr int TX = NDIM == 3 ? (TB == 2 ? 64 : TB == 4 ? 32 : 16)
                                      : 2 * ((128 * TB - TB * (TB - 1) / 2) / TB);
  static constexpr int TY = NDIM == 3 ? (TB == 2 ? (BOX ? 32 : 16) : TX) : 1;
};

// Stage schedule.  LAG = 2: stage s produces plane k - 2s in iteration k, so
// no stage reads what another writes in the same iteration and one barrier
// per input plane covers all stages (rings of 4 planes).  LAG = 1: stage s
// produces plane k - s - 1, reading what stage s - 1 wrote just before, with
// a barrier between stages (rings of 3 planes).  The 3D star at Tb = 2 takes
// LAG = 1: its 72 KB of rings let three CTAs share an SM, whose barriers then
// overlap (measured at 512^3: 77.2 GStencil/s against 74.9 for LAG = 2 at two
// CTAs per SM and 67.5 at one).  The 27-point box keeps its 27 weights in
// registers, which leaves room for one CTA of 16 warps: LAG = 2 (20.5 against
// 19.9 GStencil/s at 384^3).
template <int NDIM, int TB, bool BOX>
constexpr int temporal_lag() { return NDIM == 3 && TB == 2 && !BOX ? 1 : 2; }

// Threads per CTA and CTAs per SM.  3D star at Tb = 2: 8 warps, three CTAs per
// SM; other 3D kernels: one CTA of 16 warps (rings of 147-172 KB); 2D: 8
// warps, several CTAs.
template <int NDIM, bool BOX, int TB>
constexpr int temporal_threads() { return NDIM == 3 && (TB > 2 || BOX) ? 512 : 256; }
template <int NDIM, bool BOX, int TB>
constexpr int temporal_min_blocks() { return NDIM == 3 ? (TB == 2 && !BOX ? 3 : 1) : 2; }

// Shared-memory layout.  Plane coordinates (py, px) cover the tile and a halo
// of Tb cells per side.  Stage q = 0 .. Tb-1 (q = 0: the input) keeps a ring
// of planes over its region [q, PX-q) x [q, PY-q) (2D: the row [q, PX-q)),
// stored compactly with row stride W(q): the input ring holds 4 (three that
// stage 1 reads and one landing), the stage rings 4 (LAG = 2: three read by
// the next stage, one being written) or 3 (LAG = 1).
template <int NDIM, int TB, bool BOX>
struct Lay {
  static constexpr int PX = Geo<NDIM, TB, BOX>::TX + 2 * TB;
  static constexpr int PY = NDIM == 3 ? Geo<NDIM, TB, BOX>::TY + 2 * TB : 1;
  static constexpr int P = PX * PY;
  static constexpr int kIn = 4;
  static constexpr int kRing = temporal_lag<NDIM, TB, BOX>() == 2 ? 4 : 3;
  __host__ __device__ static constexpr int W(int q) { return PX - 2 * q; }
  __host__ __device__ static constexpr int H(int q) { return NDIM == 3 ? PY - 2 * q : 1; }
  __host__ __device__ static constexpr int N(int q) { return W(q) * H(q); }
  // N(0) + ... + N(q-1), in closed form
  __host__ __device__ static constexpr int cells_before(int q) {
    return NDIM == 3 ? q * PX * PY - (PX + PY) * q * (q - 1) + 2 * (q - 1) * q * (2 * q - 1) / 3
                     : q * PX - q * (q - 1);
  }
  // first double of stage q's ring
  __host__ __device__ static constexpr int off(int q) {
    return q == 0 ? 0 : kIn * P + kRing * (cells_before(q) - P);
  }
  // ring slot of plane i of stage q
  __host__ __device__ static constexpr int slot(int q, int i) { return q == 0 || kRing == 4 ? (i & 3) : i % 3; }
  static constexpr size_t bytes = (size_t)off(TB) * sizeof(double);
  // jobs: pairs of y-neighbours in 3D (H(q) is even: a pair never leaves the
  // region, and a warp reads 32 consecutive doubles of a row per load), pairs
  // of x-neighbours in 2D (W(q) is even)
  __host__ __device__ static constexpr int pairs(int q) { return N(q) / 2; }
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
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Issues the copies of input plane w (global streaming coordinate) of the tile
// whose output origin is (y0, x0) into `slot`.
template <int NDIM, int TB, bool BOX, bool PERIODIC, int NTH>
__device__ __forceinline__ void load_plane(double* slot, const TParams& P, int w, int y0, int x0) {
  using L = Lay<NDIM, TB, BOX>;
  bool win = true;
  int ww = w;
  if (PERIODIC) ww = wrapn(w, P.nw);
  else win = (unsigned)w < (unsigned)P.nw;
  for (int c = threadIdx.x; c < L::P; c += NTH) {
    const int px = c % L::PX, py = c / L::PX;
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

// Two neighbouring cells of a stage (3D: along y; 2D: along x): taps over
// planes (pm, p0, pp) of the previous stage (row stride sw) around the cells
// at (ly, lx) and (ly + 1, lx) (2D: (0, lx) and (0, lx + 1)) of that stage's
// region.  Two independent chains, each in tap order.
// EQ (2D 9-point box whose weights are all equal, w): the pair shares partial
// sums instead: the four column sums C(x) = u(y-1, x) + (u(y, x) + u(y+1, x))
// it needs, then u'(x) = w C(x-1) + w (C(x) + C(x+1)) and u'(x+1) =
// w C(x+2) + w (C(x) + C(x+1)): 12 FP64 instructions for the two cells
// instead of 18 (additions as FMAs against a register holding 1).  The sum
// is taken in another order than the tap list, so the result is within
// rounding of the other kernels, not bitwise equal to them.
template <int NDIM, int NT, bool BOX, bool EQ = false>
__device__ __forceinline__ void pair_update(const RegWeights<NT>& W, const double* pm, const double* p0,
                                            const double* pp, int sw, int ly, int lx, double& a0,
                                            double& a1) {
  if constexpr (NDIM == 2 && EQ) {
    double C[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int x = lx - 1 + k;
      C[k] = W.add(pm[x], W.add(p0[x], pp[x], k & 1), 2 + (k & 1));
    }
    const double wt = fma(W.w[4], W.add(C[1], C[2], 0), W.z[0]);
    a0 = fma(W.w[0], C[0], wt);
    a1 = fma(W.w[8], C[3], wt);
    return;
  }
  const double* pl[3] = {pm, p0, pp};
  const int de = NDIM == 3 ? sw : 1;  // the second cell
#pragma unroll
  for (int dw = -1; dw <= 1; ++dw) {
#pragma unroll
    for (int dv = -1; dv <= 1; ++dv) {
      if (NDIM == 2 && dv != 0) continue;
#pragma unroll
      for (int du = -1; du <= 1; ++du) {
        if (!BOX && (dw != 0) + (dv != 0) + (du != 0) > 1) continue;
        const double* q = pl[dw + 1] + (ly + dv) * sw + lx + du;
        const int t = tidx<NDIM, BOX>(dw, dv, du);
        W.tap(a0, t, q[0], 0);
        W.tap(a1, t, q[de], 1);
      }
    }
  }
}

// Pair c of stage s's region, plane i: computed from the three planes of
// stage s-1 around it and written to stage s's ring, or (s = Tb) to global
// memory.
template <int NDIM, int NT, bool BOX, bool PERIODIC, int TB, bool EQ = false>
__device__ __forceinline__ void stage_pair(const TParams& P, const RegWeights<NT>& W, double* sm, int s,
                                           int c, int i, int wa, int y0, int x0) {
  using L = Lay<NDIM, TB, BOX>;
  const int ws = L::W(s);
  int qy, qx;  // the pair's first cell, as an offset in stage s's region
  if (NDIM == 3) {
    qy = c / ws;
    qx = c - qy * ws;
    qy *= 2;
  } else {
    qy = 0;
    qx = 2 * c;
  }
  const int sn = L::N(s - 1);
  const double* src = sm + L::off(s - 1);
  const double* pm = src + L::slot(s - 1, i - 1) * sn;
  const double* p0 = src + L::slot(s - 1, i) * sn;
  const double* pp = src + L::slot(s - 1, i + 1) * sn;
  double a0, a1;
  pair_update<NDIM, NT, BOX, EQ>(W, pm, p0, pp, L::W(s - 1), NDIM == 3 ? qy + 1 : 0, qx + 1, a0, a1);
  const int w = wa - TB + i;
  const int x = x0 - TB + s + qx;
  const int y = NDIM == 3 ? y0 - TB + s + qy : 0;
  if (s < TB) {
    double* out = sm + L::off(s) + L::slot(s, i) * L::N(s) + qy * ws + qx;
    if (NDIM == 3) {
      if (!PERIODIC) {
        const bool g = (unsigned)w >= (unsigned)P.nw || (unsigned)x >= (unsigned)P.nx;
        if (g || (unsigned)y >= (unsigned)P.ny) a0 = 0.0;
        if (g || (unsigned)(y + 1) >= (unsigned)P.ny) a1 = 0.0;
      }
      out[0] = a0;
      out[ws] = a1;
    } else {
      if (!PERIODIC) {
        const bool g = (unsigned)w >= (unsigned)P.nw;
        if (g || (unsigned)x >= (unsigned)P.nx) a0 = 0.0;
        if (g || (unsigned)(x + 1) >= (unsigned)P.nx) a1 = 0.0;
      }
      *reinterpret_cast<double2*>(out) = make_double2(a0, a1);  // 16-byte aligned
    }
  } else if (NDIM == 3) {
    // the tile itself (x >= 0, y >= 0, w in range): straight to global memory
    if (x < P.nx) {
      double* g = P.dst + ((int64_t)w * P.ny + y) * P.nx + x;
      if (y < P.ny) g[0] = a0;
      if (y + 1 < P.ny) g[P.nx] = a1;
    }
  } else {
    double* g = P.dst + (int64_t)w * P.nx + x;
    if (x + 1 < P.nx && (reinterpret_cast<uintptr_t>(g) & 15) == 0) {
      *reinterpret_cast<double2*>(g) = make_double2(a0, a1);
    } else {
      if (x < P.nx) g[0] = a0;
      if (x + 1 < P.nx) g[1] = a1;
    }
  }
}

template <int NDIM, int NT, bool BOX, bool PERIODIC, int TB, bool EQ = false>
__global__ void __launch_bounds__(temporal_threads<NDIM, BOX, TB>(), temporal_min_blocks<NDIM, BOX, TB>())
    k_temporal(const TParams P) {
  using L = Lay<NDIM, TB, BOX>;
  constexpr int NTH = temporal_threads<NDIM, BOX, TB>();
  constexpr int LAG = temporal_lag<NDIM, TB, BOX>();
  constexpr int TX = Geo<NDIM, TB, BOX>::TX, TY = Geo<NDIM, TB, BOX>::TY;
  extern __shared__ __align__(16) double sm[];
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
    // input planes i = 0 .. nin-1 are streaming coordinates wa-TB .. wb+TB-1;
    // stage s produces its planes i in [s, nin-s), plane i in iteration
    // i + 2s (LAG = 2) or i + s + 1 (LAG = 1)
    const int nin = (wb - wa) + 2 * TB;
    load_plane<NDIM, TB, BOX, PERIODIC, NTH>(sm, P, wa - TB, y0, x0);
    cp_async_commit();
    const int k_end = LAG == 2 ? nin + TB : nin + 1;
    for (int k = 1; k < k_end; ++k) {
      cp_async_wait_all();  // input plane k-1 has landed
      __syncthreads();      // ... for every thread, and iteration k-1's stage planes are written
      if (k < nin) load_plane<NDIM, TB, BOX, PERIODIC, NTH>(sm + (k & 3) * L::P, P, wa - TB + k, y0, x0);
      cp_async_commit();
      if (LAG == 2) {
        // one flat job list: stage s contributes its pairs when its plane
        // k - 2s is in range, i.e. for s_lo <= s <= s_hi
        const int s_lo = max(1, k - nin + 1), s_hi = min(TB, k / 3);
        int njobs = 0;
        for (int s = s_lo; s <= s_hi; ++s) njobs += L::pairs(s);
        for (int j = threadIdx.x; j < njobs; j += NTH) {
          int s = s_lo, c = j;
          while (c >= L::pairs(s)) {
            c -= L::pairs(s);
            ++s;
          }
          stage_pair<NDIM, NT, BOX, PERIODIC, TB, EQ>(P, W, sm, s, c, k - 2 * s, wa, y0, x0);
        }
      } else {
        // stage by stage: plane k - s - 1 is in range for s <= (k - 1) / 2
        const int s_hi = min(TB, (k - 1) / 2);
        for (int s = 1; s <= s_hi; ++s) {
          if (s > 1) __syncthreads();  // stage s-1's plane of this iteration is written
          for (int j = threadIdx.x; j < L::pairs(s); j += NTH)
            stage_pair<NDIM, NT, BOX, PERIODIC, TB, EQ>(P, W, sm, s, j, k - s - 1, wa, y0, x0);
        }
      }
    }
    __syncthreads();  // the next tile's first plane reuses input slot 0
  }
}

template <int NDIM, int NT, bool BOX, bool PERIODIC, int TB, bool EQ = false>
cudaError_t launch_tb(const Geom& g, const double* wdev, const double* src, double* dst, int sms,
                      cudaStream_t stream) {
  using L = Lay<NDIM, TB, BOX>;
  constexpr int NTH = temporal_threads<NDIM, BOX, TB>();
  static_assert(L::bytes <= 227 * 1024, "stage rings exceed shared memory");
  auto kern = k_temporal<NDIM, NT, BOX, PERIODIC, TB, EQ>;
  static std::atomic<int> cache[kMaxDeviceOrdinals];
  const int occ = cached_per_device(cache, [kern] {
    int n = 0;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::bytes) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, NTH, L::bytes) != cudaSuccess)
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
  P.tiles_x = (g.nx + Geo<NDIM, TB, BOX>::TX - 1) / Geo<NDIM, TB, BOX>::TX;
  P.tiles_y = NDIM == 3 ? (g.ny + Geo<NDIM, TB, BOX>::TY - 1) / Geo<NDIM, TB, BOX>::TY : 1;
  P.work = (long long)P.tiles_x * P.tiles_y * P.nw;
  P.wdev = wdev;
  long long grid = (long long)sms * occ;
  if (grid > P.work) grid = P.work;
  kern<<<(unsigned)grid, NTH, L::bytes, stream>>>(P);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

template <int NDIM, int NT, bool BOX, bool PERIODIC, bool EQ = false>
cudaError_t by_tb(int Tb, const Geom& g, const double* wdev, const double* src, double* dst, int sms,
                  cudaStream_t stream) {
  switch (Tb) {
    case 2: return launch_tb<NDIM, NT, BOX, PERIODIC, 2, EQ>(g, wdev, src, dst, sms, stream);
    case 4: return launch_tb<NDIM, NT, BOX, PERIODIC, 4, EQ>(g, wdev, src, dst, sms, stream);
    case 8: return launch_tb<NDIM, NT, BOX, PERIODIC, 8, EQ>(g, wdev, src, dst, sms, stream);
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
  return (ndim == 2 || ndim == 3) && (Tb == 2 || Tb == 4 || Tb == 8);
}

cudaError_t launch_temporal(int ndim, int radius, Shape shape, int boundary, int Tb, const Geom& g,
                            const double* wdev, const double* src, double* dst, int sms,
                            cudaStream_t stream, bool equal) {
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
  if (box && equal) return per ? by_tb<2, 9, true, true, true>(Tb, g, wdev, src, dst, sms, stream)
                               : by_tb<2, 9, true, false, true>(Tb, g, wdev, src, dst, sms, stream);
  if (box) return per ? by_tb<2, 9, true, true>(Tb, g, wdev, src, dst, sms, stream)
                      : by_tb<2, 9, true, false>(Tb, g, wdev, src, dst, sms, stream);
  return per ? by_tb<2, 5, false, true>(Tb, g, wdev, src, dst, sms, stream)
             : by_tb<2, 5, false, false>(Tb, g, wdev, src, dst, sms, stream);
}

}  // namespace gbst
