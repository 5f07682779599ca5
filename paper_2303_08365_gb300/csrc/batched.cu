// batched.cu -- many independent 2D heat grids (Eq. 3 weights, each grid its
// own alpha and step count T) advanced by ONE persistent cooperative launch.
//
// Work list: every grid is cut into tiles; the tile list is sorted by the
// grid's T, largest first, so the tiles still active at step t always form a
// prefix of the list.  Step t: block b takes tiles b, b+G, b+2G, ... of that
// prefix (equal shares, whatever the mix of grid sizes), then all blocks meet
// at a device-wide barrier before step t+1 reads the neighbours written in
// step t.  The barrier's wait is bounded by wall time (%globaltimer): a block
// that waits too long records STENCIL_ERR_TIMEOUT and every block returns.
//
// Each grid alternates between the caller's buffer (even steps read it) and a
// library-owned partner; grids with odd T get their result copied back after
// the last barrier.  The per-cell arithmetic is the tap order of the generic
// sweep (lexicographic offsets: north, west, centre, east, south; the first
// product is a plain multiply), so a batched grid is bitwise equal to the
// same grid advanced by stencil_run.
#include "internal.h"
#include "taps.cuh"

namespace gbst {
namespace {

constexpr int kThreads = 256;
constexpr int kTileH = 8;
constexpr int kTileW = 64;  // kThreads = kTileW * 4 rows; each thread does 2 rows

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Device-wide barrier for a cooperative launch (all blocks co-resident).
// bar[0] counts arrivals, bar[1] is the generation.  Thread 0 of each block
// reads the generation, releases the block's writes (fence), arrives, and
// spins with acquire loads until the last arriver bumps the generation.
// The wait is bounded by wall time; returns false when it gave up or
// another block already reported an error.
__device__ bool grid_barrier(unsigned int* bar, unsigned int nblocks, long long limit_ns,
                             int* status) {
  __syncthreads();
  __shared__ int ok;
  if (threadIdx.x == 0) {
    ok = 1;
    unsigned int gen, arrived;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(gen) : "l"(bar + 1) : "memory");
    // arrival: releases this block's writes (ordered by the CTA barrier above)
    // and, for the last arriver, acquires every other block's
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(arrived) : "l"(bar) : "memory");
    if (arrived == nblocks - 1) {
      asm volatile("st.relaxed.gpu.global.u32 [%0], 0;" ::"l"(bar) : "memory");
      asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(bar + 1) : "memory");
    } else {
      const unsigned long long t0 = global_ns();
      for (unsigned int spin = 0;; ++spin) {
        unsigned int g;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(g) : "l"(bar + 1) : "memory");
        if (g != gen) break;
        if ((spin & 63) == 63) {
          if (*(volatile int*)status != 0) break;
          if ((long long)(global_ns() - t0) > limit_ns) {
            atomicCAS(status, 0, (int)-5 /* STENCIL_ERR_TIMEOUT */);
            break;
          }
        }
      }
    }
    if (*(volatile int*)status != 0) ok = 0;
  }
  __syncthreads();
  return ok != 0;
}

// One step of one tile: rows y0 .. y0+kTileH-1, columns x0 .. x0+kTileW-1.
__device__ __forceinline__ void tile_step(const BatchItemDev& it, const double* __restrict__ src,
                                          double* __restrict__ dst, int y0, int x0, bool periodic) {
  const int tx = threadIdx.x % kTileW;
  const int ty = threadIdx.x / kTileW;  // 0..3
  const int x = x0 + tx;
  if (x >= it.nx) return;
  const int ny = it.ny, nx = it.nx;
  int xw = x - 1, xe = x + 1;
  bool inw = true, ine = true;
  if (periodic) {
    xw = xw < 0 ? xw + nx : xw;
    xe = xe >= nx ? xe - nx : xe;
  } else {
    inw = xw >= 0;
    ine = xe < nx;
  }
#pragma unroll
  for (int r = 0; r < kTileH / 4; ++r) {
    const int y = y0 + ty + 4 * r;
    if (y >= ny) break;
    int yn = y - 1, ys = y + 1;
    bool inn = true, ins = true;
    if (periodic) {
      yn = yn < 0 ? yn + ny : yn;
      ys = ys >= ny ? ys - ny : ys;
    } else {
      inn = yn >= 0;
      ins = ys < ny;
    }
    const double* row = src + (int64_t)y * nx;
    const double vn = inn ? __ldcg(src + (int64_t)yn * nx + x) : 0.0;
    const double vw = inw ? __ldcg(row + xw) : 0.0;
    const double vc = __ldcg(row + x);
    const double ve = ine ? __ldcg(row + xe) : 0.0;
    const double vs = ins ? __ldcg(src + (int64_t)ys * nx + x) : 0.0;
    double acc = fma(it.w[0], vn, it.zero[r]);
    acc = fma(it.w[1], vw, acc);
    acc = fma(it.w[2], vc, acc);
    acc = fma(it.w[3], ve, acc);
    acc = fma(it.w[4], vs, acc);
    dst[(int64_t)y * nx + x] = acc;
  }
}

__global__ void __launch_bounds__(kThreads) k_batched(BatchLaunch L) {
  const unsigned int G = gridDim.x;
  const unsigned int arrivals = L.barrier_blocks > 0 ? (unsigned int)L.barrier_blocks : G;
  const bool periodic = L.boundary == kPeriodic;
  for (int t = 0; t < L.max_T; ++t) {
    for (int j = blockIdx.x; j < L.ntiles; j += G) {
      const BatchTile tl = L.tiles[j];
      const BatchItemDev it = L.items[tl.item];
      if (it.T <= t) break;  // tiles are sorted by T, largest first
      const double* src = (t & 1) ? it.b : it.a;
      double* dst = (t & 1) ? it.a : it.b;
      tile_step(it, src, dst, tl.y0, tl.x0, periodic);
    }
    if (!grid_barrier(L.barrier, arrivals, L.spin_limit, L.status)) return;
  }
  // grids with odd T hold their result in the partner buffer: copy it back
  for (int j = blockIdx.x; j < L.ntiles; j += G) {
    const BatchTile tl = L.tiles[j];
    const BatchItemDev it = L.items[tl.item];
    if ((it.T & 1) == 0) continue;
    const int tx = threadIdx.x % kTileW, ty = threadIdx.x / kTileW;
    const int x = tl.x0 + tx;
    if (x >= it.nx) continue;
    for (int r = 0; r < kTileH / 4; ++r) {
      const int y = tl.y0 + ty + 4 * r;
      if (y >= it.ny) break;
      const int64_t k = (int64_t)y * it.nx + x;
      it.a[k] = __ldcg(it.b + k);
    }
  }
}


// ---------------------------------------------------------------------------
// Persistent temporal blocking for one small 2D grid: every CTA owns tiles of
// kPTH x kPTW cells, loads each with a halo of Tb cells, advances it Tb steps
// in shared memory (the region shrinks by one cell per side per step: the
// overlapped-tile recompute of the paper's temporal tiling, Sec. 4.1), writes
// the tile back, and only then meets the other CTAs at the device-wide
// barrier -- one barrier per Tb steps instead of one per step.  Every cell
// applies the lexicographic tap chain of the single-step kernels (bitwise
// equal results).  Loads after a barrier bypass L1 (other SMs wrote them).
constexpr int kPTH = 16, kPTW = 32;
constexpr int kPThreads = 512;  // one CTA per SM on small grids: 16 warps to hide FP64 latency

template <int NT, bool BOX, bool PERIODIC, int TB>
__device__ __forceinline__ double ptb_cell(const RegWeights<NT>& W, const double* in, int ry, int rx,
                                           int y, int x, int ny, int nx, int chain) {
  constexpr int RW = kPTW + 2 * TB;
  double acc = 0.0;
  if (PERIODIC || ((unsigned)y < (unsigned)ny && (unsigned)x < (unsigned)nx)) {
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) {
        if (!BOX && dy != 0 && dx != 0) continue;
        const int k = BOX ? (dy + 1) * 3 + (dx + 1) : (dy < 0 ? 0 : dy > 0 ? 4 : 2 + dx);
        W.tap(acc, k, in[(ry + dy) * RW + rx + dx], chain);
      }
  }
  return acc;
}

template <int NT, bool BOX, bool PERIODIC, int TB>
__global__ void __launch_bounds__(kPThreads) k_persist_tb(PersistTbLaunch L) {
  constexpr int RH = kPTH + 2 * TB, RW = kPTW + 2 * TB;
  __shared__ double buf[2][RH * RW];
  RegWeights<NT> W;
  W.load(L.wdev);
  const unsigned int G = gridDim.x;
  const int ny = L.ny, nx = L.nx;
  const int tiles_x = (nx + kPTW - 1) / kPTW, tiles_y = (ny + kPTH - 1) / kPTH;
  const int ntiles = tiles_x * tiles_y;
  double* src = L.a;
  double* dst = L.b;
  for (long long t0 = 0; t0 < L.T; t0 += TB) {
    const int tb = (int)(L.T - t0 < TB ? L.T - t0 : TB);
    for (int j = blockIdx.x; j < ntiles; j += G) {
      const int y0 = (j / tiles_x) * kPTH, x0 = (j % tiles_x) * kPTW;
      // load the tile with a halo of tb cells (region offset TB - tb inside the buffer)
      const int off = TB - tb;
      const int lh = kPTH + 2 * tb, lw = kPTW + 2 * tb;
      for (int c = threadIdx.x; c < lh * lw; c += kPThreads) {
        const int ry = c / lw, rx = c % lw;
        int y = y0 - tb + ry, x = x0 - tb + rx;
        double v = 0.0;
        if (PERIODIC) {
          y %= ny; y += y < 0 ? ny : 0;
          x %= nx; x += x < 0 ? nx : 0;
          v = __ldcg(src + (int64_t)y * nx + x);
        } else if ((unsigned)y < (unsigned)ny && (unsigned)x < (unsigned)nx) {
          v = __ldcg(src + (int64_t)y * nx + x);
        }
        buf[0][(off + ry) * RW + off + rx] = v;
      }
      __syncthreads();
      int cur = 0;
      for (int s = 1; s <= tb; ++s) {
        const int m = tb - s;  // remaining halo after this step
        const int h = kPTH + 2 * m, w = kPTW + 2 * m;
        const double* in = buf[cur];
        double* out = buf[cur ^ 1];
        // two cells per thread per pass: two independent FMA chains in flight
        for (int c = threadIdx.x; c < h * w; c += 2 * kPThreads) {
          const int c2 = c + kPThreads;
          const int ry = TB - m + c / w, rx = TB - m + c % w;  // buffer coordinates
          const int ry2 = TB - m + c2 / w, rx2 = TB - m + c2 % w;
          const double v1 = ptb_cell<NT, BOX, PERIODIC, TB>(W, in, ry, rx, y0 - TB + ry, x0 - TB + rx, ny,
                                                           nx, 0);
          double v2 = 0.0;
          if (c2 < h * w)
            v2 = ptb_cell<NT, BOX, PERIODIC, TB>(W, in, ry2, rx2, y0 - TB + ry2, x0 - TB + rx2, ny, nx, 1);
          out[ry * RW + rx] = v1;
          if (c2 < h * w) out[ry2 * RW + rx2] = v2;
        }
        __syncthreads();
        cur ^= 1;
      }
      // the tile itself back to global memory
      for (int c = threadIdx.x; c < kPTH * kPTW; c += kPThreads) {
        const int ry = c / kPTW, rx = c % kPTW;
        const int y = y0 + ry, x = x0 + rx;
        if (y < ny && x < nx) dst[(int64_t)y * nx + x] = buf[cur][(TB + ry) * RW + TB + rx];
      }
      __syncthreads();
    }
    if (!grid_barrier(L.barrier, G, L.spin_limit, L.status)) return;
    double* tmp = src;
    src = dst;
    dst = tmp;
  }
  // the result is in `src`; if that is the partner buffer, copy it back
  if (src != L.a) {
    for (int j = blockIdx.x; j < ntiles; j += G) {
      const int y0 = (j / tiles_x) * kPTH, x0 = (j % tiles_x) * kPTW;
      for (int c = threadIdx.x; c < kPTH * kPTW; c += kPThreads) {
        const int y = y0 + c / kPTW, x = x0 + c % kPTW;
        if (y < ny && x < nx) L.a[(int64_t)y * nx + x] = __ldcg(src + (int64_t)y * nx + x);
      }
    }
  }
}

template <int NT, bool BOX, bool PERIODIC, int TB>
cudaError_t launch_ptb(const PersistTbLaunch& L, int sms, cudaStream_t stream) {
  auto kern = k_persist_tb<NT, BOX, PERIODIC, TB>;
  static int occ = -1;
  if (occ < 0 && cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kPThreads, 0) != cudaSuccess)
    occ = 0;
  if (occ < 1) return cudaErrorInvalidConfiguration;
  const int tiles = ((L.nx + kPTW - 1) / kPTW) * ((L.ny + kPTH - 1) / kPTH);
  int grid = sms * (occ < 2 ? occ : 2);
  if (tiles < grid) grid = tiles;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid, 1, 1);
  cfg.blockDim = dim3(kPThreads, 1, 1);
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelEx(&cfg, kern, L);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return e;
}

template <int NT, bool BOX, bool PERIODIC>
cudaError_t ptb_by_tb(int Tb, const PersistTbLaunch& L, int sms, cudaStream_t stream) {
  switch (Tb) {
    case 2: return launch_ptb<NT, BOX, PERIODIC, 2>(L, sms, stream);
    case 4: return launch_ptb<NT, BOX, PERIODIC, 4>(L, sms, stream);
    case 8: return launch_ptb<NT, BOX, PERIODIC, 8>(L, sms, stream);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t launch_persist_tb(Shape shape, int boundary, int Tb, const PersistTbLaunch& L, int sms,
                              cudaStream_t stream) {
  const bool per = boundary == kPeriodic;
  if (shape == Shape::kBox)
    return per ? ptb_by_tb<9, true, true>(Tb, L, sms, stream) : ptb_by_tb<9, true, false>(Tb, L, sms, stream);
  return per ? ptb_by_tb<5, false, true>(Tb, L, sms, stream) : ptb_by_tb<5, false, false>(Tb, L, sms, stream);
}

namespace {
}  // namespace

int batched_block_size() { return kThreads; }
int batched_tile_h() { return kTileH; }
int batched_tile_w() { return kTileW; }

cudaError_t launch_batched(const BatchLaunch& L, int grid_blocks, cudaStream_t stream) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid_blocks, 1, 1);
  cfg.blockDim = dim3(kThreads, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelEx(&cfg, k_batched, L);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return e;
}

// Blocks of k_batched that fit on one SM at once (for the cooperative grid size).
int batched_blocks_per_sm() {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batched, kThreads, 0) != cudaSuccess)
    return 0;
  return n;
}

}  // namespace gbst
