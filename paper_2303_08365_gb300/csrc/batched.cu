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
    if (!grid_barrier(L.barrier, G, L.spin_limit, L.status)) return;
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
