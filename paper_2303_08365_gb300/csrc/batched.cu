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
// product is an FMA onto 0.0), so a batched grid is bitwise equal to the
// same grid advanced by stencil_run.
#include "internal.h"
#include "taps.cuh"

namespace gbst {
namespace {

constexpr int kThreads = kBatchThreads;
// A tile is a run of CPT * kThreads consecutive cells of one grid in row-major
// order (CPT cells per thread, kThreads apart), so every warp is full except
// at a grid's last tile: the FP64 unit charges a warp instruction the same
// time whatever the number of active lanes.  CPT (1, 2 or 4) is chosen by the
// batch autotuner; 2 is the default.
constexpr int kDefaultCpt = 2;

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

// One step of one tile: cells k0 .. k0+n-1 of the item (row-major), CPT per
// thread.  The per-cell chain is the generic sweep's tap order.
template <int CPT>
__device__ __forceinline__ void tile_step(const BatchItemDev& it, const double* __restrict__ src,
                                          double* __restrict__ dst, int k0, int n, bool periodic) {
  const int ny = it.ny, nx = it.nx;
#pragma unroll
  for (int r = 0; r < CPT; ++r) {
    const int c = threadIdx.x + r * kThreads;
    if (c >= n) break;
    const int k = k0 + c;
    const int y = k / nx, x = k - y * nx;
    int xw = x - 1, xe = x + 1, yn = y - 1, ys = y + 1;
    bool inw = true, ine = true, inn = true, ins = true;
    if (periodic) {
      xw = xw < 0 ? xw + nx : xw;
      xe = xe >= nx ? xe - nx : xe;
      yn = yn < 0 ? yn + ny : yn;
      ys = ys >= ny ? ys - ny : ys;
    } else {
      inw = xw >= 0;
      ine = xe < nx;
      inn = yn >= 0;
      ins = ys < ny;
    }
    const double* row = src + (int64_t)y * nx;
    const double vn = inn ? __ldcg(src + (int64_t)yn * nx + x) : 0.0;
    const double vw = inw ? __ldcg(row + xw) : 0.0;
    const double vc = __ldcg(row + x);
    const double ve = ine ? __ldcg(row + xe) : 0.0;
    const double vs = ins ? __ldcg(src + (int64_t)ys * nx + x) : 0.0;
    double acc = fma(it.w[0], vn, it.zero[r & 1]);
    acc = fma(it.w[1], vw, acc);
    acc = fma(it.w[2], vc, acc);
    acc = fma(it.w[3], ve, acc);
    acc = fma(it.w[4], vs, acc);
    dst[k] = acc;
  }
}

template <int CPT>
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
      tile_step<CPT>(it, src, dst, tl.k0, tl.n, periodic);
    }
    if (!grid_barrier(L.barrier, arrivals, L.spin_limit, L.status)) return;
  }
  // grids with odd T hold their result in the partner buffer: copy it back
  for (int j = blockIdx.x; j < L.ntiles; j += G) {
    const BatchTile tl = L.tiles[j];
    const BatchItemDev it = L.items[tl.item];
    if ((it.T & 1) == 0) continue;
    for (int c = threadIdx.x; c < tl.n; c += kThreads) {
      const int k = tl.k0 + c;
      it.a[k] = __ldcg(it.b + k);
    }
  }
}


// ---------------------------------------------------------------------------
// Persistent temporal blocking for one small 2D grid.  The grid is cut into
// tiles_y x tiles_x tiles of near-equal size (at most kPTH x kPTW; the host
// picks the cut so that the tiles cover the SMs evenly).  Every CTA owns
// tiles, loads each with a halo of Tb cells, advances it Tb steps in shared
// memory (the region shrinks by one cell per side per step: the overlapped-
// tile recompute of the paper's temporal tiling, Sec. 4.1) and writes the tile
// back.  There is no device-wide barrier: each tile publishes the number of
// blocks it has finished in its own flag, and a tile starts block k once every
// tile its halo reaches has finished block k-1.  That also keeps a tile from
// overwriting data a slower neighbour is still reading, since the neighbour's
// reads of block k-1 come before its flag.  Every cell applies the
// lexicographic tap chain of the single-step kernels (bitwise equal
// results).  Loads of other tiles' data bypass L1 (other SMs wrote them).
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

// Waits until every tile within (reach_y, reach_x) tiles of (ty, tx) has
// published at least `target` finished blocks.  The wait is bounded by wall
// time and gives up at once when another CTA has reported an error; returns
// false (for every thread of the CTA) when it gave up.
// (flags: the grid's tiles_y x tiles_x flag words, row-major.)
template <bool PERIODIC>
__device__ bool wait_tiles(const unsigned int* flags, int tiles_y, int tiles_x, int reach_y, int reach_x,
                           int ty, int tx, unsigned int target, int* status, long long spin_limit) {
  const int wy = 2 * reach_y + 1, wx = 2 * reach_x + 1;
  int ok = 1;
  for (int i = threadIdx.x; i < wy * wx; i += blockDim.x) {
    int yy = ty + i / wx - reach_y, xx = tx + i % wx - reach_x;
    if (PERIODIC) {
      yy %= tiles_y;
      yy += yy < 0 ? tiles_y : 0;
      xx %= tiles_x;
      xx += xx < 0 ? tiles_x : 0;
    } else if ((unsigned)yy >= (unsigned)tiles_y || (unsigned)xx >= (unsigned)tiles_x) {
      continue;
    }
    const unsigned int* f = flags + yy * tiles_x + xx;
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(f) : "memory");
    if (v >= target) continue;
    const unsigned long long t0 = global_ns();
    for (unsigned int spin = 0;; ++spin) {
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(f) : "memory");
      if (v >= target) break;
      if ((spin & 31) == 31) {
        if (*(volatile int*)status != 0) {
          ok = 0;
          break;
        }
        if ((long long)(global_ns() - t0) > spin_limit) {
          atomicCAS(status, 0, (int)-5 /* STENCIL_ERR_TIMEOUT */);
          ok = 0;
          break;
        }
      }
    }
    if (!ok) break;
  }
  return __syncthreads_and(ok) != 0;
}

template <bool PERIODIC>
__device__ bool wait_reach(const PersistTbLaunch& L, int ty, int tx, unsigned int target) {
  return wait_tiles<PERIODIC>(L.flags, L.tiles_y, L.tiles_x, L.reach_y, L.reach_x, ty, tx, target, L.status,
                              L.spin_limit);
}

// Rows [y0, y1) of tile row ty when ny rows are cut into `tiles` near-equal parts.
__device__ __forceinline__ int cut(int i, int n, int tiles) {
  return (int)((long long)i * n / tiles);
}

// Row and column of a flat index k = r * w + c that advances by a fixed
// stride: one division when the walk starts, none per step.
struct FlatWalk {
  int r, c, dr, dc, w;
  __device__ __forceinline__ FlatWalk(int start, int stride, int width)
      : r(start / width), c(start % width), dr(stride / width), dc(stride % width), w(width) {}
  __device__ __forceinline__ void next() {
    r += dr;
    c += dc;
    if (c >= w) {
      c -= w;
      ++r;
    }
  }
};

__device__ __forceinline__ int wrap_into(int v, int n) {
  while (v < 0) v += n;
  while (v >= n) v -= n;
  return v;
}

template <int NT, bool BOX, bool PERIODIC, int TB>
__global__ void __launch_bounds__(kPThreads, 2) k_persist_tb(PersistTbLaunch L) {
  constexpr int RW = kPTW + 2 * TB;
  constexpr int RH = kPTH + 2 * TB;
  __shared__ double buf[2][RH * RW];
  RegWeights<NT> W;
  W.load(L.wdev);
  const int G = gridDim.x;
  const int ny = L.ny, nx = L.nx;
  const int ntiles = L.tiles_y * L.tiles_x;
  const long long nblk = (L.T + TB - 1) / TB;
  // the geometry of this CTA's first tile, worked out once: most CTAs own one
  // tile, and its divisions sit on the path between two blocks
  const int fty = blockIdx.x / L.tiles_x, ftx = blockIdx.x % L.tiles_x;
  const int fy0 = cut(fty, ny, L.tiles_y), fx0 = cut(ftx, nx, L.tiles_x);
  const int fth = cut(fty + 1, ny, L.tiles_y) - fy0, ftw = cut(ftx + 1, nx, L.tiles_x) - fx0;
  for (long long blk = 0; blk < nblk; ++blk) {
    const int tb = (int)(L.T - blk * TB < TB ? L.T - blk * TB : TB);
    const double* src = (blk & 1) ? L.b : L.a;
    double* dst = (blk & 1) ? L.a : L.b;
    for (int j = blockIdx.x; j < ntiles; j += G) {
      const bool first = j == (int)blockIdx.x;
      const int ty = first ? fty : j / L.tiles_x, tx = first ? ftx : j % L.tiles_x;
      const int y0 = first ? fy0 : cut(ty, ny, L.tiles_y), x0 = first ? fx0 : cut(tx, nx, L.tiles_x);
      const int th = first ? fth : cut(ty + 1, ny, L.tiles_y) - y0;
      const int tw = first ? ftw : cut(tx + 1, nx, L.tiles_x) - x0;
      if (blk > 0 && !wait_reach<PERIODIC>(L, ty, tx, (unsigned int)blk)) return;
      // load the tile with a halo of tb cells (region offset TB - tb inside the
      // buffer): every load of this thread first, then the shared-memory
      // stores, so the loads' L2 round trips overlap
      const int off = TB - tb;
      const int lh = th + 2 * tb, lw = tw + 2 * tb;
      constexpr int KL = (RH * RW + kPThreads - 1) / kPThreads;
      double lv[KL];
      int li[KL];
      FlatWalk lwk(threadIdx.x, kPThreads, lw);
#pragma unroll
      for (int k = 0; k < KL; ++k, lwk.next()) {
        const int c = threadIdx.x + k * kPThreads;
        lv[k] = 0.0;
        li[k] = -1;
        if (c < lh * lw) {
          const int ry = lwk.r, rx = lwk.c;
          int y = y0 - tb + ry, x = x0 - tb + rx;
          if (PERIODIC) {
            y = wrap_into(y, ny);
            x = wrap_into(x, nx);
            lv[k] = __ldcg(src + (int64_t)y * nx + x);
          } else if ((unsigned)y < (unsigned)ny && (unsigned)x < (unsigned)nx) {
            lv[k] = __ldcg(src + (int64_t)y * nx + x);
          }
          li[k] = (off + ry) * RW + off + rx;
        }
      }
#pragma unroll
      for (int k = 0; k < KL; ++k)
        if (li[k] >= 0) buf[0][li[k]] = lv[k];
      __syncthreads();
      int cur = 0;
      for (int s = 1; s <= tb; ++s) {
        const int m = tb - s;  // remaining halo after this step
        const int h = th + 2 * m, w = tw + 2 * m;
        const double* in = buf[cur];
        double* out = buf[cur ^ 1];
        // two cells per thread per pass: two independent FMA chains in flight
        FlatWalk wa(threadIdx.x, 2 * kPThreads, w), wb(threadIdx.x + kPThreads, 2 * kPThreads, w);
        for (int c = threadIdx.x; c < h * w; c += 2 * kPThreads, wa.next(), wb.next()) {
          const int c2 = c + kPThreads;
          const int ry = TB - m + wa.r, rx = TB - m + wa.c;  // buffer coordinates
          const int ry2 = TB - m + wb.r, rx2 = TB - m + wb.c;
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
      // the tile itself back to global memory, then its flag (release: the
      // CTA barrier orders every thread's stores before thread 0's release)
      FlatWalk swk(threadIdx.x, kPThreads, tw);
      for (int c = threadIdx.x; c < th * tw; c += kPThreads, swk.next()) {
        const int ry = swk.r, rx = swk.c;
        dst[(int64_t)(y0 + ry) * nx + x0 + rx] = buf[cur][(TB + ry) * RW + TB + rx];
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        __threadfence();
        asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(L.flags + j), "r"((unsigned int)(blk + 1))
                     : "memory");
      }
    }
  }
  // an odd number of blocks leaves the result in the partner buffer: copy each
  // tile back once every tile that reads it in the last block is done
  if (nblk & 1) {
    for (int j = blockIdx.x; j < ntiles; j += G) {
      const int ty = j / L.tiles_x, tx = j % L.tiles_x;
      const int y0 = cut(ty, ny, L.tiles_y), x0 = cut(tx, nx, L.tiles_x);
      const int th = cut(ty + 1, ny, L.tiles_y) - y0, tw = cut(tx + 1, nx, L.tiles_x) - x0;
      if (!wait_reach<PERIODIC>(L, ty, tx, (unsigned int)nblk)) return;
      for (int c = threadIdx.x; c < th * tw; c += kPThreads) {
        const int64_t k = (int64_t)(y0 + c / tw) * nx + x0 + c % tw;
        L.a[k] = __ldcg(L.b + k);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Batched temporal blocking: the persistent temporal kernel over the tiles of
// many 2D 5-point grids at once (each grid its own weights and T).  A tile of
// an item whose blocks are done sits out; a tile waits only on the tiles of
// its own item that its halo reaches, so items never wait on each other.
static_assert(kBatchTbTileH == kPTH && kBatchTbTileW == kPTW, "tile bounds of the batched temporal kernel");

template <bool PERIODIC, int TB>
__global__ void __launch_bounds__(kPThreads, 2) k_batched_tb(BatchTbLaunch L) {
  constexpr int RW = kPTW + 2 * TB;
  constexpr int RH = kPTH + 2 * TB;
  __shared__ double buf[2][RH * RW];
  const int G = gridDim.x;
  for (int blk = 0; blk < L.max_blocks; ++blk) {
    for (int j = blockIdx.x; j < L.ntiles; j += G) {
      const BatchTbTile tl = L.tiles[j];
      const BatchTbItemDev& it = L.items[tl.item];
      const int ny = it.ny, nx = it.nx, T = it.T;
      if (blk >= (T + TB - 1) / TB) continue;  // this item is done
      const int tb = T - blk * TB < TB ? T - blk * TB : TB;
      const double* src = (blk & 1) ? it.b : it.a;
      double* dst = (blk & 1) ? it.a : it.b;
      const int ty = tl.ty, tx = tl.tx;
      const int y0 = cut(ty, ny, it.tiles_y), x0 = cut(tx, nx, it.tiles_x);
      const int th = cut(ty + 1, ny, it.tiles_y) - y0, tw = cut(tx + 1, nx, it.tiles_x) - x0;
      unsigned int* flags = L.flags + it.tile_base;
      if (blk > 0 && !wait_tiles<PERIODIC>(flags, it.tiles_y, it.tiles_x, it.reach_y, it.reach_x, ty, tx,
                                           (unsigned int)blk, L.status, L.spin_limit))
        return;
      const double w0 = it.w[0], w1 = it.w[1], w2 = it.w[2], w3 = it.w[3], w4 = it.w[4], zero = it.zero;
      // the tile with a halo of tb cells (region offset TB - tb inside the buffer)
      const int off = TB - tb;
      const int lh = th + 2 * tb, lw = tw + 2 * tb;
      FlatWalk lwk(threadIdx.x, kPThreads, lw);
      for (int c = threadIdx.x; c < lh * lw; c += kPThreads, lwk.next()) {
        int y = y0 - tb + lwk.r, x = x0 - tb + lwk.c;
        double v = 0.0;
        if (PERIODIC) {
          y = wrap_into(y, ny);
          x = wrap_into(x, nx);
          v = __ldcg(src + (int64_t)y * nx + x);
        } else if ((unsigned)y < (unsigned)ny && (unsigned)x < (unsigned)nx) {
          v = __ldcg(src + (int64_t)y * nx + x);
        }
        buf[0][(off + lwk.r) * RW + off + lwk.c] = v;
      }
      __syncthreads();
      int cur = 0;
      for (int s = 1; s <= tb; ++s) {
        const int m = tb - s;
        const int h = th + 2 * m, w = tw + 2 * m;
        const double* in = buf[cur];
        double* out = buf[cur ^ 1];
        FlatWalk wk(threadIdx.x, kPThreads, w);
        for (int c = threadIdx.x; c < h * w; c += kPThreads, wk.next()) {
          const int ry = TB - m + wk.r, rx = TB - m + wk.c;
          const int y = y0 - TB + ry, x = x0 - TB + rx;
          double acc = 0.0;  // Dirichlet ghosts stay zero at every time level
          if (PERIODIC || ((unsigned)y < (unsigned)ny && (unsigned)x < (unsigned)nx)) {
            const double* p = in + ry * RW + rx;
            acc = fma(w0, p[-RW], zero);  // north
            acc = fma(w1, p[-1], acc);    // west
            acc = fma(w2, p[0], acc);     // centre
            acc = fma(w3, p[1], acc);     // east
            acc = fma(w4, p[RW], acc);    // south
          }
          out[ry * RW + rx] = acc;
        }
        __syncthreads();
        cur ^= 1;
      }
      FlatWalk swk(threadIdx.x, kPThreads, tw);
      for (int c = threadIdx.x; c < th * tw; c += kPThreads, swk.next())
        dst[(int64_t)(y0 + swk.r) * nx + x0 + swk.c] = buf[cur][(TB + swk.r) * RW + TB + swk.c];
      __syncthreads();
      if (threadIdx.x == 0) {
        __threadfence();
        asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(L.flags + j), "r"((unsigned int)(blk + 1))
                     : "memory");
      }
    }
  }
  // items with an odd number of blocks hold their result in the partner
  // buffer: copy each tile back once the tiles that read it are done
  for (int j = blockIdx.x; j < L.ntiles; j += G) {
    const BatchTbTile tl = L.tiles[j];
    const BatchTbItemDev& it = L.items[tl.item];
    const int nblk = (it.T + TB - 1) / TB;
    if ((nblk & 1) == 0) continue;
    const int ty = tl.ty, tx = tl.tx;
    const int y0 = cut(ty, it.ny, it.tiles_y), x0 = cut(tx, it.nx, it.tiles_x);
    const int th = cut(ty + 1, it.ny, it.tiles_y) - y0, tw = cut(tx + 1, it.nx, it.tiles_x) - x0;
    if (!wait_tiles<PERIODIC>(L.flags + it.tile_base, it.tiles_y, it.tiles_x, it.reach_y, it.reach_x, ty, tx,
                              (unsigned int)nblk, L.status, L.spin_limit))
      return;
    for (int c = threadIdx.x; c < th * tw; c += kPThreads) {
      const int64_t k = (int64_t)(y0 + c / tw) * it.nx + x0 + c % tw;
      it.a[k] = __ldcg(it.b + k);
    }
  }
}

template <bool PERIODIC, int TB>
cudaError_t launch_btb(const BatchTbLaunch& L, int grid_blocks, cudaStream_t stream) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid_blocks, 1, 1);
  cfg.blockDim = dim3(kPThreads, 1, 1);
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelEx(&cfg, k_batched_tb<PERIODIC, TB>, L);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return e;
}

template <bool PERIODIC, int TB>
int btb_occupancy() {
  static std::atomic<int> cache[kMaxDeviceOrdinals];
  return cached_per_device(cache, [] {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batched_tb<PERIODIC, TB>, kPThreads, 0) !=
        cudaSuccess)
      n = 0;
    return n;
  });
}

template <int NT, bool BOX, bool PERIODIC, int TB>
cudaError_t launch_ptb(const PersistTbLaunch& L, int sms, cudaStream_t stream) {
  auto kern = k_persist_tb<NT, BOX, PERIODIC, TB>;
  static std::atomic<int> cache[kMaxDeviceOrdinals];
  const int occ = cached_per_device(cache, [kern] {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, kPThreads, 0) != cudaSuccess) n = 0;
    return n;
  });
  if (occ < 1) return cudaErrorInvalidConfiguration;
  const int tiles = L.tiles_y * L.tiles_x;
  if (L.tiles_y < 1 || L.tiles_x < 1 || (L.ny + L.tiles_y - 1) / L.tiles_y > kPTH ||
      (L.nx + L.tiles_x - 1) / L.tiles_x > kPTW)
    return cudaErrorInvalidValue;
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

void persist_tiling(int ny, int nx, int Tb, int sms, int* tiles_y, int* tiles_x, int* reach_y,
                    int* reach_x) {
  const int ty0 = (ny + kPTH - 1) / kPTH, tx0 = (nx + kPTW - 1) / kPTW;
  long long best = -1;
  int bty = ty0, btx = tx0;
  for (int ty = ty0; ty <= ny && ty <= 3 * ty0 + 8; ++ty)
    for (int tx = tx0; tx <= nx && tx <= 3 * tx0 + 8; ++tx) {
      const long long h = (ny + ty - 1) / ty, w = (nx + tx - 1) / tx;
      long long work = 0;  // cell updates of the largest tile over one block
      for (int m = 0; m < Tb; ++m) work += (h + 2 * m) * (w + 2 * m);
      const long long per_sm = ((long long)ty * tx + sms - 1) / sms;
      const long long cost = per_sm * work;
      if (best < 0 || cost < best || (cost == best && (long long)ty * tx < (long long)bty * btx)) {
        best = cost;
        bty = ty;
        btx = tx;
      }
    }
  *tiles_y = bty;
  *tiles_x = btx;
  const int hmin = ny / bty, wmin = nx / btx;
  *reach_y = (Tb + hmin - 1) / hmin;
  *reach_x = (Tb + wmin - 1) / wmin;
}

cudaError_t launch_persist_tb(Shape shape, int boundary, int Tb, const PersistTbLaunch& L, int sms,
                              cudaStream_t stream) {
  const bool per = boundary == kPeriodic;
  if (shape == Shape::kBox)
    return per ? ptb_by_tb<9, true, true>(Tb, L, sms, stream) : ptb_by_tb<9, true, false>(Tb, L, sms, stream);
  return per ? ptb_by_tb<5, false, true>(Tb, L, sms, stream) : ptb_by_tb<5, false, false>(Tb, L, sms, stream);
}

cudaError_t launch_batched_tb(const BatchTbLaunch& L, int grid_blocks, int Tb, int boundary,
                              cudaStream_t stream) {
  const bool per = boundary == kPeriodic;
  switch (Tb) {
    case 2: return per ? launch_btb<true, 2>(L, grid_blocks, stream) : launch_btb<false, 2>(L, grid_blocks, stream);
    case 4: return per ? launch_btb<true, 4>(L, grid_blocks, stream) : launch_btb<false, 4>(L, grid_blocks, stream);
    case 8: return per ? launch_btb<true, 8>(L, grid_blocks, stream) : launch_btb<false, 8>(L, grid_blocks, stream);
    default: return cudaErrorInvalidValue;
  }
}

int batched_tb_blocks_per_sm(int Tb, int boundary) {
  const bool per = boundary == kPeriodic;
  switch (Tb) {
    case 2: return per ? btb_occupancy<true, 2>() : btb_occupancy<false, 2>();
    case 4: return per ? btb_occupancy<true, 4>() : btb_occupancy<false, 4>();
    case 8: return per ? btb_occupancy<true, 8>() : btb_occupancy<false, 8>();
    default: return 0;
  }
}

int batched_block_size() { return kThreads; }
int batched_default_cpt() { return kDefaultCpt; }
int batched_tile_cells(int cpt) { return cpt * kThreads; }

namespace {
template <int CPT>
cudaError_t launch_batched_cpt(const BatchLaunch& L, int grid_blocks, cudaStream_t stream) {
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
  cudaError_t e = cudaLaunchKernelEx(&cfg, k_batched<CPT>, L);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return e;
}
}  // namespace

cudaError_t launch_batched(const BatchLaunch& L, int grid_blocks, int cpt, cudaStream_t stream) {
  switch (cpt) {
    case 1: return launch_batched_cpt<1>(L, grid_blocks, stream);
    case 2: return launch_batched_cpt<2>(L, grid_blocks, stream);
    case 4: return launch_batched_cpt<4>(L, grid_blocks, stream);
    default: return cudaErrorInvalidValue;
  }
}

// Blocks of k_batched<cpt> that fit on one SM at once (for the cooperative grid size).
int batched_blocks_per_sm(int cpt) {
  int n = 0;
  cudaError_t e = cudaErrorInvalidValue;
  if (cpt == 1) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batched<1>, kThreads, 0);
  if (cpt == 2) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batched<2>, kThreads, 0);
  if (cpt == 4) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batched<4>, kThreads, 0);
  return e == cudaSuccess ? n : 0;
}

}  // namespace gbst
