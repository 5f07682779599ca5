// stream2d.cu -- 2D sweep (radius 1: 5-point star or 9-point box; radius 2:
// 9-point star or 25-point box) that streams along y through a TMA-fed ring
// of row blocks in shared memory.
//
// One step of u'(x) = sum_o w_o u~(x+o) (paper Sec. 2.1, Listing 1; Eq. 3 for
// the heat weights).  A CTA owns a 64-column strip and walks down it in blocks
// of 16 rows.  Shared memory holds a ring of 4 blocks = 64 consecutive rows,
// so the row above / below any row is simply the previous / next ring row;
// one TMA box (16 rows x 64 columns, y wrapped for periodic grids, zeros out
// of range for Dirichlet) fills a block, two blocks are in flight while the
// CTA computes a third.  A producer warp posts the TMA boxes and loads the
// x-halo columns with plain loads; eight consumer warps compute, releasing
// ring slots through per-slot mbarriers (no CTA-wide barrier in the loop).
// Each lane owns two adjacent columns (16-byte shared loads and global
// stores) and exchanges its edge values with the adjacent lanes by shuffle.
//
// Two arithmetic forms:
//   - general weights: the taps in the direct kernel's lexicographic order
//     (the first an FMA onto a register holding 0.0, then FMAs), bitwise
//     equal to it;
//   - equal box weights w (e.g. 1/9): u' = w * sum of the 9 values, with the
//     sums shared between neighbouring cells -- each warp owns two adjacent
//     rows, so the column sums of 3 rows share their middle pair, and the two
//     cells of a lane share the middle pair of the row sum:
//         s  = u[r][c] + u[r+1][c]
//         V[r][c] = u[r-1][c] + s,  V[r+1][c] = s + u[r+2][c]
//         t  = V[x] + V[x+1],  wt = w * t
//         u'[x] = fma(w, V[x-1], wt),  u'[x+1] = fma(w, V[x+2], wt)
//     3.5 FP64 operations per cell instead of 9 (plus the strip-edge columns).
#include <cudaTypedefs.h>

#include "internal.h"
#include "ptx.cuh"
#include "taps.cuh"

namespace gbst {

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder();

namespace {

constexpr int kTX = 64;
constexpr int kRB = 16;             // rows per block
constexpr int kSlots = 4;
constexpr int kRing = kSlots * kRB; // 64 ring rows
constexpr int kThreads = 256;
constexpr unsigned long long kWaitLimitNs = 2000000000ull;
constexpr uint32_t kBlockBytes = kRB * kTX * sizeof(double);

template <int R>
struct __align__(128) Smem2 {
  double row[kRing][kTX];    // TMA destination (block s = rows 16s .. 16s+15)
  double halo[kRing][2 * R]; // columns x0-R .. x0-1 and x0+64 .. x0+63+R of each ring row
  uint64_t full[kSlots];     // TMA bytes + producer arrivals
  uint64_t empty[kSlots];    // one arrival per consumer warp
  int abort;
};

template <int NT>
struct Params2 {
  CUtensorMap map;  // box {64, 16} over src
  const double* src;
  double* dst;
  int ny, nx;
  int strips, blocks;  // per strip: ceil(ny / 16) blocks
  long long work;      // strips * blocks
  int* status;
  const double* wdev;  // NT weights, then the zero and one slots of taps.cuh (device)
};

__device__ __forceinline__ int wrapc(int c, int n) { return c < 0 ? c + n : (c >= n ? c - n : c); }

template <int NT, int R, bool PERIODIC>
__device__ __forceinline__ void issue_block(Smem2<R>& S, const Params2<NT>& P, int slot, int blk,
                                            int x0) {
  int y = blk * kRB;
  if (PERIODIC) y = wrapc(y, P.ny);  // ny % 16 == 0: a block never straddles the edge
  mbar_arrive_expect_tx(&S.full[slot], kBlockBytes);
  tma_load_2d(&S.row[slot * kRB][0], &P.map, x0, y, &S.full[slot]);
}

// Position of offset (dy, dx) in the lexicographic tap list of the shape
// class of radius R (box: all (2R+1)^2; star: the 4R+1 axis offsets).
template <bool BOX, int R>
__device__ __forceinline__ constexpr int tap_index2(int dy, int dx) {
  if (BOX) return (dy + R) * (2 * R + 1) + (dx + R);
  return dy < 0 ? dy + R : dy > 0 ? 3 * R + dy : 2 * R + dx;
}

// General weights: cells (x, x+1) of ring row q.  A row's values x-R ..
// x+1+R come from the lane's own pair and the adjacent lanes' pairs by
// shuffle (each lane holds two columns, so R <= 2 reaches one lane away);
// the warp's edge lanes take the halo columns instead.
template <int NT, bool BOX, int R>
__device__ __forceinline__ void pair_general(const Smem2<R>& S, const RegWeights<NT>& W, int q, int lane,
                                             int c0, double& a0, double& a1) {
#pragma unroll
  for (int dy = -R; dy <= R; ++dy) {
    const int rr = (q + dy + kRing) % kRing;
    const double2 p = *reinterpret_cast<const double2*>(&S.row[rr][2 * lane]);
    if (BOX || dy == 0) {
      double v[2 * R + 2];  // columns x-R .. x+1+R
      const double lx = __shfl_up_sync(0xffffffffu, p.x, 1), ly = __shfl_up_sync(0xffffffffu, p.y, 1);
      const double rx = __shfl_down_sync(0xffffffffu, p.x, 1), ry = __shfl_down_sync(0xffffffffu, p.y, 1);
      if (R == 2) {
        v[0] = lane == 0 ? S.halo[rr][0] : lx;
        v[1] = lane == 0 ? S.halo[rr][1] : ly;
        v[4] = lane == 31 ? S.halo[rr][2] : rx;
        v[5] = lane == 31 ? S.halo[rr][3] : ry;
      } else {
        v[0] = lane == 0 ? S.halo[rr][0] : ly;
        v[2 * R + 1] = lane == 31 ? S.halo[rr][1] : rx;
      }
      v[R] = p.x;
      v[R + 1] = p.y;
#pragma unroll
      for (int dx = -R; dx <= R; ++dx) W.tap(a0, tap_index2<BOX, R>(dy, dx), v[R + dx], c0);
#pragma unroll
      for (int dx = -R; dx <= R; ++dx) W.tap(a1, tap_index2<BOX, R>(dy, dx), v[R + 1 + dx], c0 + 1);
    } else {
      W.tap(a0, tap_index2<BOX, R>(dy, 0), p.x, c0);
      W.tap(a1, tap_index2<BOX, R>(dy, 0), p.y, c0 + 1);
    }
  }
}

// Equal weights: rows q and q+1 (cells x, x+1 of each).  out[row][cell].
// Every addition is an FMA against a register holding 1.0 (same rounding,
// full FP64 rate); the common weight comes from the register copies W.w[k].
template <int NT>
__device__ __forceinline__ void quad_equal(const Smem2<1>& S, const RegWeights<NT>& W, int q, int lane,
                                           double out[2][2]) {
  const int qm = (q - 1 + kRing) % kRing, q1 = (q + 1) % kRing, q2 = (q + 2) % kRing;
  const double2 a = *reinterpret_cast<const double2*>(&S.row[qm][2 * lane]);
  const double2 b = *reinterpret_cast<const double2*>(&S.row[q][2 * lane]);
  const double2 c = *reinterpret_cast<const double2*>(&S.row[q1][2 * lane]);
  const double2 d = *reinterpret_cast<const double2*>(&S.row[q2][2 * lane]);
  // column sums of 3 rows for the lane's two columns, rows q and q+1
  const double s0 = W.add(b.x, c.x, 0), s1 = W.add(b.y, c.y, 1);
  const double V00 = W.add(a.x, s0, 2), V01 = W.add(a.y, s1, 3);   // row q, columns x, x+1
  const double V10 = W.add(s0, d.x, 0), V11 = W.add(s1, d.y, 1);   // row q+1
  // column sums at the strip-edge columns (lanes 0 and 31 only)
  double H0 = 0.0, H1 = 0.0;
  if (lane == 0 || lane == 31) {
    const int side = lane == 0 ? 0 : 1;
    const double hs = W.add(S.halo[q][side], S.halo[q1][side], 2);
    H0 = W.add(S.halo[qm][side], hs, 3);
    H1 = W.add(hs, S.halo[q2][side], 0);
  }
  // neighbours' column sums: x-1 from the lane below, x+2 from the lane above
  double L0 = __shfl_up_sync(0xffffffffu, V01, 1), L1 = __shfl_up_sync(0xffffffffu, V11, 1);
  double R0 = __shfl_down_sync(0xffffffffu, V00, 1), R1 = __shfl_down_sync(0xffffffffu, V10, 1);
  if (lane == 0) { L0 = H0; L1 = H1; }
  if (lane == 31) { R0 = H0; R1 = H1; }
  const double wt0 = fma(W.w[0], W.add(V00, V01, 2), W.z[0]);
  const double wt1 = fma(W.w[1], W.add(V10, V11, 3), W.z[1]);
  out[0][0] = fma(W.w[2], L0, wt0);
  out[0][1] = fma(W.w[3], R0, wt0);
  out[1][0] = fma(W.w[4], L1, wt1);
  out[1][1] = fma(W.w[5], R1, wt1);
}

// Warp-specialised: warp 8 produces (waits for the consumers to release
// block g-4 on the slot's `empty` barrier, posts the TMA box with its byte
// count, loads its part of the x-halo columns, arrives on `full`); warps 0..7
// consume (wait on `full` for the blocks a step reads, compute, release block
// k-1 with one arrival per warp).  No CTA-wide barrier in the loop.
template <int NT, bool BOX, int R, bool PERIODIC, bool EQUAL>
__global__ void __launch_bounds__(kThreads + 32, 2) k_stream2d(const __grid_constant__ Params2<NT> P) {
  __shared__ Smem2<R> S;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kSlots; ++s) {
      mbar_init(&S.full[s], 33);
      mbar_init(&S.empty[s], 8);
    }
    S.abort = 0;
    fence_mbar_init();
    prefetch_tmap(&P.map);
  }
  __syncthreads();
  const long long G = gridDim.x;
  const long long f_begin = P.work * blockIdx.x / G;
  const long long f_end = P.work * (blockIdx.x + 1) / G;
  volatile int* abort_flag = &S.abort;

  if (warp == 8) {
    // ------------------------------------------------------------ producer
    uint32_t g = 0;
    for (long long f = f_begin; f < f_end;) {
      const int strip = (int)(f / P.blocks);
      const int ba = (int)(f % P.blocks);
      const long long rem = f_end - f;
      const int bb = (long long)P.blocks < ba + rem ? P.blocks : (int)(ba + rem);
      f += bb - ba;
      const int x0 = strip * kTX;
      const int nblk = bb - ba + 2;
      for (int j = 0; j < nblk; ++j, ++g) {
        const int slot = g % kSlots;
        if (g >= kSlots &&
            !mbar_wait_bounded(&S.empty[slot], ((g - kSlots) / kSlots) & 1, kWaitLimitNs)) {
          *abort_flag = 1;
          atomicCAS(P.status, 0, -5 /* STENCIL_ERR_TIMEOUT */);
        }
        if (*abort_flag) {
          for (uint32_t q = g > kSlots ? g - kSlots : 0; q < g; ++q)
            mbar_wait_bounded(&S.full[q % kSlots], (q / kSlots) & 1, kWaitLimitNs);
          return;
        }
        const int blk = ba - 1 + j;
        if (lane == 0) {
          fence_proxy_async_smem();
          issue_block<NT, R, PERIODIC>(S, P, slot, blk, x0);
        }
        for (int t = lane; t < 2 * R * kRB; t += 32) {
          const int h = t / kRB, r = t % kRB;
          int x = h < R ? x0 - R + h : x0 + kTX + (h - R);
          int y = blk * kRB + r;
          double v = 0.0;
          if (PERIODIC) {
            x = wrapc(x, P.nx);
            y = wrapc(y, P.ny);
            v = __ldg(P.src + (int64_t)y * P.nx + x);
          } else if ((unsigned)x < (unsigned)P.nx && (unsigned)y < (unsigned)P.ny) {
            v = __ldg(P.src + (int64_t)y * P.nx + x);
          }
          S.halo[slot * kRB + r][h] = v;
        }
        mbar_arrive(&S.full[slot]);
      }
    }
    return;
  }

  // -------------------------------------------------------------- consumers
  RegWeights<NT> W;
  W.load(P.wdev);
  uint32_t seq = 0;
  for (long long f = f_begin; f < f_end;) {
    const int strip = (int)(f / P.blocks);
    const int ba = (int)(f % P.blocks);
    const long long rem = f_end - f;
    const int bb = (long long)P.blocks < ba + rem ? P.blocks : (int)(ba + rem);
    f += bb - ba;
    const int x0 = strip * kTX;
    const int nblk = bb - ba + 2;  // blocks ba-1 .. bb
    const uint32_t base = seq;
    seq += nblk;
    for (int k = 1; k <= nblk - 2; ++k) {
      const int jfirst = (k == 1) ? 0 : k + 1;
      for (int j = jfirst; j <= k + 1; ++j) {
        const uint32_t gq = base + j;
        if (!mbar_wait_bounded(&S.full[gq % kSlots], (gq / kSlots) & 1, kWaitLimitNs)) {
          *abort_flag = 1;
          atomicCAS(P.status, 0, -5 /* STENCIL_ERR_TIMEOUT */);
        }
      }
      if (*abort_flag) return;
      const int slot = (base + k) % kSlots;
      const int blk = ba + k - 1;
      const int x = x0 + 2 * lane;
      if (EQUAL) {
        const int r = 2 * warp;  // rows r, r+1 of the block
        double out[2][2];
        if constexpr (R == 1) quad_equal<NT>(S, W, slot * kRB + r, lane, out);
#pragma unroll
        for (int i = 0; i < 2; ++i) {
          const int y = blk * kRB + r + i;
          if (y < P.ny && x < P.nx) st_global_v2(P.dst + (int64_t)y * P.nx + x, out[i][0], out[i][1]);
        }
      } else {
#pragma unroll
        for (int i = 0; i < 2; ++i) {
          const int r = warp + 8 * i;
          double a0 = 0.0, a1 = 0.0;
          pair_general<NT, BOX, R>(S, W, slot * kRB + r, lane, 2 * i, a0, a1);
          const int y = blk * kRB + r;
          if (y < P.ny && x < P.nx) st_global_v2(P.dst + (int64_t)y * P.nx + x, a0, a1);
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&S.empty[(base + k - 1) % kSlots]);  // block k-1 is not read again
    }
    __syncwarp();
    if (lane == 0) {
      mbar_arrive(&S.empty[(base + nblk - 2) % kSlots]);
      mbar_arrive(&S.empty[(base + nblk - 1) % kSlots]);
    }
  }
}

bool encode_2d(CUtensorMap* map, const double* base, int ny, int nx) {
  auto enc = tensor_map_encoder();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)nx, (cuuint64_t)ny};
  cuuint64_t strides[1] = {(cuuint64_t)nx * sizeof(double)};
  cuuint32_t box[2] = {(cuuint32_t)kTX, (cuuint32_t)kRB};
  cuuint32_t estr[2] = {1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<double*>(base), dims, strides, box,
             estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int NT, bool BOX, int R, bool PERIODIC, bool EQUAL>
cudaError_t launch2(const Geom& g, const double* wdev, const double* src, double* dst, int* status,
                    int sms, cudaStream_t stream) {
  Params2<NT> P;
  if (!encode_2d(&P.map, src, g.ny, g.nx)) return cudaErrorInvalidValue;
  P.src = src;
  P.dst = dst;
  P.ny = g.ny;
  P.nx = g.nx;
  P.strips = (g.nx + kTX - 1) / kTX;
  P.blocks = (g.ny + kRB - 1) / kRB;
  P.work = (long long)P.strips * P.blocks;
  P.status = status;
  P.wdev = wdev;
  static std::atomic<int> cache[kMaxDeviceOrdinals];
  const int occ = cached_per_device(cache, [] {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_stream2d<NT, BOX, R, PERIODIC, EQUAL>,
                                                      kThreads + 32, 0) != cudaSuccess)
      n = 0;
    return n;
  });
  if (occ < 1) return cudaErrorInvalidConfiguration;
  long long grid = (long long)sms * occ;
  if (grid > P.work) grid = P.work;
  k_stream2d<NT, BOX, R, PERIODIC, EQUAL><<<(unsigned)grid, kThreads + 32, 0, stream>>>(P);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

}  // namespace

bool stream2d_shape_ok(int ndim, int radius, int boundary, const Geom& g) {
  if (ndim != 2 || (radius != 1 && radius != 2)) return false;
  if (g.nx % 2 != 0) return false;
  return !(boundary == kPeriodic && (g.nx % kTX != 0 || g.ny % kRB != 0));
}

bool stream2d_eligible(int ndim, int radius, int boundary, const Geom& g, const void* a,
                       const void* b) {
  if (!stream2d_shape_ok(ndim, radius, boundary, g)) return false;
  if (((uintptr_t)a & 15) || ((uintptr_t)b & 15)) return false;
  return tensor_map_encoder() != nullptr;
}

bool taps_all_equal(const HostTaps& t) {
  for (int k = 1; k < t.n; ++k)
    if (t.w[k] != t.w[0]) return false;
  return t.n > 0;
}

cudaError_t launch_stream2d(Shape shape, int radius, int boundary, bool equal, const Geom& g,
                            const HostTaps& taps, const double* wdev, const double* src, double* dst,
                            int* status, int sms, cudaStream_t stream) {
  const bool per = boundary == kPeriodic;
  if (radius == 2) {
    if (shape == Shape::kBox) {
      if (taps.n != 25) return cudaErrorInvalidValue;
      return per ? launch2<25, true, 2, true, false>(g, wdev, src, dst, status, sms, stream)
                 : launch2<25, true, 2, false, false>(g, wdev, src, dst, status, sms, stream);
    }
    if (taps.n != 9) return cudaErrorInvalidValue;
    return per ? launch2<9, false, 2, true, false>(g, wdev, src, dst, status, sms, stream)
               : launch2<9, false, 2, false, false>(g, wdev, src, dst, status, sms, stream);
  }
  if (shape == Shape::kBox) {
    if (taps.n != 9) return cudaErrorInvalidValue;
    if (equal)
      return per ? launch2<9, true, 1, true, true>(g, wdev, src, dst, status, sms, stream)
                 : launch2<9, true, 1, false, true>(g, wdev, src, dst, status, sms, stream);
    return per ? launch2<9, true, 1, true, false>(g, wdev, src, dst, status, sms, stream)
               : launch2<9, true, 1, false, false>(g, wdev, src, dst, status, sms, stream);
  }
  if (taps.n != 5) return cudaErrorInvalidValue;
  return per ? launch2<5, false, 1, true, false>(g, wdev, src, dst, status, sms, stream)
             : launch2<5, false, 1, false, false>(g, wdev, src, dst, status, sms, stream);
}

}  // namespace gbst
