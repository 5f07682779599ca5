// stream.cu -- 3D radius-1 sweep (7-point star or 27-point box) that streams
// along z through a TMA-fed ring of shared-memory planes.
//
// One step of u'(x) = sum_o w_o u~(x+o) (paper Sec. 2.1, Listing 1).  The
// paper's GPU design keeps a tile in shared memory so that global accesses
// are coalesced (Sec. 4.2, checkerboard blocking); here the tile is a 64 x TY
// (x, y) slab (TY = 32 for the 7-point star, 16 for the 27-point box) that
// advances plane by plane along z:
//   - a 4-slot ring of planes (rows y0-1 .. y0+TY, columns x0 .. x0+63), each
//     filled by three TMA boxes (halo row above, TY rows, halo row below)
//     whose y and z coordinates are wrapped for periodic grids; out-of-range
//     boxes read zeros, which is exactly the Dirichlet-zero ghost rule;
//   - a producer warp posts the TMA boxes and loads the x-halo columns
//     (x0-1 and x0+64) with plain loads, while 8 consumer warps compute; two
//     planes are in flight while a third is computed (mbarrier transaction
//     counts signal arrival, per-slot `empty` barriers release slots);
//   - every lane owns two adjacent x cells (one 16-byte shared load, one
//     16-byte global store); the x-1 / x+2 neighbours come from the adjacent
//     lanes by warp shuffle, the warp's edge lanes take the halo column;
//   - every consumer warp owns rows w, w+8, ...: 4 (box) or 8 (star)
//     independent FMA chains per thread keep the FP64 pipe, the bound of this
//     kernel, busy.
// The taps are applied in the same lexicographic order as the direct sweep,
// starting with an FMA onto zero, so the two kernels agree bitwise.
// Work split: the (tile, z) planes of the grid are cut into equal contiguous
// ranges, one per persistent CTA (a CTA may finish one tile's z-column and
// start the next one's).
#include <cudaTypedefs.h>

#include "internal.h"
#include "ptx.cuh"
#include "taps.cuh"

namespace gbst {

// cuTensorMapEncodeTiled from the driver, fetched once through the runtime's
// entry-point query (no link-time dependency on libcuda).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  // a function-local static: initialised once, thread-safe
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    return nullptr;
  }();
  return fn;
}

namespace {

constexpr int kTX = 64;
constexpr int kSlots = 4;
constexpr int kThreads = 256;

// Tile height TY (8, 16 or 32 rows of 64 columns; a tuning choice).  The
// default: the 7-point star takes 32 rows (4 per warp, 8 FMA chains per
// thread, one barrier per 2048 cells); the 27-point box keeps 16 rows (its 27
// register-resident weights leave room for fewer chains).
template <int TY_>
struct Tile {
  static constexpr int TY = TY_;
  static constexpr int Rows = TY + 2;
  static constexpr int RowsPerWarp = TY / 8;
  static constexpr uint32_t PlaneBytes = Rows * kTX * sizeof(double);
};
template <bool BOX>
constexpr int default_ty() { return BOX ? 16 : 32; }

template <int NT>
struct StreamParams {
  CUtensorMap map_row;   // box {64, 1, 1} over src
  CUtensorMap map_main;  // box {64, TY, 1} over src
  const double* src;
  double* dst;
  int nz, ny, nx;
  int tiles_x, tiles_y;
  long long work;  // tiles * nz plane-tiles
  int* status;
  const double* wdev;  // NT weights then kZeroSlots zeros (device)
  unsigned long long wait_ns;  // limit of every mbarrier wait (2 s; the self-test sets less)
  long long skip_plane;        // self-test only: the producer posts no copy for this plane (-1: none)
};

__device__ __forceinline__ int wrap_or_keep(int c, int n, bool periodic) {
  if (!periodic) return c;
  return c < 0 ? c + n : (c >= n ? c - n : c);
}

template <int NT, int TY, bool PERIODIC, class Smem>
__device__ __forceinline__ void issue_plane(Smem& S, const StreamParams<NT>& P, int slot,
                                            int z, int y0, int x0) {
  constexpr int kRows = Tile<TY>::Rows;
  const int zc = wrap_or_keep(z, P.nz, PERIODIC);
  const int ya = wrap_or_keep(y0 - 1, P.ny, PERIODIC);
  const int yb = wrap_or_keep(y0 + TY, P.ny, PERIODIC);
  mbar_arrive_expect_tx(&S.full[slot], Tile<TY>::PlaneBytes);
  tma_load_3d(&S.plane[slot][0][0], &P.map_row, x0, ya, zc, &S.full[slot]);
  tma_load_3d(&S.plane[slot][1][0], &P.map_main, x0, y0, zc, &S.full[slot]);
  tma_load_3d(&S.plane[slot][kRows - 1][0], &P.map_row, x0, yb, zc, &S.full[slot]);
}

// Tap index of offset (dz, dy, dx) in the lexicographic tap list of the
// shape class (box: all 27; star: the 7 axis offsets).
template <bool BOX>
__device__ __forceinline__ constexpr int tap_index(int dz, int dy, int dx) {
  if (BOX) return ((dz + 1) * 3 + (dy + 1)) * 3 + (dx + 1);
  return dz < 0 ? 0 : dz > 0 ? 6 : dy < 0 ? 1 : dy > 0 ? 5 : 3 + dx;
}

// Two adjacent cells (x, x+1) of tile row ry in the plane whose neighbours are
// in slots (sm, s0, sp).
template <int NT, bool BOX, class Smem>
__device__ __forceinline__ void compute_pair(const Smem& S, const RegWeights<NT>& W, int sm,
                                             int s0, int sp, int ry, int lane, int c0, double& a0,
                                             double& a1) {
  const int slots[3] = {sm, s0, sp};
#pragma unroll
  for (int dz = -1; dz <= 1; ++dz) {
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy) {
      if (!BOX && dz != 0 && dy != 0) continue;
      const int sl = slots[dz + 1];
      const int row = ry + 1 + dy;
      const double2 p = *reinterpret_cast<const double2*>(&S.plane[sl][row][2 * lane]);
      const bool need_x = BOX || (dz == 0 && dy == 0);
      if (need_x) {
        double wv = __shfl_up_sync(0xffffffffu, p.y, 1);
        double ev = __shfl_down_sync(0xffffffffu, p.x, 1);
        if (lane == 0) wv = S.halo[sl][0][row];
        if (lane == 31) ev = S.halo[sl][1][row];
        W.tap(a0, tap_index<BOX>(dz, dy, -1), wv, c0);
        W.tap(a0, tap_index<BOX>(dz, dy, 0), p.x, c0);
        W.tap(a0, tap_index<BOX>(dz, dy, 1), p.y, c0);
        W.tap(a1, tap_index<BOX>(dz, dy, -1), p.x, c0 + 1);
        W.tap(a1, tap_index<BOX>(dz, dy, 0), p.y, c0 + 1);
        W.tap(a1, tap_index<BOX>(dz, dy, 1), ev, c0 + 1);
      } else {
        W.tap(a0, tap_index<BOX>(dz, dy, 0), p.x, c0);
        W.tap(a1, tap_index<BOX>(dz, dy, 0), p.y, c0 + 1);
      }
    }
  }
}

// Warp-specialised form of the same sweep (used for the 7-point star): warp 8
// produces, warps 0..7 consume, and no CTA-wide barrier remains in the loop.
//   - producer: for plane g (slot g % 4) it waits until the 8 consumer warps
//     have released plane g-4 (`empty` mbarrier, 8 arrivals), then lane 0
//     posts the TMA boxes with their byte count and every lane loads part of
//     the x-halo into shared memory and arrives on `full` (1 + 32 arrivals);
//   - consumers: wait on `full` for the planes a step reads, compute, and
//     release plane k-1 with one arrival per warp on `empty`.
template <int TY>
struct __align__(128) WsSmem {
  double plane[kSlots][Tile<TY>::Rows][kTX];
  double halo[kSlots][2][Tile<TY>::Rows];
  uint64_t full[kSlots];
  uint64_t empty[kSlots];
  int abort;
};

template <int NT, bool BOX, bool PERIODIC, int TY>
__global__ void __launch_bounds__(kThreads + 32, BOX ? 2 : 3)
    k_stream3d_ws(const __grid_constant__ StreamParams<NT> P) {
  constexpr int kTY = TY;
  constexpr int kRows = Tile<TY>::Rows;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  WsSmem<TY>& S = *reinterpret_cast<WsSmem<TY>*>(smem_raw);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kSlots; ++s) {
      mbar_init(&S.full[s], 33);
      mbar_init(&S.empty[s], 8);
    }
    S.abort = 0;
    fence_mbar_init();
    prefetch_tmap(&P.map_row);
    prefetch_tmap(&P.map_main);
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
      const int tile = (int)(f / P.nz);
      const int za = (int)(f % P.nz);
      const long long rem = f_end - f;
      const int zb = (long long)P.nz < za + rem ? P.nz : (int)(za + rem);
      f += zb - za;
      const int x0 = (tile % P.tiles_x) * kTX;
      const int y0 = (tile / P.tiles_x) * kTY;
      const int nplanes = zb - za + 2;
      for (int j = 0; j < nplanes; ++j, ++g) {
        const int slot = g % kSlots;
        if (g >= kSlots &&
            !mbar_wait_bounded(&S.empty[slot], ((g - kSlots) / kSlots) & 1, P.wait_ns)) {
          *abort_flag = 1;
          atomicCAS(P.status, 0, -5 /* STENCIL_ERR_TIMEOUT */);
        }
        if (*abort_flag) {
          // let the copies already posted land (bounded), then leave
          for (uint32_t q = g > kSlots ? g - kSlots : 0; q < g; ++q)
            mbar_wait_bounded(&S.full[q % kSlots], (q / kSlots) & 1, P.wait_ns);
          return;
        }
        const int z = za - 1 + j;
        // (the self-test's skipped plane gets neither its copies nor the
        // arrival that announces them: its consumers' wait can only run out)
        if (lane == 0 && (long long)g != P.skip_plane) {
          fence_proxy_async_smem();
          issue_plane<NT, TY, PERIODIC>(S, P, slot, z, y0, x0);
        }
        for (int h = lane; h < 2 * kRows; h += 32) {
          const int side = h / kRows, r = h % kRows;
          int x = side ? x0 + kTX : x0 - 1;
          int y = y0 - 1 + r, zz = z;
          double v = 0.0;
          if (PERIODIC) {
            x = wrap_or_keep(x, P.nx, true);
            y = wrap_or_keep(y, P.ny, true);
            zz = wrap_or_keep(zz, P.nz, true);
            v = __ldg(P.src + ((int64_t)zz * P.ny + y) * P.nx + x);
          } else if ((unsigned)x < (unsigned)P.nx && (unsigned)y < (unsigned)P.ny &&
                     (unsigned)zz < (unsigned)P.nz) {
            v = __ldg(P.src + ((int64_t)zz * P.ny + y) * P.nx + x);
          }
          S.halo[slot][side][r] = v;
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
    const int tile = (int)(f / P.nz);
    const int za = (int)(f % P.nz);
    const long long rem = f_end - f;
    const int zb = (long long)P.nz < za + rem ? P.nz : (int)(za + rem);
    f += zb - za;
    const int x0 = (tile % P.tiles_x) * kTX;
    const int y0 = (tile / P.tiles_x) * kTY;
    const int nplanes = zb - za + 2;
    const uint32_t base = seq;
    seq += nplanes;
    for (int k = 1; k <= nplanes - 2; ++k) {
      const int jfirst = (k == 1) ? 0 : k + 1;
      for (int j = jfirst; j <= k + 1; ++j) {
        const uint32_t gq = base + j;
        if (!mbar_wait_bounded(&S.full[gq % kSlots], (gq / kSlots) & 1, P.wait_ns)) {
          *abort_flag = 1;
          atomicCAS(P.status, 0, -5 /* STENCIL_ERR_TIMEOUT */);
        }
      }
      if (*abort_flag) return;
      const int sm = (base + k - 1) % kSlots, s0 = (base + k) % kSlots, sp = (base + k + 1) % kSlots;
      const int z = za + k - 1;
#pragma unroll
      for (int r = 0; r < Tile<TY>::RowsPerWarp; ++r) {
        const int ry = warp + 8 * r;
        double a0 = 0.0, a1 = 0.0;
        compute_pair<NT, BOX>(S, W, sm, s0, sp, ry, lane, (2 * r) & 3, a0, a1);
        const int y = y0 + ry, x = x0 + 2 * lane;
        if (y < P.ny && x < P.nx) st_global_v2(P.dst + ((int64_t)z * P.ny + y) * P.nx + x, a0, a1);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&S.empty[sm]);  // plane k-1 is not read again
    }
    __syncwarp();
    if (lane == 0) {
      mbar_arrive(&S.empty[(base + nplanes - 2) % kSlots]);
      mbar_arrive(&S.empty[(base + nplanes - 1) % kSlots]);
    }
  }
}

bool encode_3d(CUtensorMap* map, const double* base, int nz, int ny, int nx, int box_y) {
  auto enc = tensor_map_encoder();
  if (!enc) return false;
  cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
  cuuint64_t strides[2] = {(cuuint64_t)nx * sizeof(double), (cuuint64_t)nx * ny * sizeof(double)};
  cuuint32_t box[3] = {(cuuint32_t)kTX, (cuuint32_t)box_y, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, const_cast<double*>(base), dims, strides,
                   box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

template <int TY>
constexpr size_t ws_smem_bytes() { return sizeof(WsSmem<TY>); }

template <int NT, bool BOX, bool PERIODIC, int TY>
int ws_occupancy() {
  static std::atomic<int> cache[kMaxDeviceOrdinals];
  const int n = cached_per_device(cache, [] {
    int occ = 0;
    auto kern = k_stream3d_ws<NT, BOX, PERIODIC, TY>;
    cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ws_smem_bytes<TY>()) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kThreads + 32, ws_smem_bytes<TY>()) !=
            cudaSuccess)
      occ = 0;
    return occ;
  });
  return n;
}

template <int NT, bool BOX, bool PERIODIC, int TY>
cudaError_t launch_t(const Geom& g, const double* wdev, const double* src, double* dst, int* status,
                     int sms, cudaStream_t stream, unsigned long long wait_ns, long long skip_plane) {
  constexpr int kTY = TY;
  StreamParams<NT> P;
  if (!encode_3d(&P.map_row, src, g.nz, g.ny, g.nx, 1) ||
      !encode_3d(&P.map_main, src, g.nz, g.ny, g.nx, kTY))
    return cudaErrorInvalidValue;
  P.src = src;
  P.dst = dst;
  P.nz = g.nz;
  P.ny = g.ny;
  P.nx = g.nx;
  P.tiles_x = (g.nx + kTX - 1) / kTX;
  P.tiles_y = (g.ny + kTY - 1) / kTY;
  P.work = (long long)P.tiles_x * P.tiles_y * g.nz;
  P.status = status;
  P.wdev = wdev;
  P.wait_ns = wait_ns;
  P.skip_plane = skip_plane;
  int occ = ws_occupancy<NT, BOX, PERIODIC, TY>();
  if (occ < 1) return cudaErrorInvalidConfiguration;
  long long grid = (long long)sms * occ;
  if (grid > P.work) grid = P.work;
  k_stream3d_ws<NT, BOX, PERIODIC, TY><<<(unsigned)grid, kThreads + 32, ws_smem_bytes<TY>(), stream>>>(P);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

}  // namespace

int stream3d_tile_y(Shape shape, int tile_y) {
  if (tile_y == 0) return shape == Shape::kBox ? default_ty<true>() : default_ty<false>();
  return (tile_y == 8 || tile_y == 16 || tile_y == 32) ? tile_y : -1;
}

bool stream3d_shape_ok(int ndim, int radius, Shape shape, int boundary, const Geom& g, int tile_y) {
  if (ndim != 3 || radius != 1) return false;
  if (g.nx % 2 != 0) return false;  // TMA: row pitch multiple of 16 bytes
  const int ty = stream3d_tile_y(shape, tile_y);
  if (ty < 0) return false;
  return !(boundary == kPeriodic && (g.nx % kTX != 0 || g.ny % ty != 0));
}

bool stream3d_eligible(int ndim, int radius, Shape shape, int boundary, const Geom& g, const void* a,
                       const void* b, int tile_y) {
  if (!stream3d_shape_ok(ndim, radius, shape, boundary, g, tile_y)) return false;
  if (((uintptr_t)a & 15) || ((uintptr_t)b & 15)) return false;  // TMA base and 16-byte stores
  return tensor_map_encoder() != nullptr;
}

namespace {
template <int NT, bool BOX, bool PERIODIC>
cudaError_t launch_ty(int ty, const Geom& g, const double* wdev, const double* src, double* dst, int* status,
                      int sms, cudaStream_t stream, unsigned long long wait_ns, long long skip_plane) {
  switch (ty) {
    case 8: return launch_t<NT, BOX, PERIODIC, 8>(g, wdev, src, dst, status, sms, stream, wait_ns, skip_plane);
    case 16: return launch_t<NT, BOX, PERIODIC, 16>(g, wdev, src, dst, status, sms, stream, wait_ns, skip_plane);
    case 32: return launch_t<NT, BOX, PERIODIC, 32>(g, wdev, src, dst, status, sms, stream, wait_ns, skip_plane);
    default: return cudaErrorInvalidValue;
  }
}
}  // namespace

cudaError_t launch_stream3d(Shape shape, int boundary, const Geom& g, const HostTaps& taps,
                            const double* wdev, const double* src, double* dst, int* status,
                            int sms, cudaStream_t stream, unsigned long long wait_ns, long long skip_plane,
                            int tile_y) {
  const bool per = boundary == kPeriodic;
  const int ty = stream3d_tile_y(shape, tile_y);
  if (shape == Shape::kBox) {
    if (taps.n != 27) return cudaErrorInvalidValue;
    return per ? launch_ty<27, true, true>(ty, g, wdev, src, dst, status, sms, stream, wait_ns, skip_plane)
               : launch_ty<27, true, false>(ty, g, wdev, src, dst, status, sms, stream, wait_ns, skip_plane);
  }
  if (taps.n != 7) return cudaErrorInvalidValue;
  return per ? launch_ty<7, false, true>(ty, g, wdev, src, dst, status, sms, stream, wait_ns, skip_plane)
             : launch_ty<7, false, false>(ty, g, wdev, src, dst, status, sms, stream, wait_ns, skip_plane);
}

}  // namespace gbst
