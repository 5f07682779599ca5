// exchange.cu -- temporal blocking without redundant computation for 3D
// radius-1 stencils (7-point star, 27-point box): Tb time steps per HBM round
// trip, every cell of every intermediate time level computed exactly once.
//
// The paper's tessellate tiling (Sec. 4.1) fuses Tb steps over space-time
// tiles that are computed concurrently "without redundant computation"; its
// overlapped alternative recomputes a halo that grows with Tb.  On this chip
// the FP64 pipe is the bound for every stencil, so a recomputed halo costs its
// share of the roofline one for one (1.20x the work at Tb = 4 and 2.15x at
// Tb = 8 for the 3D overlapped tiles).  Here the tiles do not recompute; they
// hand each other their intermediate time levels through L2:
//
//   - one persistent CTA per tile of the (y, x) plane (64 columns by h rows,
//     h near-equal over the tile rows, h <= 32), all CTAs co-resident
//     (cooperative launch), each streaming its whole z column once.  On a
//     Dirichlet grid whose nx is not a multiple of 64 the last tile column is
//     ragged: its lanes beyond nx read zeros (TMA out-of-bounds fill, the
//     ghost value) and store nothing;
//   - stage s = 1 .. Tb holds time level t+s.  In iteration i stage s computes
//     plane q_s(i) = i + qoff - L(s-1) of its tile from planes q-1, q, q+1 of
//     stage s-1 (the input grid for s = 1); stage s < Tb writes its plane to
//     an L2-resident ring of K planes per stage (the whole plane of the band
//     of rows the launch covers, so neighbouring tiles can read their halo
//     from it), stage Tb writes the
//     output grid.  The stage skew of L >= 2 planes (2; 4 at Tb = 2) means a
//     stage only reads planes written in earlier iterations: unit (i, s)
//     needs unit (i-L+1, s-1);
//   - a consumer thread fences its stores into the async proxy and bumps its
//     warp's shared-memory count of stage s (release) once it has written its
//     share of unit (i, s), s < Tb (the levels other tiles
//     read; stage Tb only writes the output); a publisher warp waits until
//     every warp's count shows unit (i, s) (acquire; per warp, because warps
//     run up to four units apart), fences and publishes the CTA's progress counter
//     of stage s (i+1) with a release store, so neither the consumers nor the
//     producer stall on a GPU-scope fence.  Before unit (i, s), s >= 2, the
//     producer makes sure (one lane: relaxed loads of every stage's counters
//     at once, then an acquire fence; the minimum per stage is kept, so most
//     units need no poll; bounded by wall time) that the CTA itself and every
//     neighbour whose cells the tile's halo touches have published i-L+2 for
//     stage s-1 (the TMA reads its own rows back through L2 too).  A level is
//     published (L-1) Tb units before it is needed (L = 2: units
//     (i-1, s+1 .. Tb) and (i, 1 .. s) lie in between; at Tb = 2 those would
//     be two units only, hence L = 4 there; stage 1 reads the caller's grid,
//     which is prefetched into L2 an iteration ahead), which covers the
//     hand-over;
//   - the producer warp fills a 4-slot shared-memory ring of "stage units"
//     (three planes of tile + halo rows, each one TMA box of its exact height,
//     with x-halo column pairs by 16-byte cp.async through L2) under mbarrier
//     transaction counts; 16 consumer warps compute rows of 64 cells (two adjacent cells
//     per lane, x-neighbours by warp shuffle; a warp takes rows r and r+16
//     together, four FMA chains per lane), rotating rows over the warps from
//     unit to unit, and store with 16-byte st.global.v2 (ring planes with an
//     L2 evict-last policy, the output as streaming stores);
//   - a plane taller than the co-resident tiles cover (at most 32 rows each)
//     is cut into bands of rows, one launch each.  A band carries Tb - 1
//     margin rows toward each neighbouring band: rows it computes but does
//     not write to the output.  The ring holds the band's rows only, and a
//     row beyond the band's edge reads as zero; stage s reads one row further
//     out than stage s - 1 wrote (stage 1 reads the input, which has every
//     row), so the zeros reach at most Tb - 1 rows into the last stage, all
//     of them margin rows;
//   - periodic z: each stage also computes Tb - s extra planes beyond each
//     end of the z column (from wrapped input planes), so no stage needs a
//     plane computed at the other end of the sweep: (Tb-1)/nz of the work
//     (1.4% at 512 planes, Tb = 8).  Dirichlet: planes outside the grid are
//     zero at every level (TMA out-of-bounds fill), nothing extra is computed;
//   - ring slot reuse: plane p of stage s, written in iteration j, is read in
//     iterations j+L-1 .. j+L+1 (by other tiles up to j+L for the star, whose
//     plane q-1 is read at the tile's own cells only; the tile's own reads
//     precede its own later writes) and rewritten in j+K.  Unit (i, s),
//     s >= 2, is posted once every neighbour has finished (i-L+1, s-1), so all
//     of iteration i-L; unit (i, 1) after the wait of the last such unit of
//     iteration i-1, so all of iteration i-L-1: K = 2L+1 planes (star) or
//     2L+2 (box) keep every read ahead of the rewrite (5 / 6 at L = 2, 9 / 10
//     at L = 4).
// Each cell applies its taps in the direct kernel's lexicographic order with
// register-resident weights, so a Tb-fused sweep is bitwise equal to Tb
// single steps.  Every wait is bounded (2 s of wall time): a CTA that gives up
// writes STENCIL_ERR_TIMEOUT to the status word, lets its posted copies land
// and returns; the others see the status word and return too.
#include <cudaTypedefs.h>

#include "internal.h"
#include "ptx.cuh"
#include "taps.cuh"

namespace gbst {

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder();  // stream.cu

namespace {

constexpr int kXW = 64;            // tile width: one warp row of 32 cell pairs
constexpr int kHMax = 32;          // tallest tile
constexpr int kRows = kHMax + 2;   // tile rows and the two y-halo rows
constexpr int kSlots = 4;          // stage units in flight
constexpr int kWarps = 16;         // consumer warps
constexpr int kProducer = kWarps;  // warp that fills the unit ring
constexpr int kPublisher = kWarps + 1;  // warp that publishes the CTA's progress
constexpr int kThreadsX = (kWarps + 2) * 32;
constexpr int kMaps = 5;           // TMA box heights: 1, h_lo, h_lo+1, h_lo+2, h_lo+3 rows
constexpr int kMaxStages = 8;      // largest Tb; progress counters per CTA
constexpr unsigned long long kWaitNs = 2000000000ull;
// Stage skew L in planes: 4 at Tb = 2 (a level is published 3 Tb units
// before it is needed instead of Tb), else 2 (a skew of 3 measured the same
// at Tb = 4 and 8, with a larger ring).
inline int stage_lag(int Tb) { return Tb == 2 ? 4 : 2; }
// Ring planes per stage for skew L (see the slot-reuse rule above).
inline int ring_k(bool box, int lag) { return box ? 2 * lag + 2 : 2 * lag + 1; }

// One stage unit: planes q-1, q, q+1 of the previous stage over the tile's
// rows and the y-halo rows (row r <-> y0 - 1 + r), and the x-halo column
// pairs (x0-2, x0-1) and (x0+64, x0+65) of every row.
struct __align__(1024) XSlot {
  double plane[3][kRows][kXW];
  double2 halo[3][kRows][2];
};
// The copies of one unit that do not change from unit to unit, worked out
// once per launch by the producer warp (it shares its issue slots with FP64
// consumer warps, so per-unit integer work delays the copies).  A segment:
// smem rows r .. r+n-1 from source rows y .. y+n-1, one box of map `map`
// (its exact height), or n one-row boxes of map 0 when map == 0.
struct XSeg {
  int r, y, n, map;
};
// One x-halo pair: slot element dst (double2 index into halo), plane j, the
// source row in the input grid (yin) and in the ring band (yring), column x;
// flags bit 0 / 1: the pair exists in the input / the ring (Dirichlet edges,
// band edges).
struct XHalo {
  int yin, yring, x;
  short dst;
  unsigned char j, flags;
};
constexpr int kSegMax = 4;           // a unit spans at most ny + 2 rows: three segments
constexpr int kHaloMax = 2 * 3 * kRows;

struct XSmem {
  XSlot slot[kSlots];
  uint64_t full[kSlots];
  uint64_t empty[kSlots];
  // per stage s < Tb and consumer warp: lane-units (i, s) written.  Counted per
  // warp: warps run up to kSlots units apart, so a total over the CTA could
  // count one warp's unit (i+1, s) in place of another's (i, s)
  unsigned int done[kMaxStages][kWarps];
  int abort;
  // producer tables: [source: 0 input, 1 ring][rows: 0 = 1 .. h, 1 = 0 .. h+1]
  XSeg seg[2][2][kSegMax];
  int nseg[2][2];
  XHalo hal[kHaloMax];
};
static_assert(sizeof(XSmem) <= 227 * 1024, "the unit ring and tables exceed the shared memory of one CTA");

struct XParams {
  // boxes of 64 columns by 1, h_lo, h_lo+1, h_lo+2 and h_lo+3 rows: every
  // plane of a unit (h or h+2 rows, h in {h_lo, h_lo+1}) is one box, or up to
  // three at a periodic grid's wrap
  CUtensorMap map_in[kMaps];    // the input grid {nx, ny, nz}
  CUtensorMap map_ring[kMaps];  // the ring {nx, ny, K, Tb-1}
  const double* src;
  double* dst;
  double* ring;
  unsigned int* counters;  // [CTA][kMaxStages]: [s] = iterations whose stage s is written
  int* status;
  const double* wdev;
  int nz, ny, nx;
  // the band of rows this launch covers: band row b is grid row yb + b
  // (periodic grids wrap, so yb may be negative), b in [0, nyb); rows
  // [own_lo, own_hi) go to the output, the others are a margin that the
  // neighbouring band owns.  The ring holds band rows; ring_wrap: the band is
  // the whole periodic grid, so band rows wrap too (else a row outside the
  // band reads as zero: only margin rows depend on it)
  int yb, nyb, own_lo, own_hi, ring_wrap;
  int tiles_x, h_lo, h_extra;  // tile row j: h_lo + (j < h_extra) rows
  int tiles_y;
  int Tb, iters, qoff;
  int lag, K;  // stage skew in planes; ring planes per stage
  long long spin_limit;
};

__device__ __forceinline__ int wrapi(int c, int n) {
  int m = c % n;
  return m < 0 ? m + n : m;
}

template <bool BOX>
__device__ __forceinline__ constexpr int tap_at(int dz, int dy, int dx) {
  if (BOX) return ((dz + 1) * 3 + (dy + 1)) * 3 + (dx + 1);
  return dz < 0 ? 0 : dz > 0 ? 6 : dy < 0 ? 1 : dy > 0 ? 5 : 3 + dx;
}

// Range of planes stage s computes.
__device__ __forceinline__ void stage_range(const XParams& P, bool periodic, int s, int& lo, int& hi) {
  if (periodic) {
    lo = -(P.Tb - s);
    hi = P.nz - 1 + (P.Tb - s);
  } else {
    lo = 0;
    hi = P.nz - 1;
  }
}

// Cells (x0 + 2 lane, x0 + 2 lane + 1) of tile rows r[0 .. R) from the unit
// in `sl`: 2R independent FMA chains, interleaved tap by tap.
template <int NT, bool BOX, int R>
__device__ __forceinline__ void unit_rows(const XSlot& sl, const RegWeights<NT>& W, const int (&r)[R], int lane,
                                          double (&a)[R][2]) {
#pragma unroll
  for (int dz = -1; dz <= 1; ++dz) {
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy) {
      if (!BOX && dz != 0 && dy != 0) continue;
      const int j = dz + 1;
      double2 p[R];
#pragma unroll
      for (int k = 0; k < R; ++k) p[k] = *reinterpret_cast<const double2*>(&sl.plane[j][r[k] + 1 + dy][2 * lane]);
      if (BOX || (dz == 0 && dy == 0)) {
        double wv[R], ev[R];
#pragma unroll
        for (int k = 0; k < R; ++k) {
          wv[k] = __shfl_up_sync(0xffffffffu, p[k].y, 1);
          ev[k] = __shfl_down_sync(0xffffffffu, p[k].x, 1);
          if (lane == 0) wv[k] = sl.halo[j][r[k] + 1 + dy][0].y;
          if (lane == 31) ev[k] = sl.halo[j][r[k] + 1 + dy][1].x;
        }
#pragma unroll
        for (int k = 0; k < R; ++k) {
          W.tap(a[k][0], tap_at<BOX>(dz, dy, -1), wv[k], 2 * k);
          W.tap(a[k][1], tap_at<BOX>(dz, dy, -1), p[k].x, 2 * k + 1);
        }
#pragma unroll
        for (int k = 0; k < R; ++k) {
          W.tap(a[k][0], tap_at<BOX>(dz, dy, 0), p[k].x, 2 * k);
          W.tap(a[k][1], tap_at<BOX>(dz, dy, 0), p[k].y, 2 * k + 1);
        }
#pragma unroll
        for (int k = 0; k < R; ++k) {
          W.tap(a[k][0], tap_at<BOX>(dz, dy, 1), p[k].y, 2 * k);
          W.tap(a[k][1], tap_at<BOX>(dz, dy, 1), ev[k], 2 * k + 1);
        }
      } else {
#pragma unroll
        for (int k = 0; k < R; ++k) {
          W.tap(a[k][0], tap_at<BOX>(dz, dy, 0), p[k].x, 2 * k);
          W.tap(a[k][1], tap_at<BOX>(dz, dy, 0), p[k].y, 2 * k + 1);
        }
      }
    }
  }
}

// Waits until every CTA in nb[0 .. nnb) has published `target` for `stage`.
// Lane 0 keeps, in ready[], the smallest counter of every stage over those
// CTAs as last observed and acquired; when that already covers the target
// nothing is read.  Otherwise it polls every stage's counters of every CTA at
// once (relaxed vector loads, one L2 round trip per poll, a short sleep
// between polls so that 150 polling CTAs do not crowd L2), and makes what it
// saw an acquire with a fence; the warp barrier after it orders the other
// lanes' reads behind it.  Returns false (the whole warp) when the wait gave
// up: wall-time limit, or another CTA already reported an error.
__device__ __forceinline__ bool wait_counters(const XParams& P, const int (&nb)[9], int nnb, int stage,
                                              unsigned int target, unsigned int (&ready)[kMaxStages]) {
  int verdict = 0;  // 1 ready, -1 gave up
  if ((threadIdx.x & 31) == 0) {
    if (ready[stage] >= target) {
      verdict = 1;
    } else {
      const unsigned long long t0 = globaltimer_ns();
      for (;;) {
        unsigned int m[kMaxStages];
#pragma unroll
        for (int k = 0; k < kMaxStages; ++k) m[k] = 0xffffffffu;
#pragma unroll
        for (int c = 0; c < 9; ++c) {
          if (c < nnb) {
            const uint4 a = ld_relaxed_gpu_v4(P.counters + nb[c] * kMaxStages);
            const uint4 b = ld_relaxed_gpu_v4(P.counters + nb[c] * kMaxStages + 4);
            m[0] = min(m[0], a.x); m[1] = min(m[1], a.y); m[2] = min(m[2], a.z); m[3] = min(m[3], a.w);
            m[4] = min(m[4], b.x); m[5] = min(m[5], b.y); m[6] = min(m[6], b.z); m[7] = min(m[7], b.w);
          }
        }
        if (m[stage] >= target) {
          fence_acq_rel_gpu();
#pragma unroll
          for (int k = 0; k < kMaxStages; ++k) ready[k] = m[k];
          verdict = 1;
          break;
        }
        if (*(volatile int*)P.status != 0) {
          verdict = -1;
          break;
        }
        if ((long long)(globaltimer_ns() - t0) > P.spin_limit) {
          atomicCAS(P.status, 0, -5 /* STENCIL_ERR_TIMEOUT */);
          verdict = -1;
          break;
        }
        __nanosleep(128);
      }
    }
  }
  verdict = __shfl_sync(0xffffffffu, verdict, 0);
  __syncwarp();
  return verdict > 0;
}

// The segments of smem rows ra .. rb, which hold source rows ytop + ra ..
// ytop + rb (grid rows of the input; band rows of the ring).  With wrap > 0
// those rows wrap modulo wrap (a periodic axis): contiguous segments split
// at the wrap, at most three since a unit spans at most wrap + 2 rows.  Each
// segment is one box of its exact height when the maps have one (and it
// fits the source's `limit` rows), else row by row.  Rows outside a source
// that does not wrap read as zeros (TMA out-of-bounds fill).  Returns the
// count, or -1 if the segments do not fit the table.
__device__ int build_segs(const XParams& P, int ra, int rb, int ytop, int wrap, int limit, XSeg* out) {
  int ns = 0;
  for (int a = ra; a <= rb;) {
    int y = ytop + a;
    int n = rb - a + 1;
    if (wrap > 0) {
      y = wrapi(y, wrap);
      n = min(n, wrap - y);
    }
    if (ns == kSegMax) return -1;
    const int k = n - P.h_lo + 1;  // the box of exactly n rows, if there is one
    const bool whole = n > 1 && k >= 1 && k < kMaps && n <= limit;
    out[ns++] = XSeg{a, y, n, whole ? k : 0};
    a += n;
  }
  return ns;
}

template <int NT, bool BOX, bool PERIODIC>
__global__ void __launch_bounds__(kThreadsX, 1) k_exchange3d(const __grid_constant__ XParams P) {
  const int K = P.K;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  XSmem& S = *reinterpret_cast<XSmem*>(smem_raw);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int tx = blockIdx.x % P.tiles_x, ty = blockIdx.x / P.tiles_x;
  const int x0 = tx * kXW;
  const int yl0 = ty * P.h_lo + min(ty, P.h_extra);  // band row of the tile's first row
  const int y0 = P.yb + yl0;                           // its grid row (periodic margins: may lie outside)
  const int h = P.h_lo + (ty < P.h_extra ? 1 : 0);
  const int Tb = P.Tb;
  if (threadIdx.x == 0) {
    for (int k = 0; k < kSlots; ++k) {
      mbar_init(&S.full[k], 1 + 32);  // expect_tx arrival + one cp.async arrival per producer lane
      mbar_init(&S.empty[k], kWarps);
    }
    for (int k = 0; k < kMaxStages; ++k)
      for (int w = 0; w < kWarps; ++w) S.done[k][w] = 0;
    S.abort = 0;
    fence_mbar_init();
    for (int k = 0; k < kMaps; ++k) {
      prefetch_tmap(&P.map_in[k]);
      prefetch_tmap(&P.map_ring[k]);
    }
  }
  __syncthreads();
  volatile int* abort_flag = &S.abort;

  if (warp == kProducer) {
    // ------------------------------------------------------------ producer
    // this CTA (its own rows of the previous stage are read back by TMA, so
    // they must be visible at GPU scope: the publisher's counter says so) and
    // the CTAs whose cells the halo touches
    int nb[9];
    int nnb = 0;
    nb[nnb++] = blockIdx.x;
    for (int dy = -1; dy <= 1; ++dy) {
      for (int dx = -1; dx <= 1; ++dx) {
        if ((dy == 0 && dx == 0) || (!BOX && dy != 0 && dx != 0)) continue;
        int jy = ty + dy, jx = tx + dx;
        if (PERIODIC) jx = wrapi(jx, P.tiles_x);
        else if (jx < 0 || jx >= P.tiles_x) continue;
        if (P.ring_wrap) jy = wrapi(jy, P.tiles_y);
        else if (jy < 0 || jy >= P.tiles_y) continue;  // the band's edge: no tile beyond it
        nb[nnb++] = jy * P.tiles_x + jx;
      }
    }
    // the unit-invariant part of every copy
    if (lane < 4) {
      const int src = lane >> 1, kind = lane & 1;
      const int ra = kind ? 0 : 1, rb = kind ? h + 1 : h;
      S.nseg[src][kind] = src == 0 ? build_segs(P, ra, rb, y0 - 1, PERIODIC ? P.ny : 0, P.ny, S.seg[0][kind])
                                   : build_segs(P, ra, rb, yl0 - 1, P.ring_wrap ? P.nyb : 0, P.nyb, S.seg[1][kind]);
    }
    // x-halo pairs: box: every plane and row; star: plane q at the tile's rows
    const int nh = 2 * (BOX ? 3 * (h + 2) : h);
    for (int e = lane; e < nh; e += 32) {
      const int side = e & 1;
      const int k = e >> 1;
      const int j = BOX ? k / (h + 2) : 1;
      const int r = BOX ? k % (h + 2) : k + 1;
      int x = side ? x0 + kXW : x0 - 2;
      bool xv = true;
      if (PERIODIC) x = wrapi(x, P.nx);
      else xv = x >= 0 && x < P.nx;
      int yin = y0 - 1 + r, yring = yl0 - 1 + r;
      bool vin = xv, vring = xv;
      if (PERIODIC) yin = wrapi(yin, P.ny);
      else vin = vin && yin >= 0 && yin < P.ny;
      if (P.ring_wrap) yring = wrapi(yring, P.nyb);
      else vring = vring && yring >= 0 && yring < P.nyb;
      S.hal[e] = XHalo{yin, yring, x, (short)((j * kRows + r) * 2 + side), (unsigned char)j,
                       (unsigned char)((vin ? 1 : 0) | (vring ? 2 : 0))};
    }
    // the next input plane's rows for the L2 prefetch of stage-1 units
    const int pf_y = PERIODIC ? wrapi(y0 - 1, P.ny) : y0 - 1;
    const bool pf_whole = (pf_y + h + 2 <= P.ny || !PERIODIC) && h + 2 <= P.ny;
    __syncwarp();
    uint32_t u = 0;
    bool failed = __any_sync(0xffffffffu, lane < 4 && S.nseg[lane >> 1][lane & 1] < 0);
    if (failed && lane == 0) atomicCAS(P.status, 0, -2 /* STENCIL_ERR_UNSUPPORTED */);
    const uint64_t keep = policy_evict_last();
    unsigned int ready[kMaxStages];  // lane 0: acquired minimum of the counters per stage
#pragma unroll
    for (int k = 0; k < kMaxStages; ++k) ready[k] = 0;
    for (int i = 0; i < P.iters && !failed; ++i) {
      for (int s = 1; s <= Tb; ++s) {
        const int q = i + P.qoff - P.lag * (s - 1);
        int lo, hi;
        stage_range(P, PERIODIC, s, lo, hi);
        if (q < lo || q > hi) continue;
        if (s >= 2) {
          // plane q+1 of stage s-1 (iteration i-L+1) is written here and at
          // every neighbour: its counter has reached i-L+2
          const int need = i - P.lag + 2;
          if (need > 0 && !wait_counters(P, nb, nnb, s - 1, (unsigned int)need, ready)) {
            failed = true;
            break;
          }
          fence_proxy_async_global();
        }
        const int slot = u % kSlots;
        const bool free_slot = u < kSlots || mbar_wait_bounded(&S.empty[slot], ((u / kSlots) - 1) & 1, kWaitNs);
        if (!__all_sync(0xffffffffu, free_slot)) {
          if (lane == 0) atomicCAS(P.status, 0, -5 /* STENCIL_ERR_TIMEOUT */);
          failed = true;
          break;
        }
        XSlot& sl = S.slot[slot];
        // rows loaded: the star reads planes q-1 and q+1 only at the tile's
        // own cells; the box reads every plane with its halo rows
        const int rows_side = BOX ? h + 2 : h;
        const int nrows = 2 * rows_side + (h + 2);
        if (lane == 0) mbar_arrive_expect_tx(&S.full[slot], (uint32_t)nrows * kXW * sizeof(double));
        __syncwarp();
        if (s == 1 && lane == 3) {
          // the input plane stage 1 reads next iteration: into L2 now
          const int qn = q + 2;
          if (PERIODIC || (qn >= 0 && qn < P.nz)) {
            const int zn = PERIODIC ? wrapi(qn, P.nz) : qn;
            if (pf_whole) {
              tma_prefetch_3d(&P.map_in[h - P.h_lo + 3], x0, pf_y, zn);  // h + 2 rows
            } else {
              for (int r = 0; r < h + 2; ++r) tma_prefetch_3d(&P.map_in[0], x0, wrapi(y0 - 1 + r, P.ny), zn);
            }
          }
        }
        // planes q-1, q, q+1 of the previous stage: z in the input (s == 1) or
        // ring slot (-1: a plane of zeros outside a Dirichlet grid)
        auto plane_z = [&](int j) {
          const int qq = q - 1 + j;
          const bool exists = PERIODIC || (qq >= 0 && qq < P.nz);
          return s == 1 ? (PERIODIC ? wrapi(qq, P.nz) : qq) : (exists ? wrapi(qq, K) : -1);
        };
        const int z0 = plane_z(0), z1 = plane_z(1), z2 = plane_z(2);
        // (selected, not indexed: a register array indexed by a lane-dependent
        // value would live in local memory)
        auto zsel = [&](int j) { return j == 0 ? z0 : j == 1 ? z1 : z2; };
        if (lane < 3) {
          const int j = lane;
          const int src = s == 1 ? 0 : 1, kind = (BOX || j == 1) ? 1 : 0;
          const int nsg = S.nseg[src][kind];
          for (int g = 0; g < nsg; ++g) {
            const XSeg sg = S.seg[src][kind][g];
            for (int e = 0; e < (sg.map ? 1 : sg.n); ++e) {
              if (s == 1)
                tma_load_3d(&sl.plane[j][sg.r + e][0], &P.map_in[sg.map], x0, sg.y + e, zsel(j), &S.full[slot]);
              else  // ring lines stay in L2 until their slot is rewritten
                tma_load_4d_hint(&sl.plane[j][sg.r + e][0], &P.map_ring[sg.map], x0, sg.y + e, zsel(j), s - 2,
                                 &S.full[slot], keep);
            }
          }
        }
        double2* const hbase = &sl.halo[0][0][0];
        for (int e = lane; e < nh; e += 32) {
          const XHalo t = S.hal[e];
          const int qq = q - 1 + t.j;
          const bool zv = PERIODIC || (qq >= 0 && qq < P.nz);
          if (s == 1) {
            const bool valid = (t.flags & 1) && zv;
            const double* g = valid ? P.src + ((int64_t)zsel(t.j) * P.ny + t.yin) * P.nx + t.x : P.src;
            cp_async16_cg(hbase + t.dst, g, valid);
          } else {
            const bool valid = (t.flags & 2) && zv;
            const double* g =
                valid ? P.ring + (((int64_t)(s - 2) * K + zsel(t.j)) * P.nyb + t.yring) * P.nx + t.x : P.src;
            cp_async16_cg_hint(hbase + t.dst, g, valid, keep);
          }
        }
        cp_async_arrive_noinc(&S.full[slot]);
        ++u;
      }
    }
    if (failed) {
      *abort_flag = 1;
      // let the units already posted land (bounded) before leaving
      for (uint32_t v = u > kSlots ? u - kSlots : 0; v < u; ++v)
        mbar_wait_bounded(&S.full[v % kSlots], (v / kSlots) & 1, kWaitNs);
    }
    return;
  }

  if (warp == kPublisher) {
    // ----------------------------------------------------------- publisher
    // once every consumer thread has written its share of unit (i, s), s < Tb,
    // make those writes visible at GPU scope and publish i+1 for stage s
    if (lane == 0) {
      bool late = false;
      for (int i = 0; i + 1 < P.iters && !late; ++i) {
        for (int s = 1; s < Tb; ++s) {
          const unsigned int need = 32u * (unsigned int)(i + 1);
          const unsigned long long t0 = globaltimer_ns();
          for (int w = 0; w < kWarps && !late; ++w) {
            while (ld_acquire_cta_shared(&S.done[s][w]) < need) {
              if (*abort_flag || (long long)(globaltimer_ns() - t0) > (long long)kWaitNs) {
                late = true;
                break;
              }
              __nanosleep(32);
            }
          }
          if (late) break;
          const int q = i + P.qoff - P.lag * (s - 1);
          int lo, hi;
          stage_range(P, PERIODIC, s, lo, hi);
          if (q >= lo && q <= hi) {  // the unit wrote a plane
            fence_proxy_async_global();
            fence_acq_rel_gpu();
          }
          st_release_gpu(P.counters + blockIdx.x * kMaxStages + s, (unsigned int)(i + 1));
        }
      }
      if (late) {
        if (!*abort_flag) atomicCAS(P.status, 0, -5 /* STENCIL_ERR_TIMEOUT */);
        *abort_flag = 1;
      }
    }
    return;
  }

  // -------------------------------------------------------------- consumers
  RegWeights<NT> W;
  W.load(P.wdev);
  // the ring is re-read within a few iterations: keep its lines in L2; the
  // output is not re-read: streaming stores
  const uint64_t keep = policy_evict_last();
  // this lane's cell pair lies in the grid (a ragged last tile column computes
  // its lanes beyond nx from zeros and stores nothing there)
  const bool xin = x0 + 2 * lane < P.nx;
  uint32_t u = 0;
  int rot = 0;
  for (int i = 0; i < P.iters; ++i) {
    for (int s = 1; s <= Tb; ++s) {
      const int q = i + P.qoff - P.lag * (s - 1);
      int lo, hi;
      stage_range(P, PERIODIC, s, lo, hi);
      if (q < lo || q > hi) {
        if (s < Tb) red_release_cta_shared_add(&S.done[s][warp], 1u);
        continue;
      }
      const int slot = u % kSlots;
      // warp-uniform: every lane leaves together or none does
      if (!__all_sync(0xffffffffu, mbar_wait_bounded(&S.full[slot], (u / kSlots) & 1, kWaitNs))) {
        *abort_flag = 1;
        if (lane == 0) atomicCAS(P.status, 0, -5 /* STENCIL_ERR_TIMEOUT */);
      }
      if (__any_sync(0xffffffffu, *abort_flag != 0)) return;
      const XSlot& sl = S.slot[slot];
      // this warp's rows: r0 and r0 + 16 (tiles have at most 32 rows),
      // computed together (four FMA chains per lane)
      int r0 = warp - rot;
      if (r0 < 0) r0 += kWarps;
      const bool last = s == Tb;
      // stage Tb: the output, grid rows (only the band's own); else the ring, band rows
      // (element offset of the tile's row 0; a margin tile's may be negative
      // in the output, whose rows it does not write)
      const int64_t base = (last ? ((int64_t)q * P.ny + y0) * P.nx
                                 : (((int64_t)(s - 1) * K + wrapi(q, K)) * P.nyb + yl0) * P.nx) +
                           x0 + 2 * lane;
      if (r0 + kWarps < h) {
        const int rr[2] = {r0, r0 + kWarps};
        double a[2][2];
        unit_rows<NT, BOX, 2>(sl, W, rr, lane, a);
        if (xin) {
#pragma unroll
          for (int k = 0; k < 2; ++k) {
            const int64_t off = base + (int64_t)rr[k] * P.nx;
            if (!last) st_global_v2_hint(P.ring + off, a[k][0], a[k][1], keep);
            else if (y0 + rr[k] >= P.own_lo && y0 + rr[k] < P.own_hi) st_global_v2_cs(P.dst + off, a[k][0], a[k][1]);
          }
        }
      } else if (r0 < h) {
        const int rr[1] = {r0};
        double a[1][2];
        unit_rows<NT, BOX, 1>(sl, W, rr, lane, a);
        const int64_t off = base + (int64_t)r0 * P.nx;
        if (!xin) {
        } else if (!last) {
          st_global_v2_hint(P.ring + off, a[0][0], a[0][1], keep);
        } else if (y0 + r0 >= P.own_lo && y0 + r0 < P.own_hi) {
          st_global_v2_cs(P.dst + off, a[0][0], a[0][1]);
        }
      }
      // this thread's share of unit (i, s) is written (stage Tb: the output).
      // Its stores are generic-proxy writes that TMA (the async proxy) reads
      // back: the proxy fence is the writing thread's, before the release
      if (s < Tb) {
        fence_proxy_async_global();
        red_release_cta_shared_add(&S.done[s][warp], 1u);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&S.empty[slot]);
      rot += h % kWarps;
      if (rot >= kWarps) rot -= kWarps;
      ++u;
    }
  }
}

bool encode_in(CUtensorMap* map, const double* base, const Geom& g, int rows) {
  auto enc = tensor_map_encoder();
  if (!enc) return false;
  cuuint64_t dims[3] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz};
  cuuint64_t strides[2] = {(cuuint64_t)g.nx * sizeof(double), (cuuint64_t)g.nx * g.ny * sizeof(double)};
  cuuint32_t box[3] = {(cuuint32_t)kXW, (cuuint32_t)rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, const_cast<double*>(base), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The ring: {nx, band rows, K slots, stages}.
bool encode_ring(CUtensorMap* map, const double* base, int nx, int nyb, int K, int stages, int rows) {
  auto enc = tensor_map_encoder();
  if (!enc) return false;
  cuuint64_t dims[4] = {(cuuint64_t)nx, (cuuint64_t)nyb, (cuuint64_t)K, (cuuint64_t)stages};
  cuuint64_t strides[3] = {(cuuint64_t)nx * sizeof(double), (cuuint64_t)nx * nyb * sizeof(double),
                           (cuuint64_t)K * nx * nyb * sizeof(double)};
  cuuint32_t box[4] = {(cuuint32_t)kXW, (cuuint32_t)rows, 1, 1};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 4, const_cast<double*>(base), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int NT, bool BOX, bool PERIODIC>
int x_occupancy() {
  static std::atomic<int> cache[kMaxDeviceOrdinals];
  return cached_per_device(cache, [] {
    int occ = 0;
    auto kern = k_exchange3d<NT, BOX, PERIODIC>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(XSmem)) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kThreadsX, sizeof(XSmem)) != cudaSuccess)
      occ = 0;
    return occ;
  });
}

template <int NT, bool BOX, bool PERIODIC>
cudaError_t launch_x(const ExchangeLaunch& L, cudaStream_t stream) {
  if (x_occupancy<NT, BOX, PERIODIC>() < 1) return cudaErrorInvalidConfiguration;
  XParams P;
  const Geom& g = L.g;
  const ExchangeBand& b = L.band;
  if (b.tiles_y < 1 || b.rows < 1 || (b.rows + b.tiles_y - 1) / b.tiles_y > kHMax || b.own_lo < 0 ||
      b.own_hi > g.ny || b.own_lo >= b.own_hi || b.own_lo < b.y_base || b.own_hi > b.y_base + b.rows ||
      (b.whole && (b.y_base != 0 || b.rows != g.ny)))
    return cudaErrorInvalidValue;
  const int stages = L.Tb - 1 > 0 ? L.Tb - 1 : 1;
  const int h_lo = b.rows / b.tiles_y;
  for (int k = 0; k < kMaps; ++k) {
    // a box taller than its tensor is never used (the kernel checks n against
    // the grid's rows for the input and the band's rows for the ring)
    const int rows = k == 0 ? 1 : h_lo + k - 1;
    if (!encode_in(&P.map_in[k], L.src, g, rows > g.ny ? 1 : rows) ||
        !encode_ring(&P.map_ring[k], L.ring, g.nx, b.rows, ring_k(BOX, stage_lag(L.Tb)), stages,
                     rows > b.rows ? 1 : rows))
      return cudaErrorInvalidValue;
  }
  P.src = L.src;
  P.dst = L.dst;
  P.ring = L.ring;
  P.counters = L.counters;
  P.status = L.status;
  P.wdev = L.wdev;
  P.nz = g.nz;
  P.ny = g.ny;
  P.nx = g.nx;
  P.yb = b.y_base;
  P.nyb = b.rows;
  P.own_lo = b.own_lo;
  P.own_hi = b.own_hi;
  P.ring_wrap = PERIODIC && b.whole ? 1 : 0;
  P.tiles_x = L.tiles_x;
  P.tiles_y = b.tiles_y;
  P.h_lo = h_lo;
  P.h_extra = b.rows % b.tiles_y;
  P.Tb = L.Tb;
  P.lag = stage_lag(L.Tb);
  P.K = ring_k(BOX, P.lag);
  P.qoff = PERIODIC ? -(L.Tb - 1) : 0;
  // the last stage reaches its last plane (nz - 1, periodic: plus none) in
  // iteration nz - 1 - qoff + lag (Tb - 1)
  P.iters = g.nz - P.qoff + P.lag * (L.Tb - 1);
  P.spin_limit = L.spin_limit;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(L.tiles_x * b.tiles_y), 1, 1);
  cfg.blockDim = dim3(kThreadsX, 1, 1);
  cfg.dynamicSmemBytes = sizeof(XSmem);
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelEx(&cfg, k_exchange3d<NT, BOX, PERIODIC>, P);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return e;
}

}  // namespace

int exchange_tiles_x(const Geom& g) { return (int)((g.nx + kXW - 1) / kXW); }

bool exchange_fits(int ndim, int radius, const Geom& g, bool periodic, int sms) {
  // a ragged last tile column reads zeros beyond nx (TMA out-of-bounds fill),
  // which is the Dirichlet ghost but not the periodic wrap; rows must start
  // on 16 bytes (nx even) for the paired stores
  return ndim == 3 && radius == 1 && g.nx % 2 == 0 && (!periodic || g.nx % kXW == 0) &&
         exchange_tiles_x(g) <= sms && g.ny >= 1 && g.nz >= 1;
}

std::vector<ExchangeBand> exchange_bands(const Geom& g, bool periodic, int Tb, int sms) {
  std::vector<ExchangeBand> out;
  const int tx = exchange_tiles_x(g);
  const int ty_max = sms / tx;                 // tile rows that are co-resident with every column
  const int max_rows = ty_max * kHMax;
  if (g.ny <= max_rows) {
    out.push_back({0, g.ny, 0, g.ny, g.ny < ty_max ? g.ny : ty_max, true});
    return out;
  }
  // interior bands carry a margin of Tb - 1 rows on each side (radius 1:
  // stage s reads rows one further out than stage s-1 wrote; the first stage
  // reads the input, which holds every row)
  const int H = Tb - 1;
  const int room = max_rows - 2 * H;          // owned rows of a band with two margins (>= 18)
  const int nb = (g.ny + room - 1) / room;
  for (int k = 0; k < nb; ++k) {
    const int lo = (int)((int64_t)k * g.ny / nb), hi = (int)((int64_t)(k + 1) * g.ny / nb);
    const int top = periodic || k > 0 ? H : 0, bot = periodic || k < nb - 1 ? H : 0;
    const int rows = hi - lo + top + bot;
    out.push_back({lo - top, rows, lo, hi, rows < ty_max ? rows : ty_max, false});
  }
  return out;
}

int exchange_counter_words(int tiles) { return tiles * kMaxStages; }

size_t exchange_ring_cells(const Geom& g, int Tb, int band_rows) {
  return (size_t)(Tb > 1 ? Tb - 1 : 1) * ring_k(true, stage_lag(Tb)) * (size_t)band_rows * (size_t)g.nx;
}

cudaError_t launch_exchange(Shape shape, int boundary, const ExchangeLaunch& L, cudaStream_t stream) {
  const bool per = boundary == kPeriodic;
  if (L.Tb < 2 || L.Tb > kMaxStages || L.tiles_x < 1 || L.band.tiles_y < 1) return cudaErrorInvalidValue;
  if (shape == Shape::kBox)
    return per ? launch_x<27, true, true>(L, stream) : launch_x<27, true, false>(L, stream);
  return per ? launch_x<7, false, true>(L, stream) : launch_x<7, false, false>(L, stream);
}

}  // namespace gbst
