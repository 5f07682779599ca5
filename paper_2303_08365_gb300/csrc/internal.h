// internal.h -- declarations shared by the C-ABI layer (api.cpp) and the
// CUDA translation units of the stencil library.  Not installed, not part of
// the ABI; nothing here is visible outside libstencil_gb300.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <vector>

namespace gbst {

// Largest tap set: a radius-2 box in 3D.
constexpr int kMaxTaps = 125;

// Stencil classes the plan recognises from the non-zero pattern of the
// weights.  The class fixes the compile-time tap list of the kernels.
enum class Shape : int {
  kStar = 0,  // taps only on the axes through the centre (2*d*r + 1 taps)
  kBox = 1,   // every offset in [-r, r]^d ((2r+1)^d taps)
};

// Boundary rule (same values as stencil_boundary).
enum Boundary : int { kDirichlet = 0, kPeriodic = 1 };

// Kernel variants selectable through stencil_set_tuning.  Ids are ABI-stable.
enum Variant : int {
  kVariantAuto = 0,
  kVariantDirect = 1,     // one cell per thread per plane, taps from L1
  kVariantStream = 2,     // slowest-axis streaming through a TMA-fed SMEM ring
  kVariantTemporal = 3,   // Tb fused steps per HBM round trip (overlapped tiles)
  kVariantPersistent = 4, // one launch for all steps: barrier per step (Tb 1) or tile flags (Tb > 1)
  kVariantExchange = 5,   // Tb fused steps per launch, 3D, no recompute: tiles hand over levels through L2
  kVariantCount = 6
};

// Tap list for a launch, passed by value (kernel parameter space lives in the
// constant bank, so the weights are constant-bank operands of the FMAs).
template <int NT>
struct TapList {
  double w[NT];
  int8_t dz[NT], dy[NT], dx[NT];
};

// Grid geometry padded to three axes (leading axes of length 1).
struct Geom {
  int nz, ny, nx;
  int64_t cells() const { return (int64_t)nz * ny * nx; }
};

// Host-side description of the taps (any count up to kMaxTaps).
struct HostTaps {
  int n = 0;
  double w[kMaxTaps];
  int8_t dz[kMaxTaps], dy[kMaxTaps], dx[kMaxTaps];
};

// Launchers implemented in the .cu files.  Each returns a cudaError_t from
// the launch (cudaSuccess when nothing failed) and enqueues on `stream`.
// wdev: the plan's weights on the device (taps.n weights in tap order, then
// zero and one slots; see taps.cuh).
cudaError_t launch_direct(int ndim, int radius, Shape shape, int boundary, const Geom& g,
                          const HostTaps& taps, const double* wdev, const double* src, double* dst,
                          cudaStream_t stream);

// FP32 twin of the direct sweep (accuracy studies only; up to 27 taps).
cudaError_t launch_direct_f32(int ndim, int radius, int boundary, const Geom& g, const HostTaps& taps,
                              const float* src, float* dst, cudaStream_t stream);

// 3D radius-1 streaming sweep (TMA-fed shared-memory plane ring) over tiles
// of 64 columns by tile_y rows (8, 16 or 32; 0 = the default: 32 for the
// star, 16 for the box).  Eligible when nx is even, both buffers are 16-byte
// aligned and, for periodic grids, nx % 64 == 0 and ny % tile_y == 0.
bool stream3d_eligible(int ndim, int radius, Shape shape, int boundary, const Geom& g, const void* a,
                       const void* b, int tile_y = 0);
// The shape part of that rule (no buffers, no driver query).
bool stream3d_shape_ok(int ndim, int radius, Shape shape, int boundary, const Geom& g, int tile_y = 0);
// The tile height a tile_y request resolves to (-1: not a supported height).
int stream3d_tile_y(Shape shape, int tile_y);
// wait_ns bounds every mbarrier wait (kSpinLimitNs in normal runs); skip_plane
// >= 0 is the self-test's starved plane (the producer posts no copy for it).
cudaError_t launch_stream3d(Shape shape, int boundary, const Geom& g, const HostTaps& taps,
                            const double* wdev, const double* src, double* dst, int* status,
                            int sms, cudaStream_t stream, unsigned long long wait_ns = 2000000000ull,
                            long long skip_plane = -1, int tile_y = 0);

// 2D radius-1 or radius-2 streaming sweep (TMA-fed ring of 16-row blocks).  Same
// eligibility rules with ny % 16 == 0 for periodic grids.  `equal` selects
// the shared-partial-sum form for a box whose weights are all equal.
bool stream2d_eligible(int ndim, int radius, int boundary, const Geom& g, const void* a,
                       const void* b);
bool stream2d_shape_ok(int ndim, int radius, int boundary, const Geom& g);
bool taps_all_equal(const HostTaps& t);
cudaError_t launch_stream2d(Shape shape, int radius, int boundary, bool equal, const Geom& g,
                            const HostTaps& taps, const double* wdev, const double* src, double* dst,
                            int* status, int sms, cudaStream_t stream);

// Temporal blocking: Tb fused steps per launch (2D and 3D: radius 1, any
// shape and boundary; 1D: radius 1 or 2; Tb in {2, 4, 8}).
bool temporal_supported(int ndim, int radius, int Tb);
// equal: a 2D box whose weights are all equal takes the shared-partial-sum
// form (within rounding of the tap-order kernels, not bitwise equal).
cudaError_t launch_temporal(int ndim, int radius, Shape shape, int boundary, int Tb, const Geom& g,
                            const double* wdev, const double* src, double* dst, int sms,
                            cudaStream_t stream, bool equal = false);

// Temporal blocking without recomputation (3D radius 1, star or box, Tb >= 2):
// one co-resident CTA per 64-column tile of a band of rows of the (y, x)
// plane, intermediate time levels handed between tiles through a ring of
// Tb-1 x K band planes (K = 5 / 6 for the star / box; 9 / 10 at Tb = 2).  A
// plane taller than the co-resident tiles cover (32 rows each) is cut into
// bands, one launch each, every band with a margin of Tb-1 rows toward each
// neighbouring band: the rows its last stage may get wrong at an edge whose
// neighbour rows it does not compute.
struct ExchangeBand {
  int y_base;          // grid row of the band's first row (periodic: may be negative)
  int rows;            // rows of the band, margins included
  int own_lo, own_hi;  // grid rows the band writes to the output
  int tiles_y;         // tile rows (tiles of at most 32 rows)
  bool whole;          // the band is the whole plane (periodic rows wrap within it)
};
struct ExchangeLaunch {
  Geom g;
  const double* src;       // time t (16-byte aligned)
  double* dst;             // time t + Tb (16-byte aligned, not src)
  double* ring;            // exchange_ring_cells(g, Tb, band.rows) doubles
  unsigned int* counters;  // exchange_counter_words(tiles) words, zero before the launch
  int* status;
  const double* wdev;
  int Tb;
  int tiles_x;             // exchange_tiles_x(g): ceil(nx / 64)
  ExchangeBand band;
  long long spin_limit;    // ns
};
// True when the kernel takes the shape: 3D radius 1, nx even (a multiple of
// 64 on a periodic grid), at most `sms` tile columns of 64.
bool exchange_fits(int ndim, int radius, const Geom& g, bool periodic, int sms);
int exchange_tiles_x(const Geom& g);
// The bands of a shape that fits, for `sms` co-resident CTAs and Tb steps.
std::vector<ExchangeBand> exchange_bands(const Geom& g, bool periodic, int Tb, int sms);
size_t exchange_ring_cells(const Geom& g, int Tb, int band_rows);
int exchange_counter_words(int tiles);
cudaError_t launch_exchange(Shape shape, int boundary, const ExchangeLaunch& L, cudaStream_t stream);

// Variable-coefficient diffusion: coefficient preparation, one forward step,
// one fused adjoint step, gradient finalisation and the loss reduction.
struct VarcoefBufs {
  // per-cell coefficients: centre c0 = 1 - sum of face coefficients, and the
  // coefficient of the +x, +y, +z face of each cell (dt * face diffusivity)
  double* c0;
  double* cx;
  double* cy;
  double* cz;
};
cudaError_t launch_varcoef_prepare(int ndim, int boundary, const Geom& g, const double* kappa,
                                   double dt, VarcoefBufs b, cudaStream_t stream);
cudaError_t launch_varcoef_step(int ndim, int boundary, const Geom& g, VarcoefBufs b,
                                const double* src, double* dst, const double* zero,
                                cudaStream_t stream);
// lam_out = A^T lam_in, and for every +face f=(i,n): G_f += (u_n - u_i)(lam_i - lam_n)
// (lam = lam_in = lambda^{t+1}, u = u^t); ghost faces: Gg_i -= k_i * u_i * lam_i
// where k_i is the number of ghost faces of cell i (Dirichlet only).
cudaError_t launch_adjoint_step(int ndim, int boundary, const Geom& g, VarcoefBufs b,
                                const double* lam_in, const double* u, double* lam_out,
                                double* gx, double* gy, double* gz, double* gg, const double* zero,
                                cudaStream_t stream);
// grad_kappa_i = (dt/2) * sum_{faces f of i} G_f + dt * Gg_i
cudaError_t launch_adjoint_finalize(int ndim, int boundary, const Geom& g, double dt,
                                    const double* gx, const double* gy, const double* gz,
                                    const double* gg, double* grad_kappa, cudaStream_t stream);
// lam = u - target, and block partial sums of 0.5*(u - target)^2 into partials
// (nblocks entries); then a single-block pass sums the partials in order.
cudaError_t launch_loss_residual(int64_t n, const double* u, const double* target, double* lam,
                                 double* partials, int nblocks, double* loss_out,
                                 cudaStream_t stream);

// Batched persistent sweep over many 2D heat grids.
struct BatchTile {
  int item;     // index into the item table
  int k0;       // first cell of the tile (row-major index within the item)
  int n;        // cells in the tile (batched_tile_cells(), fewer at an item's end)
};
struct BatchItemDev {
  double* a;     // the caller's grid (time level parity 0)
  double* b;     // library-owned partner buffer (parity 1)
  int ny, nx;
  int T;
  // 5-point star weights in lexicographic tap order: north (y-1), west (x-1),
  // centre, east (x+1), south (y+1); Eq. 3 gives alpha, alpha, 1-4 alpha, alpha, alpha
  double w[5];
  double zero[2];  // 0.0: the addends of the first FMA of each row's chain
};
struct BatchLaunch {
  const BatchItemDev* items;
  const BatchTile* tiles;
  int ntiles;
  int max_T;
  int boundary;
  unsigned int* barrier;  // two words: arrival count, generation
  int* status;            // 0 ok, else a stencil_status
  long long spin_limit;   // bounded waits: wall-time limit in ns
  int barrier_blocks;     // arrivals a device-wide barrier waits for (0: the grid size)
};
// Threads per block of the batched kernel; a tile is cpt * kBatchThreads
// consecutive cells, so the smallest tile (cpt = 1) holds kBatchThreads cells.
constexpr int kBatchThreads = 256;
constexpr int kBatchMinTileCells = kBatchThreads;
// cpt: cells per thread of the kernel (1, 2 or 4); a tile holds cpt * 256 cells.
cudaError_t launch_batched(const BatchLaunch& L, int grid_blocks, int cpt, cudaStream_t stream);
int batched_block_size();
int batched_default_cpt();
int batched_tile_cells(int cpt);
int batched_blocks_per_sm(int cpt);

// Persistent temporal blocking for one small 2D grid (radius 1, star or box):
// Tb in {2, 4, 8} steps per exchange, tiles synchronised by per-tile flags.
struct PersistTbLaunch {
  double* a;             // the caller's grid
  double* b;             // partner buffer
  int ny, nx;
  long long T;
  const double* wdev;    // weights, then the zero and one slots
  int tiles_y, tiles_x;  // near-equal cut of the grid (from persist_tiling)
  int reach_y, reach_x;  // tiles a Tb-cell halo can reach on each side
  unsigned int* flags;   // tiles_y * tiles_x words, zero before the launch
  int* status;
  long long spin_limit;  // ns
};
// Batched temporal blocking: many 2D 5-point heat grids advanced Tb steps in
// shared memory per exchange, one launch, tiles synchronised by per-tile
// flags (each item cut into tiles of at most 16 x 32 cells).
struct BatchTbItemDev {
  double* a;              // the caller's grid
  double* b;              // partner buffer
  int ny, nx, T;
  int tiles_y, tiles_x;   // near-equal cut of the item
  int reach_y, reach_x;   // tiles a Tb-cell halo can reach on each side
  int tile_base;          // the item's first tile (its flag words start there)
  double w[5];            // north, west, centre, east, south (lexicographic taps)
  double zero;            // 0.0, the addend of each chain's first FMA
};
struct BatchTbTile {
  int item, ty, tx;       // tile (ty, tx) of item `item`
};
struct BatchTbLaunch {
  const BatchTbItemDev* items;
  const BatchTbTile* tiles;
  int ntiles;
  int max_blocks;         // the largest ceil(T / Tb) over the items
  unsigned int* flags;    // ntiles words, zero before the launch
  int* status;
  long long spin_limit;   // ns
};
cudaError_t launch_batched_tb(const BatchTbLaunch& L, int grid_blocks, int Tb, int boundary,
                              cudaStream_t stream);
int batched_tb_blocks_per_sm(int Tb, int boundary);
// Largest tile of the batched temporal kernel.
constexpr int kBatchTbTileH = 16, kBatchTbTileW = 32;

// Picks the cut of an ny x nx grid into tiles of at most 16 x 32 cells that
// minimises the FP64 work of the busiest SM for Tb steps per block, and the
// reach of a Tb-cell halo in tiles.
void persist_tiling(int ny, int nx, int Tb, int sms, int* tiles_y, int* tiles_x, int* reach_y, int* reach_x);
cudaError_t launch_persist_tb(Shape shape, int boundary, int Tb, const PersistTbLaunch& L, int sms,
                              cudaStream_t stream);

// FP64 peak microbenchmark: `iters` rounds of 8 independent DFMA chains in
// blocks x 256 threads; out receives one double per thread.
cudaError_t launch_fp64_peak(int blocks, int iters, double* out, cudaStream_t stream);

// Wall-time limit of every bounded device-side wait the host configures
// (barriers of the persistent kernels): 2 s.
constexpr long long kSpinLimitNs = 2000000000LL;

// Launch accounting (every kernel launch of the library adds one).
extern std::atomic<int64_t> g_launches;

// Ordinal of the current device, clamped to [0, kMaxDeviceOrdinals).
constexpr int kMaxDeviceOrdinals = 64;
int device_ordinal();

// Per-device cache of a kernel's launch property (occupancy after its
// attributes are set): `compute` runs on the first call for each device and
// must be idempotent (concurrent first calls may both run it).  `cache` is a
// zero-initialised static array owned by the call site.
template <typename F>
int cached_per_device(std::atomic<int> (&cache)[kMaxDeviceOrdinals], F&& compute) {
  const int dev = device_ordinal();
  int v = cache[dev].load(std::memory_order_acquire);
  if (v == 0) {
    v = compute() + 1;
    cache[dev].store(v, std::memory_order_release);
  }
  return v - 1;
}

}  // namespace gbst
