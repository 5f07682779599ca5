// static_entry.cu -- stencil_run_2d_static: the persistent single-grid 2D sweep
// with all of its scratch in one array reserved when the library is loaded.
//
// Some callers cannot allocate device memory at the point where they want a
// sweep: code whose device memory is entirely owned by another allocator
// (a framework's caching pool that has already reserved most of HBM, so a
// cudaMalloc behind its back fails), and latency-critical loops in which the
// implicit device-wide synchronisation of cudaMalloc / cudaFree is not
// acceptable.  For them this entry point runs the same cooperative persistent
// kernel as the library's persistent path, but its ping-pong partner grid,
// tile list, item descriptor and barrier words live in g_static_scratch below.
//
// Properties the caller relies on:
//   - nothing is allocated: no cudaMalloc / cudaFree / allocating library call;
//   - the array is shared by every call in the process on that GPU and keeps
//     the last call's contents; the barrier words are cleared on the stream
//     before every launch;
//   - calls whose work overlaps on the GPU (different streams, or threads
//     without ordering) race on the array and must be serialised by the caller;
//   - the first call on a device looks up the array's device address
//     (cudaGetSymbolAddress) and the kernel's occupancy with that device
//     current; make that first call before any stream capture begins;
//   - the kernel's device-wide barrier is a bounded wait: if it gives up it
//     writes STENCIL_ERR_TIMEOUT into a status word inside the array, which
//     stencil_static_status reads back (no allocation either).
#include "../../include/stencil.h"
#include "internal.h"

#include <cstdio>
#include <cstring>
#include <mutex>

namespace gbst {
int set_error(int code, const char* msg);  // api.cpp: thread-local message for stencil_last_error
}

using namespace gbst;

namespace {

constexpr int64_t kMaxCells = STENCIL_STATIC_MAX_CELLS;
// Tiles of the persistent kernel are runs of cpt * kBatchThreads consecutive
// cells; sized for the smallest tile (cpt = 1), the list holds the tiles of
// any grid within the limit whatever the kernel's cells per thread.
constexpr int64_t kMaxTiles = kMaxCells / kBatchMinTileCells + 1;
constexpr size_t kPartnerBytes = (size_t)kMaxCells * sizeof(double);
constexpr size_t kItemOff = kPartnerBytes;
constexpr size_t kTileOff = kItemOff + 256;
constexpr size_t kCtlOff = kTileOff + ((kMaxTiles * sizeof(BatchTile) + 255) / 256) * 256;
constexpr size_t kScratchBytes = kCtlOff + 256;

static_assert(sizeof(BatchItemDev) <= 256, "item descriptor slot");

// The reserved scratch: partner grid | item descriptor | tile list | barrier
// words ([0] arrivals, [1] generation, [2] status word of the last launch).
static __device__ __align__(256) unsigned char g_static_scratch[kScratchBytes];

struct DeviceSetup {
  bool ready = false;
  unsigned char* base = nullptr;  // device address of g_static_scratch
  int blocks = 0;                 // cooperative grid size
};
constexpr int kMaxDevices = 64;
DeviceSetup g_setup[kMaxDevices];
std::mutex g_setup_mu;

int sfail(int code, const char* msg) { return set_error(code, msg); }

// The persistent launch over the static scratch: fills the item descriptor and
// tile list for a grid of `cells` cells, clears the barrier words on the
// stream and launches `blocks` (at most the cooperative grid) blocks whose
// device-wide barrier waits for `barrier_blocks` arrivals (0: the launch's own
// block count) for at most `spin_limit_ns`.
int static_launch(const DeviceSetup& s, const BatchItemDev& item, int64_t cells, int boundary,
                  int barrier_blocks, long long spin_limit_ns, cudaStream_t stream);

// Writes the item descriptor and the tile list (runs of `tc` consecutive
// cells -- the persistent kernel's tile) into the static scratch on the device.
__global__ void k_fill_static(BatchItemDev item, BatchItemDev* __restrict__ d_item,
                              BatchTile* __restrict__ d_tiles, int ntiles, int cells, int tc) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < ntiles; j += gridDim.x * blockDim.x) {
    const int k0 = j * tc;
    d_tiles[j] = BatchTile{0, k0, cells - k0 < tc ? cells - k0 : tc};
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *d_item = item;
}

int setup_device(int dev, DeviceSetup& out) {
  std::lock_guard<std::mutex> lock(g_setup_mu);
  DeviceSetup& s = g_setup[dev];
  if (!s.ready) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
    if (e != cudaSuccess) return sfail(STENCIL_ERR_CUDA, "cudaGetSymbolAddress of the static scratch failed");
    int per_sm = batched_blocks_per_sm(batched_default_cpt()), sms = 0;
    if (per_sm < 1 || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return sfail(STENCIL_ERR_CUDA, "querying the persistent kernel's occupancy failed");
    s.base = static_cast<unsigned char*>(ptr);
    s.blocks = sms * (per_sm < 4 ? per_sm : 4);
    s.ready = true;
  }
  out = s;
  return STENCIL_OK;
}

int static_launch(const DeviceSetup& s, const BatchItemDev& item, int64_t cells, int boundary,
                  int barrier_blocks, long long spin_limit_ns, cudaStream_t stream) {
  // the tile list is a pure function of the shape: runs of tc consecutive cells
  const int tc = batched_tile_cells(batched_default_cpt());
  const int64_t ntiles = (cells + tc - 1) / tc;
  if (ntiles > kMaxTiles) return sfail(STENCIL_ERR_UNSUPPORTED, "tile list exceeds the static scratch");
  BatchTile* d_tiles = reinterpret_cast<BatchTile*>(s.base + kTileOff);
  BatchItemDev* d_item = reinterpret_cast<BatchItemDev*>(s.base + kItemOff);
  unsigned int* d_ctl = reinterpret_cast<unsigned int*>(s.base + kCtlOff);
  {
    const int fill_blocks = (int)((ntiles + 255) / 256 < 1024 ? (ntiles + 255) / 256 : 1024);
    k_fill_static<<<fill_blocks, 256, 0, stream>>>(item, d_item, d_tiles, (int)ntiles, (int)cells, tc);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if (cudaGetLastError() != cudaSuccess)
      return sfail(STENCIL_ERR_CUDA, "launching the static scratch fill failed");
  }
  if (cudaMemsetAsync(d_ctl, 0, 4 * sizeof(unsigned int), stream) != cudaSuccess)
    return sfail(STENCIL_ERR_CUDA, "clearing the barrier words failed");
  BatchLaunch L;
  L.items = d_item;
  L.tiles = d_tiles;
  L.ntiles = (int)ntiles;
  L.max_T = item.T;
  L.boundary = boundary;
  L.barrier = d_ctl;
  L.status = reinterpret_cast<int*>(d_ctl + 2);
  L.spin_limit = spin_limit_ns;
  L.barrier_blocks = barrier_blocks;
  int blocks = s.blocks;
  if (ntiles < blocks) blocks = (int)ntiles;
  if (launch_batched(L, blocks, batched_default_cpt(), stream) != cudaSuccess)
    return sfail(STENCIL_ERR_CUDA, "launching the persistent kernel failed");
  return STENCIL_OK;
}

}  // namespace

extern "C" {

int stencil_run_2d_static(int64_t ny, int64_t nx, const double* weights, int boundary,
                          double* d_grid, int64_t T, void* cuda_stream) {
  if (ny < 1 || nx < 1) return sfail(STENCIL_ERR_ARG, "ny and nx must be >= 1");
  if (ny > kMaxCells || nx > kMaxCells || ny * nx > kMaxCells) {
    char buf[160];
    snprintf(buf, sizeof(buf), "a %lld x %lld grid exceeds the static scratch limit of %lld cells",
             (long long)ny, (long long)nx, (long long)kMaxCells);
    return sfail(STENCIL_ERR_UNSUPPORTED, buf);
  }
  if (!weights || !d_grid) return sfail(STENCIL_ERR_ARG, "NULL weights or d_grid");
  if ((uintptr_t)d_grid & 7) return sfail(STENCIL_ERR_ARG, "d_grid is not 8-byte aligned");
  if (boundary != STENCIL_DIRICHLET_ZERO && boundary != STENCIL_PERIODIC)
    return sfail(STENCIL_ERR_ARG, "unknown boundary");
  if (T < 0 || T > (1 << 30)) return sfail(STENCIL_ERR_ARG, "T must be in [0, 2^30]");
  for (int k = 0; k < 9; ++k) {
    if (!(weights[k] - weights[k] == 0.0)) return sfail(STENCIL_ERR_ARG, "weights must be finite");
    if ((k == 0 || k == 2 || k == 6 || k == 8) && weights[k] != 0.0)
      return sfail(STENCIL_ERR_UNSUPPORTED, "only the 5-point star (zero corner weights) is supported");
  }
  if (T == 0) return STENCIL_OK;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return sfail(STENCIL_ERR_CUDA, "no current CUDA device");
  DeviceSetup s;
  int rc = setup_device(dev, s);
  if (rc) return rc;
  cudaStream_t stream = (cudaStream_t)cuda_stream;

  BatchItemDev item;
  memset(&item, 0, sizeof(item));
  item.a = d_grid;
  item.b = reinterpret_cast<double*>(s.base);
  item.ny = (int)ny;
  item.nx = (int)nx;
  item.T = (int)T;
  item.w[0] = weights[1];  // north (y-1)
  item.w[1] = weights[3];  // west (x-1)
  item.w[2] = weights[4];  // centre
  item.w[3] = weights[5];  // east (x+1)
  item.w[4] = weights[7];  // south (y+1)
  return static_launch(s, item, ny * nx, boundary, 0, kSpinLimitNs, stream);
}

int stencil_static_status(void* cuda_stream) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return sfail(STENCIL_ERR_CUDA, "no current CUDA device");
  DeviceSetup s;
  int rc = setup_device(dev, s);
  if (rc) return rc;
  if (cudaStreamSynchronize((cudaStream_t)cuda_stream) != cudaSuccess)
    return sfail(STENCIL_ERR_CUDA, "waiting for the stream failed");
  int* word = reinterpret_cast<int*>(s.base + kCtlOff) + 2;
  int st = 0;
  // a device-to-host copy into a stack variable: no allocation
  if (cudaMemcpy(&st, word, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return sfail(STENCIL_ERR_CUDA, "reading the static status word failed");
  if (st == 0) return STENCIL_OK;
  if (cudaMemset(word, 0, sizeof(int)) != cudaSuccess)
    return sfail(STENCIL_ERR_CUDA, "clearing the static status word failed");
  char buf[128];
  snprintf(buf, sizeof(buf), "the static-scratch sweep reported status %d (a bounded wait gave up)", st);
  return sfail(st, buf);
}

int stencil_selftest_static_timeout(double limit_ms, void* cuda_stream) {
  if (!(limit_ms > 0.0) || limit_ms > 2000.0) return sfail(STENCIL_ERR_ARG, "limit_ms must be in (0, 2000]");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return sfail(STENCIL_ERR_CUDA, "no current CUDA device");
  DeviceSetup s;
  int rc = setup_device(dev, s);
  if (rc) return rc;
  // a 1 x 64 grid inside the static partner region (cells 64 .. 127; the
  // kernel's partner is cells 0 .. 63), advanced by one block whose barrier
  // counts on one block more than the launch has
  double* partner = reinterpret_cast<double*>(s.base);
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  if (cudaMemsetAsync(partner, 0, 128 * sizeof(double), stream) != cudaSuccess)
    return sfail(STENCIL_ERR_CUDA, "clearing the self-test grid failed");
  BatchItemDev item;
  memset(&item, 0, sizeof(item));
  item.a = partner + 64;
  item.b = partner;
  item.ny = 1;
  item.nx = 64;
  item.T = 2;
  item.w[2] = 1.0;
  DeviceSetup one = s;
  one.blocks = 1;
  rc = static_launch(one, item, 64, STENCIL_DIRICHLET_ZERO, 2, (long long)(limit_ms * 1e6), stream);
  if (rc) return rc;
  rc = stencil_static_status(cuda_stream);
  if (rc == STENCIL_ERR_TIMEOUT) return rc;
  if (rc == STENCIL_OK) return sfail(STENCIL_ERR_CUDA, "the bounded wait did not report a timeout");
  return rc;
}

}  // extern "C"
