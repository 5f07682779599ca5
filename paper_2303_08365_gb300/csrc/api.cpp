// api.cpp -- the C ABI of include/stencil.h: argument checks, plans, buffer
// ownership, kernel selection and the host loops over time steps.
#include "../../include/stencil.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "internal.h"
#include "taps.cuh"

namespace gbst {
std::atomic<int64_t> g_launches{0};
int set_error(int code, const char* msg);
}  // namespace gbst

using namespace gbst;

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  int code = (e == cudaErrorMemoryAllocation) ? STENCIL_ERR_OOM : STENCIL_ERR_CUDA;
  return fail(code, "%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
}

#define CUDA_TRY(call, what)                  \
  do {                                        \
    cudaError_t e_ = (call);                  \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

// Host-side fault injection for tests (stencil_debug_fail_allocations): when
// g_fail_after >= 0, that many more device allocations succeed and the next
// one reports cudaErrorMemoryAllocation without calling the driver.
std::atomic<int> g_fail_after{-1};

cudaError_t dev_malloc(void** ptr, size_t bytes) {
  int left = g_fail_after.load();
  while (left >= 0) {
    if (left == 0) {
      *ptr = nullptr;
      return cudaErrorMemoryAllocation;
    }
    if (g_fail_after.compare_exchange_weak(left, left - 1)) break;
  }
  return cudaMalloc(ptr, bytes);
}
template <typename T>
cudaError_t dev_malloc(T** ptr, size_t bytes) {
  return dev_malloc(reinterpret_cast<void**>(ptr), bytes);
}

bool is_finite(double v) { return std::isfinite(v); }

// Pads a shape to three axes; rejects axes beyond the kernels' 32-bit indexing.
int make_geom(int ndim, const int64_t* dims, Geom& g) {
  if (ndim < 1 || ndim > 3) return fail(STENCIL_ERR_ARG, "ndim must be 1, 2 or 3 (got %d)", ndim);
  if (!dims) return fail(STENCIL_ERR_ARG, "dims is NULL");
  int64_t n[3] = {1, 1, 1};
  for (int d = 0; d < ndim; ++d) {
    if (dims[d] < 1) return fail(STENCIL_ERR_ARG, "dims[%d] = %lld < 1", d, (long long)dims[d]);
    if (dims[d] > (int64_t)1 << 30)
      return fail(STENCIL_ERR_UNSUPPORTED, "dims[%d] = %lld exceeds 2^30", d, (long long)dims[d]);
    n[3 - ndim + d] = dims[d];
  }
  if (n[0] > 65535) return fail(STENCIL_ERR_UNSUPPORTED, "slowest axis of a 3D grid exceeds 65535");
  if (n[1] > 65535 * 8) return fail(STENCIL_ERR_UNSUPPORTED, "second-slowest axis exceeds 524280");
  g.nz = (int)n[0];
  g.ny = (int)n[1];
  g.nx = (int)n[2];
  return STENCIL_OK;
}

}  // namespace

int gbst::device_ordinal() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDeviceOrdinals) dev = 0;
  return dev;
}

// Lets other translation units report through stencil_last_error.
int gbst::set_error(int code, const char* msg) {
  g_err = msg ? msg : "";
  return code;
}

constexpr int kPersistCache = 8;

struct stencil_plan_s {
  int ndim = 0;
  Geom g{1, 1, 1};
  int radius = 0;
  int boundary = 0;
  bool varcoef = false;
  Shape shape = Shape::kStar;
  HostTaps taps;
  // library-owned device buffers
  double* d_tmp = nullptr;     // ping-pong partner of the caller's grid
  double* d_stage = nullptr;   // host-entry staging (grid, then kappa)
  double* d_coef = nullptr;    // varcoef: c0, cx, cy, cz (4 x cells)
  double* d_adj = nullptr;     // adjoint scratch
  size_t adj_cells = 0;
  int* d_status = nullptr;     // device status word (bounded waits that gave up)
  unsigned int* d_flags = nullptr;  // per-tile flags of the persistent temporal kernel
  int flags_cap = 0;
  double* d_ring = nullptr;         // exchange kernel: ring of intermediate time levels
  size_t ring_cells = 0;
  unsigned int* d_xcnt = nullptr;   // exchange kernel: per-CTA progress counters
  int xcnt_cap = 0;
  double* d_w = nullptr;       // weights in tap order, then kZeroSlots zeros and kOneSlots ones
  // one-item batches of the one-step persistent path, one per (grid, T) the
  // plan has run recently (least recently used evicted beyond kPersistCache):
  // a CUDA graph captured around a run keeps using its entry's buffers
  struct PersistEntry {
    const double* grid;
    int64_t T;
    stencil_batch_s* batch;
    uint64_t last_use;
  };
  std::vector<PersistEntry> persist;
  uint64_t persist_clock = 0;
  // tuning
  int user_Tb = 0, user_variant = 0;
  int tuned_Tb = 0, tuned_variant = 0;
  int user_tile_y = 0, tuned_tile_y = 0;  // streaming kernel's tile height (0: its default)

  int64_t cells() const { return g.cells(); }
};

struct stencil_batch_s {
  int n = 0;
  int boundary = 0;
  std::vector<stencil_batch_item> items;
  BatchItemDev* d_items = nullptr;
  BatchTile* d_tiles = nullptr;
  double* d_partner = nullptr;
  unsigned int* d_ctl = nullptr;  // [0] arrivals, [1] generation, [2] status
  int ntiles = 0;
  int max_T = 0;
  int blocks = 0;
  int64_t updates = 0;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t capture_stream = nullptr;
  cudaStream_t last_stream = nullptr;
  bool use_graph = true;
  // kernel configuration (stencil_batch_set_tuning / stencil_batch_autotune)
  int Tb = 1;              // 1: one step per device-wide barrier; 2, 4, 8: Tb steps per exchange
  int cpt = 0;             // cells per thread (1, 2, 4; Tb = 1 only); 0 = the default
  int per_sm = 0;          // cooperative blocks per SM (Tb = 1 only); 0 = min(occupancy, 4)
  // Tb > 1: per-item tiles and per-tile flags of the batched temporal kernel
  BatchTbItemDev* d_tb_items = nullptr;
  BatchTbTile* d_tb_tiles = nullptr;
  unsigned int* d_tb_flags = nullptr;
  int ntb_tiles = 0;
  int tb_max_blocks = 0;
  std::vector<BatchItemDev> hi;  // the item descriptors, kept to rebuild the tile list
  bool ready = false;      // the work list is complete (the last build succeeded)
};

namespace {

int batch_init(stencil_batch_s* b, const std::vector<BatchItemDev>& hi, int boundary);
int batch_enqueue(stencil_batch_s* b, cudaStream_t s);

// Builds the compile-time tap list of the plan's shape class: every offset of
// the class in lexicographic order (slowest axis first), with its weight
// (possibly zero) from the dense array.
void build_taps(stencil_plan_s* p, const double* w) {
  const int r = p->radius, side = 2 * r + 1, nd = p->ndim;
  int64_t total = 1;
  for (int d = 0; d < nd; ++d) total *= side;
  p->taps.n = 0;
  for (int64_t k = 0; k < total; ++k) {
    int off[3] = {0, 0, 0};
    int64_t rem = k;
    for (int d = nd - 1; d >= 0; --d) {
      off[3 - nd + d] = (int)(rem % side) - r;
      rem /= side;
    }
    int nonzero_axes = (off[0] != 0) + (off[1] != 0) + (off[2] != 0);
    if (p->shape == Shape::kStar && nonzero_axes > 1) continue;
    int i = p->taps.n++;
    p->taps.w[i] = w[k];
    p->taps.dz[i] = (int8_t)off[0];
    p->taps.dy[i] = (int8_t)off[1];
    p->taps.dx[i] = (int8_t)off[2];
  }
}

std::string device_name();

std::string plan_key(const stencil_plan_s* p) {
  char buf[256];
  bool equal = p->shape == Shape::kBox;
  for (int k = 1; equal && k < p->taps.n; ++k) equal = p->taps.w[k] == p->taps.w[0];
  std::snprintf(buf, sizeof(buf), "%s/d%d/%dx%dx%d/r%d/%s%s/b%d", device_name().c_str(), p->ndim, p->g.nz,
                p->g.ny, p->g.nx, p->radius, p->shape == Shape::kBox ? "box" : "star", equal ? "eq" : "",
                p->boundary);
  return buf;
}

int ensure(double** buf, size_t count, const char* what) {
  if (*buf) return STENCIL_OK;
  cudaError_t e = dev_malloc(buf, count * sizeof(double));
  if (e != cudaSuccess) {
    *buf = nullptr;
    return cuda_fail(e, what);
  }
  return STENCIL_OK;
}

constexpr int kMaxDevices = kMaxDeviceOrdinals;

int current_device() { return device_ordinal(); }

// SM count of the current device (cached per device).
int sm_count() {
  static std::atomic<int> cache[kMaxDevices];
  const int dev = current_device();
  int n = cache[dev].load(std::memory_order_relaxed);
  if (n <= 0) {
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 1;
    cache[dev].store(n, std::memory_order_relaxed);
  }
  return n;
}

// ------------------------------------------------------------ tuning record
// Process-wide record of autotuned choices, keyed by the GPU name and the
// plan's shape (ndim, dims, radius, stencil class, equal-weight box,
// boundary).  STENCIL_TUNE_CACHE=<file> persists it across processes (one
// line per key: key Tb variant rate); STENCIL_TUNE=off ignores it,
// STENCIL_TUNE=full tunes a plan on its first run when no record exists.
struct TuneRec {
  int Tb, variant, tile_y;
};
std::mutex g_tune_mu;
std::map<std::string, TuneRec> g_tune;
bool g_tune_loaded = false;

// Name of the current device with blanks replaced (cached per device).
std::string device_name() {
  static std::mutex mu;
  static std::string cache[kMaxDevices];
  const int dev = current_device();
  std::lock_guard<std::mutex> lock(mu);
  std::string& name = cache[dev];
  if (name.empty()) {
    cudaDeviceProp prop;
    name = cudaGetDeviceProperties(&prop, dev) == cudaSuccess ? std::string(prop.name) : "unknown";
    for (char& c : name)
      if (c == ' ') c = '_';
  }
  return name;
}

std::string tune_mode() {
  const char* m = std::getenv("STENCIL_TUNE");
  return m ? std::string(m) : std::string("cached");
}

void tune_load_locked() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  const char* path = std::getenv("STENCIL_TUNE_CACHE");
  if (!path) return;
  FILE* f = std::fopen(path, "r");
  if (!f) return;
  // one line per key: key Tb variant tile_y rate (older records: key Tb variant rate)
  char line[1024];
  while (std::fgets(line, sizeof(line), f)) {
    char key[512];
    int tb = 0, v = 0, ty = 0;
    double rate = 0.0;
    const int got = std::sscanf(line, "%511s %d %d %d %lf", key, &tb, &v, &ty, &rate);
    if (got == 4) ty = 0;  // key Tb variant rate
    if (got >= 4 && tb > 0 && v > 0 && v < kVariantCount && ty >= 0) g_tune[key] = {tb, v, ty};
  }
  std::fclose(f);
}

void tune_store(const std::string& key, int tb, int v, int ty, double rate) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  tune_load_locked();
  g_tune[key] = {tb, v, ty};
  const char* path = std::getenv("STENCIL_TUNE_CACHE");
  if (!path) return;
  FILE* f = std::fopen(path, "a");
  if (!f) return;
  std::fprintf(f, "%s %d %d %d %.3f\n", key.c_str(), tb, v, ty, rate);
  std::fclose(f);
}

bool tune_lookup(const std::string& key, int& tb, int& v, int& ty) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  tune_load_locked();
  auto it = g_tune.find(key);
  if (it == g_tune.end()) return false;
  tb = it->second.Tb;
  v = it->second.variant;
  ty = it->second.tile_y;
  return true;
}

// The kernel (and Tb) a constant-weight plan uses when nothing was tuned or
// forced.  Small 2D grids are latency-bound: they run as one persistent launch,
// with Tb = 4 steps in shared memory per exchange up to 2^18 cells, and one
// step per device-wide barrier (5-point star) up to 3 * 2^20 cells; larger
// grids stream one launch per step (measured on GB300, 2D 5-point heat,
// T = 100: 512^2 53.6 vs 43.3 GStencil/s, 1024^2 76.2 vs 54.3 and 68.1 for
// streaming, 2048^2 streaming 102.3 vs 99.7).
int default_variant(const stencil_plan_s* p, int* Tb = nullptr) {
  if (Tb) *Tb = 1;
  // shapes the streaming kernels cannot take (odd nx; periodic sizes off their tile) go direct
  if (p->ndim == 3 && p->radius == 1)
    return stream3d_shape_ok(p->ndim, p->radius, p->shape, p->boundary, p->g) ? kVariantStream
                                                                               : kVariantDirect;
  const bool stream2d = stream2d_shape_ok(p->ndim, p->radius, p->boundary, p->g);
  if (p->ndim == 2 && p->radius == 1) {
    if (p->cells() <= ((int64_t)1 << 18)) {
      if (Tb) *Tb = 4;
      return kVariantPersistent;
    }
    if (p->cells() <= ((int64_t)3 << 20) && p->shape == Shape::kStar && p->taps.n == 5)
      return kVariantPersistent;
    return stream2d ? kVariantStream : kVariantDirect;
  }
  if (p->ndim == 2 && p->radius == 2) return stream2d ? kVariantStream : kVariantDirect;
  if (p->ndim == 1) {
    if (Tb) *Tb = 8;  // 8 steps per launch in shared memory, 0.4-0.8% halo recompute
    return kVariantTemporal;
  }
  return kVariantDirect;
}

// The kernel for a fused step count Tb > 1 that the caller fixed without a
// variant: the exchange kernel (no recomputed halo) for 3D radius-1 grids
// its tiling covers, the persistent temporal kernel for the small 2D grids
// it serves by default, else the overlapped temporal kernel (1D, 2D and 3D
// radius 1; other plans have no fused kernel and the run reports that).
int fused_variant(const stencil_plan_s* p) {
  if (p->ndim == 3 && p->radius == 1)
    return exchange_fits(p->ndim, p->radius, p->g, p->boundary == kPeriodic, sm_count()) ? kVariantExchange
                                                                                            : kVariantTemporal;
  if (p->ndim == 2 && p->radius == 1 && p->cells() <= ((int64_t)1 << 18) && (p->taps.n == 5 || p->taps.n == 9))
    return kVariantPersistent;
  return kVariantTemporal;
}

bool persistent_eligible(const stencil_plan_s* p) {
  return p->ndim == 2 && p->radius == 1 && p->shape == Shape::kStar && p->taps.n == 5;
}

// The kernel for one step per launch (Tb = 1 fixed without a variant): the
// default where it is a one-step kernel, else the streaming or direct sweep.
int one_step_variant(const stencil_plan_s* p) {
  const int v = default_variant(p);
  if (v == kVariantTemporal) return kVariantDirect;  // 1D: fused by default
  if (v == kVariantPersistent && !persistent_eligible(p))
    return stream2d_shape_ok(p->ndim, p->radius, p->boundary, p->g) ? kVariantStream : kVariantDirect;
  return v;
}

// Resolved (Tb, variant, streaming tile height; 0 = the kernel's default) for
// the next run of a constant-weight plan.
void choose(const stencil_plan_s* p, int& Tb, int& variant, int& tile_y) {
  tile_y = p->user_tile_y;
  if (p->user_Tb > 0 || p->user_variant > 0) {
    Tb = p->user_Tb > 0 ? p->user_Tb : 1;
    variant = p->user_variant > 0 ? p->user_variant : Tb > 1 ? fused_variant(p) : one_step_variant(p);
    return;
  }
  if (p->tuned_Tb > 0) {
    Tb = p->tuned_Tb;
    variant = p->tuned_variant;
    if (!tile_y) tile_y = p->tuned_tile_y;
    return;
  }
  int ty = 0;
  if (tune_mode() != "off" && tune_lookup(plan_key(p), Tb, variant, ty)) {
    if (!tile_y) tile_y = ty;
    return;
  }
  variant = default_variant(p, &Tb);
}
void choose(const stencil_plan_s* p, int& Tb, int& variant) {
  int ty;
  choose(p, Tb, variant, ty);
}

// Uploads the plan's weights (and the zero slots) to the device once.
int ensure_weights(stencil_plan_s* p) {
  if (p->d_w) return STENCIL_OK;
  std::vector<double> h(p->taps.n + kExtraSlots, 0.0);
  for (int k = 0; k < p->taps.n; ++k) h[k] = p->taps.w[k];
  for (int k = 0; k < kOneSlots; ++k) h[p->taps.n + kZeroSlots + k] = 1.0;
  CUDA_TRY(dev_malloc(&p->d_w, h.size() * sizeof(double)), "allocating the weight array");
  cudaError_t e = cudaMemcpy(p->d_w, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {  // leave no half-initialised array behind
    cudaFree(p->d_w);
    p->d_w = nullptr;
    return cuda_fail(e, "copying the weights");
  }
  return STENCIL_OK;
}

int ensure_status(stencil_plan_s* p) {
  if (p->d_status) return STENCIL_OK;
  CUDA_TRY(dev_malloc(&p->d_status, sizeof(int)), "allocating the status word");
  cudaError_t e = cudaMemset(p->d_status, 0, sizeof(int));
  if (e != cudaSuccess) {
    cudaFree(p->d_status);
    p->d_status = nullptr;
    return cuda_fail(e, "clearing the status word");
  }
  return STENCIL_OK;
}

// STENCIL_TUNE=full: the first run of an untuned shape times the candidates
// on a scratch copy of the grid (their runs destroy it) and records the best.
void tune_on_first_run(stencil_plan_s* p, const double* d_grid, cudaStream_t s) {
  if (tune_mode() != "full" || p->user_Tb != 0 || p->user_variant != 0 || p->tuned_Tb != 0) return;
  int tb0, v0, ty0;
  if (tune_lookup(plan_key(p), tb0, v0, ty0)) return;
  double* scratch = nullptr;
  if (dev_malloc(&scratch, (size_t)p->cells() * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  cudaMemcpyAsync(scratch, d_grid, (size_t)p->cells() * sizeof(double), cudaMemcpyDeviceToDevice, s);
  stencil_autotune(p, scratch, 4, s, nullptr);
  cudaStreamSynchronize(s);
  cudaFree(scratch);
}

// Persistent temporal kernel: Tb steps in shared memory per exchange, tiles
// synchronised by per-tile flags, one launch for all T steps.
int run_persistent_tb(stencil_plan_s* p, double* d_grid, int64_t T, int Tb, cudaStream_t s) {
  PersistTbLaunch L;
  persist_tiling(p->g.ny, p->g.nx, Tb, sm_count(), &L.tiles_y, &L.tiles_x, &L.reach_y, &L.reach_x);
  const int ntiles = L.tiles_y * L.tiles_x;
  if (p->flags_cap < ntiles) {
    cudaFree(p->d_flags);
    p->d_flags = nullptr;
    p->flags_cap = 0;
    CUDA_TRY(dev_malloc(&p->d_flags, ntiles * sizeof(unsigned int)), "allocating the tile flags");
    p->flags_cap = ntiles;
  }
  CUDA_TRY(cudaMemsetAsync(p->d_flags, 0, ntiles * sizeof(unsigned int), s), "clearing the tile flags");
  L.a = d_grid;
  L.b = p->d_tmp;
  L.ny = p->g.ny;
  L.nx = p->g.nx;
  L.T = T;
  L.wdev = p->d_w;
  L.flags = p->d_flags;
  L.status = p->d_status;
  L.spin_limit = kSpinLimitNs;
  cudaError_t e = launch_persist_tb(p->shape, p->boundary, Tb, L, sm_count(), s);
  if (e != cudaSuccess) return cuda_fail(e, "launching the persistent temporal kernel");
  return STENCIL_OK;
}

// One-step persistent kernel (the batched kernel with a single item): its
// device work list for (d_grid, T) comes from the plan's LRU cache.
int run_persistent_step(stencil_plan_s* p, double* d_grid, int64_t T, cudaStream_t s) {
  stencil_batch_s* hit = nullptr;
  for (auto& e : p->persist)
    if (e.grid == d_grid && e.T == T) {
      e.last_use = ++p->persist_clock;
      hit = e.batch;
    }
  if (!hit) {
    if ((int)p->persist.size() >= kPersistCache) {
      auto lru = std::min_element(p->persist.begin(), p->persist.end(),
                                  [](const auto& x, const auto& y) { return x.last_use < y.last_use; });
      lru->batch->d_partner = nullptr;  // the plan's own ping-pong buffer
      stencil_batch_destroy(lru->batch);
      p->persist.erase(lru);
    }
    auto* b = new (std::nothrow) stencil_batch_s();
    if (!b) return fail(STENCIL_ERR_OOM, "allocating the persistent plan");
    BatchItemDev it;
    it.a = d_grid;
    it.b = p->d_tmp;
    it.ny = p->g.ny;
    it.nx = p->g.nx;
    it.T = (int)T;
    for (int k = 0; k < 5; ++k) it.w[k] = p->taps.w[k];
    it.zero[0] = it.zero[1] = 0.0;
    const int rc = batch_init(b, std::vector<BatchItemDev>{it}, p->boundary);
    if (rc) {
      stencil_batch_destroy(b);
      return rc;
    }
    p->persist.push_back({d_grid, T, b, ++p->persist_clock});
    hit = b;
  }
  return batch_enqueue(hit, s);
}

// The exchange kernel's ring (for bands of up to band_rows rows) and
// progress counters for Tb (grown on demand).
int ensure_exchange(stencil_plan_s* p, int Tb, int band_rows, int ntiles) {
  const size_t cells = exchange_ring_cells(p->g, Tb, band_rows);
  if (p->ring_cells < cells) {
    cudaFree(p->d_ring);
    p->d_ring = nullptr;
    p->ring_cells = 0;
    CUDA_TRY(dev_malloc(&p->d_ring, cells * sizeof(double)), "allocating the exchange ring");
    p->ring_cells = cells;
  }
  const int words = exchange_counter_words(ntiles);
  if (p->xcnt_cap < words) {
    cudaFree(p->d_xcnt);
    p->d_xcnt = nullptr;
    p->xcnt_cap = 0;
    CUDA_TRY(dev_malloc(&p->d_xcnt, words * sizeof(unsigned int)), "allocating the exchange counters");
    p->xcnt_cap = words;
  }
  return STENCIL_OK;
}

// One Tb-step block of the exchange kernel from a to b: one launch per band
// of rows (one band unless the plane is taller than the co-resident tiles
// cover), each after clearing the progress counters.
int launch_exchange_block(stencil_plan_s* p, const double* a, double* b, int Tb, cudaStream_t s) {
  const int sms = sm_count();
  if (!exchange_fits(p->ndim, p->radius, p->g, p->boundary == kPeriodic, sms))
    return fail(STENCIL_ERR_UNSUPPORTED, "the grid does not fit the exchange kernel's tiling");
  const std::vector<ExchangeBand> bands = exchange_bands(p->g, p->boundary == kPeriodic, Tb, sms);
  ExchangeLaunch L;
  L.tiles_x = exchange_tiles_x(p->g);
  int max_rows = 0, max_ty = 0;
  for (const ExchangeBand& band : bands) {
    max_rows = std::max(max_rows, band.rows);
    max_ty = std::max(max_ty, band.tiles_y);
  }
  int rc = ensure_exchange(p, Tb, max_rows, max_ty * L.tiles_x);
  if (rc) return rc;
  L.g = p->g;
  L.src = a;
  L.dst = b;
  L.ring = p->d_ring;
  L.counters = p->d_xcnt;
  L.status = p->d_status;
  L.wdev = p->d_w;
  L.Tb = Tb;
  L.spin_limit = kSpinLimitNs;
  for (const ExchangeBand& band : bands) {
    CUDA_TRY(cudaMemsetAsync(p->d_xcnt, 0, exchange_counter_words(band.tiles_y * L.tiles_x) * sizeof(unsigned int),
                             s),
             "clearing the exchange counters");
    L.band = band;
    cudaError_t e = launch_exchange(p->shape, p->boundary, L, s);
    if (e != cudaSuccess) return cuda_fail(e, "launching the exchange kernel");
  }
  return STENCIL_OK;
}

// One launch per step (direct or streaming) or per Tb steps (temporal or
// exchange, with single steps for the remainder), ping-ponging with the
// plan's buffer; the result ends in d_grid.
int run_steps(stencil_plan_s* p, double* d_grid, int64_t T, int Tb, int variant, bool stream_ok,
              int tile_y, cudaStream_t s) {
  const int sms = sm_count();
  const bool equal_box = p->shape == Shape::kBox && taps_all_equal(p->taps);
  // the single-step kernel for the steps that do not fill a whole Tb block
  const int single = stream_ok ? kVariantStream : kVariantDirect;
  double* a = d_grid;
  double* b = p->d_tmp;
  int64_t t = 0;
  while (t < T) {
    cudaError_t e;
    int steps = 1;
    if (variant == kVariantExchange && T - t >= Tb) {
      const int rc = launch_exchange_block(p, a, b, Tb, s);
      if (rc) return rc;
      e = cudaSuccess;
      steps = Tb;
    } else if (variant == kVariantTemporal && T - t >= Tb) {
      e = launch_temporal(p->ndim, p->radius, p->shape, p->boundary, Tb, p->g, p->d_w, a, b, sms, s,
                          equal_box && p->ndim == 2 && p->radius == 1);
      steps = Tb;
    } else {
      const int v = variant == kVariantTemporal || variant == kVariantExchange ? single : variant;
      if (v == kVariantStream && p->ndim == 3)
        e = launch_stream3d(p->shape, p->boundary, p->g, p->taps, p->d_w, a, b, p->d_status, sms, s,
                            (unsigned long long)kSpinLimitNs, -1, tile_y);
      else if (v == kVariantStream)
        e = launch_stream2d(p->shape, p->radius, p->boundary, equal_box && p->radius == 1, p->g, p->taps,
                            p->d_w, a, b, p->d_status, sms, s);
      else
        e = launch_direct(p->ndim, p->radius, p->shape, p->boundary, p->g, p->taps, p->d_w, a, b, s);
    }
    if (e != cudaSuccess) return cuda_fail(e, "launching the sweep");
    std::swap(a, b);
    t += steps;
  }
  if (a != d_grid)
    CUDA_TRY(cudaMemcpyAsync(d_grid, a, (size_t)p->cells() * sizeof(double), cudaMemcpyDeviceToDevice, s),
             "copying the result back");
  return STENCIL_OK;
}

// A constant-weight sweep: resolve (Tb, variant), make sure the plan's
// buffers exist, fall back from a variant the grid cannot use (an error when
// the caller forced it) and dispatch.
int run_const(stencil_plan_s* p, double* d_grid, int64_t T, cudaStream_t s) {
  tune_on_first_run(p, d_grid, s);
  int Tb, variant, tile_y;
  choose(p, Tb, variant, tile_y);
  // a variant the caller named is an error when the grid cannot use it; a
  // Tb > 1 fixed without a variant is an error when no fused kernel covers
  // the plan; any other choice falls back quietly
  const bool v_user = p->user_variant > 0;
  const bool tb_user = p->user_Tb > 1 && !v_user;
  int rc = ensure(&p->d_tmp, (size_t)p->cells(), "allocating the ping-pong buffer");
  if (rc) return rc;
  rc = ensure_status(p);
  if (rc) return rc;
  rc = ensure_weights(p);
  if (rc) return rc;
  if (p->ndim == 3 && tile_y && !stream3d_eligible(p->ndim, p->radius, p->shape, p->boundary, p->g, d_grid,
                                                      p->d_tmp, tile_y)) {
    if (p->user_tile_y)
      return fail(STENCIL_ERR_UNSUPPORTED, "tile height %d does not fit this grid (periodic grids need ny a "
                  "multiple of it)", tile_y);
    tile_y = 0;  // a tuned tile that no longer fits: the default
  }
  const bool stream_ok = p->ndim == 3
                             ? stream3d_eligible(p->ndim, p->radius, p->shape, p->boundary, p->g, d_grid,
                                                 p->d_tmp, tile_y)
                             : stream2d_eligible(p->ndim, p->radius, p->boundary, p->g, d_grid, p->d_tmp);
  if (variant == kVariantStream && !stream_ok) {
    if (p->user_variant == kVariantStream)
      return fail(STENCIL_ERR_UNSUPPORTED,
                  "the streaming kernel needs a 2D or 3D radius-1 plan, even nx, 16-byte aligned "
                  "buffers and, for periodic grids, nx %% 64 == 0 and ny a multiple of the tile "
                  "height (16; 32 for the 3D star)");
    variant = kVariantDirect;
  }
  if (variant == kVariantPersistent && Tb > 1) {
    if (p->ndim == 2 && p->radius == 1 && (p->taps.n == 5 || p->taps.n == 9) && Tb <= 8)
      return run_persistent_tb(p, d_grid, T, Tb, s);
    if (v_user) return fail(STENCIL_ERR_UNSUPPORTED, "the persistent temporal kernel covers 2D radius-1 plans");
    variant = kVariantTemporal;  // keeps Tb where the overlapped kernel covers the plan (checked next)
  }
  if (variant == kVariantPersistent) {
    if (persistent_eligible(p) && T <= (1 << 30)) return run_persistent_step(p, d_grid, T, s);
    if (v_user) return fail(STENCIL_ERR_UNSUPPORTED, "the persistent kernel covers 2D 5-point star plans");
    variant = stream_ok ? kVariantStream : kVariantDirect;
  }
  if (variant == kVariantTemporal && !temporal_supported(p->ndim, p->radius, Tb)) {
    if (v_user || tb_user)
      return fail(STENCIL_ERR_UNSUPPORTED,
                  "temporal blocking covers 2D and 3D radius-1 plans with Tb in {2, 4, 8}, "
                  "and 1D plans of radius 1 or 2 with Tb in {2, 4, 8}");
    variant = default_variant(p) == kVariantStream && stream_ok ? kVariantStream : kVariantDirect;
  }
  if (variant == kVariantExchange) {
    const bool ok = Tb >= 2 && Tb <= 8 && exchange_fits(p->ndim, p->radius, p->g, p->boundary == kPeriodic, sm_count()) &&
                    ((uintptr_t)d_grid & 15) == 0 && ((uintptr_t)p->d_tmp & 15) == 0;
    if (!ok) {
      if (v_user)
        return fail(STENCIL_ERR_UNSUPPORTED,
                    "the exchange kernel covers 3D radius-1 plans with Tb in {2, 4, 8}, nx even (a "
                    "multiple of 64 on a periodic grid) and at most %d tile columns of 64, on 16-byte "
                    "aligned buffers", sm_count());
      // a Tb fixed without a variant keeps its Tb on the overlapped kernel;
      // a tuned choice falls back to one step per launch
      if (tb_user && temporal_supported(p->ndim, p->radius, Tb))
        variant = kVariantTemporal;
      else
        variant = stream_ok ? kVariantStream : kVariantDirect;
    }
  }
  if (variant != kVariantTemporal && variant != kVariantExchange) Tb = 1;
  if (variant != kVariantDirect && variant != kVariantStream && variant != kVariantTemporal &&
      variant != kVariantExchange)
    return fail(STENCIL_ERR_UNSUPPORTED, "variant %s is not available", stencil_variant_name(variant));
  return run_steps(p, d_grid, T, Tb, variant, stream_ok, tile_y, s);
}

VarcoefBufs coef_bufs(stencil_plan_s* p) {
  size_t n = (size_t)p->cells();
  return VarcoefBufs{p->d_coef, p->d_coef + n, p->d_coef + 2 * n, p->d_coef + 3 * n};
}

int run_varcoef(stencil_plan_s* p, double* d_grid, int64_t T, const double* d_kappa, double dt,
                cudaStream_t s) {
  if (!d_kappa) return fail(STENCIL_ERR_ARG, "variable-coefficient plan needs d_kappa");
  if (!(dt > 0.0) || !is_finite(dt)) return fail(STENCIL_ERR_ARG, "dt must be finite and > 0");
  int rc = ensure(&p->d_tmp, (size_t)p->cells(), "allocating the ping-pong buffer");
  if (rc) return rc;
  rc = ensure(&p->d_coef, 4 * (size_t)p->cells(), "allocating the coefficient arrays");
  if (rc) return rc;
  rc = ensure_weights(p);
  if (rc) return rc;
  VarcoefBufs cb = coef_bufs(p);
  cudaError_t e = launch_varcoef_prepare(p->ndim, p->boundary, p->g, d_kappa, dt, cb, s);
  if (e != cudaSuccess) return cuda_fail(e, "launching the coefficient preparation");
  double* a = d_grid;
  double* b = p->d_tmp;
  for (int64_t t = 0; t < T; ++t) {
    e = launch_varcoef_step(p->ndim, p->boundary, p->g, cb, a, b, p->d_w, s);
    if (e != cudaSuccess) return cuda_fail(e, "launching the variable-coefficient step");
    std::swap(a, b);
  }
  if (a != d_grid)
    CUDA_TRY(cudaMemcpyAsync(d_grid, a, (size_t)p->cells() * sizeof(double),
                             cudaMemcpyDeviceToDevice, s),
             "copying the result back");
  return STENCIL_OK;
}

// Fills a batch from device item descriptors (buffers and weights set):
// the T-sorted tile list, the item table, the barrier words and the
// cooperative grid size.
// Tb > 1: every item cut into near-equal tiles of at most 16 x 32 cells (the
// fewest such tiles: least halo recompute), listed item by item in the
// order of decreasing T, with the reach of a Tb-cell halo in tiles.
int batch_init_tb(stencil_batch_s* b, const std::vector<BatchItemDev>& hi, const std::vector<int>& order) {
  const int n = (int)hi.size();
  const int Tb = b->Tb;
  std::vector<BatchTbItemDev> items(n);
  std::vector<BatchTbTile> tiles;
  b->tb_max_blocks = 0;
  for (int i : order) {
    BatchTbItemDev& d = items[i];
    d.a = hi[i].a;
    d.b = hi[i].b;
    d.ny = hi[i].ny;
    d.nx = hi[i].nx;
    d.T = hi[i].T;
    for (int k = 0; k < 5; ++k) d.w[k] = hi[i].w[k];
    d.zero = 0.0;
    d.tiles_y = (d.ny + kBatchTbTileH - 1) / kBatchTbTileH;
    d.tiles_x = (d.nx + kBatchTbTileW - 1) / kBatchTbTileW;
    const int hmin = d.ny / d.tiles_y, wmin = d.nx / d.tiles_x;
    d.reach_y = (Tb + hmin - 1) / hmin;
    d.reach_x = (Tb + wmin - 1) / wmin;
    d.tile_base = (int)tiles.size();
    if (d.T == 0) continue;
    b->tb_max_blocks = std::max(b->tb_max_blocks, (d.T + Tb - 1) / Tb);
    for (int ty = 0; ty < d.tiles_y; ++ty)
      for (int tx = 0; tx < d.tiles_x; ++tx) tiles.push_back(BatchTbTile{i, ty, tx});
  }
  b->ntb_tiles = 0;  // set once every list below exists
  CUDA_TRY(dev_malloc(&b->d_tb_items, sizeof(BatchTbItemDev) * (size_t)std::max(n, 1)),
           "allocating the item table");
  CUDA_TRY(cudaMemcpy(b->d_tb_items, items.data(), sizeof(BatchTbItemDev) * (size_t)n, cudaMemcpyHostToDevice),
           "copying the item table");
  CUDA_TRY(dev_malloc(&b->d_tb_tiles, sizeof(BatchTbTile) * std::max<size_t>(1, tiles.size())),
           "allocating the tile list");
  if (!tiles.empty())
    CUDA_TRY(cudaMemcpy(b->d_tb_tiles, tiles.data(), sizeof(BatchTbTile) * tiles.size(), cudaMemcpyHostToDevice),
             "copying the tile list");
  CUDA_TRY(dev_malloc(&b->d_tb_flags, sizeof(unsigned int) * std::max<size_t>(1, tiles.size())),
           "allocating the tile flags");
  const int occ = batched_tb_blocks_per_sm(Tb, b->boundary);
  if (occ < 1) return fail(STENCIL_ERR_CUDA, "the batched temporal kernel does not fit on an SM");
  b->ntb_tiles = (int)tiles.size();
  b->blocks = sm_count() * std::min(occ, 2);
  if (b->ntb_tiles > 0 && b->ntb_tiles < b->blocks) b->blocks = b->ntb_tiles;
  b->ready = true;
  return STENCIL_OK;
}

int batch_init(stencil_batch_s* b, const std::vector<BatchItemDev>& hi, int boundary) {
  b->ready = false;
  const int n = (int)hi.size();
  b->n = n;
  b->boundary = boundary;
  b->max_T = 0;
  b->updates = 0;
  for (const BatchItemDev& it : hi) {
    b->max_T = std::max(b->max_T, it.T);
    b->updates += (int64_t)it.ny * it.nx * it.T;
  }
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return hi[a].T > hi[c].T; });
  if (b->cpt == 0) b->cpt = batched_default_cpt();
  b->hi = hi;
  CUDA_TRY(dev_malloc(&b->d_ctl, 4 * sizeof(unsigned int)), "allocating the barrier words");
  CUDA_TRY(cudaMemset(b->d_ctl, 0, 4 * sizeof(unsigned int)), "clearing the barrier words");
  if (b->Tb > 1) return batch_init_tb(b, hi, order);
  std::vector<BatchTile> tiles;
  const int tc = batched_tile_cells(b->cpt);
  for (int i : order) {
    if (hi[i].T == 0) continue;
    const int64_t cells = (int64_t)hi[i].ny * hi[i].nx;
    for (int64_t k0 = 0; k0 < cells; k0 += tc)
      tiles.push_back(BatchTile{i, (int)k0, (int)std::min<int64_t>(tc, cells - k0)});
  }
  b->ntiles = 0;  // set once every list below exists
  CUDA_TRY(dev_malloc(&b->d_items, sizeof(BatchItemDev) * (size_t)n), "allocating the item table");
  CUDA_TRY(cudaMemcpy(b->d_items, hi.data(), sizeof(BatchItemDev) * (size_t)n, cudaMemcpyHostToDevice),
           "copying the item table");
  CUDA_TRY(dev_malloc(&b->d_tiles, sizeof(BatchTile) * std::max<size_t>(1, tiles.size())),
           "allocating the tile list");
  if (!tiles.empty())
    CUDA_TRY(cudaMemcpy(b->d_tiles, tiles.data(), sizeof(BatchTile) * tiles.size(), cudaMemcpyHostToDevice),
             "copying the tile list");
  const int occ = batched_blocks_per_sm(b->cpt);
  if (occ < 1) return fail(STENCIL_ERR_CUDA, "the batched kernel does not fit on an SM");
  b->ntiles = (int)tiles.size();
  const int per_sm = b->per_sm > 0 ? std::min(b->per_sm, occ) : std::min(occ, 4);
  b->blocks = sm_count() * per_sm;
  if (b->ntiles > 0 && b->ntiles < b->blocks) b->blocks = b->ntiles;
  b->ready = true;
  return STENCIL_OK;
}

int batch_enqueue(stencil_batch_s* b, cudaStream_t s) {
  // a batch whose last (re)build failed part-way has no complete work list
  if (!b->ready) return fail(STENCIL_ERR_ARG, "the batch has no complete work list (an earlier call failed)");
  if (b->Tb > 1) {
    if (b->ntb_tiles == 0) return STENCIL_OK;  // every item has T = 0
    BatchTbLaunch L;
    L.items = b->d_tb_items;
    L.tiles = b->d_tb_tiles;
    L.ntiles = b->ntb_tiles;
    L.max_blocks = b->tb_max_blocks;
    L.flags = b->d_tb_flags;
    L.status = (int*)(b->d_ctl + 2);
    L.spin_limit = kSpinLimitNs;
    CUDA_TRY(cudaMemsetAsync(b->d_ctl, 0, 4 * sizeof(unsigned int), s), "clearing the status word");
    CUDA_TRY(cudaMemsetAsync(b->d_tb_flags, 0, sizeof(unsigned int) * b->ntb_tiles, s), "clearing the tile flags");
    cudaError_t e = launch_batched_tb(L, b->blocks, b->Tb, b->boundary, s);
    if (e != cudaSuccess) return cuda_fail(e, "launching the batched temporal kernel");
    return STENCIL_OK;
  }
  BatchLaunch L;
  L.items = b->d_items;
  L.tiles = b->d_tiles;
  L.ntiles = b->ntiles;
  L.max_T = b->max_T;
  L.boundary = b->boundary;
  L.barrier = b->d_ctl;
  L.status = (int*)(b->d_ctl + 2);
  L.spin_limit = kSpinLimitNs;
  L.barrier_blocks = 0;
  CUDA_TRY(cudaMemsetAsync(b->d_ctl, 0, 4 * sizeof(unsigned int), s), "clearing the barrier words");
  cudaError_t e = launch_batched(L, b->blocks, b->cpt, s);
  if (e != cudaSuccess) return cuda_fail(e, "launching the batched kernel");
  return STENCIL_OK;
}


}  // namespace

extern "C" {

const char* stencil_last_error(void) { return g_err.c_str(); }

void stencil_debug_fail_allocations(int after) { g_fail_after.store(after < 0 ? -1 : after); }

int64_t stencil_launch_count(void) { return g_launches.load(); }

const char* stencil_variant_name(int v) {
  switch (v) {
    case kVariantAuto: return "auto";
    case kVariantDirect: return "direct";
    case kVariantStream: return "stream";
    case kVariantTemporal: return "temporal";
    case kVariantPersistent: return "persistent";
    case kVariantExchange: return "exchange";
    default: return "";
  }
}

int stencil_create(int ndim, const int64_t* dims, int radius, const double* weights, int boundary,
                   stencil_plan* out) {
  g_err.clear();
  if (!out) return fail(STENCIL_ERR_ARG, "out is NULL");
  *out = nullptr;
  Geom g;
  int rc = make_geom(ndim, dims, g);
  if (rc) return rc;
  if (radius < 1 || radius > 2) return fail(STENCIL_ERR_ARG, "radius must be 1 or 2 (got %d)", radius);
  if (boundary != STENCIL_DIRICHLET_ZERO && boundary != STENCIL_PERIODIC)
    return fail(STENCIL_ERR_ARG, "unknown boundary %d", boundary);
  if (!weights) return fail(STENCIL_ERR_ARG, "weights is NULL");
  const int side = 2 * radius + 1;
  int64_t total = 1;
  for (int d = 0; d < ndim; ++d) total *= side;
  bool star = true;
  for (int64_t k = 0; k < total; ++k) {
    if (!is_finite(weights[k])) return fail(STENCIL_ERR_ARG, "weights[%lld] is not finite", (long long)k);
    if (weights[k] == 0.0) continue;
    int64_t rem = k;
    int nz_axes = 0;
    for (int d = ndim - 1; d >= 0; --d) {
      nz_axes += (rem % side) != radius;
      rem /= side;
    }
    if (nz_axes > 1) star = false;
  }
  auto* p = new (std::nothrow) stencil_plan_s();
  if (!p) return fail(STENCIL_ERR_OOM, "allocating the plan");
  p->ndim = ndim;
  p->g = g;
  p->radius = radius;
  p->boundary = boundary;
  p->shape = (star || ndim == 1) ? Shape::kStar : Shape::kBox;
  build_taps(p, weights);
  *out = p;
  return STENCIL_OK;
}

int stencil_create_varcoef(int ndim, const int64_t* dims, int boundary, stencil_plan* out) {
  g_err.clear();
  if (!out) return fail(STENCIL_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (ndim < 2 || ndim > 3) return fail(STENCIL_ERR_ARG, "variable-coefficient plans are 2D or 3D");
  Geom g;
  int rc = make_geom(ndim, dims, g);
  if (rc) return rc;
  if (boundary != STENCIL_DIRICHLET_ZERO && boundary != STENCIL_PERIODIC)
    return fail(STENCIL_ERR_ARG, "unknown boundary %d", boundary);
  auto* p = new (std::nothrow) stencil_plan_s();
  if (!p) return fail(STENCIL_ERR_OOM, "allocating the plan");
  p->ndim = ndim;
  p->g = g;
  p->radius = 1;
  p->boundary = boundary;
  p->varcoef = true;
  *out = p;
  return STENCIL_OK;
}

void stencil_destroy(stencil_plan p) {
  if (!p) return;
  cudaDeviceSynchronize();
  cudaFree(p->d_tmp);
  cudaFree(p->d_stage);
  cudaFree(p->d_coef);
  cudaFree(p->d_adj);
  cudaFree(p->d_status);
  cudaFree(p->d_flags);
  cudaFree(p->d_ring);
  cudaFree(p->d_xcnt);
  cudaFree(p->d_w);
  for (auto& e : p->persist) {
    e.batch->d_partner = nullptr;  // the plan's own ping-pong buffer
    stencil_batch_destroy(e.batch);
  }
  delete p;
}

int stencil_run(stencil_plan p, double* d_grid, int64_t T, const double* d_kappa, double dt,
                void* cuda_stream) {
  g_err.clear();
  if (!p) return fail(STENCIL_ERR_ARG, "plan is NULL");
  if (!d_grid) return fail(STENCIL_ERR_ARG, "d_grid is NULL");
  if (((uintptr_t)d_grid & 7) != 0) return fail(STENCIL_ERR_ARG, "d_grid is not 8-byte aligned");
  if (T < 0) return fail(STENCIL_ERR_ARG, "T must be >= 0");
  if (T == 0) return STENCIL_OK;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  if (p->varcoef) return run_varcoef(p, d_grid, T, d_kappa, dt, s);
  return run_const(p, d_grid, T, s);
}

int stencil_run_host(stencil_plan p, double* h_grid, int64_t T, const double* h_kappa, double dt,
                     void* cuda_stream) {
  g_err.clear();
  if (!p) return fail(STENCIL_ERR_ARG, "plan is NULL");
  if (!h_grid) return fail(STENCIL_ERR_ARG, "h_grid is NULL");
  if (p->varcoef && !h_kappa) return fail(STENCIL_ERR_ARG, "variable-coefficient plan needs h_kappa");
  if (T < 0) return fail(STENCIL_ERR_ARG, "T must be >= 0");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const size_t n = (size_t)p->cells();
  int rc = ensure(&p->d_stage, p->varcoef ? 2 * n : n, "allocating the staging buffer");
  if (rc) return rc;
  CUDA_TRY(cudaMemcpyAsync(p->d_stage, h_grid, n * sizeof(double), cudaMemcpyHostToDevice, s),
           "copying the grid to the device");
  if (p->varcoef)
    CUDA_TRY(cudaMemcpyAsync(p->d_stage + n, h_kappa, n * sizeof(double), cudaMemcpyHostToDevice, s),
             "copying kappa to the device");
  rc = stencil_run(p, p->d_stage, T, p->varcoef ? p->d_stage + n : nullptr, dt, cuda_stream);
  if (rc) return rc;
  CUDA_TRY(cudaMemcpyAsync(h_grid, p->d_stage, n * sizeof(double), cudaMemcpyDeviceToHost, s),
           "copying the result to the host");
  CUDA_TRY(cudaStreamSynchronize(s), "waiting for the host-buffer sweep");
  return STENCIL_OK;
}

}  // extern "C"

namespace {

// The adjoint sweep shared by stencil_adjoint (loss form: lambda^T = u^T - target,
// loss reduced on the device) and stencil_adjoint_vjp (lambda^T given).
int adjoint_core(stencil_plan_s* p, const double* d_u0, const double* d_kappa, double dt,
                 const double* d_target, const double* d_lambda_T, int64_t T, int ckpt_every,
                 double* d_grad_u0, double* d_grad_kappa, double* h_loss, cudaStream_t s) {
  if (!p->varcoef) return fail(STENCIL_ERR_ARG, "the adjoint needs a variable-coefficient plan");
  if (!d_u0 || !d_kappa || !d_grad_u0 || !d_grad_kappa) return fail(STENCIL_ERR_ARG, "NULL buffer");
  if (!(dt > 0.0) || !is_finite(dt)) return fail(STENCIL_ERR_ARG, "dt must be finite and > 0");
  if (T < 0) return fail(STENCIL_ERR_ARG, "T must be >= 0");
  if (ckpt_every < 0) return fail(STENCIL_ERR_ARG, "ckpt_every must be >= 0");
  const size_t n = (size_t)p->cells();
  // automatic interval: about sqrt(T), so the scratch grows with sqrt(T)
  // (every state, c = 1, is an explicit choice of the caller)
  const int64_t c_sqrt = std::max<int64_t>(1, (int64_t)llround(std::sqrt((double)T)));
  int64_t c = ckpt_every == 0 ? c_sqrt : ckpt_every;
  if (T > 0 && c > T) c = T;
  const int64_t nck = T / c + 1;        // u at t = 0, c, 2c, ... (<= T)
  const int64_t nseg_states = c;        // u^{t0} .. u^{t0+c-1} of one segment
  const int nblocks = 4 * sm_count();
  // scratch: checkpoints, segment states, 2 lambda, 4 gradient accumulators,
  // the running state pair and the loss partials
  const size_t need = n * (size_t)(nck + nseg_states + 2 + 4 + 2) + (size_t)nblocks + 8;
  // the plan keeps its scratch between calls; one left from a call with a
  // shorter interval (more states kept) than this one needs is given back
  if (p->d_adj && (p->adj_cells < need || p->adj_cells > 2 * need)) {
    cudaFree(p->d_adj);
    p->d_adj = nullptr;
  }
  int rc = ensure(&p->d_adj, need, "allocating the adjoint scratch (checkpoints)");
  if (rc) return rc;
  p->adj_cells = need;
  rc = ensure(&p->d_coef, 4 * n, "allocating the coefficient arrays");
  if (rc) return rc;
  rc = ensure_weights(p);
  if (rc) return rc;
  double* ck = p->d_adj;
  double* seg = ck + n * nck;
  double* lam = seg + n * nseg_states;
  double* lam2 = lam + n;
  double* gx = lam2 + n;
  double* gy = gx + n;
  double* gz = gy + n;
  double* gg = gz + n;
  double* cur = gg + n;
  double* nxt = cur + n;
  double* partials = nxt + n;
  double* d_loss = partials + nblocks;
  VarcoefBufs cb = coef_bufs(p);
  cudaError_t e = launch_varcoef_prepare(p->ndim, p->boundary, p->g, d_kappa, dt, cb, s);
  if (e != cudaSuccess) return cuda_fail(e, "launching the coefficient preparation");
  const size_t bytes = n * sizeof(double);
  // forward sweep, keeping u at every multiple of c; the states inside the
  // last segment go straight to the segment buffer, so the reverse sweep
  // starts without recomputing them
  const int64_t nseg = (T + c - 1) / c;
  const int64_t t_last = (nseg - 1) * c;  // first step of the last segment
  CUDA_TRY(cudaMemcpyAsync(ck, d_u0, bytes, cudaMemcpyDeviceToDevice, s), "copying u0");
  const double* src = ck;
  for (int64_t t = 0; t < T; ++t) {
    const int64_t k = t + 1;  // index of the state this step produces
    double* dst = (k % c == 0)            ? ck + n * (size_t)(k / c)
                  : (k > t_last && k < T) ? seg + n * (size_t)(k - t_last)
                                          : (src == cur ? nxt : cur);
    e = launch_varcoef_step(p->ndim, p->boundary, p->g, cb, src, dst, p->d_w, s);
    if (e != cudaSuccess) return cuda_fail(e, "launching the forward step");
    src = dst;
  }
  if (d_target) {
    // loss and lambda^T = u^T - target
    e = launch_loss_residual((int64_t)n, src, d_target, lam, partials, nblocks, d_loss, s);
    if (e != cudaSuccess) return cuda_fail(e, "launching the loss reduction");
  } else {
    CUDA_TRY(cudaMemcpyAsync(lam, d_lambda_T, bytes, cudaMemcpyDeviceToDevice, s), "copying lambda^T");
  }
  CUDA_TRY(cudaMemsetAsync(gx, 0, 4 * bytes, s), "clearing the gradient accumulators");
  // reverse sweep, one segment [t0, t1) at a time
  for (int64_t sg = nseg - 1; sg >= 0; --sg) {
    const int64_t t0 = sg * c, t1 = std::min(T, t0 + c);
    const double* base = ck + n * (size_t)sg;
    // seg[k] = u^{t0+k} for k = 1 .. t1-t0-1 (k = 0 is the checkpoint itself);
    // the forward sweep already left the last segment's states there
    for (int64_t t = t0 + 1; t < t1 && sg < nseg - 1; ++t) {
      const double* from = (t == t0 + 1) ? base : seg + n * (size_t)(t - t0 - 1);
      e = launch_varcoef_step(p->ndim, p->boundary, p->g, cb, from, seg + n * (size_t)(t - t0), p->d_w, s);
      if (e != cudaSuccess) return cuda_fail(e, "launching the segment recompute");
    }
    for (int64_t t = t1 - 1; t >= t0; --t) {
      const double* ut = (t == t0) ? base : seg + n * (size_t)(t - t0);
      e = launch_adjoint_step(p->ndim, p->boundary, p->g, cb, lam, ut, lam2, gx, gy, gz, gg, p->d_w, s);
      if (e != cudaSuccess) return cuda_fail(e, "launching the adjoint step");
      std::swap(lam, lam2);
    }
  }
  e = launch_adjoint_finalize(p->ndim, p->boundary, p->g, dt, gx, gy, gz, gg, d_grad_kappa, s);
  if (e != cudaSuccess) return cuda_fail(e, "launching the gradient finalisation");
  CUDA_TRY(cudaMemcpyAsync(d_grad_u0, lam, bytes, cudaMemcpyDeviceToDevice, s), "copying dL/du0");
  if (d_target) {
    CUDA_TRY(cudaMemcpyAsync(h_loss, d_loss, sizeof(double), cudaMemcpyDeviceToHost, s),
             "copying the loss");
    CUDA_TRY(cudaStreamSynchronize(s), "waiting for the adjoint");
  }
  return STENCIL_OK;
}

}  // namespace

extern "C" {

int stencil_adjoint(stencil_plan p, const double* d_u0, const double* d_kappa, double dt,
                    const double* d_target, int64_t T, int ckpt_every, double* d_grad_u0,
                    double* d_grad_kappa, double* h_loss, void* cuda_stream) {
  g_err.clear();
  if (!p) return fail(STENCIL_ERR_ARG, "plan is NULL");
  if (!d_target || !h_loss) return fail(STENCIL_ERR_ARG, "NULL target or loss");
  return adjoint_core(p, d_u0, d_kappa, dt, d_target, nullptr, T, ckpt_every, d_grad_u0, d_grad_kappa,
                      h_loss, (cudaStream_t)cuda_stream);
}

int stencil_adjoint_vjp(stencil_plan p, const double* d_u0, const double* d_kappa, double dt,
                        int64_t T, int ckpt_every, const double* d_lambda_T, double* d_grad_u0,
                        double* d_grad_kappa, void* cuda_stream) {
  g_err.clear();
  if (!p) return fail(STENCIL_ERR_ARG, "plan is NULL");
  if (!d_lambda_T) return fail(STENCIL_ERR_ARG, "d_lambda_T is NULL");
  return adjoint_core(p, d_u0, d_kappa, dt, nullptr, d_lambda_T, T, ckpt_every, d_grad_u0, d_grad_kappa,
                      nullptr, (cudaStream_t)cuda_stream);
}

int stencil_run_f32(stencil_plan p, float* d_grid, float* d_work, int64_t T, void* cuda_stream) {
  g_err.clear();
  if (!p || !d_grid || !d_work) return fail(STENCIL_ERR_ARG, "NULL argument");
  if (p->varcoef) return fail(STENCIL_ERR_ARG, "the FP32 twin covers constant-weight plans");
  if (p->taps.n > 27) return fail(STENCIL_ERR_UNSUPPORTED, "the FP32 twin covers up to 27 taps");
  if (T < 0) return fail(STENCIL_ERR_ARG, "T must be >= 0");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  float* a = d_grid;
  float* b = d_work;
  for (int64_t t = 0; t < T; ++t) {
    cudaError_t e = launch_direct_f32(p->ndim, p->radius, p->boundary, p->g, p->taps, a, b, s);
    if (e != cudaSuccess) return cuda_fail(e, "launching the FP32 sweep");
    std::swap(a, b);
  }
  if (a != d_grid)
    CUDA_TRY(cudaMemcpyAsync(d_grid, a, (size_t)p->cells() * sizeof(float), cudaMemcpyDeviceToDevice, s),
             "copying the FP32 result back");
  return STENCIL_OK;
}

int stencil_plan_status(stencil_plan p, void* cuda_stream) {
  g_err.clear();
  if (!p) return fail(STENCIL_ERR_ARG, "plan is NULL");
  CUDA_TRY(cudaStreamSynchronize((cudaStream_t)cuda_stream), "waiting for the stream");
  if (!p->d_status) return STENCIL_OK;
  int st = 0;
  CUDA_TRY(cudaMemcpy(&st, p->d_status, sizeof(int), cudaMemcpyDeviceToHost), "reading the status");
  if (st != 0) {
    CUDA_TRY(cudaMemset(p->d_status, 0, sizeof(int)), "clearing the status word");
    return fail(st, "a kernel of this plan reported status %d (a bounded wait gave up)", st);
  }
  return STENCIL_OK;
}

int stencil_set_tuning(stencil_plan p, int Tb, int variant) {
  g_err.clear();
  if (!p) return fail(STENCIL_ERR_ARG, "plan is NULL");
  if (Tb != 0 && Tb != 1 && Tb != 2 && Tb != 4 && Tb != 8)
    return fail(STENCIL_ERR_ARG, "Tb must be 0, 1, 2, 4 or 8 (got %d)", Tb);
  if (variant < 0 || variant >= kVariantCount)
    return fail(STENCIL_ERR_ARG, "unknown variant %d", variant);
  p->user_Tb = Tb;
  p->user_variant = Tb == 0 ? 0 : variant;
  return STENCIL_OK;
}

int stencil_set_tile(stencil_plan p, int tile_x, int tile_y) {
  g_err.clear();
  if (!p) return fail(STENCIL_ERR_ARG, "plan is NULL");
  if (tile_x != 0 && tile_x != 64) return fail(STENCIL_ERR_ARG, "tile_x must be 0 or 64 (got %d)", tile_x);
  if (tile_y != 0 && stream3d_tile_y(p->shape, tile_y) < 0)
    return fail(STENCIL_ERR_ARG, "tile_y must be 0, 8, 16 or 32 (got %d)", tile_y);
  p->user_tile_y = tile_y;
  return STENCIL_OK;
}

int stencil_get_tile(stencil_plan p, int* tile_x, int* tile_y) {
  g_err.clear();
  if (!p || !tile_x || !tile_y) return fail(STENCIL_ERR_ARG, "NULL argument");
  int Tb, v, ty;
  choose(p, Tb, v, ty);
  *tile_x = 0;
  *tile_y = 0;
  if (v == kVariantStream && p->ndim == 3 && p->radius == 1) {
    *tile_x = 64;
    *tile_y = stream3d_tile_y(p->shape, ty);
  }
  return STENCIL_OK;
}

int stencil_get_tuning(stencil_plan p, int* Tb, int* variant) {
  g_err.clear();
  if (!p || !Tb || !variant) return fail(STENCIL_ERR_ARG, "NULL argument");
  choose(p, *Tb, *variant);
  return STENCIL_OK;
}

int stencil_exchange_layout(stencil_plan p, int Tb, int* nbands, int64_t* rows_computed) {
  g_err.clear();
  if (!p || !nbands || !rows_computed) return fail(STENCIL_ERR_ARG, "NULL argument");
  if (Tb != 2 && Tb != 4 && Tb != 8) return fail(STENCIL_ERR_ARG, "Tb must be 2, 4 or 8 (got %d)", Tb);
  const int sms = sm_count();
  if (p->varcoef || !exchange_fits(p->ndim, p->radius, p->g, p->boundary == kPeriodic, sms))
    return fail(STENCIL_ERR_UNSUPPORTED, "the exchange kernel does not take this plan");
  const std::vector<ExchangeBand> bands = exchange_bands(p->g, p->boundary == kPeriodic, Tb, sms);
  int64_t rows = 0;
  for (const ExchangeBand& b : bands) rows += b.rows;
  *nbands = (int)bands.size();
  *rows_computed = rows;
  return STENCIL_OK;
}

int stencil_autotune(stencil_plan p, double* d_grid, int64_t probe_steps, void* cuda_stream,
                     double* best_gstencils) {
  g_err.clear();
  if (!p || !d_grid) return fail(STENCIL_ERR_ARG, "NULL argument");
  if (p->varcoef) return fail(STENCIL_ERR_UNSUPPORTED, "autotune covers constant-weight plans");
  if (probe_steps < 1) return fail(STENCIL_ERR_ARG, "probe_steps must be >= 1");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  struct Cand { int Tb, variant, tile_y; };
  std::vector<Cand> cands = {{1, kVariantDirect, 0}, {1, kVariantStream, 0}, {1, kVariantPersistent, 0},
                             {2, kVariantPersistent, 0}, {4, kVariantPersistent, 0}, {8, kVariantPersistent, 0},
                             {2, kVariantTemporal, 0}, {4, kVariantTemporal, 0}, {8, kVariantTemporal, 0},
                             {2, kVariantExchange, 0}, {4, kVariantExchange, 0}, {8, kVariantExchange, 0}};
  if (p->ndim == 3 && p->radius == 1)  // the streaming kernel's tile heights
    for (int ty : {8, 16, 32})
      if (ty != stream3d_tile_y(p->shape, 0)) cands.push_back({1, kVariantStream, ty});
  cudaEvent_t e0, e1;
  CUDA_TRY(cudaEventCreate(&e0), "creating an event");
  CUDA_TRY(cudaEventCreate(&e1), "creating an event");
  const int saved_Tb = p->user_Tb, saved_v = p->user_variant, saved_ty = p->user_tile_y;
  double best = -1.0;
  Cand best_c = cands[0];
  for (const Cand& c : cands) {
    p->user_Tb = c.Tb;
    p->user_variant = c.variant;
    p->user_tile_y = c.tile_y;
    int rc = stencil_run(p, d_grid, c.Tb, nullptr, 0.0, cuda_stream);  // warm-up
    if (rc == STENCIL_ERR_UNSUPPORTED) continue;
    if (rc) break;
    cudaEventRecord(e0, s);
    rc = stencil_run(p, d_grid, probe_steps, nullptr, 0.0, cuda_stream);
    cudaEventRecord(e1, s);
    if (rc) break;
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    double rate = (double)p->cells() * (double)probe_steps / (ms * 1e-3) / 1e9;
    if (rate > best) {
      best = rate;
      best_c = c;
    }
  }
  p->user_Tb = saved_Tb;
  p->user_variant = saved_v;
  p->user_tile_y = saved_ty;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (best < 0) return g_err.empty() ? fail(STENCIL_ERR_CUDA, "no candidate ran") : STENCIL_ERR_CUDA;
  p->tuned_Tb = best_c.Tb;
  p->tuned_variant = best_c.variant;
  p->tuned_tile_y = best_c.tile_y;
  tune_store(plan_key(p), best_c.Tb, best_c.variant, best_c.tile_y, best);
  if (best_gstencils) *best_gstencils = best;
  return STENCIL_OK;
}

// ------------------------------------------------------------------ batches

int stencil_batch_create(const stencil_batch_item* items, int n, int boundary, stencil_batch* out) {
  g_err.clear();
  if (!out) return fail(STENCIL_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!items || n < 1) return fail(STENCIL_ERR_ARG, "a batch needs at least one item");
  if (boundary != STENCIL_DIRICHLET_ZERO && boundary != STENCIL_PERIODIC)
    return fail(STENCIL_ERR_ARG, "unknown boundary %d", boundary);
  int64_t total_cells = 0;
  for (int i = 0; i < n; ++i) {
    const stencil_batch_item& it = items[i];
    if (it.ny < 1 || it.nx < 1 || it.ny > (1 << 30) || it.nx > (1 << 30))
      return fail(STENCIL_ERR_ARG, "item %d: bad shape %lld x %lld", i, (long long)it.ny, (long long)it.nx);
    if (it.ny * it.nx > INT32_MAX)
      return fail(STENCIL_ERR_UNSUPPORTED, "item %d: a batched grid holds at most 2^31 - 1 cells", i);
    if (it.T < 0 || it.T > (1 << 30)) return fail(STENCIL_ERR_ARG, "item %d: bad T", i);
    if (!is_finite(it.alpha)) return fail(STENCIL_ERR_ARG, "item %d: alpha not finite", i);
    if (!it.d_grid || ((uintptr_t)it.d_grid & 7)) return fail(STENCIL_ERR_ARG, "item %d: bad d_grid", i);
    total_cells += it.ny * it.nx;
  }
  auto* b = new (std::nothrow) stencil_batch_s();
  if (!b) return fail(STENCIL_ERR_OOM, "allocating the batch");
  b->items.assign(items, items + n);
  cudaError_t e = dev_malloc(&b->d_partner, (size_t)total_cells * sizeof(double));
  if (e != cudaSuccess) {
    int rc = cuda_fail(e, "allocating the partner buffers");
    stencil_batch_destroy(b);
    return rc;
  }
  std::vector<BatchItemDev> hi(n);
  int64_t off = 0;
  for (int i = 0; i < n; ++i) {
    const stencil_batch_item& it = items[i];
    hi[i].a = it.d_grid;
    hi[i].b = b->d_partner + off;
    hi[i].ny = (int)it.ny;
    hi[i].nx = (int)it.nx;
    hi[i].T = (int)it.T;
    hi[i].w[0] = it.alpha;             // Eq. 3: alpha at the four neighbours,
    hi[i].w[1] = it.alpha;
    hi[i].w[2] = 1.0 - 4.0 * it.alpha; // 1 - 4 alpha at the centre
    hi[i].w[3] = it.alpha;
    hi[i].w[4] = it.alpha;
    hi[i].zero[0] = hi[i].zero[1] = 0.0;
    off += it.ny * it.nx;
  }
  int rc = batch_init(b, hi, boundary);
  if (rc) {
    stencil_batch_destroy(b);
    return rc;
  }
  *out = b;
  return STENCIL_OK;
}

int stencil_batch_run(stencil_batch b, void* cuda_stream) {
  g_err.clear();
  if (!b) return fail(STENCIL_ERR_ARG, "batch is NULL");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  b->last_stream = s;
  if (b->use_graph && !b->exec) {
    if (!b->capture_stream)
      CUDA_TRY(cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking), "creating a stream");
    cudaGraph_t graph = nullptr;
    bool ok = cudaStreamBeginCapture(b->capture_stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
      int rc = batch_enqueue(b, b->capture_stream);
      ok = cudaStreamEndCapture(b->capture_stream, &graph) == cudaSuccess && rc == STENCIL_OK;
      g_launches.fetch_sub(1, std::memory_order_relaxed);  // captured, not launched
    }
    if (ok) ok = cudaGraphInstantiate(&b->exec, graph, 0) == cudaSuccess;
    if (graph) cudaGraphDestroy(graph);
    if (!ok) {
      cudaGetLastError();
      b->exec = nullptr;
      b->use_graph = false;  // fall back to direct cooperative launches
    }
  }
  if (b->exec) {
    CUDA_TRY(cudaGraphLaunch(b->exec, s), "launching the batch graph");
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return STENCIL_OK;
  }
  return batch_enqueue(b, s);
}

int stencil_batch_status(stencil_batch b) {
  g_err.clear();
  if (!b) return fail(STENCIL_ERR_ARG, "batch is NULL");
  CUDA_TRY(cudaStreamSynchronize(b->last_stream), "waiting for the batch");
  int st = 0;
  CUDA_TRY(cudaMemcpy(&st, b->d_ctl + 2, sizeof(int), cudaMemcpyDeviceToHost), "reading the status");
  if (st != 0) return fail(st, "the batched kernel reported status %d (a bounded wait gave up)", st);
  return STENCIL_OK;
}

}  // extern "C"

namespace {

// Frees a batch's tile list, item table and barrier words and drops its graph
// (the partner buffer stays), after the device has finished with them.
void batch_release_lists(stencil_batch_s* b) {
  cudaDeviceSynchronize();
  if (b->exec) cudaGraphExecDestroy(b->exec);
  b->exec = nullptr;
  b->use_graph = true;
  cudaFree(b->d_items);
  cudaFree(b->d_tiles);
  cudaFree(b->d_ctl);
  cudaFree(b->d_tb_items);
  cudaFree(b->d_tb_tiles);
  cudaFree(b->d_tb_flags);
  b->d_items = nullptr;
  b->d_tiles = nullptr;
  b->d_ctl = nullptr;
  b->d_tb_items = nullptr;
  b->d_tb_tiles = nullptr;
  b->d_tb_flags = nullptr;
  b->ntiles = b->ntb_tiles = 0;
  b->ready = false;
}

// Rebuilds the tile list for the batch's current kernel configuration.
int batch_rebuild(stencil_batch_s* b) {
  batch_release_lists(b);
  const std::vector<BatchItemDev> hi = b->hi;
  return batch_init(b, hi, b->boundary);
}

}  // namespace

extern "C" {

int stencil_batch_set_tuning(stencil_batch b, int Tb, int cells_per_thread, int blocks_per_sm) {
  g_err.clear();
  if (!b) return fail(STENCIL_ERR_ARG, "batch is NULL");
  if (Tb != 0 && Tb != 1 && Tb != 2 && Tb != 4 && Tb != 8) return fail(STENCIL_ERR_ARG, "Tb must be 0, 1, 2, 4 or 8");
  if (cells_per_thread != 0 && cells_per_thread != 1 && cells_per_thread != 2 && cells_per_thread != 4)
    return fail(STENCIL_ERR_ARG, "cells_per_thread must be 0, 1, 2 or 4");
  if (blocks_per_sm < 0 || blocks_per_sm > 32) return fail(STENCIL_ERR_ARG, "blocks_per_sm must be in [0, 32]");
  b->Tb = Tb == 0 ? 1 : Tb;
  b->cpt = cells_per_thread;
  b->per_sm = blocks_per_sm;
  return batch_rebuild(b);
}

int stencil_batch_get_tuning(stencil_batch b, int* Tb, int* cells_per_thread, int* blocks_per_sm) {
  g_err.clear();
  if (!b || !Tb || !cells_per_thread || !blocks_per_sm) return fail(STENCIL_ERR_ARG, "NULL argument");
  *Tb = b->Tb;
  *cells_per_thread = b->Tb > 1 ? 0 : b->cpt;
  *blocks_per_sm = (b->blocks + sm_count() - 1) / std::max(1, sm_count());
  return STENCIL_OK;
}

int stencil_batch_autotune(stencil_batch b, int64_t probe_steps, void* cuda_stream, double* best_gstencils) {
  g_err.clear();
  if (!b) return fail(STENCIL_ERR_ARG, "batch is NULL");
  if (probe_steps < 1 || probe_steps > (1 << 20)) return fail(STENCIL_ERR_ARG, "probe_steps must be in [1, 2^20]");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  // scratch copies of every item (grid and partner): the probes leave the
  // caller's grids untouched
  int64_t total = 0, updates = 0;
  for (const BatchItemDev& it : b->hi) total += (int64_t)it.ny * it.nx;
  double* scratch = nullptr;
  CUDA_TRY(dev_malloc(&scratch, 2 * (size_t)std::max<int64_t>(total, 1) * sizeof(double)),
           "allocating the autotuner's scratch grids");
  std::vector<BatchItemDev> probe = b->hi;
  int64_t off = 0;
  int rc = STENCIL_OK;
  // each item's T scaled by probe_steps / max T (rounded up): the probe keeps
  // the batch's mix of step counts, so the tail where few items are still
  // active weighs in as it does in a full run
  const int64_t max_T = std::max<int64_t>(1, b->max_T);
  for (size_t i = 0; i < probe.size(); ++i) {
    const int64_t cells = (int64_t)probe[i].ny * probe[i].nx;
    probe[i].a = scratch + off;
    probe[i].b = scratch + total + off;
    probe[i].T = probe[i].T == 0 ? 0
                                 : (int)std::max<int64_t>(1, (probe[i].T * std::min(probe_steps, max_T) + max_T - 1) /
                                                                 max_T);
    updates += cells * probe[i].T;
    if (cudaMemcpyAsync(probe[i].a, b->hi[i].a, cells * sizeof(double), cudaMemcpyDeviceToDevice, s) !=
        cudaSuccess)
      rc = fail(STENCIL_ERR_CUDA, "copying the items to the autotuner's scratch");
    off += cells;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (!rc && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
    rc = fail(STENCIL_ERR_CUDA, "creating events");
  double best = -1.0;
  int best_Tb = 1, best_cpt = batched_default_cpt(), best_per_sm = 0;
  struct Cand { int Tb, cpt, per_sm; };
  std::vector<Cand> cands;
  for (int cpt : {1, 2, 4})
    for (int per_sm = 1; per_sm <= std::min(batched_blocks_per_sm(cpt), 4); ++per_sm) cands.push_back({1, cpt, per_sm});
  for (int Tb : {2, 4, 8}) cands.push_back({Tb, 0, 0});
  for (const Cand& cd : cands) {
    if (rc) break;
    auto* t = new (std::nothrow) stencil_batch_s();
    if (!t) {
      rc = fail(STENCIL_ERR_OOM, "allocating a probe batch");
      break;
    }
    t->Tb = cd.Tb;
    t->cpt = cd.cpt;
    t->per_sm = cd.per_sm;
    rc = batch_init(t, probe, b->boundary);
    if (!rc) rc = batch_enqueue(t, s);  // warm-up
    float best_ms = -1.f;               // the fastest of three timed runs
    for (int rep = 0; rep < 3 && !rc; ++rep) {
      cudaEventRecord(e0, s);
      rc = batch_enqueue(t, s);
      cudaEventRecord(e1, s);
      if (rc) break;
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (best_ms < 0.f || ms < best_ms) best_ms = ms;
    }
    if (!rc) {
      const double rate = (double)updates / (std::max(best_ms, 1e-3f) * 1e-3) / 1e9;
      if (rate > best) {
        best = rate;
        best_Tb = cd.Tb;
        best_cpt = cd.cpt;
        best_per_sm = cd.per_sm;
      }
    }
    t->d_partner = nullptr;  // scratch, freed below
    stencil_batch_destroy(t);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(scratch);
  if (rc) return rc;
  if (best < 0) return fail(STENCIL_ERR_CUDA, "no batch configuration ran");
  b->Tb = best_Tb;
  b->cpt = best_cpt;
  b->per_sm = best_per_sm;
  rc = batch_rebuild(b);
  if (rc) return rc;
  if (best_gstencils) *best_gstencils = best;
  return STENCIL_OK;
}

void stencil_batch_destroy(stencil_batch b) {
  if (!b) return;
  cudaDeviceSynchronize();
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
  cudaFree(b->d_items);
  cudaFree(b->d_tiles);
  cudaFree(b->d_partner);
  cudaFree(b->d_ctl);
  cudaFree(b->d_tb_items);
  cudaFree(b->d_tb_tiles);
  cudaFree(b->d_tb_flags);
  delete b;
}

int stencil_run_batched(const stencil_batch_item* items, int n, int boundary, void* cuda_stream) {
  stencil_batch b = nullptr;
  int rc = stencil_batch_create(items, n, boundary, &b);
  if (rc) return rc;
  rc = stencil_batch_run(b, cuda_stream);
  if (rc == STENCIL_OK) rc = stencil_batch_status(b);
  std::string keep = g_err;
  stencil_batch_destroy(b);
  g_err = keep;
  return rc;
}

// ------------------------------------------------------------ self-test

int stencil_selftest_barrier_timeout(double limit_ms, void* cuda_stream) {
  g_err.clear();
  if (!(limit_ms > 0.0) || limit_ms > 2000.0) return fail(STENCIL_ERR_ARG, "limit_ms must be in (0, 2000]");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  // one 1 x 64 grid whose single tile is advanced by one block, while the
  // barrier counts on one block more than the launch has: no wait can end
  // except by its wall-time limit
  double* grid = nullptr;
  unsigned int* ctl = nullptr;
  BatchItemDev* d_item = nullptr;
  BatchTile* d_tile = nullptr;
  int rc = STENCIL_OK;
  auto cleanup = [&]() {
    cudaFree(grid);
    cudaFree(ctl);
    cudaFree(d_item);
    cudaFree(d_tile);
  };
  if (dev_malloc(&grid, 2 * 64 * sizeof(double)) != cudaSuccess ||
      dev_malloc(&ctl, 4 * sizeof(unsigned int)) != cudaSuccess ||
      dev_malloc(&d_item, sizeof(BatchItemDev)) != cudaSuccess ||
      dev_malloc(&d_tile, sizeof(BatchTile)) != cudaSuccess) {
    cleanup();
    return fail(STENCIL_ERR_OOM, "allocating the self-test buffers");
  }
  BatchItemDev it{};
  it.a = grid;
  it.b = grid + 64;
  it.ny = 1;
  it.nx = 64;
  it.T = 2;
  it.w[2] = 1.0;
  BatchTile tl{0, 0, 64};
  cudaMemsetAsync(grid, 0, 2 * 64 * sizeof(double), s);
  cudaMemsetAsync(ctl, 0, 4 * sizeof(unsigned int), s);
  cudaMemcpyAsync(d_item, &it, sizeof(it), cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(d_tile, &tl, sizeof(tl), cudaMemcpyHostToDevice, s);
  BatchLaunch L;
  L.items = d_item;
  L.tiles = d_tile;
  L.ntiles = 1;
  L.max_T = 2;
  L.boundary = 0;
  L.barrier = ctl;
  L.status = reinterpret_cast<int*>(ctl + 2);
  L.spin_limit = (long long)(limit_ms * 1e6);
  L.barrier_blocks = 2;  // the launch below has one block
  cudaError_t e = launch_batched(L, 1, batched_default_cpt(), s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  int st = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&st, ctl + 2, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) rc = cuda_fail(e, "running the self-test");
  cleanup();
  if (rc) return rc;
  if (st != STENCIL_ERR_TIMEOUT)
    return fail(STENCIL_ERR_CUDA, "the bounded wait did not report a timeout (status %d)", st);
  return st;
}

int stencil_selftest_flag_timeout(double limit_ms, void* cuda_stream) {
  g_err.clear();
  if (!(limit_ms > 0.0) || limit_ms > 2000.0) return fail(STENCIL_ERR_ARG, "limit_ms must be in (0, 2000]");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  // one 32 x 64 grid cut into 2 x 2 tiles of the batched temporal kernel
  // (Tb = 2, T = 4), launched with only three of the four tiles: the fourth
  // tile's flag is never set, so the second block's waits can only end by
  // their wall-time limit
  double* grid = nullptr;
  unsigned int* ctl = nullptr;
  unsigned int* flags = nullptr;
  BatchTbItemDev* d_item = nullptr;
  BatchTbTile* d_tiles = nullptr;
  int rc = STENCIL_OK;
  auto cleanup = [&]() {
    cudaFree(grid);
    cudaFree(ctl);
    cudaFree(flags);
    cudaFree(d_item);
    cudaFree(d_tiles);
  };
  const int ny = 32, nx = 64, n = ny * nx;
  if (dev_malloc(&grid, 2 * n * sizeof(double)) != cudaSuccess ||
      dev_malloc(&ctl, 4 * sizeof(unsigned int)) != cudaSuccess ||
      dev_malloc(&flags, 4 * sizeof(unsigned int)) != cudaSuccess ||
      dev_malloc(&d_item, sizeof(BatchTbItemDev)) != cudaSuccess ||
      dev_malloc(&d_tiles, 3 * sizeof(BatchTbTile)) != cudaSuccess) {
    cleanup();
    return fail(STENCIL_ERR_OOM, "allocating the self-test buffers");
  }
  BatchTbItemDev it{};
  it.a = grid;
  it.b = grid + n;
  it.ny = ny;
  it.nx = nx;
  it.T = 4;
  it.tiles_y = 2;
  it.tiles_x = 2;
  it.reach_y = 1;
  it.reach_x = 1;
  it.tile_base = 0;
  it.w[2] = 1.0;
  it.zero = 0.0;
  const BatchTbTile tl[3] = {{0, 0, 0}, {0, 0, 1}, {0, 1, 0}};  // tile (1, 1) left out
  cudaMemsetAsync(grid, 0, 2 * n * sizeof(double), s);
  cudaMemsetAsync(ctl, 0, 4 * sizeof(unsigned int), s);
  cudaMemsetAsync(flags, 0, 4 * sizeof(unsigned int), s);
  cudaMemcpyAsync(d_item, &it, sizeof(it), cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(d_tiles, tl, sizeof(tl), cudaMemcpyHostToDevice, s);
  BatchTbLaunch L;
  L.items = d_item;
  L.tiles = d_tiles;
  L.ntiles = 3;
  L.max_blocks = 2;
  L.flags = flags;
  L.status = reinterpret_cast<int*>(ctl + 2);
  L.spin_limit = (long long)(limit_ms * 1e6);
  cudaError_t e = launch_batched_tb(L, 3, 2, STENCIL_DIRICHLET_ZERO, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  int st = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&st, ctl + 2, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) rc = cuda_fail(e, "running the self-test");
  cleanup();
  if (rc) return rc;
  if (st != STENCIL_ERR_TIMEOUT)
    return fail(STENCIL_ERR_CUDA, "the bounded wait did not report a timeout (status %d)", st);
  return st;
}

int stencil_selftest_tma_timeout(double limit_ms, void* cuda_stream) {
  g_err.clear();
  if (!(limit_ms > 0.0) || limit_ms > 2000.0) return fail(STENCIL_ERR_ARG, "limit_ms must be in (0, 2000]");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  // an 8 x 32 x 128 periodic grid on the TMA-fed streaming kernel (7-point
  // star), whose producer warp posts no copy -- and not the arrival that
  // announces its bytes -- for the second plane of every CTA: the consumers'
  // mbarrier waits for that plane can only end by their wall-time limit
  const Geom g{8, 32, 128};
  const size_t cells = (size_t)g.cells();
  double* a = nullptr;
  double* b = nullptr;
  double* w = nullptr;
  int* status = nullptr;
  auto cleanup = [&]() {
    cudaFree(a);
    cudaFree(b);
    cudaFree(w);
    cudaFree(status);
  };
  if (dev_malloc(&a, cells * sizeof(double)) != cudaSuccess ||
      dev_malloc(&b, cells * sizeof(double)) != cudaSuccess ||
      dev_malloc(&w, (7 + kExtraSlots) * sizeof(double)) != cudaSuccess ||
      dev_malloc(&status, sizeof(int)) != cudaSuccess) {
    cleanup();
    return fail(STENCIL_ERR_OOM, "allocating the self-test buffers");
  }
  HostTaps taps;
  taps.n = 7;
  for (int k = 0; k < 7; ++k) {
    taps.w[k] = k == 3 ? 1.0 : 0.0;
    taps.dz[k] = taps.dy[k] = taps.dx[k] = 0;
  }
  std::vector<double> hw(7 + kExtraSlots, 0.0);
  hw[3] = 1.0;
  for (int k = 0; k < kOneSlots; ++k) hw[7 + kZeroSlots + k] = 1.0;
  cudaMemsetAsync(a, 0, cells * sizeof(double), s);
  cudaMemsetAsync(status, 0, sizeof(int), s);
  cudaMemcpyAsync(w, hw.data(), hw.size() * sizeof(double), cudaMemcpyHostToDevice, s);
  int rc = STENCIL_OK;
  cudaError_t e = launch_stream3d(Shape::kStar, kPeriodic, g, taps, w, a, b, status, sm_count(), s,
                                  (unsigned long long)(limit_ms * 1e6), 1);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  int st = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&st, status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) rc = cuda_fail(e, "running the self-test");
  cleanup();
  if (rc) return rc;
  if (st != STENCIL_ERR_TIMEOUT)
    return fail(STENCIL_ERR_CUDA, "the bounded mbarrier wait did not report a timeout (status %d)", st);
  return st;
}

// ------------------------------------------------------------ measurement

int stencil_fp64_peak(double millis, double* dfma_per_s, void* cuda_stream) {
  g_err.clear();
  if (!dfma_per_s || !(millis > 0)) return fail(STENCIL_ERR_ARG, "bad argument");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const int blocks = sm_count() * 8;
  double* out = nullptr;
  CUDA_TRY(dev_malloc(&out, sizeof(double) * blocks * 256), "allocating the output");
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int iters = 256;
  double rate = 0.0;
  int rc = STENCIL_OK;
  for (int round = 0; round < 8; ++round) {
    cudaEventRecord(e0, s);
    cudaError_t e = launch_fp64_peak(blocks, iters, out, s);
    cudaEventRecord(e1, s);
    if (e != cudaSuccess) { rc = cuda_fail(e, "launching the peak kernel"); break; }
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    rate = (double)blocks * 256.0 * 8.0 * iters / (ms * 1e-3);
    if (ms >= millis * 0.5) break;
    double scale = millis / std::max(0.01, (double)ms);
    iters = (int)std::min(1.0e8, iters * scale);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (rc) return rc;
  *dfma_per_s = rate;
  return STENCIL_OK;
}

}  // extern "C"
