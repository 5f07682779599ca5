/*
 * stencil.h -- C ABI of the GB300 (sm_103a) FP64 iterative-stencil library.
 *
 * The operation (paper Sec. 2.1, Listing 1 "Heat-2D Stencil", Eq. 3): every
 * point of a d-dimensional grid is replaced, once per time step, by a weighted
 * sum of itself and its neighbours at the previous step,
 *
 *     u^{t+1}(x) = sum_{o in [-r, r]^d} w_o * u~^t(x + o),
 *
 * where u~ is u extended by the boundary rule.  The update order inside a step
 * is free (Sec. 1, first key observation), which is what makes the library's
 * spatial and temporal tiling legal.  Arithmetic is IEEE binary64 throughout.
 *
 * Conventions for every entry point:
 *   - dims are listed slowest axis first; the last axis is contiguous in
 *     memory (row-major, C order).  ndim is 1, 2 or 3.
 *   - weights is a dense (2r+1)^ndim array of doubles in the same axis order;
 *     entry k along an axis is offset k - r.  A zero entry is not a tap.
 *     The update is a correlation: u'(x) = sum_o w_o u(x+o).
 *   - boundary: STENCIL_DIRICHLET_ZERO updates every cell and reads 0 for a
 *     neighbour outside the grid; STENCIL_PERIODIC wraps indices.
 *   - d_* pointers are device memory owned by the caller (for example torch
 *     tensors): contiguous FP64, at least 8-byte aligned.  h_* pointers are host
 *     memory owned by the caller.  The library owns plans, their ping-pong and
 *     checkpoint buffers and their tuning records; scratch is allocated on the
 *     first call that needs it and freed by stencil_destroy.
 *   - cuda_stream is a cudaStream_t (NULL = the legacy default stream).  Calls
 *     are asynchronous on that stream unless stated otherwise.
 *   - Every call returns a stencil_status.  On failure, stencil_last_error()
 *     returns a message for the calling thread.  A plan is not thread-safe.
 */
#ifndef GB300_STENCIL_H
#define GB300_STENCIL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct stencil_plan_s* stencil_plan;   /* opaque, library-owned */
typedef struct stencil_batch_s* stencil_batch; /* opaque, library-owned */

typedef enum {
  STENCIL_DIRICHLET_ZERO = 0,
  STENCIL_PERIODIC = 1
} stencil_boundary;

typedef enum {
  STENCIL_OK = 0,
  STENCIL_ERR_ARG = -1,          /* invalid argument (nothing was launched) */
  STENCIL_ERR_UNSUPPORTED = -2,  /* valid but not supported by this build */
  STENCIL_ERR_OOM = -3,          /* device or host allocation failed */
  STENCIL_ERR_CUDA = -4,         /* a CUDA runtime or driver call failed */
  STENCIL_ERR_TIMEOUT = -5       /* a bounded device-side wait gave up */
} stencil_status;

/* ------------------------------------------------------------------ plans */

/* Creates a plan for the constant-weight stencil of Sec. 2.1 / Listing 1.
 * ndim in {1,2,3}; dims[ndim] >= 1; radius in {1, 2}; weights as above
 * (copied, host memory); boundary a stencil_boundary.  *out receives the
 * plan.  Errors: STENCIL_ERR_ARG for a bad shape, radius, boundary or a
 * non-finite weight; STENCIL_ERR_UNSUPPORTED for an axis longer than 2^30
 * cells, or a grid whose slowest of three axes exceeds 65535 cells or whose
 * middle axis exceeds 524280 (limits of the kernels' launch grids).  The
 * total cell count may exceed 2^31 (64-bit offsets).  No device memory is
 * allocated here. */
int stencil_create(int ndim, const int64_t* dims, int radius, const double* weights,
                   int boundary, stencil_plan* out);

/* Creates a plan for the variable-coefficient diffusion step (an explicit
 * step of du/dt = div(kappa grad u), the heat equation of Eq. 1 with a
 * per-cell diffusivity):
 *   u'_i = u_i + dt * sum_{faces n} 0.5*(kappa_i + kappa_n) * (u_n - u_i)
 * over the 2*ndim face neighbours.  Periodic wraps; Dirichlet zero uses
 * u_n = 0 and the face coefficient kappa_i outside the grid.  ndim in {2,3}. */
int stencil_create_varcoef(int ndim, const int64_t* dims, int boundary, stencil_plan* out);

/* Frees the plan and everything it owns (synchronises the device first). */
void stencil_destroy(stencil_plan p);

/* ------------------------------------------------------------------ sweeps */

/* Advances d_grid (device, dims of the plan, in place) by T >= 0 steps.
 * Constant-weight plans ignore d_kappa and dt.  Variable-coefficient plans
 * need d_kappa (device, same shape) and dt > 0.  The library alternates
 * between d_grid and a plan-owned buffer and leaves the result in d_grid.
 * The fused step count Tb and kernel variant come from stencil_set_tuning,
 * the autotuner record, or a default (see stencil_variant).
 * CUDA graphs: the first run of a plan allocates its scratch; later runs only
 * enqueue stream-ordered work (kernels, memsets, device-to-device copies) on
 * cuda_stream, so they can be captured in a CUDA graph and replayed.  The
 * graph uses the plan's buffers: it stays valid until the plan is destroyed
 * or re-tuned.  (The one-step persistent variant keeps a work list for each
 * of the last 8 (grid, T) pairs it ran; a graph captured around a run whose
 * pair has since been evicted by 8 newer pairs is no longer valid.) */
int stencil_run(stencil_plan p, double* d_grid, int64_t T, const double* d_kappa, double dt,
                void* cuda_stream);

/* The same sweep on a HOST buffer: copies h_grid to a plan-owned device
 * buffer, runs T steps, copies the result back into h_grid and waits for the
 * stream.  Pinned host memory makes the copies asynchronous DMA. */
int stencil_run_host(stencil_plan p, double* h_grid, int64_t T, const double* h_kappa,
                     double dt, void* cuda_stream);

/* FP32 twin of stencil_run, for accuracy studies only: the paper compares an
 * FP32 run of its thermal-diffusion case with FP64 (Sec. 5.5, Table 4) to
 * show why the method keeps FP64.  Same plan (constant weights, up to 27
 * taps), same tap order, weights rounded to float.  d_grid and d_work are
 * device float arrays of the plan's shape (caller-owned); the result is left
 * in d_grid.  No FP64 entry point uses this path. */
int stencil_run_f32(stencil_plan p, float* d_grid, float* d_work, int64_t T, void* cuda_stream);

/* Loss and gradients of the variable-coefficient sweep (the adjoint, or
 * transposed stencil swept backward in time):
 *   u^0 = d_u0, u^{t+1} = A(kappa) u^t, L = 0.5 * sum_i (u^T_i - target_i)^2,
 *   lambda^T = u^T - target, lambda^t = A^T lambda^{t+1},
 *   dL/du0 = lambda^0,
 *   dL/dkappa_i = -(dt/2) sum_t sum_{faces n} (lambda^{t+1}_i - lambda^{t+1}_n)(u^t_i - u^t_n)
 *   (ghost faces under Dirichlet: -dt sum_t lambda^{t+1}_i u^t_i per face),
 * with dt held constant.  The forward states are checkpointed every
 * ckpt_every steps and recomputed one segment at a time in reverse, so
 * device memory grows with sqrt(T) rather than T when ckpt_every is about
 * sqrt(T); the last segment's states are kept by the forward sweep and never
 * recomputed.  ckpt_every = 1 keeps every state (no recompute, T + 10 grids
 * of scratch: 126 GiB for 256^3 and T = 1000, which an HBM3e part of 288 GB
 * holds).  ckpt_every = 0 takes round(sqrt(T)).  The results do not depend on
 * the interval (bitwise).  The plan keeps its adjoint scratch (checkpoints,
 * segment states, adjoint fields: (T/c + c + 8) grids) for the next call, so
 * repeated calls allocate nothing; a call that needs less than half of it
 * gives it back and allocates its own size, and stencil_destroy frees it.
 * d_grad_u0 and d_grad_kappa (device, caller-owned, same shape) are
 * overwritten; *h_loss (host) receives L and the call waits for the stream. */
int stencil_adjoint(stencil_plan p, const double* d_u0, const double* d_kappa, double dt,
                    const double* d_target, int64_t T, int ckpt_every, double* d_grad_u0,
                    double* d_grad_kappa, double* h_loss, void* cuda_stream);

/* The same reverse sweep for any upstream gradient: given lambda^T = dL/du^T
 * (device, same shape) for some scalar L of u^T, writes dL/du0 = lambda^0
 * and dL/dkappa (formulas above) into d_grad_u0 and d_grad_kappa.
 * Asynchronous on cuda_stream (the vector-Jacobian product behind the
 * torch.autograd.Function of the binding). */
int stencil_adjoint_vjp(stencil_plan p, const double* d_u0, const double* d_kappa, double dt,
                        int64_t T, int ckpt_every, const double* d_lambda_T, double* d_grad_u0,
                        double* d_grad_kappa, void* cuda_stream);

/* ----------------------------------------------------------- batched form */

/* One independent 2D heat grid of a batch: ny x nx cells (row-major, device,
 * in place; at most 2^31 - 1 cells, STENCIL_ERR_UNSUPPORTED otherwise), Eq. 3
 * weights (1-4*alpha at the centre, alpha at the four neighbours), T >= 0
 * steps. */
typedef struct {
  int64_t ny, nx;
  double alpha;
  int64_t T;
  double* d_grid;
} stencil_batch_item;

/* Builds a batch plan: cuts every item into tiles of 512 consecutive cells,
 * lists them by the item's T (largest first) as one persistent kernel's
 * device work list, allocates one partner buffer for all items, the item
 * table and the barrier words, and captures the whole advance (every item
 * by its own T, a bounded device-wide barrier between steps) as one CUDA
 * graph on first run.  items is copied.  All items share the boundary rule. */
int stencil_batch_create(const stencil_batch_item* items, int n, int boundary,
                         stencil_batch* out);

/* Advances every item of the batch by its own T, in place, by replaying the
 * captured graph on cuda_stream.  Device-side waits are bounded; if one
 * gives up, the batch records STENCIL_ERR_TIMEOUT, which stencil_batch_status
 * and the next stencil_batch_run return. */
int stencil_batch_run(stencil_batch b, void* cuda_stream);

/* Waits for the batch's last run and returns its device status word. */
int stencil_batch_status(stencil_batch b);

void stencil_batch_destroy(stencil_batch b);

/* Kernel configuration of a batch.  Tb = 1 (or 0): one step per device-wide
 * barrier, with cells_per_thread (1, 2 or 4; a tile is 256 *
 * cells_per_thread consecutive cells of one item) and cooperative blocks per
 * SM (1 .. the kernel's occupancy; 0 restores the defaults 2 and
 * min(occupancy, 4)).  Tb = 2, 4 or 8: Tb steps in shared memory per
 * exchange, every item cut into tiles of at most 16 x 32 cells that
 * synchronise through per-tile flags with the tiles of the same item their
 * halo reaches (cells_per_thread and blocks_per_sm are then ignored).
 * Rebuilds the work list and recaptures the graph on the next run; waits for
 * the device.  Results do not depend on it (bitwise). */
int stencil_batch_set_tuning(stencil_batch b, int Tb, int cells_per_thread, int blocks_per_sm);

/* Reports the batch's Tb, cells per thread (0 when Tb > 1) and blocks per SM. */
int stencil_batch_get_tuning(stencil_batch b, int* Tb, int* cells_per_thread, int* blocks_per_sm);

/* The batch autotuner: times every configuration (Tb = 1 with each
 * (cells_per_thread, blocks_per_sm) pair, and Tb = 2, 4, 8) on
 * scratch copies of the items (the caller's grids are not modified), each
 * item advanced ceil(T * probe_steps / max T) steps so the probe keeps the
 * batch's mix of step counts, keeps the fastest and rebuilds the batch for
 * it.  Synchronous; allocates and frees two copies of the items' cells.
 * *best_gstencils (may be NULL) receives the winner's rate in 1e9 cell
 * updates per second. */
int stencil_batch_autotune(stencil_batch b, int64_t probe_steps, void* cuda_stream,
                           double* best_gstencils);

/* Convenience: create, run once, wait, destroy. */
int stencil_run_batched(const stencil_batch_item* items, int n, int boundary,
                        void* cuda_stream);

/* Waits for cuda_stream and returns the plan's device status word: STENCIL_OK,
 * or STENCIL_ERR_TIMEOUT when a bounded device-side wait of one of the plan's
 * kernels gave up since the last call (the word is then cleared). */
int stencil_plan_status(stencil_plan p, void* cuda_stream);

/* ------------------------------------------------------------- tuning */

/* Kernel variants (ids are stable).  Defaults when nothing is forced or
 * tuned: 3D radius 1 -> STREAM; 2D radius 1 -> PERSISTENT with Tb = 4 up to
 * 2^18 cells, PERSISTENT with Tb = 1 (5-point star) up to 3 * 2^20 cells,
 * else STREAM; 2D radius 2 -> STREAM; 1D -> TEMPORAL with Tb = 8; anything
 * else -> DIRECT.  STREAM needs an even nx and, for periodic grids, nx a
 * multiple of 64 and ny a multiple of the tile height (32 for the 3D star,
 * 16 otherwise); other shapes default to DIRECT.  A variant a plan cannot
 * use (including STREAM on buffers not 16-byte aligned) falls back to DIRECT
 * unless it was forced, in which case stencil_run returns
 * STENCIL_ERR_UNSUPPORTED. */
typedef enum {
  STENCIL_VARIANT_AUTO = 0,
  STENCIL_VARIANT_DIRECT = 1,     /* one launch per step, any shape */
  STENCIL_VARIANT_STREAM = 2,     /* one launch per step, TMA-fed tiles streamed
                                     along the slowest axis (2D/3D, radius 1;
                                     2D radius 2) */
  STENCIL_VARIANT_TEMPORAL = 3,   /* Tb fused steps per launch (overlapped
                                     tiles): Tb 2, 4 or 8 (1D; 2D and 3D
                                     radius 1) */
  STENCIL_VARIANT_PERSISTENT = 4, /* one launch for all T steps (2D radius 1):
                                     Tb = 1 with a device-wide barrier per step
                                     (5-point star), Tb > 1 with Tb steps in
                                     shared memory per exchange */
  STENCIL_VARIANT_EXCHANGE = 5    /* Tb fused steps per launch with no
                                     recomputed halo (3D radius 1, Tb 2, 4 or
                                     8): the space-time tiles of Sec. 4.1
                                     computed "without redundant computation",
                                     one co-resident CTA per 64-column tile,
                                     intermediate time levels handed between
                                     tiles through an L2-resident ring of
                                     (Tb-1) x K grid planes (plan-owned; K =
                                     5 for a star, 6 for a box, 9 / 10 at
                                     Tb = 2).
                                     Needs nx even (a multiple of 64 on a
                                     periodic grid) and at most one 64-column
                                     tile column per SM.  A plane taller
                                     than the co-resident tiles cover (32
                                     rows each) runs as bands of rows, one
                                     launch each, every band with a margin of
                                     Tb-1 rows toward each neighbouring band
                                     that both bands compute */
} stencil_variant;

/* Fixes the fused step count Tb (1, 2, 4 or 8) and kernel variant (a
 * stencil_variant; 0 = let the library choose) for later runs of p.
 * Tb = 0 returns the plan to the tuned / default choice.  With variant 0 the
 * library keeps the Tb: for Tb > 1 the exchange kernel (3D radius 1, nx
 * even -- a multiple of 64 when periodic -- and at most 64 columns per SM),
 * the persistent temporal kernel (2D radius 1 up to 2^18 cells) or the
 * overlapped temporal kernel; for Tb = 1 a one-step kernel.  A run reports
 * STENCIL_ERR_UNSUPPORTED when the plan has no fused kernel for the Tb (2D
 * and 3D radius 2), and when a variant named here cannot take the grid (the
 * kernels' limits are listed with stencil_variant): neither a named variant
 * nor a fixed Tb is dropped silently. */
int stencil_set_tuning(stencil_plan p, int Tb, int variant);

/* Reports the Tb and variant the next stencil_run of p will use. */
int stencil_get_tuning(stencil_plan p, int* Tb, int* variant);

/* Tile shape of the 3D TMA-fed streaming kernel (STENCIL_VARIANT_STREAM,
 * radius 1): tiles of tile_x = 64 columns (one warp's 32 lanes x 2 cells; 0
 * also means 64) by tile_y rows, tile_y in {8, 16, 32}, or 0 for the default
 * (32 for a star, 16 for a box).  Periodic grids need ny a multiple of
 * tile_y (STENCIL_ERR_UNSUPPORTED at the next run otherwise).  The paper's
 * blocking sizes are per-benchmark tuning parameters too (Table 1); results
 * do not depend on the tile (bitwise).  The temporal kernels' tiles follow
 * from Tb and, for STENCIL_VARIANT_EXCHANGE, from the SM count (one
 * co-resident tile per SM), and are not set here.  stencil_autotune tries
 * every tile height of the streaming kernel. */
int stencil_set_tile(stencil_plan p, int tile_x, int tile_y);

/* Reports the tile of the kernel the next run of p will use: (64, tile_y)
 * for the 3D streaming kernel, (0, 0) for kernels whose tile is not a tuning
 * choice. */
int stencil_get_tile(stencil_plan p, int* tile_x, int* tile_y);

/* How the exchange kernel (STENCIL_VARIANT_EXCHANGE) cuts p's (y, x) plane
 * for Tb (2, 4 or 8) on the current device: *nbands receives the number of
 * bands of rows (one launch each per Tb-step block) and *rows_computed the
 * rows the bands compute in total -- ny, plus the Tb-1 margin rows that two
 * neighbouring bands both compute.  Errors: STENCIL_ERR_ARG for a NULL
 * argument or another Tb; STENCIL_ERR_UNSUPPORTED when the kernel does not
 * take the plan. */
int stencil_exchange_layout(stencil_plan p, int Tb, int* nbands, int64_t* rows_computed);

/* Times the candidate (Tb, variant) pairs -- and, for the 3D streaming
 * kernel, each tile height -- on d_grid (device, contents are destroyed) for
 * probe_steps steps each, after a warm-up, and keeps the fastest for p (and
 * in the tuning record: key Tb variant tile_y rate).  Synchronous.
 * *best_gstencils (may be NULL) receives its rate in 1e9 cell updates per
 * second. */
int stencil_autotune(stencil_plan p, double* d_grid, int64_t probe_steps, void* cuda_stream,
                     double* best_gstencils);

/* Name of a kernel variant id ("" for an unknown id). */
const char* stencil_variant_name(int variant);

/* ------------------------------------------------ allocation-free entry */

/* Largest grid, in cells, that stencil_run_2d_static accepts. */
#define STENCIL_STATIC_MAX_CELLS (1 << 20)

/* The paper has no counterpart: this entry point serves callers that cannot
 * allocate device memory at the moment they want a sweep -- for example code
 * whose GPU memory is owned by another allocator's pool (a framework cache
 * that has already reserved the HBM, so a cudaMalloc behind its back fails),
 * or a latency-critical loop that must not take the device-wide
 * synchronisation of cudaMalloc / cudaFree.
 *
 * Advances d_grid (device, ny x nx row-major doubles, in place) by T steps of
 * the 2D 5-point star stencil given by the dense 3x3 weights (host; the four
 * corner weights must be 0), with the given boundary rule, in one launch of
 * the persistent kernel.  It allocates nothing: the partner grid, tile list
 * and barrier words live in one array of about 8.4 MB (8.0 MiB) that every GPU loading
 * the library reserves until the process exits.
 *   - ny * nx must not exceed STENCIL_STATIC_MAX_CELLS (STENCIL_ERR_UNSUPPORTED
 *     otherwise, with a message naming the limit).
 *   - Every call shares that array and it keeps the last call's contents (the
 *     barrier words are cleared before each launch): calls whose work
 *     overlaps on the GPU race and must be serialised by the caller.
 *   - The first call on a device looks up the array's device address and the
 *     kernel's occupancy with that device current; make that first call before
 *     any stream capture begins.
 * Asynchronous on cuda_stream.  Argument and launch errors are returned at
 * once (message in stencil_last_error).  The kernel's device-wide barrier is a
 * bounded wait (2 s): if it gives up, the grid is left part-advanced and the
 * kernel records STENCIL_ERR_TIMEOUT in a status word inside the array, which
 * stencil_static_status returns. */
int stencil_run_2d_static(int64_t ny, int64_t nx, const double* weights, int boundary,
                          double* d_grid, int64_t T, void* cuda_stream);

/* Waits for cuda_stream and returns the status word of the last
 * stencil_run_2d_static launch on the current device: STENCIL_OK, or
 * STENCIL_ERR_TIMEOUT when its bounded barrier wait gave up (the word is then
 * cleared).  Copies 4 bytes to the host; allocates nothing. */
int stencil_static_status(void* cuda_stream);

/* Failure-path self-test of the allocation-free entry: launches its kernel on
 * a 1 x 64 grid held inside the static array with a device-wide barrier that
 * waits for one block more than the launch has, so the wait can only end by
 * its wall-time limit (limit_ms, at most 2000), then reads the status word.
 * Returns STENCIL_ERR_TIMEOUT when the kernel gave up and reported it as
 * designed.  Synchronous; allocates nothing; overwrites the array like any
 * other call (serialise it with them). */
int stencil_selftest_static_timeout(double limit_ms, void* cuda_stream);

/* ---------------------------------------------------------- diagnostics */

/* Message for the last failing call on this thread ("" if none). */
const char* stencil_last_error(void);

/* Number of kernels this library has launched in this process (all plans,
 * all streams), for launch accounting in benchmarks. */
int64_t stencil_launch_count(void);

/* Failure-path self-test: launches the persistent kernel (one block, a 1 x 64
 * grid) with a device-wide barrier that waits for one block more than the
 * launch has, so its wait can only end by its wall-time limit (limit_ms, at
 * most 2000).  Synchronous.  Returns STENCIL_ERR_TIMEOUT when the kernel gave
 * up and reported it as designed (the context stays usable); any other code
 * means the failure path did not behave.  Allocates and frees a few hundred
 * bytes of device memory. */
int stencil_selftest_barrier_timeout(double limit_ms, void* cuda_stream);

/* The same for the tile-flag waits of the temporal persistent kernels:
 * launches the batched temporal kernel on a 32 x 64 grid cut into 2 x 2
 * tiles with one tile left out of the work list, so the flag that tile would
 * set is never set and its neighbours' waits can only end by their
 * wall-time limit.  Returns STENCIL_ERR_TIMEOUT when they gave up as
 * designed. */
int stencil_selftest_flag_timeout(double limit_ms, void* cuda_stream);

/* The same for the TMA-fed streaming kernel's mbarrier waits: launches it on
 * an 8 x 32 x 128 periodic grid with its producer warp told to post no copy
 * (and not the arrival that announces the copy's bytes) for the second plane
 * of every CTA, so the consumers' waits for that plane can only end by their
 * wall-time limit (limit_ms, at most 2000).  No copy is left half-issued, so
 * nothing can fault.  Returns STENCIL_ERR_TIMEOUT when the kernel gave up and
 * reported it as designed.  Synchronous; allocates and frees about 0.5 MB. */
int stencil_selftest_tma_timeout(double limit_ms, void* cuda_stream);

/* Host-side fault injection for tests: after `after` more device allocations
 * by this library succeed, every later one fails as if the device were out
 * of memory, without calling the driver, until the injection is turned off
 * with a negative value (the default).  The call that needed the allocation
 * returns STENCIL_ERR_OOM at that point and launches nothing after it; the
 * plan or batch keeps what it had already allocated.  Process-wide; no GPU
 * is faulted. */
void stencil_debug_fail_allocations(int after);

/* FP64 fused multiply-add throughput of the current device, measured with a
 * kernel of independent DFMA chains on every SM for about `millis` ms.
 * *dfma_per_s receives DFMA instructions per second (2 flops each). */
int stencil_fp64_peak(double millis, double* dfma_per_s, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* GB300_STENCIL_H */
