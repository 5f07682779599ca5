/*
 * oracle.c -- plain, slow, obviously correct CPU FP64 reference for the
 * iterative stencil sweep, its variable-coefficient form and that form's
 * adjoint.  See oracle.h for the conventions.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by tests/, by the smoke check and by the
 * benchmark's CPU-baseline leg, never by the product library.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -fPIC -shared (see build.py).
 * No fused multiply-add, no reassociation: every sum is evaluated left to
 * right in the order written here.
 */
#include "oracle.h"

#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define MAXD 3

/* One stencil tap: its offset along each of the three (padded) axes and its
 * weight.  Paper Sec. 2.1: a point's new value is a weighted sum of itself and
 * its neighbours at the previous step; Listing 1 names the weights c1..c5. */
typedef struct {
  int64_t off[MAXD];
  double w;
} tap_t;

static int64_t wrap(int64_t a, int64_t n) {
  int64_t m = a % n;
  return m < 0 ? m + n : m;
}

static int use_threads(int nthreads) {
#ifdef _OPENMP
  if (nthreads <= 0) return omp_get_num_procs();
  return nthreads;
#else
  (void)nthreads;
  return 1;
#endif
}

/* Pads an ndim-axis shape to three axes (leading axes of length 1). */
static int pad_dims(int ndim, const int64_t* dims, int64_t n[MAXD]) {
  if (ndim < 1 || ndim > MAXD || dims == NULL) return -1;
  for (int d = 0; d < MAXD; ++d) n[d] = 1;
  for (int d = 0; d < ndim; ++d) {
    if (dims[d] < 1) return -1;
    n[MAXD - ndim + d] = dims[d];
  }
  return 0;
}

/* Lists the non-zero taps of the dense (2r+1)^ndim weight array in
 * lexicographic order of the offset (slowest axis first). */
static int build_taps(int ndim, int radius, const double* weights, tap_t** out) {
  if (radius < 0 || radius > 8 || weights == NULL) return -1;
  int64_t side = 2 * radius + 1, total = 1;
  for (int d = 0; d < ndim; ++d) total *= side;
  tap_t* taps = (tap_t*)malloc(sizeof(tap_t) * (size_t)total);
  if (!taps) return -1;
  int count = 0;
  for (int64_t k = 0; k < total; ++k) {
    if (weights[k] == 0.0) continue;
    tap_t t;
    for (int d = 0; d < MAXD; ++d) t.off[d] = 0;
    int64_t rem = k;
    for (int d = ndim - 1; d >= 0; --d) {
      t.off[MAXD - ndim + d] = rem % side - radius;
      rem /= side;
    }
    t.w = weights[k];
    taps[count++] = t;
  }
  *out = taps;
  return count;
}

/* One step of u'(x) = sum_o w_o * u~(x+o) over the whole grid (Listing 1
 * loop nest; Eq. 3 gives its heat-equation weights).  u~ is u extended by the
 * boundary rule. */
static void step_const(const int64_t n[MAXD], int ntaps, const tap_t* taps, int periodic,
                       const double* src, double* dst, int nthreads) {
  int64_t rows = n[0] * n[1];
#pragma omp parallel for num_threads(nthreads) schedule(static)
  for (int64_t zy = 0; zy < rows; ++zy) {
    int64_t z = zy / n[1], y = zy % n[1];
    for (int64_t x = 0; x < n[2]; ++x) {
      int64_t c[MAXD] = {z, y, x};
      double acc = 0.0;
      for (int k = 0; k < ntaps; ++k) {
        int64_t g[MAXD];
        int inside = 1;
        for (int d = 0; d < MAXD; ++d) {
          g[d] = c[d] + taps[k].off[d];
          if (periodic)
            g[d] = wrap(g[d], n[d]);
          else if (g[d] < 0 || g[d] >= n[d])
            inside = 0;
        }
        double v = inside ? src[(g[0] * n[1] + g[1]) * n[2] + g[2]] : 0.0;
        acc = acc + taps[k].w * v;
      }
      dst[(z * n[1] + y) * n[2] + x] = acc;
    }
  }
}

int oracle_run(int ndim, const int64_t* dims, int radius, const double* weights,
               int boundary, double* u, int64_t T, int nthreads) {
  int64_t n[MAXD];
  if (pad_dims(ndim, dims, n) != 0 || u == NULL || T < 0) return -1;
  if (boundary != 0 && boundary != 1) return -1;
  tap_t* taps = NULL;
  int ntaps = build_taps(ndim, radius, weights, &taps);
  if (ntaps < 0) return -1;
  int64_t cells = n[0] * n[1] * n[2];
  double* a = u;
  double* b = (double*)malloc(sizeof(double) * (size_t)cells);
  if (!b) { free(taps); return -1; }
  double* other = b;
  int th = use_threads(nthreads);
  for (int64_t t = 0; t < T; ++t) {  /* ping-pong: A[(t+1)%2] from A[t%2] */
    step_const(n, ntaps, taps, boundary == 1, a, b, th);
    double* s = a; a = b; b = s;
  }
  if (a != u) memcpy(u, a, sizeof(double) * (size_t)cells);
  free(other);
  free(taps);
  return 0;
}

/*
 * Light-cone evaluation of a box of outputs.  Along each axis the local
 * buffer covers either the whole axis (periodic axis that the widened box
 * would wrap around) or the global index range [lo - R, hi + R), R = r*T,
 * clipped to [-r, n + r) for Dirichlet.  Local cells outside [0, n) on a
 * Dirichlet axis are ghost cells: they stay 0 and are never updated.  Reads
 * that leave the local range (only at the artificial faces of the buffer)
 * return 0; after s steps the cells within r*s of those faces are wrong, and
 * after T steps none of them reaches [lo, hi).
 */
int oracle_run_window(int ndim, const int64_t* dims, int radius, const double* weights,
                      int boundary, const double* u, int64_t T,
                      const int64_t* lo_in, const int64_t* hi_in, double* out) {
  int64_t n[MAXD];
  if (pad_dims(ndim, dims, n) != 0 || u == NULL || out == NULL || T < 0) return -1;
  if (boundary != 0 && boundary != 1) return -1;
  if (lo_in == NULL || hi_in == NULL) return -1;
  int64_t lo[MAXD], hi[MAXD];
  for (int d = 0; d < MAXD; ++d) { lo[d] = 0; hi[d] = 1; }
  for (int d = 0; d < ndim; ++d) {
    lo[MAXD - ndim + d] = lo_in[d];
    hi[MAXD - ndim + d] = hi_in[d];
  }
  for (int d = 0; d < MAXD; ++d)
    if (lo[d] < 0 || hi[d] > n[d] || lo[d] >= hi[d]) return -1;
  tap_t* taps = NULL;
  int ntaps = build_taps(ndim, radius, weights, &taps);
  if (ntaps < 0) return -1;

  int64_t R = (int64_t)radius * T;
  int full[MAXD];
  int64_t start[MAXD], len[MAXD];
  for (int d = 0; d < MAXD; ++d) {
    int64_t a = lo[d] - R, b = hi[d] + R;
    if (boundary == 1) {
      full[d] = (b - a) >= n[d];
      if (full[d]) { a = 0; b = n[d]; }
    } else {
      full[d] = 0;
      if (a < -radius) a = -radius;
      if (b > n[d] + radius) b = n[d] + radius;
    }
    start[d] = a;
    len[d] = b - a;
  }
  int64_t cells = len[0] * len[1] * len[2];
  double* a = (double*)malloc(sizeof(double) * (size_t)cells);
  double* b = (double*)malloc(sizeof(double) * (size_t)cells);
  if (!a || !b) { free(a); free(b); free(taps); return -1; }

  /* initial local field */
  for (int64_t i0 = 0; i0 < len[0]; ++i0)
    for (int64_t i1 = 0; i1 < len[1]; ++i1)
      for (int64_t i2 = 0; i2 < len[2]; ++i2) {
        int64_t l[MAXD] = {i0, i1, i2}, g[MAXD];
        int inside = 1;
        for (int d = 0; d < MAXD; ++d) {
          g[d] = start[d] + l[d];
          if (boundary == 1)
            g[d] = wrap(g[d], n[d]);
          else if (g[d] < 0 || g[d] >= n[d])
            inside = 0;
        }
        a[(i0 * len[1] + i1) * len[2] + i2] =
            inside ? u[(g[0] * n[1] + g[1]) * n[2] + g[2]] : 0.0;
      }

  for (int64_t t = 0; t < T; ++t) {
    for (int64_t i0 = 0; i0 < len[0]; ++i0)
      for (int64_t i1 = 0; i1 < len[1]; ++i1)
        for (int64_t i2 = 0; i2 < len[2]; ++i2) {
          int64_t l[MAXD] = {i0, i1, i2};
          int64_t li = (i0 * len[1] + i1) * len[2] + i2;
          int ghost = 0;
          if (boundary == 0)
            for (int d = 0; d < MAXD; ++d) {
              int64_t g = start[d] + l[d];
              if (g < 0 || g >= n[d]) ghost = 1;
            }
          if (ghost) { b[li] = 0.0; continue; }
          double acc = 0.0;
          for (int k = 0; k < ntaps; ++k) {
            int64_t m[MAXD];
            int inside = 1;
            for (int d = 0; d < MAXD; ++d) {
              m[d] = l[d] + taps[k].off[d];
              if (full[d])
                m[d] = wrap(m[d], n[d]);
              else if (m[d] < 0 || m[d] >= len[d])
                inside = 0;
            }
            double v = inside ? a[(m[0] * len[1] + m[1]) * len[2] + m[2]] : 0.0;
            acc = acc + taps[k].w * v;
          }
          b[li] = acc;
        }
    double* s = a; a = b; b = s;
  }

  int64_t w1 = hi[1] - lo[1], w2 = hi[2] - lo[2];
  for (int64_t z = lo[0]; z < hi[0]; ++z)
    for (int64_t y = lo[1]; y < hi[1]; ++y)
      for (int64_t x = lo[2]; x < hi[2]; ++x) {
        int64_t l0 = full[0] ? z : z - start[0];
        int64_t l1 = full[1] ? y : y - start[1];
        int64_t l2 = full[2] ? x : x - start[2];
        out[((z - lo[0]) * w1 + (y - lo[1])) * w2 + (x - lo[2])] =
            a[(l0 * len[1] + l1) * len[2] + l2];
      }
  free(a);
  free(b);
  free(taps);
  return 0;
}

/* ---------------- variable-coefficient diffusion ---------------- */

/* Face neighbour slot s (0 .. 2*MAXD-1) of cell c: axis s/2, direction
 * -1 for even s and +1 for odd s.  Returns 1 and the neighbour's linear index
 * when it lies in the grid (after wrapping for periodic), 0 for a ghost. */
static int face_neighbour(const int64_t n[MAXD], const int64_t c[MAXD], int s, int periodic,
                          int64_t* idx) {
  int64_t g[MAXD] = {c[0], c[1], c[2]};
  int d = s / 2;
  g[d] += (s % 2 == 0) ? -1 : 1;
  if (periodic)
    g[d] = wrap(g[d], n[d]);
  else if (g[d] < 0 || g[d] >= n[d])
    return 0;
  *idx = (g[0] * n[1] + g[1]) * n[2] + g[2];
  return 1;
}

/* One forward step: u'_i = u_i + dt * sum_faces kf * (u_n - u_i),
 * kf = 0.5*(kappa_i + kappa_n), ghost face kf = kappa_i and u_n = 0. */
static void step_varcoef(int ndim, const int64_t n[MAXD], int periodic, const double* kappa,
                         double dt, const double* src, double* dst, int nthreads) {
  int64_t rows = n[0] * n[1];
#pragma omp parallel for num_threads(nthreads) schedule(static)
  for (int64_t zy = 0; zy < rows; ++zy) {
    int64_t z = zy / n[1], y = zy % n[1];
    for (int64_t x = 0; x < n[2]; ++x) {
      int64_t c[MAXD] = {z, y, x};
      int64_t i = (z * n[1] + y) * n[2] + x;
      double ui = src[i], ki = kappa[i];
      double acc = 0.0;
      for (int s = 2 * (MAXD - ndim); s < 2 * MAXD; ++s) {
        int64_t j;
        double un, kf;
        if (face_neighbour(n, c, s, periodic, &j)) {
          un = src[j];
          kf = 0.5 * (ki + kappa[j]);
        } else {
          un = 0.0;
          kf = ki;
        }
        acc = acc + kf * (un - ui);
      }
      dst[i] = ui + dt * acc;
    }
  }
}

int oracle_varcoef_run(int ndim, const int64_t* dims, int boundary, double* u,
                       const double* kappa, double dt, int64_t T, int nthreads) {
  int64_t n[MAXD];
  if (pad_dims(ndim, dims, n) != 0 || u == NULL || kappa == NULL || T < 0) return -1;
  if (boundary != 0 && boundary != 1) return -1;
  int64_t cells = n[0] * n[1] * n[2];
  double* a = u;
  double* b = (double*)malloc(sizeof(double) * (size_t)cells);
  if (!b) return -1;
  double* other = b;
  int th = use_threads(nthreads);
  for (int64_t t = 0; t < T; ++t) {
    step_varcoef(ndim, n, boundary == 1, kappa, dt, a, b, th);
    double* s = a; a = b; b = s;
  }
  if (a != u) memcpy(u, a, sizeof(double) * (size_t)cells);
  free(other);
  return 0;
}

/*
 * out = A^T lambda, written as the scatter of the rows of A: row i of A has
 * diagonal 1 - dt * sum_faces kf and, for every in-grid face slot with
 * neighbour n, the entry dt * kf in column n.  Column j of A^T lambda
 * collects A_ij * lambda_i.
 */
static void transpose_step_varcoef(int ndim, const int64_t n[MAXD], int periodic,
                                   const double* kappa, double dt, const double* lam,
                                   double* out) {
  int64_t cells = n[0] * n[1] * n[2];
  for (int64_t i = 0; i < cells; ++i) out[i] = 0.0;
  for (int64_t z = 0; z < n[0]; ++z)
    for (int64_t y = 0; y < n[1]; ++y)
      for (int64_t x = 0; x < n[2]; ++x) {
        int64_t c[MAXD] = {z, y, x};
        int64_t i = (z * n[1] + y) * n[2] + x;
        double ki = kappa[i];
        double diag_sum = 0.0;
        for (int s = 2 * (MAXD - ndim); s < 2 * MAXD; ++s) {
          int64_t j;
          double kf;
          if (face_neighbour(n, c, s, periodic, &j)) {
            kf = 0.5 * (ki + kappa[j]);
            out[j] = out[j] + dt * kf * lam[i];
          } else {
            kf = ki;
          }
          diag_sum = diag_sum + kf;
        }
        out[i] = out[i] + (1.0 - dt * diag_sum) * lam[i];
      }
}

int oracle_varcoef_transpose_step(int ndim, const int64_t* dims, int boundary,
                                  const double* kappa, double dt,
                                  const double* lambda, double* out) {
  int64_t n[MAXD];
  if (pad_dims(ndim, dims, n) != 0 || kappa == NULL || lambda == NULL || out == NULL) return -1;
  if (boundary != 0 && boundary != 1) return -1;
  transpose_step_varcoef(ndim, n, boundary == 1, kappa, dt, lambda, out);
  return 0;
}

/*
 * Adds to g the derivative of <lam, A(kappa) u> with respect to kappa.
 * Row i of A u is u_i + dt * sum_faces kf * (u_n - u_i); kf depends on kappa_i
 * and kappa_n with weight 1/2 each (ghost face: kappa_i with weight 1).
 */
static void accumulate_dkappa(int ndim, const int64_t n[MAXD], int periodic, double dt,
                              const double* lam, const double* u, double* g) {
  for (int64_t z = 0; z < n[0]; ++z)
    for (int64_t y = 0; y < n[1]; ++y)
      for (int64_t x = 0; x < n[2]; ++x) {
        int64_t c[MAXD] = {z, y, x};
        int64_t i = (z * n[1] + y) * n[2] + x;
        for (int s = 2 * (MAXD - ndim); s < 2 * MAXD; ++s) {
          int64_t j;
          if (face_neighbour(n, c, s, periodic, &j)) {
            double d = dt * lam[i] * (u[j] - u[i]);
            g[i] = g[i] + 0.5 * d;
            g[j] = g[j] + 0.5 * d;
          } else {
            double d = dt * lam[i] * (0.0 - u[i]);
            g[i] = g[i] + d;
          }
        }
      }
}

int oracle_varcoef_adjoint(int ndim, const int64_t* dims, int boundary,
                           const double* u0, const double* kappa, double dt,
                           const double* target, int64_t T, int ckpt_every,
                           double* grad_u0, double* grad_kappa, double* loss,
                           int nthreads) {
  int64_t n[MAXD];
  if (pad_dims(ndim, dims, n) != 0) return -1;
  if (!u0 || !kappa || !target || !grad_u0 || !grad_kappa || !loss) return -1;
  if (boundary != 0 && boundary != 1) return -1;
  if (T < 0 || ckpt_every < 0) return -1;
  int periodic = boundary == 1;
  int th = use_threads(nthreads);
  int64_t cells = n[0] * n[1] * n[2];
  size_t bytes = sizeof(double) * (size_t)cells;
  int64_t c = ckpt_every > 0 ? ckpt_every : 1;
  int64_t nck = T / c + 1;                 /* states at t = 0, c, 2c, ... <= T */
  double* ck = (double*)malloc(bytes * (size_t)nck);
  double* seg = (double*)malloc(bytes * (size_t)c);
  double* cur = (double*)malloc(bytes);
  double* nxt = (double*)malloc(bytes);
  double* lam = (double*)malloc(bytes);
  double* lam2 = (double*)malloc(bytes);
  if (!ck || !seg || !cur || !nxt || !lam || !lam2) {
    free(ck); free(seg); free(cur); free(nxt); free(lam); free(lam2);
    return -1;
  }
  /* forward sweep, keeping the state at every multiple of c */
  memcpy(cur, u0, bytes);
  memcpy(ck, u0, bytes);
  for (int64_t t = 0; t < T; ++t) {
    step_varcoef(ndim, n, periodic, kappa, dt, cur, nxt, th);
    double* s = cur; cur = nxt; nxt = s;
    if ((t + 1) % c == 0) memcpy(ck + (size_t)((t + 1) / c) * (size_t)cells, cur, bytes);
  }
  /* loss and the final adjoint state lambda^T = dL/du^T = u^T - target */
  double L = 0.0;
  for (int64_t i = 0; i < cells; ++i) {
    double r = cur[i] - target[i];
    L = L + 0.5 * r * r;
    lam[i] = r;
  }
  *loss = L;
  for (int64_t i = 0; i < cells; ++i) grad_kappa[i] = 0.0;
  /* reverse sweep, one checkpoint segment [t0, t1) at a time */
  int64_t nseg = (T + c - 1) / c;
  for (int64_t sgi = nseg - 1; sgi >= 0; --sgi) {
    int64_t t0 = sgi * c, t1 = t0 + c < T ? t0 + c : T;
    memcpy(seg, ck + (size_t)sgi * (size_t)cells, bytes);     /* u^{t0} */
    for (int64_t t = t0 + 1; t < t1; ++t)                       /* u^{t0+1} .. u^{t1-1} */
      step_varcoef(ndim, n, periodic, kappa, dt, seg + (size_t)(t - t0 - 1) * (size_t)cells,
                   seg + (size_t)(t - t0) * (size_t)cells, th);
    for (int64_t t = t1 - 1; t >= t0; --t) {
      const double* ut = seg + (size_t)(t - t0) * (size_t)cells;
      accumulate_dkappa(ndim, n, periodic, dt, lam, ut, grad_kappa);  /* uses lambda^{t+1}, u^t */
      transpose_step_varcoef(ndim, n, periodic, kappa, dt, lam, lam2);  /* lambda^t */
      double* s = lam; lam = lam2; lam2 = s;
    }
  }
  memcpy(grad_u0, lam, bytes);
  free(ck); free(seg); free(cur); free(nxt); free(lam); free(lam2);
  return 0;
}
