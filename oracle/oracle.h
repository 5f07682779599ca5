/*
 * oracle.h -- plain CPU FP64 reference for the iterative stencil sweep.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  The product path (the
 * CUDA library under paper_2303_08365_gb300/) shares no code, header, table
 * or helper with it.
 *
 * Definition followed (paper Sec. 2.1 and Listing 1 "Heat-2D Stencil"): the
 * value of a point at step t+1 is a weighted sum of itself and its neighbours
 * at step t, with two time levels used in ping-pong fashion.  Eq. 3 gives the
 * heat-equation weights (1-4mu at the centre, mu at the four neighbours).
 *
 * Conventions shared with the product API (restated, not included from it):
 *   - dims are listed slowest axis first, the last axis is contiguous;
 *   - weights are a dense (2r+1)^ndim array, row-major in the same axis order,
 *     offset index k along an axis maps to offset k-r; a tap with weight 0.0
 *     is not part of the stencil and is skipped;
 *   - the update is a correlation: u'(x) = sum_o w_o * u(x+o);
 *   - boundary 0 = Dirichlet zero (every cell is updated, neighbours outside
 *     the grid read 0), 1 = periodic (indices wrap modulo the axis length).
 *   - all arithmetic is IEEE binary64, round to nearest, no fused multiply-add
 *     (the library is compiled with -ffp-contract=off); the taps are summed in
 *     lexicographic order of the offset, starting from 0.0.
 *
 * Every function returns 0 on success and -1 on a bad argument.
 */
#ifndef STENCIL_ORACLE_H
#define STENCIL_ORACLE_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

/* T steps of the constant-weight stencil, in place on u (host memory). */
int oracle_run(int ndim, const int64_t* dims, int radius, const double* weights,
               int boundary, double* u, int64_t T, int nthreads);

/* Values after T steps on the box [lo, hi) of the full grid u (not modified),
 * computed from the backward light cone of the box only (the box widened by
 * radius*T per axis).  out holds prod(hi-lo) values, row-major.  Gives the
 * same numbers as oracle_run restricted to the box: the same taps in the same
 * order are evaluated for every cell whose value reaches the box. */
int oracle_run_window(int ndim, const int64_t* dims, int radius, const double* weights,
                      int boundary, const double* u, int64_t T,
                      const int64_t* lo, const int64_t* hi, double* out);

/* T steps of the variable-coefficient diffusion update (7-point in 3D,
 * 2*ndim+1 points in general), in place on u:
 *   u'_i = u_i + dt * sum_{n in N(i)} 0.5*(kappa_i + kappa_n) * (u_n - u_i)
 * N(i) = the 2*ndim face neighbours.  Periodic: indices wrap.  Dirichlet zero:
 * a neighbour outside the grid has u_n = 0 and the face uses kappa_i. */
int oracle_varcoef_run(int ndim, const int64_t* dims, int boundary, double* u,
                       const double* kappa, double dt, int64_t T, int nthreads);

/* Loss L = 0.5 * sum_i (u^T_i - target_i)^2 after T variable-coefficient
 * steps from u0, and its gradients with respect to u0 and kappa (dt held
 * fixed).  ckpt_every = 0 stores every state; ckpt_every = c > 0 keeps every
 * c-th state and recomputes the others segment by segment. */
int oracle_varcoef_adjoint(int ndim, const int64_t* dims, int boundary,
                           const double* u0, const double* kappa, double dt,
                           const double* target, int64_t T, int ckpt_every,
                           double* grad_u0, double* grad_kappa, double* loss,
                           int nthreads);

/* One application of the transposed variable-coefficient step to lambda
 * (out = A(kappa)^T lambda), for the dot-product test of the adjoint. */
int oracle_varcoef_transpose_step(int ndim, const int64_t* dims, int boundary,
                                  const double* kappa, double dt,
                                  const double* lambda, double* out);

#ifdef __cplusplus
}
#endif
#endif
