// taps.cuh -- how the sweep kernels hold their weights.
//
// On this GPU the FP64 unit reaches its full rate (2 DFMA per clock per SM)
// only when every operand of the FMA is a per-thread register; an operand
// read from the constant bank (a kernel parameter), a DMUL or a DADD runs at
// about 83% of it.  So the weights are loaded from device memory into
// registers once per thread, and the first product of each chain is an FMA
// onto a register that holds 0.0 (fma(w, v, +0) equals w*v, except that a
// product of -0 becomes +0, which does not change any later sum).
#pragma once

namespace gbst {

// Device layout of a plan's weights: NT weights in tap order, then
// kZeroSlots zeros (one per independent accumulation chain of a thread),
// then kOneSlots ones.  An addition a + b is issued as fma(a, one, b) with
// `one` a register: it rounds exactly like the addition but runs at the
// FMA's full rate (DADD runs at about 83% of it).
constexpr int kZeroSlots = 4;
constexpr int kOneSlots = 4;
constexpr int kExtraSlots = kZeroSlots + kOneSlots;

#ifdef __CUDACC__
template <int NT>
struct RegWeights {
  double w[NT];
  double z[kZeroSlots];
  double o[kOneSlots];
  __device__ __forceinline__ void load(const double* __restrict__ p) {
#pragma unroll
    for (int k = 0; k < NT; ++k) w[k] = __ldg(p + k);
#pragma unroll
    for (int k = 0; k < kZeroSlots; ++k) z[k] = __ldg(p + NT + k);
#pragma unroll
    for (int k = 0; k < kOneSlots; ++k) o[k] = __ldg(p + NT + kZeroSlots + k);
  }
  // a + b at the FMA rate (slot c of the ones)
  __device__ __forceinline__ double add(double a, double b, int c) const { return fma(a, o[c], b); }
  // acc = w_k * v + acc, the chain's first tap (k == 0) starting from zero slot c
  __device__ __forceinline__ void tap(double& acc, int k, double v, int c) const {
    acc = fma(w[k], v, k == 0 ? z[c] : acc);
  }
};
#endif

}  // namespace gbst
