// peak.cu -- FP64 FMA throughput microbenchmark (the denominator of the FP64
// roofline; the chip's DFMA rate is far below its FP32 and tensor rates).
// Eight independent chains per thread, x = fma(x, a, b) with a and b kernel
// parameters, so each DFMA has one register operand and the loop measures
// the pipe, not latency or the register file.
#include "internal.h"

namespace gbst {
namespace {

__global__ void __launch_bounds__(256) k_fp64_peak(double* out, int iters, double a, double b) {
  double x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = threadIdx.x * 1e-3 + k;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += x[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

cudaError_t launch_fp64_peak(int blocks, int iters, double* out, cudaStream_t stream) {
  k_fp64_peak<<<blocks, 256, 0, stream>>>(out, iters, 0.9999999, 1e-7);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

}  // namespace gbst
