// SIMT throughput probe: dependent FMA chains in FP64 or FP32.
//
// The material kernels are bound by FP64 (or FP32) arithmetic issue, not by
// a dense contraction, so their roofline needs the chip's measured FMA rate,
// which no library routine reports.  Each thread runs CHAINS independent
// chains x <- x * a + b for `iters` steps; with enough warps per SM the
// chains hide the pipeline latency and the kernel time is the FMA issue time.
// The caller times the launch (CUDA events on `stream`) and divides
// 2 * fmas_out by it.
#include <cuda_runtime.h>

#include "common.cuh"
#include "gsm.h"

namespace gsm {
namespace {

constexpr int kChains = 8;
constexpr int kThreads = 512;

__device__ double g_probe_sink;

template <class T>
__global__ void __launch_bounds__(kThreads) fma_chains_kernel(int64_t iters, T a, T b) {
  T x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = T(threadIdx.x + c) * T(1e-3);
  // the multiplier and addend in registers (a value the compiler cannot fold
  // back into a constant-bank operand)
  a = a + T(threadIdx.x & 1) * T(1e-30);
  b = b + T(threadIdx.x & 2) * T(1e-30);
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  T s = T(0);
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  // a store the compiler cannot prove dead: only when the sum is exactly -1
  if (s == T(-1)) g_probe_sink = double(s);
}

}  // namespace
}  // namespace gsm

using namespace gsm;

extern "C" int gsm_peak_probe(int precision, int64_t iters, int blocks_per_sm, double* fmas_out, void* stream) {
  if ((precision != 0 && precision != 1) || iters <= 0 || iters > (int64_t(1) << 32) || blocks_per_sm <= 0 ||
      blocks_per_sm > 64 || !fmas_out)
    return GSM_EINVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return GSM_ECUDA;
  const int blocks = sms * blocks_per_sm;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // a, b keep every chain bounded: x -> x a + b with |a| < 1 converges
  if (precision == 0)
    fma_chains_kernel<double><<<blocks, kThreads, 0, s>>>(iters, 0.999999, 1e-6);
  else
    fma_chains_kernel<float><<<blocks, kThreads, 0, s>>>(iters, 0.999999f, 1e-6f);
  count_launch();
  if (cudaGetLastError() != cudaSuccess) return GSM_ECUDA;
  *fmas_out = double(blocks) * kThreads * kChains * double(iters);
  return GSM_OK;
}
