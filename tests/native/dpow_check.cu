// Device build of the double-float power (dpow.cuh) for tests/test_gpu_dpow.py:
// F = ac (x 2^e)^a for host arrays through the GPU, the pairs formed from the
// doubles as host_dpow (host_solver_check.cpp) forms them.
#include <cuda_runtime.h>

#include "../../paper_2006_04391_gb300/csrc/dpow.cuh"

__global__ void dpow_kernel(const double* x, const int* e, const double* a, const double* ac, float* out, int* ok,
                            int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  using namespace gsm;
  const df xd = df_of(x[i]), ad = df_of(a[i]);
  const int ace = (int)((fpow::bits_of(ac[i]) >> 52) & 0x7ff) - 1023;
  const df acm = df_of(ac[i], -ace);
  df F{0.0f, 0.0f};
  ok[i] = dpow::pow_scaled(xd, e[i], a[i], ad, acm, ace, F) ? 1 : 0;
  out[4 * i] = xd.hi;
  out[4 * i + 1] = xd.lo;
  out[4 * i + 2] = F.hi;
  out[4 * i + 3] = F.lo;
}

extern "C" int dpow_many(const double* x, const int* e, const double* a, const double* ac, float* out, int* ok,
                         int n) {
  if (n <= 0) return -1;
  double *dx = nullptr, *da = nullptr, *dac = nullptr;
  int *de = nullptr, *dok = nullptr;
  float* dout = nullptr;
  int rc = 0;
  if (cudaMalloc(&dx, n * sizeof(double)) != cudaSuccess || cudaMalloc(&da, n * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&dac, n * sizeof(double)) != cudaSuccess || cudaMalloc(&de, n * sizeof(int)) != cudaSuccess ||
      cudaMalloc(&dok, n * sizeof(int)) != cudaSuccess || cudaMalloc(&dout, 4 * n * sizeof(float)) != cudaSuccess) {
    rc = -2;
  } else {
    cudaMemcpy(dx, x, n * sizeof(double), cudaMemcpyHostToDevice);
    cudaMemcpy(da, a, n * sizeof(double), cudaMemcpyHostToDevice);
    cudaMemcpy(dac, ac, n * sizeof(double), cudaMemcpyHostToDevice);
    cudaMemcpy(de, e, n * sizeof(int), cudaMemcpyHostToDevice);
    dpow_kernel<<<(n + 255) / 256, 256>>>(dx, de, da, dac, dout, dok, n);
    if (cudaMemcpy(out, dout, 4 * n * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(ok, dok, n * sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
      rc = -3;
  }
  cudaFree(dx);
  cudaFree(da);
  cudaFree(dac);
  cudaFree(de);
  cudaFree(dok);
  cudaFree(dout);
  return rc;
}
