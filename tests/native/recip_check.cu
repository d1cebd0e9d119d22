// Device build of the FP32-seeded Newton reciprocal recip_pos (solver.cuh)
// for tests/test_gpu_recip.py: applies it to a host array through the GPU.
#include <cuda_runtime.h>

#include "../../paper_2006_04391_gb300/csrc/solver.cuh"

__global__ void recip_kernel(const double* x, double* r, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) r[i] = gsm::recip_pos(x[i]);
}

extern "C" int recip_many(const double* x_host, double* r_host, int n) {
  double *x = nullptr, *r = nullptr;
  if (n <= 0) return -1;
  if (cudaMalloc(&x, n * sizeof(double)) != cudaSuccess) return -2;
  if (cudaMalloc(&r, n * sizeof(double)) != cudaSuccess) {
    cudaFree(x);
    return -2;
  }
  cudaMemcpy(x, x_host, n * sizeof(double), cudaMemcpyHostToDevice);
  recip_kernel<<<(n + 255) / 256, 256>>>(x, r, n);
  const cudaError_t e = cudaMemcpy(r_host, r, n * sizeof(double), cudaMemcpyDeviceToHost);
  cudaFree(x);
  cudaFree(r);
  return e == cudaSuccess ? 0 : -3;
}
