// The standalone ODE material-update kernel (AutoMat, arXiv 2006.04391,
// Sec. 4.3, Corollary 1, Sec. 4.5) and its launcher, instantiated per
// integrator in ode23.cu, ode12.cu and ode23s.cu (one translation unit each,
// compiled in parallel).  One thread per voxel; fields in HBM (or page-locked
// host memory) in structure-of-arrays layout.
#pragma once

#include <type_traits>

#include "common.cuh"
#include "ode23.cuh"

namespace gsm {

// Launch the update of n voxels with integrator PAIR (ERK_BS23, ERK_HEUN12 or
// ROS_23S) for the law of m; pointers are device addresses; tangent may be NULL.
template <int PAIR>
void ode_launch(const Material& m, int64_t n, int64_t ld, const Step& hs, const Ode23Ctl& ctl, const double* e0,
                const double* e1, const double* zi, double* so, double* zo, double* to, int32_t* sto,
                cudaStream_t s);

// Each integrator's kernels live in their own translation unit only.
#define GSM_ODE_EXTERN(PAIR)                                                                                     \
  extern template void ode_launch<PAIR>(const Material&, int64_t, int64_t, const Step&, const Ode23Ctl&,         \
                                        const double*, const double*, const double*, double*, double*, double*, \
                                        int32_t*, cudaStream_t);
GSM_ODE_EXTERN(ERK_BS23)
GSM_ODE_EXTERN(ERK_HEUN12)
GSM_ODE_EXTERN(ROS_23S)
#undef GSM_ODE_EXTERN

#ifdef GSM_ODE_KERNEL_IMPL
namespace {


constexpr int kOdeBlock = 128;

// Per-lane scheduling (without the tangent): a lane takes voxels i, i +
// stride, ... and starts its next voxel as soon as the current one has
// finished its substeps; the warp runs while any lane has work.  Voxels need
// different substep counts, and with one voxel per lane per pass the finished
// lanes would idle until the slowest voxel of their warp is done (measured:
// 23.7 of 32 lanes busy; 28.7 -> 31.2 M voxel-updates/s).
template <class Law, bool TAN, int PAIR>
__global__ void __launch_bounds__(kOdeBlock) ode23_kernel(int64_t n, int64_t ld, LawParams<double> p, Step hs,
                                                          Ode23Ctl ctl, const double* __restrict__ epsn,
                                                          const double* __restrict__ eps,
                                                          const double* __restrict__ zn, double* __restrict__ sig,
                                                          double* __restrict__ z, double* __restrict__ tan,
                                                          int32_t* __restrict__ status) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  constexpr int NZ = stored_nz<Law>();
  OdeVoxel<Law, TAN, PAIR> v;
  // with TAN: psi's second-derivative blocks, constants of the law, once per block
  __shared__ PsiBlocks<Law::NY> blk;
  if constexpr (TAN) {
    if (threadIdx.x == 0) psi_const_blocks<Law>(p, blk);
    __syncthreads();
  }
  auto start = [&](int64_t k) {
    double e0[6], e1[6], zi[NZ];
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      e0[c] = __ldg(epsn + c * ld + k);
      e1[c] = __ldg(eps + c * ld + k);
    }
#pragma unroll
    for (int c = 0; c < NZ; ++c) zi[c] = __ldg(zn + c * ld + k);
    v.init(p, e0, e1, zi, hs.h, TAN ? &blk : nullptr);
  };
  if constexpr (TAN) {
    // with the tangent the state lives mostly in local memory (register
    // spills); there one voxel per lane per pass, warp-voted, measured faster
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
      const int64_t k = base + threadIdx.x;
      const bool active = k < n;
      if (active) start(k);
      else v.done = true;
      for (;;) {
        if (all_done(v.done)) break;
        if (!v.done) v.attempt(p, hs, ctl);
      }
      if (active) {
        double s[6], zo[NZ], t36[36];
        const unsigned st = v.finish(hs.h, s, zo, t36);
#pragma unroll
        for (int c = 0; c < 6; ++c) sig[c * ld + k] = s[c];
#pragma unroll
        for (int c = 0; c < NZ; ++c) z[c * ld + k] = zo[c];
#pragma unroll
        for (int c = 0; c < 36; ++c) tan[c * ld + k] = t36[c];
        if (status) status[k] = (int32_t)st;
      }
    }
    return;
  }
  bool have = i < n;
  if (have) start(i);
  while (__any_sync(0xffffffffu, have)) {
    if (!have) continue;
    v.attempt(p, hs, ctl);
    if (v.done) {
      double s[6], zo[NZ];
      const unsigned st = v.finish(hs.h, s, zo, nullptr);
#pragma unroll
      for (int c = 0; c < 6; ++c) sig[c * ld + i] = s[c];
#pragma unroll
      for (int c = 0; c < NZ; ++c) z[c * ld + i] = zo[c];
      if (status) status[i] = (int32_t)st;
      i += stride;
      have = i < n;
      if (have) start(i);
    }
  }
}

template <auto Kernel> int ode_grid(int64_t n) {
  static const int per_sm = [] {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, Kernel, kOdeBlock, 0) != cudaSuccess || b <= 0) b = 1;
    return b;
  }();
  const int64_t need = (n + kOdeBlock - 1) / kOdeBlock;
  const int64_t cap = (int64_t)sm_count() * per_sm;
  return (int)(need < cap ? need : cap);
}

}  // namespace

template <int PAIR>
void ode_launch(const Material& m, int64_t n_vox, int64_t ld, const Step& hs, const Ode23Ctl& ctl, const double* e0,
                const double* e1, const double* zi, double* so, double* zo, double* to, int32_t* sto,
                cudaStream_t s) {
  auto launch = [&](auto law) {
    using Law = decltype(law);
    if (to)
      ode23_kernel<Law, true, PAIR><<<ode_grid<ode23_kernel<Law, true, PAIR>>(n_vox), kOdeBlock, 0, s>>>(
          n_vox, ld, m.p64, hs, ctl, e0, e1, zi, so, zo, to, sto);
    else
      ode23_kernel<Law, false, PAIR><<<ode_grid<ode23_kernel<Law, false, PAIR>>(n_vox), kOdeBlock, 0, s>>>(
          n_vox, ld, m.p64, hs, ctl, e0, e1, zi, so, zo, nullptr, sto);
  };
  if (m.psi_kind == GSM_PSI_ELASTIC_VP_DEV) launch(NortonDev{});
  else launch(MichelSuquet{});
}
#endif

}  // namespace gsm
