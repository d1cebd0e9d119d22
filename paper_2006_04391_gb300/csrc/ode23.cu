// gsm_update_ode / gsm_update_ode23: the material update by adaptive explicit Runge-Kutta
// integration of the force-potential form (AutoMat, arXiv 2006.04391,
// Sec. 4.3, Corollary 1, Sec. 4.5) on sm_103a.  One thread per voxel; fields
// in HBM (or page-locked host memory) in structure-of-arrays layout; a
// persistent grid-stride loop whose bound is uniform per block, so every lane
// takes part in the warp votes of the substep loop.
#include <type_traits>

#include "common.cuh"
#include "ode23.cuh"

namespace gsm {
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
  ErkVoxel<Law, TAN, PAIR> v;
  auto start = [&](int64_t k) {
    double e0[6], e1[6], zi[NZ];
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      e0[c] = __ldg(epsn + c * ld + k);
      e1[c] = __ldg(eps + c * ld + k);
    }
#pragma unroll
    for (int c = 0; c < NZ; ++c) zi[c] = __ldg(zn + c * ld + k);
    v.init(p, e0, e1, zi, hs.h);
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
}  // namespace gsm

using namespace gsm;

extern "C" int gsm_update_ode(gsm_handle h, int method, int64_t n_vox, const void* eps_n, const void* eps,
                              const void* z_n, int64_t ld, double step_h, double rtol, double atol, int max_substeps,
                              void* sigma, void* z, void* tangent, int32_t* status, void* stream) {
  if (!h || n_vox < 0 || ld < n_vox) return GSM_EINVAL;
  if (method != GSM_ODE23 && method != GSM_ODE12) return GSM_EINVAL;
  if (n_vox == 0) return GSM_OK;
  const Material& m = *reinterpret_cast<const Material*>(h);
  if (m.psi_kind != GSM_PSI_ELASTIC_VP_DEV && m.psi_kind != GSM_PSI_ELASTIC_VP_KIN) return GSM_ENOTSUP;
  if (!eps_n || !eps || !z_n || !sigma || !z) return GSM_EINVAL;
  if (!(std::isfinite(step_h) && step_h > 0.0) || !(rtol > 0.0) || !(atol >= 0.0) || max_substeps < 1)
    return GSM_EINVAL;
  const void* in[3] = {eps_n, eps, z_n};
  void* out[4] = {sigma, z, tangent, status};
  for (auto& q : in)
    if (!device_address(q, &q)) return GSM_EINVAL;
  for (auto& q : out) {
    const void* r = q;
    if (!device_address(r, &r)) return GSM_EINVAL;
    q = const_cast<void*>(r);
  }
  const Ode23Ctl ctl{rtol, atol, max_substeps};
  const Step hs = make_step(step_h);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const double* e0 = static_cast<const double*>(in[0]);
  const double* e1 = static_cast<const double*>(in[1]);
  const double* zi = static_cast<const double*>(in[2]);
  double* so = static_cast<double*>(out[0]);
  double* zo = static_cast<double*>(out[1]);
  double* to = static_cast<double*>(out[2]);
  int32_t* sto = static_cast<int32_t*>(out[3]);
  auto launch = [&](auto law, auto pair) {
    using Law = decltype(law);
    constexpr int PAIR = decltype(pair)::value;
    if (to)
      ode23_kernel<Law, true, PAIR><<<ode_grid<ode23_kernel<Law, true, PAIR>>(n_vox), kOdeBlock, 0, s>>>(
          n_vox, ld, m.p64, hs, ctl, e0, e1, zi, so, zo, to, sto);
    else
      ode23_kernel<Law, false, PAIR><<<ode_grid<ode23_kernel<Law, false, PAIR>>(n_vox), kOdeBlock, 0, s>>>(
          n_vox, ld, m.p64, hs, ctl, e0, e1, zi, so, zo, nullptr, sto);
  };
  using BS23 = std::integral_constant<int, ERK_BS23>;
  using HEUN12 = std::integral_constant<int, ERK_HEUN12>;
  const bool nor = m.psi_kind == GSM_PSI_ELASTIC_VP_DEV;
  if (method == GSM_ODE23) {
    if (nor) launch(NortonDev{}, BS23{});
    else launch(MichelSuquet{}, BS23{});
  } else {
    if (nor) launch(NortonDev{}, HEUN12{});
    else launch(MichelSuquet{}, HEUN12{});
  }
  count_launch();
  return cudaGetLastError() == cudaSuccess ? GSM_OK : GSM_ECUDA;
}

extern "C" int gsm_update_ode23(gsm_handle h, int64_t n_vox, const void* eps_n, const void* eps, const void* z_n,
                                int64_t ld, double step_h, double rtol, double atol, int max_substeps, void* sigma,
                                void* z, void* tangent, int32_t* status, void* stream) {
  return gsm_update_ode(h, GSM_ODE23, n_vox, eps_n, eps, z_n, ld, step_h, rtol, atol, max_substeps, sigma, z,
                        tangent, status, stream);
}
