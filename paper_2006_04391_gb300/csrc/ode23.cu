// gsm_update_ode / gsm_update_ode23: the material update by adaptive
// integration of the force-potential form (AutoMat, arXiv 2006.04391,
// Sec. 4.3, Corollary 1, Sec. 4.5) on sm_103a; this unit also instantiates
// the ode23 kernels.
#define GSM_ODE_KERNEL_IMPL
#include "ode_kernel.cuh"

namespace gsm {
template void ode_launch<ERK_BS23>(const Material&, int64_t, int64_t, const Step&, const Ode23Ctl&, const double*,
                                   const double*, const double*, double*, double*, double*, int32_t*, cudaStream_t);
}  // namespace gsm

using namespace gsm;

extern "C" int gsm_update_ode(gsm_handle h, int method, int64_t n_vox, const void* eps_n, const void* eps,
                              const void* z_n, int64_t ld, double step_h, double rtol, double atol, int max_substeps,
                              void* sigma, void* z, void* tangent, int32_t* status, void* stream) {
  if (!h || n_vox < 0 || ld < n_vox) return GSM_EINVAL;
  if (method != GSM_ODE23 && method != GSM_ODE12 && method != GSM_ODE23S) return GSM_EINVAL;
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
  if (method == GSM_ODE23) ode_launch<ERK_BS23>(m, n_vox, ld, hs, ctl, e0, e1, zi, so, zo, to, sto, s);
  else if (method == GSM_ODE12) ode_launch<ERK_HEUN12>(m, n_vox, ld, hs, ctl, e0, e1, zi, so, zo, to, sto, s);
  else ode_launch<ROS_23S>(m, n_vox, ld, hs, ctl, e0, e1, zi, so, zo, to, sto, s);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? GSM_OK : GSM_ECUDA;
}

extern "C" int gsm_update_ode23(gsm_handle h, int64_t n_vox, const void* eps_n, const void* eps, const void* z_n,
                                int64_t ld, double step_h, double rtol, double atol, int max_substeps, void* sigma,
                                void* z, void* tangent, int32_t* status, void* stream) {
  return gsm_update_ode(h, GSM_ODE23, n_vox, eps_n, eps, z_n, ld, step_h, rtol, atol, max_substeps, sigma, z,
                        tangent, status, stream);
}
