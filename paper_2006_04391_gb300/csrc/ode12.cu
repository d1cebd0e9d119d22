// Kernels of the ode12 (explicit Euler / Heun) material update (gsm_update_ode); see ode_kernel.cuh.
#define GSM_ODE_KERNEL_IMPL
#include "ode_kernel.cuh"

namespace gsm {
template void ode_launch<ERK_HEUN12>(const Material&, int64_t, int64_t, const Step&, const Ode23Ctl&, const double*,
                                const double*, const double*, double*, double*, double*, int32_t*, cudaStream_t);
}  // namespace gsm
