// Kernels of the ode23s (Shampine-Reichelt Rosenbrock triple) material update (gsm_update_ode); see ode_kernel.cuh.
#define GSM_ODE_KERNEL_IMPL
#include "ode_kernel.cuh"

namespace gsm {
template void ode_launch<ROS_23S>(const Material&, int64_t, int64_t, const Step&, const Ode23Ctl&, const double*,
                                const double*, const double*, double*, double*, double*, int32_t*, cudaStream_t);
}  // namespace gsm
