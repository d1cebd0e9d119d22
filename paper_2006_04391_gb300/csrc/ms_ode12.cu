// Basic-scheme material kernel for laws integrated by ode12; see ms_ode_impl.cuh.
#include "ms_ode_impl.cuh"

namespace gsm {
GSM_MS_ODE_INSTANTIATE_MATERIAL(1)
}  // namespace gsm
