// Basic-scheme material kernel for laws integrated by ode23s; see ms_ode_impl.cuh.
#include "ms_ode_impl.cuh"

namespace gsm {
GSM_MS_ODE_INSTANTIATE_MATERIAL(2)
}  // namespace gsm
