// Basic-scheme reference-medium kernel (tangents) for laws integrated by ode23;
// see ms_ode_impl.cuh.
#include "ms_ode_impl.cuh"

namespace gsm {
GSM_MS_ODE_INSTANTIATE_REFERENCE(0)
}  // namespace gsm
