// Basic-scheme reference-medium kernel (tangents) for laws integrated by ode23s;
// see ms_ode_impl.cuh.
#include "ms_ode_impl.cuh"

namespace gsm {
GSM_MS_ODE_INSTANTIATE_REFERENCE(2)
}  // namespace gsm
