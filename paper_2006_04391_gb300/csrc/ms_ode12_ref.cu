// Basic-scheme reference-medium kernel (tangents) for laws integrated by ode12;
// see ms_ode_impl.cuh.
#include "ms_ode_impl.cuh"

namespace gsm {
GSM_MS_ODE_INSTANTIATE_REFERENCE(1)
}  // namespace gsm
