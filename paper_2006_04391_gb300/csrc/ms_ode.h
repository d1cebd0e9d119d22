// Host launchers of the basic-scheme kernels for laws integrated over the
// load step by an ODE integrator (ms_ode_impl.cuh, instantiated in
// ms_ode{23,12,23s}.cu and ms_ode{23,12,23s}_ref.cu); used by ms_solve.cu.  `pair`: 0
// ode23, 1 ode12, 2 ode23s.  Views and tables are passed untyped: their types
// are private to each translation unit (same header, same layout).
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

namespace gsm {

template <int PAIR> int ms_ode_blocks_per_sm_p();
template <int PAIR>
void ms_launch_material_ode_p(int grid, cudaStream_t s, const void* views, int n_jobs, int64_t total_chunks);
template <int PAIR>
void ms_launch_reference_ode_p(int grid, cudaStream_t s, int64_t nvox, const uint8_t* phase, const void* tab, double h,
                               double rtol, double atol, int max_steps, const double* eps_raw, const double* eps_prev,
                               const double* zn, const double* alpha_n, double inv_n3, const double (&dE)[6],
                               double* part);

// Each integrator's kernels live in their own translation unit only.
#define GSM_MS_ODE_EXTERN(PAIR)                                                                                   \
  extern template int ms_ode_blocks_per_sm_p<PAIR>();                                                           \
  extern template void ms_launch_material_ode_p<PAIR>(int, cudaStream_t, const void*, int, int64_t);           \
  extern template void ms_launch_reference_ode_p<PAIR>(int, cudaStream_t, int64_t, const uint8_t*, const void*,  \
                                                       double, double, double, int, const double*, const double*, \
                                                       const double*, const double*, double, const double (&)[6], \
                                                       double*);
GSM_MS_ODE_EXTERN(0)
GSM_MS_ODE_EXTERN(1)
GSM_MS_ODE_EXTERN(2)
#undef GSM_MS_ODE_EXTERN

// Resident blocks per SM of the batched material kernel of the integrator.
inline int ms_ode_blocks_per_sm(int pair) {
  return pair == 0 ? ms_ode_blocks_per_sm_p<0>() : pair == 1 ? ms_ode_blocks_per_sm_p<1>() : ms_ode_blocks_per_sm_p<2>();
}

// Batched material evaluation of the jobs views[0 .. n_jobs) (device JobView array).
inline void ms_launch_material_ode(int pair, int grid, cudaStream_t s, const void* views, int n_jobs,
                                   int64_t total_chunks) {
  if (pair == 0) ms_launch_material_ode_p<0>(grid, s, views, n_jobs, total_chunks);
  else if (pair == 1) ms_launch_material_ode_p<1>(grid, s, views, n_jobs, total_chunks);
  else ms_launch_material_ode_p<2>(grid, s, views, n_jobs, total_chunks);
}

// Reference-medium partials (k, mu min/max per block into part[4][grid]) from
// the tangents at the strain eps_raw * inv_n3 + dE.
inline void ms_launch_reference_ode(int pair, int grid, cudaStream_t s, int64_t nvox, const uint8_t* phase,
                                    const void* tab, double h, double rtol, double atol, int max_steps,
                                    const double* eps_raw, const double* eps_prev, const double* zn,
                                    const double* alpha_n, double inv_n3, const double (&dE)[6], double* part) {
  if (pair == 0)
    ms_launch_reference_ode_p<0>(grid, s, nvox, phase, tab, h, rtol, atol, max_steps, eps_raw, eps_prev, zn, alpha_n,
                                 inv_n3, dE, part);
  else if (pair == 1)
    ms_launch_reference_ode_p<1>(grid, s, nvox, phase, tab, h, rtol, atol, max_steps, eps_raw, eps_prev, zn, alpha_n,
                                 inv_n3, dE, part);
  else
    ms_launch_reference_ode_p<2>(grid, s, nvox, phase, tab, h, rtol, atol, max_steps, eps_raw, eps_prev, zn, alpha_n,
                                 inv_n3, dE, part);
}

}  // namespace gsm
