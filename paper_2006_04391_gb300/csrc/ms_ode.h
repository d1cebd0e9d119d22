// Host launchers of the basic-scheme kernels for laws integrated by an
// explicit Runge-Kutta pair (ms_ode.cu); used by ms_solve.cu.  Views and
// tables are passed untyped: their types are private to each translation
// unit (same header, same layout).
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

namespace gsm {

// Resident blocks per SM of the batched material kernel of the pair.
int ms_ode_blocks_per_sm(int pair);

// Batched material evaluation of the jobs views[0 .. n_jobs) (device JobView array).
void ms_launch_material_ode(int pair, int grid, cudaStream_t s, const void* views, int n_jobs, int64_t total_chunks);

// Reference-medium partials (k, mu min/max per block into part[4][grid]) from
// the tangents at the strain eps_raw * inv_n3 + dE.
void ms_launch_reference_ode(int pair, int grid, cudaStream_t s, int64_t nvox, const uint8_t* phase, const void* tab,
                             double h, double rtol, double atol, int max_steps, const double* eps_raw,
                             const double* eps_prev, const double* zn, const double* alpha_n, double inv_n3,
                             const double (&dE)[6], double* part);

}  // namespace gsm
