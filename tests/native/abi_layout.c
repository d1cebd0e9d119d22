/* Prints the size and field offsets of the C-ABI structs of include/gsm.h
 * as "struct field offset" lines (and "struct . size"), for the check that
 * the Python binding's ctypes mirrors match the header. */
#include <stddef.h>
#include <stdio.h>

#include "../../include/gsm.h"

#define F(S, M) printf(#S " " #M " %zu\n", offsetof(S, M))
#define Z(S) printf(#S " . %zu\n", sizeof(S))

int main(void) {
  Z(ms_problem);
  F(ms_problem, N); F(ms_problem, phase); F(ms_problem, n_phases); F(ms_problem, laws); F(ms_problem, precision);
  Z(ms_load);
  F(ms_load, n_steps); F(ms_load, E); F(ms_load, h); F(ms_load, tol); F(ms_load, max_iter);
  F(ms_load, forced_iters); F(ms_load, switch_tol); F(ms_load, stress_mask); F(ms_load, Sigma);
  F(ms_load, ref_update); F(ms_load, integrator); F(ms_load, ode_rtol); F(ms_load, ode_atol);
  F(ms_load, ode_max_substeps);
  Z(ms_state);
  F(ms_state, eps); F(ms_state, z); F(ms_state, resume); F(ms_state, E_prev);
  Z(ms_result);
  F(ms_result, Sigma); F(ms_result, iters); F(ms_result, final_error); F(ms_result, fp32_iters);
  F(ms_result, total_iters); F(ms_result, E); F(ms_result, reference);
  Z(serve_job);
  F(serve_job, N); F(serve_job, phase); F(serve_job, n_phases); F(serve_job, laws); F(serve_job, precision);
  F(serve_job, n_steps); F(serve_job, E); F(serve_job, h); F(serve_job, tol); F(serve_job, max_iter);
  F(serve_job, switch_tol); F(serve_job, integrator); F(serve_job, ode_rtol); F(serve_job, ode_atol);
  F(serve_job, ode_max_substeps);
  return 0;
}
