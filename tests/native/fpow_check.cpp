// Test-only host build of the table-driven FP64 power (fpow.cuh).
#include "../../paper_2006_04391_gb300/csrc/fpow.cuh"

extern "C" void host_pow(int n, const double* x, const double* p, double* out) {
  for (int i = 0; i < n; ++i) out[i] = gsm::fpow::pow_pos(x[i], p[i]);
}
