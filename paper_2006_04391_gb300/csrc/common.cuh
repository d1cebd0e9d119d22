// Internal definitions shared by the translation units of the library.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <cstdint>

#include "../../include/gsm.h"
#include "laws.cuh"

namespace gsm {

// Material handle behind gsm_handle.
struct Material {
  int psi_kind, phi_kind, precision;
  double params[8];
  LawParams<double> p64;
  LawParams<float> p32;
};

// kind: 0 elastic (E, nu); 1 Norton (E, nu, sigma0, edot0, n);
// 2 Michel-Suquet (E, nu, sigma_Y, H, edot0, sigma_d, n).
inline LawParams<double> make_params(const double* prm, int kind) {
  LawParams<double> p;
  const double E = prm[0], nu = prm[1];
  p.lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  p.mu = E / (2.0 * (1.0 + nu));
  p.H_kin = 0.0;
  p.sig_Y = 0.0;
  if (kind == 2) {
    const double sY = prm[2], H = prm[3], e0 = prm[4], sd = prm[5], n = prm[6];
    p.a_phi = 1.0;
    p.c_phi = 0.0;
    p.b_Psi = n + 1.0;
    p.c_Psi = sd * e0 / (n + 1.0) * std::pow(sd, -(n + 1.0));
    p.H_kin = H;
    p.sig_Y = sY;
  } else if (kind == 1) {
    const double s0 = prm[2], e0 = prm[3], n = prm[4];
    p.a_phi = (n + 1.0) / (2.0 * n);
    p.c_phi = s0 * e0 * n / (n + 1.0) * std::pow(e0, -(n + 1.0) / n);
    p.b_Psi = (n + 1.0) / 2.0;
    p.c_Psi = s0 * e0 / (n + 1.0) * std::pow(s0, -(n + 1.0));
  } else {
    p.a_phi = 1.0;
    p.c_phi = 0.0;
    p.b_Psi = 1.0;
    p.c_Psi = 0.0;
  }
  return p;
}

inline LawParams<float> to_float(const LawParams<double>& p) {
  LawParams<float> q;
  q.lam = (float)p.lam;
  q.mu = (float)p.mu;
  q.c_phi = (float)p.c_phi;
  q.a_phi = (float)p.a_phi;
  q.c_Psi = (float)p.c_Psi;
  q.b_Psi = (float)p.b_Psi;
  q.H_kin = (float)p.H_kin;
  q.sig_Y = (float)p.sig_Y;
  return q;
}

// The address under which the current device reaches p (device, managed or
// page-locked host memory); false for memory the device cannot reach.
bool device_address(const void* p, const void** out);

// Process-wide count of kernel launches made by this library.
extern std::atomic<int64_t> g_launches;
inline void count_launch(int n = 1) { g_launches.fetch_add(n, std::memory_order_relaxed); }

inline int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

}  // namespace gsm
