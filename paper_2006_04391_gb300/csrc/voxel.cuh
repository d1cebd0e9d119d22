// One voxel's material update in the three precision modes, plus the
// consistent tangent.  Used by the batch kernel (gsm_update) and by the
// material kernel of the basic scheme.
//
//   MODE_FP64       every step in FP64.
//   MODE_FP32_FIX   FP32 line search and Newton (the bulk of the work), then
//                   FP64 Newton corrections: FP64 residual, FP32 Newton matrix
//                   re-evaluated at the FP64 rate, until the correction is
//                   below 1e-6 of the increment (normally one).  A Newton step
//                   whose matrix is accurate to FP32 and whose residual is
//                   FP64 lands within ~1e-13 of the FP64 root.
//   MODE_FP32       FP32 only (for FP32 bulk iterations of the basic scheme).
#pragma once

#include "solver.cuh"

namespace gsm {

enum { MODE_FP64 = 0, MODE_FP32_FIX = 1, MODE_FP32 = 2 };

template <class T> struct LawPair {
  LawParams<T> p;
};

// z = P y (Voigt, engineering shears), z33 = -z11 - z22.
template <class T> AD_HD void z_of_y(const T (&y)[5], T (&z)[6]) {
  z[0] = y[0];
  z[1] = y[1];
  z[2] = -(y[0] + y[1]);
  z[3] = y[2];
  z[4] = y[3];
  z[5] = y[4];
}

// Consistent tangent at the converged state (Eq. tangent_formula), packed
// upper triangle row-major (21 entries).  `flows` = false means y = y_n with
// an unbounded dissipation Hessian: dy/deps = 0 and C_t = psi_ee.
template <class Law, class T>
AD_HD void tangent(const LawParams<T>& p, const T (&eps)[6], const T (&y)[5], const T (&w)[5], T h,
                   bool flows, T (&C21)[21]) {
  T sig[6], Cee[6][6], Cey[6][5], Cye[5][6];
  psi_blocks<Law>(p, eps, y, sig, Cee, Cey, Cye);
  if (flows) {
    T g[5], K[5][5], gv[5], Hv[5][5], v[5];
    const T inv_h = T(1) / h;
#pragma unroll
    for (int a = 0; a < 5; ++a) v[a] = w[a] * inv_h;
    psi_y_yy<Law>(p, eps, y, g, K);
    phi_v_vv<Law>(p, v, gv, Hv);
#pragma unroll
    for (int a = 0; a < 5; ++a)
#pragma unroll
      for (int b = 0; b < 5; ++b) K[a][b] += Hv[a][b] * inv_h;
    Chol5<T> ch;
    ch.factor(K);
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      T rhs[5], dy[5];
#pragma unroll
      for (int a = 0; a < 5; ++a) rhs[a] = -Cye[a][j];
      ch.solve(rhs, dy);
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        T s = Cee[i][j];
#pragma unroll
        for (int a = 0; a < 5; ++a) s += Cey[i][a] * dy[a];
        Cee[i][j] = s;
      }
    }
  }
  int c = 0;
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int j = i; j < 6; ++j) C21[c++] = T(0.5) * (Cee[i][j] + Cee[j][i]);
}

// Viscoplastic voxel, FP64 arithmetic.
template <class Law>
AD_HD unsigned voxel_fp64(const LawParams<double>& p, const double (&eps)[6], const double (&zn)[6], double h,
                          bool active, double (&sig)[6], double (&z)[6], double* C21) {
  const double yn[5] = {zn[0], zn[1], zn[3], zn[4], zn[5]};
  double w[5];
  Chol5<double> ch;
  const unsigned st = solve_increment<Law, double>(p, eps, yn, h, active, 1e-10, w, ch);
  double y[5];
#pragma unroll
  for (int a = 0; a < 5; ++a) y[a] = yn[a] + w[a];
  stress<Law>(p, eps, y, sig);
  z_of_y(y, z);
  if (C21) {
    double t[21];
    tangent<Law, double>(p, eps, y, w, h, absmax5(w) > 0.0, t);
#pragma unroll
    for (int c = 0; c < 21; ++c) C21[c] = t[c];
  }
  return st;
}

// Viscoplastic voxel, FP32 bulk + FP64 correction.
template <class Law>
AD_HD unsigned voxel_fp32_fix(const LawParams<double>& p, const LawParams<float>& pf, const double (&eps)[6],
                              const double (&zn)[6], double h, bool active, double (&sig)[6], double (&z)[6],
                              double* C21) {
  const double yn[5] = {zn[0], zn[1], zn[3], zn[4], zn[5]};
  float epsf[6], ynf[5], wf[5];
#pragma unroll
  for (int i = 0; i < 6; ++i) epsf[i] = (float)eps[i];
#pragma unroll
  for (int a = 0; a < 5; ++a) ynf[a] = (float)yn[a];
  Chol5<float> chf;
  unsigned st = solve_increment<Law, float>(pf, epsf, ynf, (float)h, active, 1e-4f, wf, chf);
  double w[5];
#pragma unroll
  for (int a = 0; a < 5; ++a) w[a] = (double)wf[a];
  const bool flows = absmax5(w) > 0.0;

  // FP64 Newton corrections.
  const double inv_h = 1.0 / h;
  bool done = !(active && flows);
  int n_fix = 0;
  bool conv = done;
  for (int it = 0; it < 4; ++it) {
    if (all_done(done)) break;
    if (!done) {
      ++n_fix;
      double y[5], v[5], R[5], gv[5];
#pragma unroll
      for (int a = 0; a < 5; ++a) {
        y[a] = yn[a] + w[a];
        v[a] = w[a] * inv_h;
      }
      psi_y<Law>(p, eps, y, R);
      phi_v<Law>(p, v, gv);
      float Rf[5], vf[5], yf[5];
#pragma unroll
      for (int a = 0; a < 5; ++a) {
        Rf[a] = (float)(-(R[a] + gv[a]));
        vf[a] = (float)v[a];
        yf[a] = (float)y[a];
      }
      float g[5], K[5][5], gvf[5], Hv[5][5];
      psi_y_yy<Law>(pf, epsf, yf, g, K);
      phi_v_vv<Law>(pf, vf, gvf, Hv);
      const float inv_hf = (float)inv_h;
#pragma unroll
      for (int a = 0; a < 5; ++a)
#pragma unroll
        for (int b = 0; b < 5; ++b) K[a][b] += Hv[a][b] * inv_hf;
      Chol5<float> ck;
      float dwf[5];
      if (ck.factor(K)) {
        ck.solve(Rf, dwf);
      } else {
        st |= ST_NOT_SPD;
#pragma unroll
        for (int a = 0; a < 5; ++a) dwf[a] = 0.0f;
        done = true;
      }
      double dw[5];
#pragma unroll
      for (int a = 0; a < 5; ++a) {
        dw[a] = (double)dwf[a];
        w[a] += dw[a];
      }
      if (absmax5(dw) <= 1e-6 * absmax5(w)) { done = true; conv = true; }
      if (!(absmax5(dw) == absmax5(dw))) { st |= ST_NONFINITE; done = true; }
    }
  }
  if (active && flows && !conv) st = (st & ~ST_CONVERGED) | ST_CAP;
  st += (unsigned)n_fix << ST_NEWTON_SHIFT;
  double y[5];
#pragma unroll
  for (int a = 0; a < 5; ++a) y[a] = yn[a] + w[a];
  stress<Law>(p, eps, y, sig);
  z_of_y(y, z);
  if (C21) {
    double t[21];
    tangent<Law, double>(p, eps, y, w, h, flows, t);
#pragma unroll
    for (int c = 0; c < 21; ++c) C21[c] = t[c];
  }
  return st;
}

// Viscoplastic voxel, FP32 only.
template <class Law>
AD_HD unsigned voxel_fp32(const LawParams<float>& pf, const float (&eps)[6], const float (&zn)[6], float h,
                          bool active, float (&sig)[6], float (&z)[6], float* C21) {
  const float yn[5] = {zn[0], zn[1], zn[3], zn[4], zn[5]};
  float w[5];
  Chol5<float> ch;
  const unsigned st = solve_increment<Law, float>(pf, eps, yn, h, active, 1e-6f, w, ch);
  float y[5];
#pragma unroll
  for (int a = 0; a < 5; ++a) y[a] = yn[a] + w[a];
  stress<Law>(pf, eps, y, sig);
  z_of_y(y, z);
  if (C21) {
    float t[21];
    tangent<Law, float>(pf, eps, y, w, h, absmax5(w) > 0.0f, t);
#pragma unroll
    for (int c = 0; c < 21; ++c) C21[c] = t[c];
  }
  return st;
}

// Elastic voxel: sigma = psi_eps, tangent = psi_ee (both by AD).
template <class T>
AD_HD void voxel_elastic(const LawParams<T>& p, const T (&eps)[6], T (&sig)[6], T* C21) {
  ad::UniformPack<ad::Var<T>, 6> E;
  ad::For<0, 6>::run([&](auto kc) { ad::get_mut<decltype(kc)::value>(E).v = eps[decltype(kc)::value]; });
  auto f = Elastic::psi(E, p);
  f.fwd();
  f.back(T(1));
  ad::For<0, 6>::run([&](auto kc) { sig[decltype(kc)::value] = ad::get<decltype(kc)::value>(E).a; });
  if (C21) {
    ad::SeededPack<ad::Var, T, 6, 0, 6> Es;
    ad::seed_unit<decltype(Es), T, 0, 6>(Es, eps);
    auto g = Elastic::psi(Es, p);
    g.fwd();
    g.back(T(1));
    T C[6][6];
    ad::For<0, 6>::run([&](auto kc) {
      constexpr int i = decltype(kc)::value;
#pragma unroll
      for (int j = 0; j < 6; ++j) C[i][j] = ad::get<i>(Es).a.d[j];
    });
    int c = 0;
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
      for (int j = i; j < 6; ++j) C21[c++] = C[i][j];
  }
}

}  // namespace gsm
