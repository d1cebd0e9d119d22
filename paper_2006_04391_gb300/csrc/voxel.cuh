// One voxel's material update in the three precision modes, plus the
// consistent tangent.  Used by the batch kernel (gsm_update) and by the
// material kernel of the basic scheme.
//
//   MODE_FP64       every step in FP64.
//   MODE_FP32_FIX   FP32 line search and Newton (the bulk of the work), then
//                   FP64 Newton corrections: FP64 residual, the FP32 Newton
//                   matrix of the last FP32 iteration, until the correction is
//                   below 1e-6 of the increment (normally one).  A Newton step
//                   whose matrix is accurate to FP32 and whose residual is
//                   FP64 lands within ~1e-13 of the FP64 root.
//   MODE_FP32       FP32 only (for FP32 bulk iterations of the basic scheme).
#pragma once

#include "dfloat.cuh"
#include "dpow.cuh"
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
AD_HD void tangent(const LawParams<T>& p, const T (&eps)[6], const T (&y)[5], const T (&w)[5], T inv_h,
                   bool flows, T (&C21)[21]) {
  T sig[6], Cee[6][6], Cey[6][5], Cye[5][6];
  psi_blocks<Law>(p, eps, y, sig, Cee, Cey, Cye);
  if (flows) {
    T g[5], K[5][5], gv[5], Hv[5][5], v[5];
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
AD_HD unsigned voxel_fp64(const LawParams<double>& p, const double (&eps)[6], const double (&zn)[6], const Step& hs,
                          bool active, double (&sig)[6], double (&z)[6], double* C21, const double* zprev = nullptr) {
  const double yn[5] = {zn[0], zn[1], zn[3], zn[4], zn[5]};
  double es[6];
  Law::trial_strain(eps, yn, es);
  double w[5], w0[5];
  if (zprev) {
    const double yp[5] = {zprev[0], zprev[1], zprev[3], zprev[4], zprev[5]};
#pragma unroll
    for (int a = 0; a < 5; ++a) w0[a] = yp[a] - yn[a];
  }
  Chol5<double> ch;
  const unsigned st = solve_increment<Law, double>(p, es, hs, active, 1e-10, w, ch, zprev ? w0 : nullptr);
  double y[5];
#pragma unroll
  for (int a = 0; a < 5; ++a) y[a] = yn[a] + w[a];
  stress<Law>(p, eps, y, sig);
  z_of_y(y, z);
  if (C21) {
    double t[21];
    tangent<Law, double>(p, eps, y, w, hs.inv_h, absmax5(w) > 0.0, t);
#pragma unroll
    for (int c = 0; c < 21; ++c) C21[c] = t[c];
  }
  return st;
}

// Residual of the Norton law's implicit-Euler step (Sec. 4.1) in double-float
// arithmetic, on the trial frame scaled by 2^-k (the frame of the FP32 solve):
//   R_s = psi_y(e_s, w_s) + phi_v(w_s / h) = 2^-k R(e_s 2^k, w_s 2^k),
// with the stress sigma_s = psi_eps(e_s, w_s) of the same sweep.  These are the
// derivatives the AD sweeps of the FP64 correction give, written out for this
// law: a = e_s - P w, tr = a0 + a1 + a2,
//   sigma_i = lam tr + 2 mu a_i (i < 3), mu a_i (shears),
//   psi_y = (sigma2 - sigma0, sigma2 - sigma1, -sigma3, -sigma4, -sigma5),
//   q = 4/3 (v0^2 + v1^2 + v0 v1) + 1/3 (v2^2 + v3^2 + v4^2),  v = w/h,
//   phi_v = a_phi c_phi q^(a_phi - 1) dq/dv.
// The power takes the unscaled q = 2^2k q_s in FP64 (the table-driven power,
// the one FP64-heavy step).  The factor F = a_phi c_phi q^(a_phi-1) is the
// same in both frames and dq/dv = 2^k dq_s/dv_s, so the scaled dissipation
// gradient is 2^-k phi_v = F dq_s/dv_s with the unscaled c_phi.
struct NortonDf {
  df lam, mu, inv_h;
  double ac;     // a_phi * c_phi (unscaled)
  double am1;    // a_phi - 1
  df am1d;       // a_phi - 1 as a pair
  df acm;        // ac = acm 2^ace, acm in [1, 2), for the double-float power
  int ace;
};

AD_HD NortonDf norton_df(const LawParams<double>& p, double inv_h) {
  const double ac = p.a_phi * p.c_phi, am1 = p.a_phi - 1.0;
  const int ace = (int)((fpow::bits_of(ac) >> 52) & 0x7ff) - 1023;
  return NortonDf{df_of(p.lam), df_of(p.mu), df_of(inv_h), ac, am1, df_of(am1), df_of(ac, -ace), ace};
}

AD_HD void norton_residual_df(const NortonDf& c, const df (&es)[6], const df (&w)[5], int k, df (&R)[5],
                              df (&sig)[6]) {
  df a[6];
  a[0] = es[0] - w[0];
  a[1] = es[1] - w[1];
  a[2] = es[2] + (w[0] + w[1]);
  a[3] = es[3] - w[2];
  a[4] = es[4] - w[3];
  a[5] = es[5] - w[4];
  const df ltr = c.lam * ((a[0] + a[1]) + a[2]);
  const df mu2 = c.mu + c.mu;
#pragma unroll
  for (int i = 0; i < 3; ++i) sig[i] = ltr + mu2 * a[i];
#pragma unroll
  for (int i = 3; i < 6; ++i) sig[i] = c.mu * a[i];
  df v[5];
#pragma unroll
  for (int j = 0; j < 5; ++j) v[j] = w[j] * c.inv_h;
  // dq/dv = (4/3 (2 v0 + v1), 4/3 (2 v1 + v0), 2/3 v_j), and q = (v . dq/dv) / 2;
  // the constants 4/3 and 2/3 in double-float (as FP32 numbers their rounding,
  // 2^-25 relative, would enter q and phi_v)
  df dq[5];
  const df c43 = df_of(4.0 / 3.0), c23 = df_of(2.0 / 3.0);
  dq[0] = (v[0] + v[0] + v[1]) * c43;
  dq[1] = (v[1] + v[1] + v[0]) * c43;
#pragma unroll
  for (int j = 2; j < 5; ++j) dq[j] = v[j] * c23;
  df q2 = v[0] * dq[0];
#pragma unroll
  for (int j = 1; j < 5; ++j) q2 = q2 + v[j] * dq[j];
  // unscaled q = 2^(2k) q_s = 2^(2k) q2 / 2; F = ac q^(a-1) by the double-float
  // power (FP32 pipe), the FP64 power where q or F leaves its fast path
  df F;
  if (!dpow::pow_scaled(q2, 2 * k - 1, c.am1, c.am1d, c.acm, c.ace, F))
    F = df_of(c.ac * fpow::pow_pos(f64_of(q2, 2 * k - 1), c.am1));
  R[0] = (sig[2] - sig[0]) + F * dq[0];
  R[1] = (sig[2] - sig[1]) + F * dq[1];
  R[2] = F * dq[2] - sig[3];
  R[3] = F * dq[3] - sig[4];
  R[4] = F * dq[4] - sig[5];
}

// Viscoplastic voxel, FP32 bulk + FP64 correction.
// The FP32 solve sees the trial strain e_s (formed in FP64) scaled by an
// exact power of two s ~ |e_s|, with c_phi rescaled to match (Law::rescale):
// its rounding is then relative to the deviatoric trial state whatever the
// hydrostatic strain, the accumulated viscous strain or the magnitude of
// e_s, and its last Newton matrix equals the unscaled one to FP32 accuracy.
// The corrections reuse that factor: each step w += K32^-1 R64 with the FP64
// residual contracts the error by ~1e-6 (normally one step).  The FP64
// reverse sweep that gives the residual also gives sigma(e_s, w); the last
// correction dw moves it by psi_ey dw (FP32 block, dw tiny), and the
// hydrostatic stress is added back.
template <class Law>
AD_HD unsigned voxel_fp32_fix(const LawParams<double>& p, const LawParams<float>& pf, const double (&eps)[6],
                              const double (&zn)[6], const Step& hs, bool active, double (&sig)[6], double (&z)[6],
                              double* C21, const double* zprev = nullptr, const NortonDf* cdf = nullptr) {
  const double yn[5] = {zn[0], zn[1], zn[3], zn[4], zn[5]};
  double es[6];
  const double tr = Law::trial_strain(eps, yn, es);
  const int k = ilog2_max(es);  // s = 2^k ~ max |e_s|, applied in the conversions
  float esf[6], wf[5], w0f[5];
#pragma unroll
  for (int i = 0; i < 6; ++i) esf[i] = f32_of(es[i], -k);
  if (zprev) {
    const double yp[5] = {zprev[0], zprev[1], zprev[3], zprev[4], zprev[5]};
#pragma unroll
    for (int a = 0; a < 5; ++a) w0f[a] = f32_of(yp[a] - yn[a], -k);
  }
  LawParams<float> ps = pf;
  const bool in_range = Law::rescale(ps, k);
  Chol5<float> chf;
  unsigned st = solve_increment<Law, float>(ps, esf, hs, active && in_range, 1e-4f, wf, chf, zprev ? w0f : nullptr);
  if (active && !in_range) st |= ST_CONVERGED;  // no resolvable flow (Law::rescale)
  const bool flows = absmax5(wf) > 0.0f;
  double w[5];
#pragma unroll
  for (int a = 0; a < 5; ++a) w[a] = f64_of(wf[a], k);

  // FP64 corrections
  const double inv_h = hs.inv_h;
  bool done = !(active && flows);
  bool conv = done;
  int n_fix = 0;
  float dwf[5] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
  if (done) {  // no flow (or padding lane): sigma at w = 0, no correction
    double R[5];
    psi_y_and_stress<Law>(p, es, w, R, sig);
  }
  if constexpr (std::is_same<Law, NortonDev>::value) {
    // the residual sweeps in double-float on the scaled frame (the FP32
    // solve's); only the power and the conversions are FP64
    if (!all_done(done)) {
      // the law's double-float constants (a caller that updates many voxels
      // of one law passes them formed once)
      const NortonDf c = cdf ? *cdf : norton_df(p, inv_h);
      df esd[6], wd[5], sd[6];
#pragma unroll
      for (int i = 0; i < 6; ++i) esd[i] = df_of(es[i], -k);
#pragma unroll
      for (int a = 0; a < 5; ++a) wd[a] = df{wf[a], 0.0f};
      for (int it = 0; it < 4; ++it) {
        if (all_done(done)) break;
        if (!done) {
          ++n_fix;
          df Rd[5];
          norton_residual_df(c, esd, wd, k, Rd, sd);
          float Rf[5];
#pragma unroll
          for (int a = 0; a < 5; ++a) Rf[a] = -(Rd[a].hi + Rd[a].lo);
          chf.solve(Rf, dwf);
          const float dmax = absmax5(dwf);
          if (!(dmax < 1e37f)) {
            st |= ST_NONFINITE;
            done = true;
#pragma unroll
            for (int a = 0; a < 5; ++a) dwf[a] = 0.0f;
          } else {
#pragma unroll
            for (int a = 0; a < 5; ++a) wd[a] = wd[a] + dwf[a];
            if (dmax <= 1e-6f * absmax5(wf)) { done = true; conv = true; }
          }
        }
      }
      if (active && flows) {
#pragma unroll
        for (int a = 0; a < 5; ++a) w[a] = f64_of(wd[a], k);
#pragma unroll
        for (int i = 0; i < 6; ++i) sig[i] = f64_of(sd[i], k);
      }
    }
  } else {
    for (int it = 0; it < 4; ++it) {
      if (all_done(done)) break;
      if (!done) {
        ++n_fix;
        double v[5], R[5], gv[5];
#pragma unroll
        for (int a = 0; a < 5; ++a) v[a] = w[a] * inv_h;
        psi_y_and_stress<Law>(p, es, w, R, sig);
        phi_v<Law>(p, v, gv);
        float Rf[5];
#pragma unroll
        for (int a = 0; a < 5; ++a) Rf[a] = f32_of(-(R[a] + gv[a]), -k);
        chf.solve(Rf, dwf);
        const float dmax = absmax5(dwf);
        if (!(dmax < 1e37f)) {
          st |= ST_NONFINITE;
          done = true;
#pragma unroll
          for (int a = 0; a < 5; ++a) dwf[a] = 0.0f;
        } else {
#pragma unroll
          for (int a = 0; a < 5; ++a) w[a] += f64_of(dwf[a], k);
          if (dmax <= 1e-6f * absmax5(wf)) { done = true; conv = true; }
        }
      }
    }
  }
  if (active && flows && !conv) st = (st & ~ST_CONVERGED) | ST_CAP;
  st += (unsigned)n_fix << ST_NEWTON_SHIFT;
  st |= (unsigned)(n_fix & 0xf) << ST_FIX_SHIFT;
  if (n_fix > 0) {
    // sigma of the last sweep was taken before the last dw: add psi_ey dw
    float B[6][5];
    psi_ey<Law>(ps, esf, wf, B);
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      float d = 0.0f;
#pragma unroll
      for (int a = 0; a < 5; ++a) d += B[i][a] * dwf[a];
      sig[i] += f64_of(d, k);
    }
  }
  const double sh = Law::hydro_stress(p, tr);
#pragma unroll
  for (int i = 0; i < 3; ++i) sig[i] += sh;
  double y[5];
#pragma unroll
  for (int a = 0; a < 5; ++a) y[a] = yn[a] + w[a];
  z_of_y(y, z);
  if (C21) {
    double t[21];
    tangent<Law, double>(p, eps, y, w, hs.inv_h, absmax5(w) > 0.0, t);
#pragma unroll
    for (int c = 0; c < 21; ++c) C21[c] = t[c];
  }
  return st;
}

// Viscoplastic voxel, FP32 only (same scaled trial frame as above).
template <class Law>
AD_HD unsigned voxel_fp32(const LawParams<float>& pf, const float (&eps)[6], const float (&zn)[6], const Step& hs,
                          bool active, float (&sig)[6], float (&z)[6], float* C21, const float* zprev = nullptr) {
  const float yn[5] = {zn[0], zn[1], zn[3], zn[4], zn[5]};
  float es[6];
  Law::trial_strain(eps, yn, es);
  const int k = ilog2_max(es) > 126 ? 126 : ilog2_max(es);
  const float s = exp2i(k, 0.0f), inv_s = exp2i(-k, 0.0f);
#pragma unroll
  for (int i = 0; i < 6; ++i) es[i] *= inv_s;
  float w0[5];
  if (zprev) {
    const float yp[5] = {zprev[0], zprev[1], zprev[3], zprev[4], zprev[5]};
#pragma unroll
    for (int a = 0; a < 5; ++a) w0[a] = (yp[a] - yn[a]) * inv_s;
  }
  LawParams<float> ps = pf;
  const bool in_range = Law::rescale(ps, k);
  float w[5];
  Chol5<float> ch;
  unsigned st = solve_increment<Law, float>(ps, es, hs, active && in_range, 1e-6f, w, ch, zprev ? w0 : nullptr);
  if (active && !in_range) st |= ST_CONVERGED;
  float y[5];
#pragma unroll
  for (int a = 0; a < 5; ++a) {
    w[a] *= s;
    y[a] = yn[a] + w[a];
  }
  stress<Law>(pf, eps, y, sig);
  z_of_y(y, z);
  if (C21) {
    float t[21];
    tangent<Law, float>(pf, eps, y, w, hs.inv_hf, absmax5(w) > 0.0f, t);
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
