// Potentials of the generalized standard materials (GSM) the library ships.
//
// AutoMat (arXiv 2006.04391) reduces a material law to two potentials
// (Sec. 2, Eq. gsm_sigma / gsm_internal); everything else -- the implicit
// Euler Newton solve, the stress and the consistent tangent -- is obtained
// by automatic differentiation (Sec. 4.1, Sec. 5).  A law here is a struct
// with two templated functions written once on AD leaf packs:
//
//   psi(eps, y, p)  free energy, eps = strain (6 leaves), y = internal
//                   variables (NY leaves);
//   phi(v, p)       dissipation potential of the rate v = (y - y_n)/h.
//
// We use the dissipation form of the evolution law, d psi/dy + d phi/dv = 0,
// which for a convex dual pair (phi = Psi*) is equivalent to the paper's
// force-potential form (the paper notes the dual exists, Sec. 2).
//
// Voigt conventions: strain-like vectors (e11,e22,e33,g23,g13,g12) with
// engineering shears g = 2 e_ij (the H = diag(H,H,H,H/2,H/2,H/2) of Eq.
// michel_suquet_omega implies them), stress-like vectors with tensor shears.
#pragma once

#include "ad.cuh"

namespace gsm {

template <class T> struct LawParams {
  T lam, mu;      // Lame constants
  T c_phi;        // phi = c_phi * q^a_phi  (see NortonDev)
  T a_phi;
  T c_Psi;        // force potential Psi = c_Psi * s_A^(2 b_Psi)  (see NortonDev, MichelSuquet)
  T b_Psi;
  T H_kin;        // kinematic hardening modulus H (MichelSuquet)
  T sig_Y;        // yield stress, K(alpha) = sigma_Y (MichelSuquet)
};

// Linear elasticity: psi = 1/2 eps^T C eps, no internal variables.
struct Elastic {
  static constexpr int NY = 0;
  template <class EP, class P> AD_HD static auto psi(const EP& e, const P& p) {
    using ad::get;
    const auto& e0 = get<0>(e); const auto& e1 = get<1>(e); const auto& e2 = get<2>(e);
    const auto& e3 = get<3>(e); const auto& e4 = get<4>(e); const auto& e5 = get<5>(e);
    auto tr = e0 + e1 + e2;
    return (p.lam * 0.5) * sq(tr) + p.mu * (sq(e0) + sq(e1) + sq(e2)) +
           (p.mu * 0.5) * (sq(e3) + sq(e4) + sq(e5));
  }
};

// Elastic-viscoplastic GSM of Sec. 3 (Eq. michel_suquet_omega / _psi) with
// sigma_Y = 0 and H = 0: the viscoplastic strain z is deviatoric and carried
// by NY = 5 unknowns y = (z11, z22, g23, g13, g12), z33 = -z11 - z22 (Sec. 6
// eliminates one component).  psi = 1/2 (eps - z)^T C (eps - z).
// phi is the Norton potential, the convex dual of the paper's Psi:
//   phi(v) = sigma0 edot0 n/(n+1) (s/edot0)^((n+1)/n),  s^2 = (2/3) zdot:zdot,
// written as c_phi * q^a_phi with q = s^2, a_phi = (n+1)/(2n),
// c_phi = sigma0 edot0 n/(n+1) edot0^(-(n+1)/n).
struct NortonDev {
  static constexpr int NY = 5;

  template <class EP, class YP, class P> AD_HD static auto psi(const EP& e, const YP& y, const P& p) {
    using ad::get;
    const auto& y0 = get<0>(y); const auto& y1 = get<1>(y); const auto& y2 = get<2>(y);
    const auto& y3 = get<3>(y); const auto& y4 = get<4>(y);
    auto a0 = get<0>(e) - y0;
    auto a1 = get<1>(e) - y1;
    auto a2 = get<2>(e) + (y0 + y1);
    auto a3 = get<3>(e) - y2;
    auto a4 = get<4>(e) - y3;
    auto a5 = get<5>(e) - y4;
    auto tr = a0 + a1 + a2;
    return (p.lam * 0.5) * sq(tr) + p.mu * (sq(a0) + sq(a1) + sq(a2)) +
           (p.mu * 0.5) * (sq(a3) + sq(a4) + sq(a5));
  }

  template <class VP, class P> AD_HD static auto phi(const VP& v, const P& p) {
    using ad::get;
    const auto& v0 = get<0>(v); const auto& v1 = get<1>(v); const auto& v2 = get<2>(v);
    const auto& v3 = get<3>(v); const auto& v4 = get<4>(v);
    using S = typename std::decay_t<decltype(v0)>::scalar;
    // q = (2/3) zdot:zdot with zdot33 = -v0 - v1 and engineering shears
    auto q = S(4.0 / 3.0) * (sq(v0) + sq(v1) + v0 * v1) + S(1.0 / 3.0) * (sq(v2) + sq(v3) + sq(v4));
    return p.c_phi * pow(q, p.a_phi);
  }

  // Force potential of Eq. michel_suquet_psi at sigma_Y = 0, H = 0, the convex
  // dual of phi, on the generalized stress A = -psi_y = (s11 - s33, s22 - s33,
  // s23, s13, s12) (Sec. 2, Eq. gsm_internal: ydot = dPsi/dA):
  //   Psi(A) = sigma0 edot0/(n+1) (s_A/sigma0)^(n+1) = c_Psi (s_A^2)^b_Psi,
  //   s_A^2 = A0^2 + A1^2 - A0 A1 + 3 (A2^2 + A3^2 + A4^2)  (von Mises stress^2,
  // the metric dual to phi's q), b_Psi = (n+1)/2.
  template <class AP, class P> AD_HD static auto Psi(const AP& A, const P& p) {
    using ad::get;
    const auto& a0 = get<0>(A); const auto& a1 = get<1>(A); const auto& a2 = get<2>(A);
    const auto& a3 = get<3>(A); const auto& a4 = get<4>(A);
    using S = typename std::decay_t<decltype(a0)>::scalar;
    auto s2 = (sq(a0) + sq(a1) - a0 * a1) + S(3) * (sq(a2) + sq(a3) + sq(a4));
    return p.c_Psi * pow(s2, p.b_Psi);
  }
  // Psi = c_Psi x^beta with x = s_A (for the hand third derivative of ode23s)
  static constexpr bool kYield = false;
  AD_HD static double Psi_beta(const LawParams<double>& p) { return 2.0 * p.b_Psi; }

  // psi depends on (eps, y) only through tr(eps) and dev(eps) - P y (P y is
  // traceless, C isotropic).  With the trial strain e_s = dev(eps) - P y_n:
  //   psi_y(eps, y_n + w)  = psi_y(e_s, w),
  //   sigma(eps, y_n + w)  = sigma(e_s, w) + kappa tr(eps) 1,  kappa = lam + 2 mu / 3.
  // The increment is solved on (e_s, w), so neither the hydrostatic strain nor
  // the accumulated viscous strain adds rounding to the residual: its
  // rounding is relative to the deviatoric trial state.  Returns tr(eps).
  template <class T> AD_HD static T trial_strain(const T (&eps)[6], const T (&yn)[5], T (&es)[6]) {
    const T tr = eps[0] + eps[1] + eps[2];
    const T m = tr * T(1.0 / 3.0);
    es[0] = (eps[0] - m) - yn[0];
    es[1] = (eps[1] - m) - yn[1];
    es[2] = (eps[2] - m) + (yn[0] + yn[1]);
    es[3] = eps[3] - yn[2];
    es[4] = eps[4] - yn[3];
    es[5] = eps[5] - yn[4];
    return tr;
  }
  template <class T> AD_HD static T hydro_stress(const LawParams<T>& p, T tr) {
    return (p.lam + p.mu * T(2.0 / 3.0)) * tr;
  }

  // phi(s v) = s^(2 a_phi) phi(v) and psi is quadratic, so the step on
  // (e_s / s, w / s) is the same problem with c_phi scaled by s^(2 a_phi - 2),
  // and has the same Newton matrix.  s = 2^k.  Returns false when the scaled
  // constant leaves the range in which the FP32 solve stays finite; that
  // happens only for trial strains so small that the dissipation dominates
  // psi by many orders and the flow, far below the resolution of y, is taken
  // as zero.
  template <class T> AD_HD static bool rescale(LawParams<T>& p, int k) {
    const T e = T(k) * (T(2) * p.a_phi - T(2));
    T f;
    if constexpr (sizeof(T) == 4) f = exp2f(e);
    else f = exp2(e);
    p.c_phi *= f;
    const T big = T(sizeof(T) == 4 ? 1e20 : 1e280);
    return p.c_phi > T(1) / big && p.c_phi < big;
  }
};

// The paper's full elasto-viscoplastic law (Sec. 3, Eq. michel_suquet_omega and
// Eq. michel_suquet_psi) with K(alpha) = sigma_Y, the paper's calibration:
// internal variables y = (z11, z22, g23, g13, g12, alpha), e_vp = P y deviatoric,
//   psi = 1/2 (eps - P y)^T C (eps - P y) + 1/3 (P y)^T Hv (P y) + sigma_Y alpha,
//   Hv = diag(H, H, H, H/2, H/2, H/2) (engineering shears: (P y)^T Hv (P y) = H e_vp:e_vp);
//   Psi(A) = sigma_d edot0/(n+1) ((s_A + A_alpha)^+ / sigma_d)^(n+1) = c_Psi ((s_A + A5)^+)^b_Psi,
//   s_A^2 = A0^2 + A1^2 - A0 A1 + 3 (A2^2 + A3^2 + A4^2) (von Mises norm of dev A_vp),
//   b_Psi = n + 1, c_Psi = sigma_d edot0/(n+1) sigma_d^-(n+1).
// The yield function is not smooth in the dual (dissipation) form, so this
// law is integrated in its force-potential form only (gsm_update_ode23).
struct MichelSuquet {
  static constexpr int NY = 6;

  template <class EP, class YP, class P> AD_HD static auto psi(const EP& e, const YP& y, const P& p) {
    using ad::get;
    const auto& y0 = get<0>(y); const auto& y1 = get<1>(y); const auto& y2 = get<2>(y);
    const auto& y3 = get<3>(y); const auto& y4 = get<4>(y); const auto& al = get<5>(y);
    using S = typename std::decay_t<decltype(y0)>::scalar;
    auto a0 = get<0>(e) - y0;
    auto a1 = get<1>(e) - y1;
    auto a2 = get<2>(e) + (y0 + y1);
    auto a3 = get<3>(e) - y2;
    auto a4 = get<4>(e) - y3;
    auto a5 = get<5>(e) - y4;
    auto tr = a0 + a1 + a2;
    auto el = (p.lam * 0.5) * sq(tr) + p.mu * (sq(a0) + sq(a1) + sq(a2)) + (p.mu * 0.5) * (sq(a3) + sq(a4) + sq(a5));
    auto kin = (p.H_kin * S(1.0 / 3.0)) * ((sq(y0) + sq(y1) + sq(y0 + y1)) + S(0.5) * (sq(y2) + sq(y3) + sq(y4)));
    return el + kin + p.sig_Y * al;
  }

  template <class AP, class P> AD_HD static auto Psi(const AP& A, const P& p) {
    using ad::get;
    const auto& a0 = get<0>(A); const auto& a1 = get<1>(A); const auto& a2 = get<2>(A);
    const auto& a3 = get<3>(A); const auto& a4 = get<4>(A); const auto& a5 = get<5>(A);
    using S = typename std::decay_t<decltype(a0)>::scalar;
    auto s2 = (sq(a0) + sq(a1) - a0 * a1) + S(3) * (sq(a2) + sq(a3) + sq(a4));
    return p.c_Psi * pospow(sqrt0(s2) + a5, p.b_Psi);
  }
  // Psi = c_Psi (x^+)^beta with x = s_A + A_alpha (for the hand third derivative of ode23s)
  static constexpr bool kYield = true;
  AD_HD static double Psi_beta(const LawParams<double>& p) { return p.b_Psi; }
};

}  // namespace gsm
