// Material update by adaptive explicit Runge-Kutta integration of the
// force-potential form (AutoMat, arXiv 2006.04391, Sec. 4.3 and Sec. 4.5).
//
// Sec. 2, Eq. gsm_internal: ydot = dPsi/dA (A), A = -d psi/dy (eps(t), y), with
// the strain interpolated linearly over the load step,
// eps(t) = eps_n + theta (eps_{n+1} - eps_n), theta = (t - t_n)/h.
// Integrators (Sec. 4.3): the Bogacki-Shampine 3(2) pair (MATLAB's ode23),
// first stage = last stage of the previous step, or ode12, the explicit Euler
// (order 1) / Heun (order 2) pair continued with Heun's solution; step sizes
// after Hairer, Norsett and Wanner (Solving ODEs I, II.4) with exponent
// 1/(q+1), q the lower order; whole interval as the first trial step.
// Error measure (Sec. 4.5, stress-driven): RMS over the stress pair the two
// embedded solutions give at the end of the substep, scaled by atol + rtol
// max(|sigma_old|, |sigma_new|); with the tangent also over the tangent pair.
// Tangent (Corollary 1): dY/dt = Psi_AA(A) dA/deps_{n+1},
// dA/deps_{n+1} = -(theta psi_ye + psi_yy Y), integrated with the same steps
// (step sizes undifferentiated); C = dsigma/deps_{n+1} = theta psi_ee + psi_ey Y.
// All derivatives of psi and Psi come from the AD sweeps; FP64 throughout.
#pragma once

#include "solver.cuh"

namespace gsm {

struct Ode23Ctl {
  double rtol, atol;
  int max_steps;  // accepted + rejected substeps
};

// Embedded explicit Runge-Kutta pairs.
enum : int { ERK_BS23 = 0, ERK_HEUN12 = 1 };

// Status word of the ode23 update: bits 0-15 accepted substeps, bits 20-30
// rejected substeps (both saturating), flags in bits 16-19 as elsewhere.
enum : unsigned { ST_ODE_REJ_SHIFT = 20 };

// Number of stored internal-variable components of a law: z (6 Voigt
// entries, z33 = -z11 - z22) plus any further scalars (alpha).
template <class Law> constexpr int stored_nz() { return Law::NY + 1; }

// psi_y at (eps, y): first-order reverse sweep over the NY internal variables.
template <class Law>
AD_HD void ode_psi_y(const LawParams<double>& p, const double (&eps)[6], const double (&y)[Law::NY],
                     double (&g)[Law::NY]) {
  constexpr int NY = Law::NY;
  EpsCst<double> E;
  fill_cst(E, eps);
  ad::UniformPack<ad::Var<double>, NY> Y;
  ad::For<0, NY>::run([&](auto kc) { ad::get_mut<decltype(kc)::value>(Y).v = y[decltype(kc)::value]; });
  auto f = Law::psi(E, Y, p);
  f.fwd();
  f.back(1.0);
  ad::For<0, NY>::run([&](auto kc) { g[decltype(kc)::value] = ad::get<decltype(kc)::value>(Y).a; });
}

// sigma = psi_eps at (eps, y).
template <class Law>
AD_HD void ode_sigma(const LawParams<double>& p, const double (&eps)[6], const double (&y)[Law::NY],
                     double (&sig)[6]) {
  constexpr int NY = Law::NY;
  ad::UniformPack<ad::Var<double>, 6> E;
  ad::For<0, 6>::run([&](auto kc) { ad::get_mut<decltype(kc)::value>(E).v = eps[decltype(kc)::value]; });
  ad::UniformPack<ad::Cst<double>, NY> Y;
  ad::For<0, NY>::run([&](auto kc) { ad::get_mut<decltype(kc)::value>(Y).v = y[decltype(kc)::value]; });
  auto f = Law::psi(E, Y, p);
  f.fwd();
  f.back(1.0);
  ad::For<0, 6>::run([&](auto kc) { sig[decltype(kc)::value] = ad::get<decltype(kc)::value>(E).a; });
}

// psi_y, psi_ye (NY x 6) and psi_yy (NY x NY) at (eps, y); with SIG also sigma and
// sigma's blocks psi_ee (6x6), psi_ey (6 x NY).  One forward-over-reverse sweep with
// 6 + NY unit directions.
template <class Law, bool SIG>
AD_HD void ode_blocks(const LawParams<double>& p, const double (&eps)[6], const double (&y)[Law::NY],
                      double (&g)[Law::NY], double (&Hye)[Law::NY][6], double (&Hyy)[Law::NY][Law::NY],
                      double (&sig)[6], double (&Cee)[6][6], double (&Cey)[6][Law::NY]) {
  constexpr int NY = Law::NY, ND = 6 + NY;
  ad::SeededPack<ad::Var, double, ND, 0, 6> E;
  ad::SeededPack<ad::Var, double, ND, 6, NY> Y;
  ad::seed_unit<decltype(E), double, 0, 6>(E, eps);
  ad::seed_unit<decltype(Y), double, 6, NY>(Y, y);
  auto f = Law::psi(E, Y, p);
  f.fwd();
  f.back(1.0);
  ad::For<0, NY>::run([&](auto kc) {
    constexpr int a = decltype(kc)::value;
    const auto& ad_ = ad::get<a>(Y).a;
    g[a] = ad_.v;
#pragma unroll
    for (int j = 0; j < 6; ++j) Hye[a][j] = ad_.d[j];
#pragma unroll
    for (int j = 0; j < NY; ++j) Hyy[a][j] = ad_.d[6 + j];
  });
  if constexpr (SIG) {
    ad::For<0, 6>::run([&](auto kc) {
      constexpr int i = decltype(kc)::value;
      const auto& ad_ = ad::get<i>(E).a;
      sig[i] = ad_.v;
#pragma unroll
      for (int j = 0; j < 6; ++j) Cee[i][j] = ad_.d[j];
#pragma unroll
      for (int j = 0; j < NY; ++j) Cey[i][j] = ad_.d[6 + j];
    });
  }
}

// Psi_A (first order) and Psi_A, Psi_AA (vector mode) of the force potential.
template <class Law>
AD_HD void force_a(const LawParams<double>& p, const double (&A)[Law::NY], double (&g)[Law::NY]) {
  constexpr int NY = Law::NY;
  ad::UniformPack<ad::Var<double>, NY> X;
  ad::For<0, NY>::run([&](auto kc) { ad::get_mut<decltype(kc)::value>(X).v = A[decltype(kc)::value]; });
  auto f = Law::Psi(X, p);
  f.fwd();
  f.back(1.0);
  ad::For<0, NY>::run([&](auto kc) { g[decltype(kc)::value] = ad::get<decltype(kc)::value>(X).a; });
}

template <class Law>
AD_HD void force_a_aa(const LawParams<double>& p, const double (&A)[Law::NY], double (&g)[Law::NY],
                      double (&H)[Law::NY][Law::NY]) {
  constexpr int NY = Law::NY;
  ad::SeededPack<ad::Var, double, NY, 0, NY> X;
  ad::seed_unit<decltype(X), double, 0, NY>(X, A);
  auto f = Law::Psi(X, p);
  f.fwd();
  f.back(1.0);
  ad::For<0, NY>::run([&](auto kc) {
    constexpr int a = decltype(kc)::value;
    const auto& ad_ = ad::get<a>(X).a;
    g[a] = ad_.v;
#pragma unroll
    for (int j = 0; j < NY; ++j) H[a][j] = ad_.d[j];
  });
}

template <int NY, bool TAN> struct OdeState {
  double y[NY];
  double Y[TAN ? NY : 1][TAN ? 6 : 1];
};

// Right-hand side at theta = t/h: f = Psi_A(A), A = -psi_y, and with TAN
// F = Psi_AA(A) dA/deps_{n+1}, dA/deps_{n+1} = -(theta psi_ye + psi_yy Y).
template <class Law, bool TAN>
AD_HD void ode_rhs(const LawParams<double>& p, const double (&epsn)[6], const double (&de)[6], double theta,
                   const OdeState<Law::NY, TAN>& s, double (&f)[Law::NY],
                   double (&F)[TAN ? Law::NY : 1][TAN ? 6 : 1]) {
  constexpr int NY = Law::NY;
  double et[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) et[i] = fma(theta, de[i], epsn[i]);
  double A[NY];
  if constexpr (!TAN) {
    double g[NY];
    ode_psi_y<Law>(p, et, s.y, g);
#pragma unroll
    for (int a = 0; a < NY; ++a) A[a] = -g[a];
    force_a<Law>(p, A, f);
  } else {
    double g[NY], Hye[NY][6], Hyy[NY][NY], sig_[6], Cee_[6][6], Cey_[6][NY];
    ode_blocks<Law, false>(p, et, s.y, g, Hye, Hyy, sig_, Cee_, Cey_);
#pragma unroll
    for (int a = 0; a < NY; ++a) A[a] = -g[a];
    double H[NY][NY];
    force_a_aa<Law>(p, A, f, H);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      double dA[NY];
#pragma unroll
      for (int a = 0; a < NY; ++a) {
        double t = theta * Hye[a][k];
#pragma unroll
        for (int b = 0; b < NY; ++b) t = fma(Hyy[a][b], s.Y[b][k], t);
        dA[a] = -t;
      }
#pragma unroll
      for (int a = 0; a < NY; ++a) {
        double t = 0.0;
#pragma unroll
        for (int b = 0; b < NY; ++b) t = fma(H[a][b], dA[b], t);
        F[a][k] = t;
      }
    }
  }
}

// Stress (and with TAN the tangent C = theta psi_ee + psi_ey Y) at theta.
template <class Law, bool TAN>
AD_HD void ode_stress(const LawParams<double>& p, const double (&epsn)[6], const double (&de)[6], double theta,
                      const OdeState<Law::NY, TAN>& s, double (&sig)[6], double (&C)[TAN ? 6 : 1][TAN ? 6 : 1]) {
  constexpr int NY = Law::NY;
  double et[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) et[i] = fma(theta, de[i], epsn[i]);
  if constexpr (!TAN) {
    ode_sigma<Law>(p, et, s.y, sig);
  } else {
    double g_[NY], Hye_[NY][6], Hyy_[NY][NY], Cee[6][6], Cey[6][NY];
    ode_blocks<Law, true>(p, et, s.y, g_, Hye_, Hyy_, sig, Cee, Cey);
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        double t = theta * Cee[i][k];
#pragma unroll
        for (int a = 0; a < NY; ++a) t = fma(Cey[i][a], s.Y[a][k], t);
        C[i][k] = t;
      }
  }
}

// (d / sc)^2 of one error-measure entry; a zero scale (atol = 0 at zero
// stress) counts a zero difference as no error.
AD_HD double scaled_sq(double d, double sc) {
  const double q = sc > 0.0 ? d * recip_pos(sc) : (d == 0.0 ? 0.0 : 1e300);
  return q * q;
}

// The ode23 integration of one voxel as a resumable state: init() at the
// start of the load step, attempt() for one trial substep (accepted or
// rejected; sets done at the end of the interval or at the substep cap),
// finish() for the outputs.  A kernel can therefore hand a lane its next voxel
// as soon as its current one is done, instead of letting the lane wait for
// the slowest voxel of its warp.
template <class Law, bool TAN, int PAIR = ERK_BS23> struct ErkVoxel {
  static constexpr int NY = Law::NY, NZ = stored_nz<Law>();
  using M56 = double[TAN ? NY : 1][TAN ? 6 : 1];
  using M66 = double[TAN ? 6 : 1][TAN ? 6 : 1];
  double epsn[6], de[6];
  OdeState<NY, TAN> s;
  double k1[NY];
  M56 K1;
  double sig_old[6];
  M66 C_old;
  double t, dt;
  int n_acc, n_rej;
  unsigned flags;
  bool last_rejected, done;

  // zn: the NZ stored internal variables (z in Voigt order, then alpha, ...)
  AD_HD void init(const LawParams<double>& p, const double (&e0)[6], const double (&e1)[6], const double (&zn)[NZ],
                  double h) {
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      epsn[i] = e0[i];
      de[i] = e1[i] - e0[i];
    }
    s.y[0] = zn[0];
    s.y[1] = zn[1];
    s.y[2] = zn[3];
    s.y[3] = zn[4];
    s.y[4] = zn[5];
#pragma unroll
    for (int a = 5; a < NY; ++a) s.y[a] = zn[a + 1];
    if constexpr (TAN) {
#pragma unroll
      for (int a = 0; a < NY; ++a)
#pragma unroll
        for (int k = 0; k < 6; ++k) s.Y[a][k] = 0.0;
    }
    ode_rhs<Law, TAN>(p, epsn, de, 0.0, s, k1, K1);
    ode_stress<Law, TAN>(p, epsn, de, 0.0, s, sig_old, C_old);
    t = 0.0;
    dt = h;
    n_acc = n_rej = 0;
    flags = 0;
    last_rejected = false;
    done = false;
  }

  AD_HD void attempt(const LawParams<double>& p, const Step& hs, const Ode23Ctl& ctl) {
    if constexpr (PAIR == ERK_BS23) attempt_bs23(p, hs, ctl);
    else attempt_heun12(p, hs, ctl);
  }

  // Error-norm entries of a stress (and tangent) pair against the last accepted
  // stress (and tangent): returns the RMS-scaled error.
  AD_HD double pair_error(const double (&s_hi)[6], const double (&s_lo)[6], const M66& C_hi, const M66& C_lo,
                          const Ode23Ctl& ctl) const {
    double sum = 0.0;
#pragma unroll
    for (int i = 0; i < 6; ++i)
      sum += scaled_sq(s_hi[i] - s_lo[i], fma(ctl.rtol, fmax_(fabs(sig_old[i]), fabs(s_hi[i])), ctl.atol));
    int m = 6;
    if constexpr (TAN) {
#pragma unroll
      for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int c = 0; c < 6; ++c)
          sum += scaled_sq(C_hi[i][c] - C_lo[i][c], fma(ctl.rtol, fmax_(fabs(C_old[i][c]), fabs(C_hi[i][c])), ctl.atol));
      m = 42;
    }
    // a trial step that overflows is rejected like one with a large error
    return finite64(sum) ? sqrt(sum / m) : 1e300;
  }

  // Accept (err <= 1: move to the new state, its right-hand side and stress)
  // or reject; next substep length after Hairer II.4 (fac 0.9, facmin 0.2,
  // facmax 5, 1 right after a rejection).
  AD_HD void conclude(double err, double tn1, bool clip, const OdeState<NY, TAN>& snew, const double (&knew)[NY],
                      const M56& Knew, const double (&s_hi)[6], const M66& C_hi) {
    const double facmax = last_rejected ? 1.0 : 5.0;
    double f;
    if constexpr (PAIR == ERK_BS23) f = err == 0.0 ? 1e300 : 0.9 * fpow::pow_pos(err, -1.0 / 3.0);
    else f = err == 0.0 ? 1e300 : 0.9 / sqrt(err);
    const double grow = fmin(facmax, fmax(0.2, f));
    if (err <= 1.0) {
      t = tn1;
#pragma unroll
      for (int a = 0; a < NY; ++a) {
        s.y[a] = snew.y[a];
        k1[a] = knew[a];
        if constexpr (TAN)
#pragma unroll
          for (int c = 0; c < 6; ++c) {
            s.Y[a][c] = snew.Y[a][c];
            K1[a][c] = Knew[a][c];
          }
      }
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        sig_old[i] = s_hi[i];
        if constexpr (TAN)
#pragma unroll
          for (int c = 0; c < 6; ++c) C_old[i][c] = C_hi[i][c];
      }
      ++n_acc;
      last_rejected = false;
      if (clip) done = true;
    } else {
      ++n_rej;
      last_rejected = true;
    }
    dt *= grow;
  }

  // ode12: y_E = y + dt k1, k2 = f(t + dt, y_E), y_H = y + dt/2 (k1 + k2); the
  // error compares the stresses of y_H and y_E; the right-hand side at y_H
  // (k1 of the next substep) is evaluated before the decision so that the
  // lanes of a warp stay together.
  AD_HD void attempt_heun12(const LawParams<double>& p, const Step& hs, const Ode23Ctl& ctl) {
    const double h = hs.h, inv_h = hs.inv_h;
    if (n_acc + n_rej >= ctl.max_steps) {
      flags |= ST_CAP;
      done = true;
      return;
    }
    const bool clip = t + dt >= h;
    if (clip) dt = h - t;
    const double tn1 = clip ? h : t + dt;
    const double th1 = clip ? 1.0 : tn1 * inv_h;
    OdeState<NY, TAN> sE, sH;
#pragma unroll
    for (int a = 0; a < NY; ++a) {
      sE.y[a] = fma(dt, k1[a], s.y[a]);
      if constexpr (TAN)
#pragma unroll
        for (int c = 0; c < 6; ++c) sE.Y[a][c] = fma(dt, K1[a][c], s.Y[a][c]);
    }
    double k[NY];
    M56 Kc;
    ode_rhs<Law, TAN>(p, epsn, de, th1, sE, k, Kc);
    const double hd = 0.5 * dt;
#pragma unroll
    for (int a = 0; a < NY; ++a) {
      sH.y[a] = fma(hd, k1[a] + k[a], s.y[a]);
      if constexpr (TAN)
#pragma unroll
        for (int c = 0; c < 6; ++c) sH.Y[a][c] = fma(hd, K1[a][c] + Kc[a][c], s.Y[a][c]);
    }
    double s_hi[6], s_lo[6];
    M66 C_hi, C_lo;
    ode_stress<Law, TAN>(p, epsn, de, th1, sH, s_hi, C_hi);
    ode_stress<Law, TAN>(p, epsn, de, th1, sE, s_lo, C_lo);
    const double err = pair_error(s_hi, s_lo, C_hi, C_lo, ctl);
    ode_rhs<Law, TAN>(p, epsn, de, th1, sH, k, Kc);
    conclude(err, tn1, clip, sH, k, Kc, s_hi, C_hi);
  }

  AD_HD void attempt_bs23(const LawParams<double>& p, const Step& hs, const Ode23Ctl& ctl) {
    // Bogacki-Shampine 3(2): c = (0, 1/2, 3/4, 1), order-3 weights (2/9, 1/3, 4/9),
    // order-2 weights (7/24, 1/4, 1/3, 1/8) on k1..k4 with k4 = f(t + dt, y3).
    constexpr double b1 = 2.0 / 9.0, b2 = 1.0 / 3.0, b3 = 4.0 / 9.0;
    constexpr double e1 = 2.0 / 9.0 - 7.0 / 24.0, e2 = 1.0 / 3.0 - 1.0 / 4.0, e3 = 4.0 / 9.0 - 1.0 / 3.0,
                     e4 = -1.0 / 8.0;
    const double h = hs.h, inv_h = hs.inv_h;
    if (n_acc + n_rej >= ctl.max_steps) {
      flags |= ST_CAP;
      done = true;
      return;
    }
    const bool clip = t + dt >= h;  // the substep that ends the interval ends at h exactly
    if (clip) dt = h - t;
    // stage 2
    OdeState<NY, TAN> st;
    double k[NY], y3[NY], e[NY];
    M56 Kc, Y3, E;
#pragma unroll
    for (int a = 0; a < NY; ++a) {
      st.y[a] = fma(0.5 * dt, k1[a], s.y[a]);
      y3[a] = fma(b1 * dt, k1[a], s.y[a]);
      e[a] = e1 * dt * k1[a];
      if constexpr (TAN)
#pragma unroll
        for (int c = 0; c < 6; ++c) {
          st.Y[a][c] = fma(0.5 * dt, K1[a][c], s.Y[a][c]);
          Y3[a][c] = fma(b1 * dt, K1[a][c], s.Y[a][c]);
          E[a][c] = e1 * dt * K1[a][c];
        }
    }
    ode_rhs<Law, TAN>(p, epsn, de, (t + 0.5 * dt) * inv_h, st, k, Kc);
    // stage 3
#pragma unroll
    for (int a = 0; a < NY; ++a) {
      st.y[a] = fma(0.75 * dt, k[a], s.y[a]);
      y3[a] = fma(b2 * dt, k[a], y3[a]);
      e[a] = fma(e2 * dt, k[a], e[a]);
      if constexpr (TAN)
#pragma unroll
        for (int c = 0; c < 6; ++c) {
          st.Y[a][c] = fma(0.75 * dt, Kc[a][c], s.Y[a][c]);
          Y3[a][c] = fma(b2 * dt, Kc[a][c], Y3[a][c]);
          E[a][c] = fma(e2 * dt, Kc[a][c], E[a][c]);
        }
    }
    ode_rhs<Law, TAN>(p, epsn, de, (t + 0.75 * dt) * inv_h, st, k, Kc);
#pragma unroll
    for (int a = 0; a < NY; ++a) {
      y3[a] = fma(b3 * dt, k[a], y3[a]);
      e[a] = fma(e3 * dt, k[a], e[a]);
      if constexpr (TAN)
#pragma unroll
        for (int c = 0; c < 6; ++c) {
          Y3[a][c] = fma(b3 * dt, Kc[a][c], Y3[a][c]);
          E[a][c] = fma(e3 * dt, Kc[a][c], E[a][c]);
        }
    }
    // last stage at the new point (k1 of the next step)
    const double tn1 = clip ? h : t + dt;
    const double th1 = clip ? 1.0 : tn1 * inv_h;
    OdeState<NY, TAN> s3;
#pragma unroll
    for (int a = 0; a < NY; ++a) {
      s3.y[a] = y3[a];
      if constexpr (TAN)
#pragma unroll
        for (int c = 0; c < 6; ++c) s3.Y[a][c] = Y3[a][c];
    }
    double k4[NY];
    M56 K4;
    ode_rhs<Law, TAN>(p, epsn, de, th1, s3, k4, K4);
#pragma unroll
    for (int a = 0; a < NY; ++a) {
      e[a] = fma(e4 * dt, k4[a], e[a]);
      if constexpr (TAN)
#pragma unroll
        for (int c = 0; c < 6; ++c) E[a][c] = fma(e4 * dt, K4[a][c], E[a][c]);
    }
    // stress pair (and tangent pair) of the two embedded solutions
    double s_hi[6], s_lo[6];
    M66 C_hi, C_lo;
    ode_stress<Law, TAN>(p, epsn, de, th1, s3, s_hi, C_hi);
    OdeState<NY, TAN> s2;
#pragma unroll
    for (int a = 0; a < NY; ++a) {
      s2.y[a] = y3[a] - e[a];
      if constexpr (TAN)
#pragma unroll
        for (int c = 0; c < 6; ++c) s2.Y[a][c] = Y3[a][c] - E[a][c];
    }
    ode_stress<Law, TAN>(p, epsn, de, th1, s2, s_lo, C_lo);
    conclude(pair_error(s_hi, s_lo, C_hi, C_lo, ctl), tn1, clip, s3, k4, K4, s_hi, C_hi);
  }

  // outputs at the end of the step (sig_old is the stress of the last accepted
  // substep); C36: row-major 6x6 (the tangent of an explicit integrator is
  // not symmetric in general), written only with TAN and when non-NULL
  AD_HD unsigned finish(double h, double (&sig)[6], double (&z)[NZ], double* C36) const {
#pragma unroll
    for (int i = 0; i < 6; ++i) sig[i] = sig_old[i];
    if constexpr (TAN) {
      if (C36)
#pragma unroll
        for (int i = 0; i < 6; ++i)
#pragma unroll
          for (int c = 0; c < 6; ++c) C36[6 * i + c] = C_old[i][c];
    }
    z[0] = s.y[0];
    z[1] = s.y[1];
    z[2] = -(s.y[0] + s.y[1]);
    z[3] = s.y[2];
    z[4] = s.y[3];
    z[5] = s.y[4];
#pragma unroll
    for (int a = 5; a < NY; ++a) z[a + 1] = s.y[a];
    unsigned st = flags;
    if (t >= h && !(flags & ST_CAP)) st |= ST_CONVERGED;
    if (!finite64(sig[0]) || !finite64(z[0])) st |= ST_NONFINITE;
    st |= (unsigned)(n_acc < 0xffff ? n_acc : 0xffff);
    st |= (unsigned)(n_rej < 0x7ff ? n_rej : 0x7ff) << ST_ODE_REJ_SHIFT;
    return st;
  }
};

template <class Law, bool TAN> using Ode23Voxel = ErkVoxel<Law, TAN, ERK_BS23>;

// One voxel, start to end (single thread; the kernel schedules ErkVoxel
// states per lane itself).
template <class Law, bool TAN, int PAIR = ERK_BS23>
AD_HD unsigned voxel_ode23(const LawParams<double>& p, const double (&epsn)[6], const double (&eps1)[6],
                           const double (&zn)[stored_nz<Law>()], const Step& hs, const Ode23Ctl& ctl,
                           double (&sig)[6], double (&z)[stored_nz<Law>()], double* C36) {
  ErkVoxel<Law, TAN, PAIR> v;
  v.init(p, epsn, eps1, zn, hs.h);
  while (!v.done) v.attempt(p, hs, ctl);
  return v.finish(hs.h, sig, z, C36);
}

}  // namespace gsm
