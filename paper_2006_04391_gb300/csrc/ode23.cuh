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

#include <type_traits>

#include "solver.cuh"

namespace gsm {

struct Ode23Ctl {
  double rtol, atol;
  int max_steps;  // accepted + rejected substeps
};

// Embedded explicit Runge-Kutta pairs, and the Rosenbrock triple of ode23s.
enum : int { ERK_BS23 = 0, ERK_HEUN12 = 1, ROS_23S = 2 };

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

// Second-derivative blocks of psi: psi_ye (NY x 6), psi_yy, psi_ee, psi_ey.
// The free energies of both laws are quadratic in (eps, y), so the blocks are
// constants of the law: one forward-over-reverse sweep (at eps = 0, y = 0)
// gives them for every voxel and substep, instead of one sweep per stage.
// (For a quadratic the sweep's second-order parts do not involve the point,
// so the blocks equal those of a sweep at the stage bit for bit.)
template <int NY> struct PsiBlocks {
  double Hye[NY][6], Hyy[NY][NY], Cee[6][6], Cey[6][NY];
};

template <class Law> struct PsiPattern;
template <class Law> AD_HD void psi_const_blocks(const LawParams<double>& p, PsiBlocks<Law::NY>& B) {
  static_assert(sizeof(PsiPattern<Law>) > 0, "");  // instantiates the quadratic check
  constexpr int NY = Law::NY;
  double e0[6], y0[NY], g[NY], sig[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) e0[i] = 0.0;
#pragma unroll
  for (int a = 0; a < NY; ++a) y0[a] = 0.0;
  ode_blocks<Law, true>(p, e0, y0, g, B.Hye, B.Hyy, sig, B.Cee, B.Cey);
}

// Structural pattern of the blocks, read off psi's expression type with the
// seeds of ode_blocks (leaves eps_0..5 then y_0..NY-1): the entries it marks
// zero are exactly -0.0 in every sweep, and the block products below skip
// them at compile time (for the laws here it marks 9 entries of psi_ye, 7 of
// psi_yy, 12 of the 36 of psi_ee and 9 of psi_ey; of these the lambda terms of
// psi_ye and psi_ey cancel numerically).
template <class Law> struct PsiPattern {
  static constexpr int NY = Law::NY, ND = 6 + NY;
  using EP = ad::SeededPack<ad::Var, double, ND, 0, 6>;
  using YP = ad::SeededPack<ad::Var, double, ND, 6, NY>;
  using Expr = decltype(Law::psi(std::declval<const EP&>(), std::declval<const YP&>(),
                                 std::declval<const LawParams<double>&>()));
  static_assert(ad::Degree<Expr>::value <= 2,
                "the constant-block tangent needs a free energy quadratic in (eps, y)");
  template <int R> static constexpr unsigned row() { return ad::hess_row<Expr, R>(); }
  template <int A, int K> static constexpr bool hye() { return ((row<6 + A>() >> K) & 1u) != 0u; }
  template <int A, int B> static constexpr bool hyy() { return ((row<6 + A>() >> (6 + B)) & 1u) != 0u; }
  template <int I, int K> static constexpr bool cee() { return ((row<I>() >> K) & 1u) != 0u; }
  template <int I, int A> static constexpr bool cey() { return ((row<I>() >> (6 + A)) & 1u) != 0u; }
};

// dA_k = -(theta psi_ye e_k + psi_yy Y e_k) over the structural non-zeros.
template <class Law, int K, class YM>
AD_HD void dA_column(const PsiBlocks<Law::NY>& B, double theta, const YM& Y, double (&dA)[Law::NY]) {
  using Pat = PsiPattern<Law>;
  ad::For<0, Law::NY>::run([&](auto ac) {
    constexpr int a = decltype(ac)::value;
    double t = 0.0;
    if constexpr (Pat::template hye<a, K>()) t = theta * B.Hye[a][K];
    ad::For<0, Law::NY>::run([&](auto bc) {
      constexpr int b = decltype(bc)::value;
      if constexpr (Pat::template hyy<a, b>()) t = fma(B.Hyy[a][b], Y[b][K], t);
    });
    dA[a] = -t;
  });
}

// C_ik = theta psi_ee,ik + sum_a psi_ey,ia Y_ak over the structural non-zeros.
template <class Law, int I, int K, class YM>
AD_HD double c_entry(const PsiBlocks<Law::NY>& B, double theta, const YM& Y) {
  using Pat = PsiPattern<Law>;
  double t = 0.0;
  if constexpr (Pat::template cee<I, K>()) t = theta * B.Cee[I][K];
  ad::For<0, Law::NY>::run([&](auto ac) {
    constexpr int a = decltype(ac)::value;
    if constexpr (Pat::template cey<I, a>()) t = fma(B.Cey[I][a], Y[a][K], t);
  });
  return t;
}

// Right-hand side at theta = t/h: f = Psi_A(A), A = -psi_y, and with TAN
// F = Psi_AA(A) dA/deps_{n+1}, dA/deps_{n+1} = -(theta psi_ye + psi_yy Y)
// (the blocks B of psi, required with TAN).
template <class Law, bool TAN>
AD_HD void ode_rhs(const LawParams<double>& p, const double (&epsn)[6], const double (&de)[6], double theta,
                   const OdeState<Law::NY, TAN>& s, double (&f)[Law::NY],
                   double (&F)[TAN ? Law::NY : 1][TAN ? 6 : 1], const PsiBlocks<Law::NY>* B = nullptr) {
  constexpr int NY = Law::NY;
  double et[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) et[i] = fma(theta, de[i], epsn[i]);
  double A[NY];
  double g[NY];
  ode_psi_y<Law>(p, et, s.y, g);
#pragma unroll
  for (int a = 0; a < NY; ++a) A[a] = -g[a];
  if constexpr (!TAN) {
    force_a<Law>(p, A, f);
  } else {
    double H[NY][NY];
    force_a_aa<Law>(p, A, f, H);
    ad::For<0, 6>::run([&](auto kc) {
      constexpr int k = decltype(kc)::value;
      double dA[NY];
      dA_column<Law, k>(*B, theta, s.Y, dA);
#pragma unroll
      for (int a = 0; a < NY; ++a) {
        double t = 0.0;
#pragma unroll
        for (int b = 0; b < NY; ++b) t = fma(H[a][b], dA[b], t);
        F[a][k] = t;
      }
    });
  }
}

// Stress (and with TAN the tangent C = theta psi_ee + psi_ey Y) at theta.
template <class Law, bool TAN>
AD_HD void ode_stress(const LawParams<double>& p, const double (&epsn)[6], const double (&de)[6], double theta,
                      const OdeState<Law::NY, TAN>& s, double (&sig)[6], double (&C)[TAN ? 6 : 1][TAN ? 6 : 1],
                      const PsiBlocks<Law::NY>* B = nullptr) {
  constexpr int NY = Law::NY;
  double et[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) et[i] = fma(theta, de[i], epsn[i]);
  ode_sigma<Law>(p, et, s.y, sig);
  if constexpr (TAN) {
    ad::For<0, 6>::run([&](auto ic) {
      constexpr int i = decltype(ic)::value;
      ad::For<0, 6>::run([&](auto kc) {
        constexpr int k = decltype(kc)::value;
        C[i][k] = c_entry<Law, i, k>(*B, theta, s.Y);
      });
    });
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
  const PsiBlocks<NY>* blk;  // psi's second-derivative blocks (with TAN)

  // zn: the NZ stored internal variables (z in Voigt order, then alpha, ...);
  // B: the law's blocks (psi_const_blocks), required with TAN
  AD_HD void init(const LawParams<double>& p, const double (&e0)[6], const double (&e1)[6], const double (&zn)[NZ],
                  double h, const PsiBlocks<NY>* B = nullptr) {
    blk = B;
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
    ode_rhs<Law, TAN>(p, epsn, de, 0.0, s, k1, K1, blk);
    ode_stress<Law, TAN>(p, epsn, de, 0.0, s, sig_old, C_old, blk);
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
    ode_rhs<Law, TAN>(p, epsn, de, th1, sE, k, Kc, blk);
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
    ode_stress<Law, TAN>(p, epsn, de, th1, sH, s_hi, C_hi, blk);
    ode_stress<Law, TAN>(p, epsn, de, th1, sE, s_lo, C_lo, blk);
    const double err = pair_error(s_hi, s_lo, C_hi, C_lo, ctl);
    ode_rhs<Law, TAN>(p, epsn, de, th1, sH, k, Kc, blk);
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
    ode_rhs<Law, TAN>(p, epsn, de, (t + 0.5 * dt) * inv_h, st, k, Kc, blk);
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
    ode_rhs<Law, TAN>(p, epsn, de, (t + 0.75 * dt) * inv_h, st, k, Kc, blk);
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
    ode_rhs<Law, TAN>(p, epsn, de, th1, s3, k4, K4, blk);
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
    ode_stress<Law, TAN>(p, epsn, de, th1, s3, s_hi, C_hi, blk);
    OdeState<NY, TAN> s2;
#pragma unroll
    for (int a = 0; a < NY; ++a) {
      s2.y[a] = y3[a] - e[a];
      if constexpr (TAN)
#pragma unroll
        for (int c = 0; c < 6; ++c) s2.Y[a][c] = Y3[a][c] - E[a][c];
    }
    ode_stress<Law, TAN>(p, epsn, de, th1, s2, s_lo, C_lo, blk);
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

// ------------------------------------------------------------------ ode23s
//
// Third derivative of the force potential contracted with two directions,
// out = Psi_AAA[u, v]: the hand partial the Rosenbrock tangent needs (the
// paper's semi-automatic strategy: the AD here stops at second order).  Both
// laws have Psi = c (x^+)^beta with x = s (Norton) or s + A_alpha
// (Michel-Suquet), s^2 = A_z^T M A_z, M = [[1, -1/2], [-1/2, 1]] + 3 I_3 (von
// Mises).  With m = M A_z / s, Q = M - m m^T and r(x) = dPsi/dx:
//   H_zz = r' m m^T + r Q/s,  H_za = r' m,  H_aa = r',
// and along u (dx = m.u_z + u_a, ds = m.u_z, dm = Q u_z / s):
//   dH_zz = r'' dx m m^T + (r' - r/s)(dm m^T + m dm^T) + (r' dx - r ds/s) Q/s,
//   dH_za = r'' dx m + r' dm,  dH_aa = r'' dx;  zero where x <= 0 or s = 0.
// The factors of Psi_AAA that depend on A alone (m, 1/s and r0..r2), formed
// once per state; apply() adds the parts along u and v.  The Rosenbrock
// tangent applies it 24 times per substep at the substep's start state.
template <class Law> struct ForceAAA {
  double m[5], inv_s, r0, r1, r2;
  bool on;  // false where x <= 0 or s = 0 (Psi_AAA = 0)

  AD_HD void setup(const LawParams<double>& p, const double (&A)[Law::NY]) {
    double MA[5];
    MA[0] = A[0] - 0.5 * A[1];
    MA[1] = A[1] - 0.5 * A[0];
    MA[2] = 3.0 * A[2];
    MA[3] = 3.0 * A[3];
    MA[4] = 3.0 * A[4];
    double s2 = 0.0;
#pragma unroll
    for (int a = 0; a < 5; ++a) s2 = fma(A[a], MA[a], s2);
    const double s = sqrt(s2);
    double x = s;
    if constexpr (Law::kYield) x += A[5];
    on = x > 0.0 && s > 0.0;
    if (!on) return;
    const double beta = Law::Psi_beta(p);
    const double px = fpow::pow_pos(x, beta - 3.0);
    r2 = p.c_Psi * beta * (beta - 1.0) * (beta - 2.0) * px;
    r1 = p.c_Psi * beta * (beta - 1.0) * px * x;
    r0 = p.c_Psi * beta * px * x * x;
    inv_s = 1.0 / s;
#pragma unroll
    for (int a = 0; a < 5; ++a) m[a] = MA[a] * inv_s;
  }

  // out = Psi_AAA[u, v]
  AD_HD void apply(const double (&u)[Law::NY], const double (&v)[Law::NY], double (&out)[Law::NY]) const {
    constexpr int NY = Law::NY;
#pragma unroll
    for (int a = 0; a < NY; ++a) out[a] = 0.0;
    if (!on) return;
    double Mu[5], Mv[5];
    Mu[0] = u[0] - 0.5 * u[1];
    Mu[1] = u[1] - 0.5 * u[0];
    Mv[0] = v[0] - 0.5 * v[1];
    Mv[1] = v[1] - 0.5 * v[0];
#pragma unroll
    for (int a = 2; a < 5; ++a) {
      Mu[a] = 3.0 * u[a];
      Mv[a] = 3.0 * v[a];
    }
    double ds = 0.0, mv = 0.0;
#pragma unroll
    for (int a = 0; a < 5; ++a) {
      ds = fma(m[a], u[a], ds);
      mv = fma(m[a], v[a], mv);
    }
    double dx = ds;
    double va = 0.0;
    if constexpr (Law::kYield) {
      dx += u[5];
      va = v[5];
    }
    // dm = Q u / s = (M u - m ds)/s;  dm.v;  Q v = M v - m mv
    double dm[5], dmv = 0.0;
#pragma unroll
    for (int a = 0; a < 5; ++a) {
      dm[a] = (Mu[a] - m[a] * ds) * inv_s;
      dmv = fma(dm[a], v[a], dmv);
    }
    const double c1 = r1 - r0 * inv_s, c2 = (r1 * dx - r0 * ds * inv_s) * inv_s;
#pragma unroll
    for (int a = 0; a < 5; ++a) {
      const double Qv = Mv[a] - m[a] * mv;
      out[a] = r2 * dx * m[a] * mv + c1 * (dm[a] * mv + m[a] * dmv) + c2 * Qv + (r2 * dx * m[a] + r1 * dm[a]) * va;
    }
    if constexpr (Law::kYield) out[5] = r2 * dx * mv + r1 * dmv + r2 * dx * va;
  }
};

template <class Law>
AD_HD void force_aaa(const LawParams<double>& p, const double (&A)[Law::NY], const double (&u)[Law::NY],
                     const double (&v)[Law::NY], double (&out)[Law::NY]) {
  ForceAAA<Law> f;
  f.setup(p, A);
  f.apply(u, v, out);
}

// W x = b for the NY x NY matrix of a Rosenbrock stage: Gaussian elimination
// with partial pivoting, factor once (multipliers below, U on and above the
// diagonal, row swaps in piv), solve many by replaying swap and elimination
// column by column; everything in registers (the row swaps are selects over
// compile-time indices).
template <int NY> struct StageLU {
  double w[NY][NY];
  int piv[NY];
  bool ok;

  AD_HD void factor() {
    ok = true;
#pragma unroll
    for (int c = 0; c < NY; ++c) {
      int pr = c;
      double best = fabs(w[c][c]);
#pragma unroll
      for (int r = c + 1; r < NY; ++r)
        if (fabs(w[r][c]) > best) {
          best = fabs(w[r][c]);
          pr = r;
        }
      piv[c] = pr;
#pragma unroll
      for (int r = c + 1; r < NY; ++r)
        if (r == pr)
#pragma unroll
          for (int j = c; j < NY; ++j) {  // (the multipliers left of c stay with their elimination step)
            const double t = w[c][j];
            w[c][j] = w[r][j];
            w[r][j] = t;
          }
      if (!(best > 0.0)) {
        ok = false;
        w[c][c] = 1.0;  // keep the arithmetic finite; the substep is rejected
      }
      const double inv = 1.0 / w[c][c];
#pragma unroll
      for (int r = c + 1; r < NY; ++r) {
        const double f = w[r][c] * inv;
        w[r][c] = f;
#pragma unroll
        for (int j = c + 1; j < NY; ++j) w[r][j] = fma(-f, w[c][j], w[r][j]);
      }
    }
  }

  AD_HD void solve(const double (&b)[NY], double (&x)[NY]) const {
    double y[NY];
#pragma unroll
    for (int i = 0; i < NY; ++i) y[i] = b[i];
#pragma unroll
    for (int c = 0; c < NY; ++c) {
#pragma unroll
      for (int r = c + 1; r < NY; ++r)
        if (r == piv[c]) {
          const double t = y[c];
          y[c] = y[r];
          y[r] = t;
        }
#pragma unroll
      for (int r = c + 1; r < NY; ++r) y[r] = fma(-w[r][c], y[c], y[r]);
    }
#pragma unroll
    for (int i = NY - 1; i >= 0; --i) {
      double t = y[i];
#pragma unroll
      for (int j = i + 1; j < NY; ++j) t = fma(-w[i][j], x[j], t);
      x[i] = t / w[i][i];
    }
  }
};

// ode23s as a resumable voxel state (same interface as ErkVoxel): the modified
// Rosenbrock triple of Shampine and Reichelt (SIAM J. Sci. Comput. 18 (1997)
// 1-22), d = 1/(2 + sqrt 2), e32 = 6 + sqrt 2, J = df/dy = Psi_AA dA/dy and
// T = df/dt = Psi_AA dA/dt at the start (t, y) of a substep, W = I - dt d J:
//   k1 = W^-1 (F0 + dt d T),  F1 = f(t + dt/2, y + dt/2 k1),
//   k2 = W^-1 (F1 - k1) + k1,  y_new = y + dt k2,  F2 = f(t + dt, y_new),
//   k3 = W^-1 (F2 - e32 (k2 - F1) - 2 (k1 - F0) + dt d T),
//   error estimate dt/6 (k1 - 2 k2 + k3), compared through the stresses of
//   y_new and y_new minus the estimate; step control as ode23's (exponent
//   1/3); F2 is F0 of the next substep; J, T re-evaluated after an acceptance.
// dA/dy = -psi_yy and dA/dt = -psi_ye (eps_{n+1} - eps_n)/h are constant for
// both laws (psi is quadratic in (eps, y)).  With TAN, each column k of Y =
// dy/deps_{n+1} follows the differentiated stages (Corollary 1, Rosenbrock
// form), with dA_k = -(theta psi_ye e_k + psi_yy Y e_k):
//   J~_k w = Psi_AAA[dA_k, dA/dy w],  T~_k = Psi_AAA[dA_k, dA/dt] - Psi_AA psi_ye e_k / h,
//   k1~ = W^-1 (F0~ + dt d (T~ + J~ k1)),
//   k2~ = k1~ + W^-1 (F1~ - k1~ + dt d J~ (k2 - k1)),
//   k3~ = W^-1 (F2~ - e32 (k2~ - F1~) - 2 (k1~ - F0~) + dt d (T~ + J~ k3)).
template <class Law, bool TAN> struct RosVoxel {
  static constexpr int NY = Law::NY, NZ = stored_nz<Law>();
  using M56 = double[TAN ? NY : 1][TAN ? 6 : 1];
  using M66 = double[TAN ? 6 : 1][TAN ? 6 : 1];
  double epsn[6], de[6];
  OdeState<NY, TAN> s;
  double F0[NY];
  M56 G0;
  double J[NY][NY], T[NY];
  // dA/dy = -psi_yy (without TAN; with TAN it is read from the law's blocks)
  double dAdy[TAN ? 1 : NY][TAN ? 1 : NY], dAdt[NY];
  // with TAN: Psi_AA and A at the substep start, psi_ye
  double H0[TAN ? NY : 1][TAN ? NY : 1];
  ForceAAA<Law> f3;  // Psi_AAA's factors at the substep start (with TAN)
  double sig_old[6];
  M66 C_old;
  double t, dt;
  int n_acc, n_rej;
  unsigned flags;
  bool last_rejected, done;
  const PsiBlocks<NY>* blk;  // psi's second-derivative blocks (with TAN)

  // Psi_AA at (theta, y): J, T (and, with TAN, H0 and the factors of Psi_AAA).
  AD_HD void refresh(const LawParams<double>& p, double theta, double inv_h) {
    double et[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) et[i] = fma(theta, de[i], epsn[i]);
    double A[NY], f[NY], H[NY][NY];
    if constexpr (TAN) {
      // psi's blocks are the law's constants (blk), their structural zeros skipped
      using Pat = PsiPattern<Law>;
      double g[NY];
      ode_psi_y<Law>(p, et, s.y, g);
#pragma unroll
      for (int a = 0; a < NY; ++a) A[a] = -g[a];
      force_a_aa<Law>(p, A, f, H);
      ad::For<0, NY>::run([&](auto ac) {
        constexpr int a = decltype(ac)::value;
        double tt = 0.0;
        ad::For<0, 6>::run([&](auto kc) {
          constexpr int k = decltype(kc)::value;
          if constexpr (Pat::template hye<a, k>()) tt = fma(blk->Hye[a][k], de[k], tt);
        });
        dAdt[a] = -tt * inv_h;
      });
#pragma unroll
      for (int a = 0; a < NY; ++a) {
        double tt = 0.0;
#pragma unroll
        for (int b = 0; b < NY; ++b) tt = fma(H[a][b], dAdt[b], tt);
        T[a] = tt;
        ad::For<0, NY>::run([&](auto bc) {
          constexpr int b = decltype(bc)::value;
          double jj = 0.0;
          ad::For<0, NY>::run([&](auto cc) {
            constexpr int c = decltype(cc)::value;
            if constexpr (Pat::template hyy<c, b>()) jj = fma(H[a][c], -blk->Hyy[c][b], jj);
          });
          J[a][b] = jj;
        });
#pragma unroll
        for (int b = 0; b < NY; ++b) H0[a][b] = H[a][b];
      }
      f3.setup(p, A);
    } else {
      double g[NY], hye[NY][6], hyy[NY][NY], sig_[6], Cee_[6][6], Cey_[6][NY];
      ode_blocks<Law, false>(p, et, s.y, g, hye, hyy, sig_, Cee_, Cey_);
#pragma unroll
      for (int a = 0; a < NY; ++a) A[a] = -g[a];
      force_a_aa<Law>(p, A, f, H);
#pragma unroll
      for (int a = 0; a < NY; ++a) {
#pragma unroll
        for (int b = 0; b < NY; ++b) dAdy[a][b] = -hyy[a][b];
        double tt = 0.0;
#pragma unroll
        for (int k = 0; k < 6; ++k) tt = fma(hye[a][k], de[k], tt);
        dAdt[a] = -tt * inv_h;
      }
#pragma unroll
      for (int a = 0; a < NY; ++a) {
        double tt = 0.0;
#pragma unroll
        for (int b = 0; b < NY; ++b) tt = fma(H[a][b], dAdt[b], tt);
        T[a] = tt;
#pragma unroll
        for (int b = 0; b < NY; ++b) {
          double jj = 0.0;
#pragma unroll
          for (int c = 0; c < NY; ++c) jj = fma(H[a][c], dAdy[c][b], jj);
          J[a][b] = jj;
        }
      }
    }
  }

  AD_HD void init(const LawParams<double>& p, const double (&e0)[6], const double (&e1)[6], const double (&zn)[NZ],
                  double h, const PsiBlocks<NY>* B = nullptr) {
    blk = B;
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
    ode_rhs<Law, TAN>(p, epsn, de, 0.0, s, F0, G0, blk);
    ode_stress<Law, TAN>(p, epsn, de, 0.0, s, sig_old, C_old, blk);
    refresh(p, 0.0, 1.0 / h);
    t = 0.0;
    dt = h;
    n_acc = n_rej = 0;
    flags = 0;
    last_rejected = false;
    done = false;
  }

  // J~_k w (column k of the tangent) into out.
  AD_HD void jtil(const LawParams<double>& p, const double (&dAk)[NY], const double (&w)[NY],
                  double (&out)[NY]) const {
    using Pat = PsiPattern<Law>;
    double v[NY];
    ad::For<0, NY>::run([&](auto ac) {
      constexpr int a = decltype(ac)::value;
      double tt = 0.0;
      ad::For<0, NY>::run([&](auto bc) {
        constexpr int b = decltype(bc)::value;
        if constexpr (Pat::template hyy<a, b>()) tt = fma(-blk->Hyy[a][b], w[b], tt);
      });
      v[a] = tt;
    });
    f3.apply(dAk, v, out);
  }

  AD_HD void attempt(const LawParams<double>& p, const Step& hs, const Ode23Ctl& ctl) {
    constexpr double d = 0.29289321881345247560;   // 1/(2 + sqrt 2)
    constexpr double e32 = 7.4142135623730950488;  // 6 + sqrt 2
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
    const double th0 = t * inv_h;
    const double hd = dt * d;
    StageLU<NY> W;
#pragma unroll
    for (int a = 0; a < NY; ++a)
#pragma unroll
      for (int b = 0; b < NY; ++b) W.w[a][b] = (a == b ? 1.0 : 0.0) - hd * J[a][b];
    W.factor();
    double rhs[NY], k1[NY], k2[NY], k3[NY], F1[NY], F2[NY];
    M56 G1, G2, K1, K2;
#pragma unroll
    for (int a = 0; a < NY; ++a) rhs[a] = fma(hd, T[a], F0[a]);
    W.solve(rhs, k1);
    OdeState<NY, TAN> st;
#pragma unroll
    for (int a = 0; a < NY; ++a) st.y[a] = fma(0.5 * dt, k1[a], s.y[a]);
    // tangent: the total dA/deps_k at the substep start, T~_k and k1~
    double dA[TAN ? 6 : 1][TAN ? NY : 1], Tt[TAN ? 6 : 1][TAN ? NY : 1];
    if constexpr (TAN) {
      // (columns one at a time: the tangent state lives in local memory anyway,
      // and unrolling the six columns multiplies the code and the compile time)
#pragma unroll 1
      for (int k = 0; k < 6; ++k) {
        ad::For<0, NY>::run([&](auto ac) {
          constexpr int a = decltype(ac)::value;
          double v = th0 * blk->Hye[a][k];
          ad::For<0, NY>::run([&](auto bc) {
            constexpr int b = decltype(bc)::value;
            if constexpr (PsiPattern<Law>::template hyy<a, b>()) v = fma(blk->Hyy[a][b], s.Y[b][k], v);
          });
          dA[k][a] = -v;
        });
        double dAt[NY];
        f3.apply(dA[k], dAdt, dAt);
        double jk[NY], r[NY], col[NY];
        jtil(p, dA[k], k1, jk);
#pragma unroll
        for (int a = 0; a < NY; ++a) {
          double hh = 0.0;
#pragma unroll
          for (int b = 0; b < NY; ++b) hh = fma(H0[a][b], blk->Hye[b][k], hh);
          Tt[k][a] = dAt[a] - hh * inv_h;
          r[a] = G0[a][k] + hd * Tt[k][a] + hd * jk[a];
        }
        W.solve(r, col);
#pragma unroll
        for (int a = 0; a < NY; ++a) {
          K1[a][k] = col[a];
          st.Y[a][k] = fma(0.5 * dt, col[a], s.Y[a][k]);
        }
      }
    }
    ode_rhs<Law, TAN>(p, epsn, de, (t + 0.5 * dt) * inv_h, st, F1, G1, blk);
    double w2[NY];
#pragma unroll
    for (int a = 0; a < NY; ++a) rhs[a] = F1[a] - k1[a];
    W.solve(rhs, w2);
    OdeState<NY, TAN> s3;
#pragma unroll
    for (int a = 0; a < NY; ++a) {
      k2[a] = w2[a] + k1[a];
      s3.y[a] = fma(dt, k2[a], s.y[a]);
    }
    if constexpr (TAN) {
      // (columns one at a time: the tangent state lives in local memory anyway,
      // and unrolling the six columns multiplies the code and the compile time)
#pragma unroll 1
      for (int k = 0; k < 6; ++k) {
        double dk[NY], jk[NY], r[NY], col[NY];
#pragma unroll
        for (int a = 0; a < NY; ++a) dk[a] = k2[a] - k1[a];
        jtil(p, dA[k], dk, jk);
#pragma unroll
        for (int a = 0; a < NY; ++a) r[a] = G1[a][k] - K1[a][k] + hd * jk[a];
        W.solve(r, col);
#pragma unroll
        for (int a = 0; a < NY; ++a) {
          K2[a][k] = K1[a][k] + col[a];
          s3.Y[a][k] = fma(dt, K2[a][k], s.Y[a][k]);
        }
      }
    }
    ode_rhs<Law, TAN>(p, epsn, de, th1, s3, F2, G2, blk);
#pragma unroll
    for (int a = 0; a < NY; ++a) rhs[a] = F2[a] - e32 * (k2[a] - F1[a]) - 2.0 * (k1[a] - F0[a]) + hd * T[a];
    W.solve(rhs, k3);
    OdeState<NY, TAN> s2;
    const double dt6 = dt * (1.0 / 6.0);
#pragma unroll
    for (int a = 0; a < NY; ++a) s2.y[a] = s3.y[a] - dt6 * (k1[a] - 2.0 * k2[a] + k3[a]);
    if constexpr (TAN) {
      // (columns one at a time: the tangent state lives in local memory anyway,
      // and unrolling the six columns multiplies the code and the compile time)
#pragma unroll 1
      for (int k = 0; k < 6; ++k) {
        double jk[NY], r[NY], col[NY];
        jtil(p, dA[k], k3, jk);
#pragma unroll
        for (int a = 0; a < NY; ++a)
          r[a] = G2[a][k] - e32 * (K2[a][k] - G1[a][k]) - 2.0 * (K1[a][k] - G0[a][k]) + hd * Tt[k][a] + hd * jk[a];
        W.solve(r, col);
#pragma unroll
        for (int a = 0; a < NY; ++a) s2.Y[a][k] = s3.Y[a][k] - dt6 * (K1[a][k] - 2.0 * K2[a][k] + col[a]);
      }
    }
    double s_hi[6], s_lo[6];
    M66 C_hi, C_lo;
    ode_stress<Law, TAN>(p, epsn, de, th1, s3, s_hi, C_hi, blk);
    ode_stress<Law, TAN>(p, epsn, de, th1, s2, s_lo, C_lo, blk);
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
    // a singular stage matrix or an overflow rejects the trial step
    const double err = W.ok && finite64(sum) ? sqrt(sum / m) : 1e300;
    const double facmax = last_rejected ? 1.0 : 5.0;
    const double f = err == 0.0 ? 1e300 : 0.9 * fpow::pow_pos(err, -1.0 / 3.0);
    const double grow = fmin(facmax, fmax(0.2, f));
    if (err <= 1.0) {
      t = tn1;
#pragma unroll
      for (int a = 0; a < NY; ++a) {
        s.y[a] = s3.y[a];
        F0[a] = F2[a];
        if constexpr (TAN)
#pragma unroll
          for (int c = 0; c < 6; ++c) {
            s.Y[a][c] = s3.Y[a][c];
            G0[a][c] = G2[a][c];
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
      else refresh(p, th1, inv_h);
    } else {
      ++n_rej;
      last_rejected = true;
    }
    dt *= grow;
  }

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

// The voxel state of integrator PAIR.
template <class Law, bool TAN, int PAIR>
using OdeVoxel = std::conditional_t<PAIR == ROS_23S, RosVoxel<Law, TAN>, ErkVoxel<Law, TAN, PAIR == ROS_23S ? 0 : PAIR>>;

// One voxel, start to end (single thread; the kernel schedules ErkVoxel
// states per lane itself).
template <class Law, bool TAN, int PAIR = ERK_BS23>
AD_HD unsigned voxel_ode23(const LawParams<double>& p, const double (&epsn)[6], const double (&eps1)[6],
                           const double (&zn)[stored_nz<Law>()], const Step& hs, const Ode23Ctl& ctl,
                           double (&sig)[6], double (&z)[stored_nz<Law>()], double* C36) {
  OdeVoxel<Law, TAN, PAIR> v;
  if constexpr (TAN) {
    PsiBlocks<Law::NY> B;
    psi_const_blocks<Law>(p, B);
    v.init(p, epsn, eps1, zn, hs.h, &B);
    while (!v.done) v.attempt(p, hs, ctl);
    return v.finish(hs.h, sig, z, C36);
  } else {
    v.init(p, epsn, eps1, zn, hs.h);
    while (!v.done) v.attempt(p, hs, ctl);
    return v.finish(hs.h, sig, z, C36);
  }
}

}  // namespace gsm
