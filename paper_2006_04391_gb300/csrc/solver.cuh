// Per-voxel implicit-Euler update of a GSM, driven entirely by AD of the two
// potentials (AutoMat, arXiv 2006.04391, Sec. 4.1 and Sec. 5).
//
// Unknowns y (NY = 5), increment w = y - y_n, rate v = w / h.  The implicit
// Euler step in dissipation form is the stationarity condition of the convex
// incremental potential Pi(y) = psi(eps, y) + h phi((y - y_n)/h):
//   R(y) = psi_y(eps, y) + phi_v(v) = 0,   K = psi_yy + phi_vv / h  (SPD).
// At y = y_n the dissipation Hessian is unbounded for power laws (n > 1), so
// the solve starts with
//   1. the psi-Newton predictor d = -psi_yy^-1 psi_y(eps, y_n),
//   2. exact minimisation of Pi on y_n + theta d, theta in (0, 1]: Newton on
//      g(theta) = d.R in the variable u = ln theta (for power-law dissipation
//      g(e^u) is convex and increasing, so Newton from u = 0 decreases
//      monotonically onto the root), safeguarded by the bracket [lo, hi];
//   3. full Newton on R with a warp-wide convergence vote.
// Any correct solver reaches the same y: Pi is strictly convex.
//
// Consistent tangent (Sec. 4.1, Eq. tangent_formula): with the converged
// Newton matrix K, dy/deps = -K^-1 psi_ye and C_t = psi_ee + psi_ey dy/deps;
// all second-order blocks come from one forward-over-reverse sweep.
#pragma once

#include "ad.cuh"
#include "laws.cuh"

namespace gsm {

// Status word per voxel.
enum : unsigned {
  ST_LINE_SHIFT = 0,     // bits 0-7: line-search iterations
  ST_NEWTON_SHIFT = 8,   // bits 8-15: Newton iterations (incl. FP64 corrections)
  ST_CONVERGED = 1u << 16,
  ST_NONFINITE = 1u << 17,
  ST_CAP = 1u << 18,
  ST_NOT_SPD = 1u << 19,
};

constexpr int kLineIterMax = 60;
constexpr int kNewtonIterMax = 12;

// ------------------------------------------------------------ small dense LA

AD_HD double fmax_(double a, double b) { return a > b ? a : b; }
AD_HD float fmax_(float a, float b) { return a > b ? a : b; }
AD_HD double sqrt_pos(double x) { return std::sqrt(x); }
AD_HD float sqrt_pos(float x) { return sqrtf(x); }


// In-place Cholesky of a 5x5 SPD matrix; keeps the inverse diagonal.
template <class T> struct Chol5 {
  T L[5][5];
  T dinv[5];
  AD_HD bool factor(const T (&A)[5][5]) {
    bool ok = true;
#pragma unroll
    for (int i = 0; i < 5; ++i) {
#pragma unroll
      for (int j = 0; j <= i; ++j) {
        T s = A[i][j];
#pragma unroll
        for (int k = 0; k < j; ++k) s -= L[i][k] * L[j][k];
        if (i == j) {
          ok = ok && (s > T(0));
          const T r = s > T(0) ? rsqrt_(s) : T(0);
          dinv[i] = r;
          L[i][i] = s * r;
        } else {
          L[i][j] = s * dinv[j];
        }
      }
    }
    return ok;
  }
  // x = A^-1 b
  AD_HD void solve(const T (&b)[5], T (&x)[5]) const {
    T t[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      T s = b[i];
#pragma unroll
      for (int k = 0; k < i; ++k) s -= L[i][k] * t[k];
      t[i] = s * dinv[i];
    }
#pragma unroll
    for (int i = 4; i >= 0; --i) {
      T s = t[i];
#pragma unroll
      for (int k = i + 1; k < 5; ++k) s -= L[k][i] * x[k];
      x[i] = s * dinv[i];
    }
  }
  static AD_HD double rsqrt_(double x) {
#if defined(__CUDA_ARCH__)
    return ::rsqrt(x);
#else
    return 1.0 / std::sqrt(x);
#endif
  }
  static AD_HD float rsqrt_(float x) {
#if defined(__CUDA_ARCH__)
    return ::rsqrtf(x);
#else
    return 1.0f / std::sqrt(x);
#endif
  }
};

// ---------------------------------------------------------- AD evaluations

// Passive strain pack.
template <class T> using EpsCst = ad::UniformPack<ad::Cst<T>, 6>;
template <class T> AD_HD void fill_cst(EpsCst<T>& p, const T (&e)[6]) {
  ad::For<0, 6>::run([&](auto kc) { ad::get_mut<decltype(kc)::value>(p).v = e[decltype(kc)::value]; });
}

// psi_y(eps, y): first-order reverse sweep.
template <class Law, class T>
AD_HD void psi_y(const LawParams<T>& p, const T (&eps)[6], const T (&y)[5], T (&g)[5]) {
  EpsCst<T> E;
  fill_cst(E, eps);
  ad::UniformPack<ad::Var<T>, 5> Y;
  ad::For<0, 5>::run([&](auto kc) { ad::get_mut<decltype(kc)::value>(Y).v = y[decltype(kc)::value]; });
  auto f = Law::psi(E, Y, p);
  f.fwd();
  f.back(T(1));
  ad::For<0, 5>::run([&](auto kc) { g[decltype(kc)::value] = ad::get<decltype(kc)::value>(Y).a; });
}

// phi_v(v): first-order reverse sweep.
template <class Law, class T>
AD_HD void phi_v(const LawParams<T>& p, const T (&v)[5], T (&g)[5]) {
  ad::UniformPack<ad::Var<T>, 5> V;
  ad::For<0, 5>::run([&](auto kc) { ad::get_mut<decltype(kc)::value>(V).v = v[decltype(kc)::value]; });
  auto f = Law::phi(V, p);
  f.fwd();
  f.back(T(1));
  ad::For<0, 5>::run([&](auto kc) { g[decltype(kc)::value] = ad::get<decltype(kc)::value>(V).a; });
}

// psi_y and psi_yy: forward-over-reverse with unit seeds (vector mode, 5 directions).
template <class Law, class T>
AD_HD void psi_y_yy(const LawParams<T>& p, const T (&eps)[6], const T (&y)[5], T (&g)[5], T (&H)[5][5]) {
  EpsCst<T> E;
  fill_cst(E, eps);
  ad::SeededPack<ad::Var, T, 5, 0, 5> Y;
  ad::seed_unit<decltype(Y), T, 0, 5>(Y, y);
  auto f = Law::psi(E, Y, p);
  f.fwd();
  f.back(T(1));
  ad::For<0, 5>::run([&](auto kc) {
    constexpr int k = decltype(kc)::value;
    const auto& a = ad::get<k>(Y).a;
    g[k] = a.v;
#pragma unroll
    for (int j = 0; j < 5; ++j) H[k][j] = a.d[j];
  });
}

// phi_v and phi_vv (vector mode).
template <class Law, class T>
AD_HD void phi_v_vv(const LawParams<T>& p, const T (&v)[5], T (&g)[5], T (&H)[5][5]) {
  ad::SeededPack<ad::Var, T, 5, 0, 5> V;
  ad::seed_unit<decltype(V), T, 0, 5>(V, v);
  auto f = Law::phi(V, p);
  f.fwd();
  f.back(T(1));
  ad::For<0, 5>::run([&](auto kc) {
    constexpr int k = decltype(kc)::value;
    const auto& a = ad::get<k>(V).a;
    g[k] = a.v;
#pragma unroll
    for (int j = 0; j < 5; ++j) H[k][j] = a.d[j];
  });
}

// Directional pass: R . d and d^T K d at y (Hessian-vector products).
template <class Law, class T>
AD_HD void line_eval(const LawParams<T>& p, const T (&eps)[6], const T (&y)[5], const T (&w)[5],
                     const T (&d)[5], T inv_h, T& g, T& gp) {
  using TT = ad::Tan<T, 1, 1u>;
  EpsCst<T> E;
  fill_cst(E, eps);
  ad::UniformPack<ad::Var<TT>, 5> Y, V;
  ad::For<0, 5>::run([&](auto kc) {
    constexpr int k = decltype(kc)::value;
    auto& ly = ad::get_mut<k>(Y);
    ly.v.v = y[k];
    ly.v.d[0] = d[k];
    auto& lv = ad::get_mut<k>(V);
    lv.v.v = w[k] * inv_h;
    lv.v.d[0] = d[k] * inv_h;
  });
  auto f = Law::psi(E, Y, p);
  f.fwd();
  f.back(T(1));
  auto q = Law::phi(V, p);
  q.fwd();
  q.back(T(1));
  T s0 = T(0), s1 = T(0);
  ad::For<0, 5>::run([&](auto kc) {
    constexpr int k = decltype(kc)::value;
    const auto& ay = ad::get<k>(Y).a;
    const auto& av = ad::get<k>(V).a;
    s0 += d[k] * (ay.v + av.v);
    s1 += d[k] * (ay.d[0] + av.d[0]);  // phi part already carries 1/h through the seed
  });
  g = s0;
  gp = s1;
}

// sigma = psi_eps(eps, y): reverse sweep with active strain leaves.
template <class Law, class T>
AD_HD void stress(const LawParams<T>& p, const T (&eps)[6], const T (&y)[5], T (&sig)[6]) {
  ad::UniformPack<ad::Var<T>, 6> E;
  ad::For<0, 6>::run([&](auto kc) { ad::get_mut<decltype(kc)::value>(E).v = eps[decltype(kc)::value]; });
  ad::UniformPack<ad::Cst<T>, 5> Y;
  ad::For<0, 5>::run([&](auto kc) { ad::get_mut<decltype(kc)::value>(Y).v = y[decltype(kc)::value]; });
  auto f = Law::psi(E, Y, p);
  f.fwd();
  f.back(T(1));
  ad::For<0, 6>::run([&](auto kc) { sig[decltype(kc)::value] = ad::get<decltype(kc)::value>(E).a; });
}

// All second-order blocks of psi at (eps, y): 11 unit directions (6 strain, 5 y).
template <class Law, class T>
AD_HD void psi_blocks(const LawParams<T>& p, const T (&eps)[6], const T (&y)[5], T (&sig)[6],
                      T (&Cee)[6][6], T (&Cey)[6][5], T (&Cye)[5][6]) {
  ad::SeededPack<ad::Var, T, 11, 0, 6> E;
  ad::SeededPack<ad::Var, T, 11, 6, 5> Y;
  ad::seed_unit<decltype(E), T, 0, 6>(E, eps);
  ad::seed_unit<decltype(Y), T, 6, 5>(Y, y);
  auto f = Law::psi(E, Y, p);
  f.fwd();
  f.back(T(1));
  ad::For<0, 6>::run([&](auto kc) {
    constexpr int i = decltype(kc)::value;
    const auto& a = ad::get<i>(E).a;
    sig[i] = a.v;
#pragma unroll
    for (int j = 0; j < 6; ++j) Cee[i][j] = a.d[j];
#pragma unroll
    for (int j = 0; j < 5; ++j) Cey[i][j] = a.d[6 + j];
  });
  ad::For<0, 5>::run([&](auto kc) {
    constexpr int i = decltype(kc)::value;
    const auto& a = ad::get<i>(Y).a;
#pragma unroll
    for (int j = 0; j < 6; ++j) Cye[i][j] = a.d[j];
  });
}

// ------------------------------------------------------------- warp voting

AD_HD bool all_done(bool done) {
#if defined(__CUDA_ARCH__)
  return __all_sync(0xffffffffu, done);
#else
  return done;
#endif
}

AD_HD double fp64_exp_step(double du) {
  // theta update factor e^du: far from the root an FP32 exponential is
  // accurate enough (the iterate only has to land in the bracket); near the
  // root a degree-4 Taylor polynomial keeps the Newton step FP64-accurate.
  if (du > -0.03 && du < 0.03) return 1.0 + du * (1.0 + du * (0.5 + du * (1.0 / 6.0 + du * (1.0 / 24.0))));
#if defined(__CUDA_ARCH__)
  return (double)__expf((float)du);
#else
  return std::exp(du);
#endif
}
AD_HD float fp64_exp_step(float du) {
#if defined(__CUDA_ARCH__)
  return __expf(du);
#else
  return std::exp(du);
#endif
}

template <class T> AD_HD T absmax5(const T (&a)[5]) {
  T m = T(0);
#pragma unroll
  for (int i = 0; i < 5; ++i) m = fmax_(m, a[i] < T(0) ? -a[i] : a[i]);
  return m;
}

// ----------------------------------------------------------------- the solve

// Solve the implicit Euler step in precision T for the increment w = y - y_n.
// Returns the Cholesky factor of the last Newton matrix in `ch` (for the
// tangent or for an FP64 correction).  `active` = false for padding lanes:
// they take part in the warp votes only.
template <class Law, class T>
AD_HD unsigned solve_increment(const LawParams<T>& p, const T (&eps)[6], const T (&yn)[5], T h,
                               bool active, T newton_tol, T (&w)[5], Chol5<T>& ch) {
  const T inv_h = T(1) / h;
  unsigned st = 0;
  int n_line = 0, n_newton = 0;
#pragma unroll
  for (int a = 0; a < 5; ++a) w[a] = T(0);

  // 1. predictor
  T r0[5];
  psi_y<Law>(p, eps, yn, r0);
  const T r0max = absmax5(r0);
  bool flows = active && (r0max > T(0));
  if (active && !(r0max == r0max)) { st |= ST_NONFINITE; flows = false; }
  T d[5];
  {
    T g0[5], Hp[5][5];
    psi_y_yy<Law>(p, eps, yn, g0, Hp);
    Chol5<T> hp;
    const bool ok = hp.factor(Hp);
    if (flows && !ok) { st |= ST_NOT_SPD; flows = false; }
    T mr[5];
#pragma unroll
    for (int a = 0; a < 5; ++a) mr[a] = -r0[a];
    hp.solve(mr, d);
  }

  // 2. segment minimisation in u = ln(theta)
  T theta = T(1), lo = T(0), hi = T(1);
  bool done = !flows;
  for (int it = 0; it < kLineIterMax; ++it) {
    if (all_done(done)) break;
    if (!done) {
      ++n_line;
      T y[5], wt[5];
#pragma unroll
      for (int a = 0; a < 5; ++a) {
        wt[a] = theta * d[a];
        y[a] = yn[a] + wt[a];
      }
      T g, gp;
      line_eval<Law>(p, eps, y, wt, d, inv_h, g, gp);
      if (g >= T(0)) hi = theta; else lo = theta;
      const T du = -g / (theta * gp);
      T tn = theta * fp64_exp_step(du);
      if (!(tn > lo && tn < hi)) tn = lo > T(0) ? sqrt_pos(lo * hi) : T(0.125) * hi;
      const bool small = (du < T(0) ? -du : du) <= T(sizeof(T) == 8 ? 1e-12 : 1e-6);
      theta = tn;
      if (small || g == T(0) || !(g == g)) done = true;
    }
  }
  if (flows) {
#pragma unroll
    for (int a = 0; a < 5; ++a) w[a] = theta * d[a];
  }

  // 3. Newton polish on the full system
  done = !flows;
  bool conv = !flows;
  for (int it = 0; it < kNewtonIterMax; ++it) {
    if (all_done(done)) break;
    if (!done) {
      ++n_newton;
      T y[5], v[5], R[5], K[5][5], gv[5], Hv[5][5];
#pragma unroll
      for (int a = 0; a < 5; ++a) {
        y[a] = yn[a] + w[a];
        v[a] = w[a] * inv_h;
      }
      psi_y_yy<Law>(p, eps, y, R, K);
      phi_v_vv<Law>(p, v, gv, Hv);
#pragma unroll
      for (int a = 0; a < 5; ++a) {
        R[a] = -(R[a] + gv[a]);
#pragma unroll
        for (int b = 0; b < 5; ++b) K[a][b] += Hv[a][b] * inv_h;
      }
      T dw[5];
      if (!ch.factor(K)) {
        st |= ST_NOT_SPD;
        done = true;
#pragma unroll
        for (int a = 0; a < 5; ++a) dw[a] = T(0);
      } else {
        ch.solve(R, dw);
      }
#pragma unroll
      for (int a = 0; a < 5; ++a) w[a] += dw[a];
      const T scale = fmax_(absmax5(w), T(sizeof(T) == 8 ? 1e-300 : 1e-30));
      if (absmax5(dw) <= newton_tol * scale) { conv = true; done = true; }
      if (!(absmax5(dw) == absmax5(dw))) { st |= ST_NONFINITE; done = true; }
    }
  }
  if (active && !conv && !(st & (ST_NOT_SPD | ST_NONFINITE))) st |= ST_CAP;
  if (conv) st |= ST_CONVERGED;
  st |= (unsigned)(n_line & 0xff) << ST_LINE_SHIFT;
  st |= (unsigned)(n_newton & 0xff) << ST_NEWTON_SHIFT;
  return st;
}

}  // namespace gsm
