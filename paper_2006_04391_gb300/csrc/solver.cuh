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

#include <cstring>

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
  ST_FIX_SHIFT = 20,     // bits 20-23: FP64 corrections (FP32-bulk mode)
  ST_MODEL_SHIFT = 24,   // bits 24-31: scalar iterations of the segment model (see solve_increment)
};

// Scalar model of the segment function g(theta) = d . R(y_n + theta d) after
// its value and slope at theta = 1 (g1 > 0, g1') are known: psi quadratic
// makes the psi part exactly -A (1 - theta) with A = -d . R(y_n) > 0, and a
// dissipation gradient homogeneous of degree p (a power law: p = 1/n) makes
// the rest B theta^p with B = g1, p = (g1' - A) / B.  The root of
//   f(u) = B e^(p u) - A (1 - e^u),  u = ln theta,
// by Newton from u = 0 (f convex and increasing: the iterates decrease
// monotonically onto the root), in FP32: the start of the segment search,
// which then needs one or two evaluations of g instead of about four.
// Returns theta in (0, 1) and the iteration count in `iters`.
AD_HD float segment_model_root(float A, float B, float pw, int& iters) {
  float u = 0.0f;
  iters = 0;
  for (int k = 0; k < 16; ++k) {
    ++iters;
#if defined(__CUDA_ARCH__)
    const float e1 = __expf(pw * u), e2 = __expf(u);
#else
    const float e1 = std::exp(pw * u), e2 = std::exp(u);
#endif
    const float f = B * e1 - A * (1.0f - e2);
    const float fp = pw * B * e1 + A * e2;
    const float du = -f / fp;
    u += du;
    if (!(du < 0.0f ? -du > 1e-7f : du > 1e-7f)) break;
  }
#if defined(__CUDA_ARCH__)
  return __expf(u);
#else
  return std::exp(u);
#endif
}

constexpr int kLineIterMax = 60;
constexpr int kNewtonIterMax = 12;

// ------------------------------------------------------------ small dense LA

AD_HD double fmax_(double a, double b) { return a > b ? a : b; }
AD_HD float fmax_(float a, float b) { return a > b ? a : b; }
AD_HD double sqrt_pos(double x) { return std::sqrt(x); }
AD_HD float sqrt_pos(float x) { return sqrtf(x); }


// Conversions between FP64 and FP32 on the integer pipe, with an optional
// exact scaling by 2^k folded into the exponent.  On GB300 an F2F conversion
// occupies the FP64 pipe (~1.7 FMA slots, measured), and the FP32-bulk update
// converts ~30 values per voxel; bit manipulation moves that work (and the
// scalings) to the integer units.  f32_of truncates (relative error < 2^-23)
// and flushes results below 2^-126 to zero; inf/nan map to inf/nan.  f64_of
// is exact for normal floats and zero (the FP32 values here are never
// subnormal) and flushes results below 2^-1022 to zero.
AD_HD float f32_of(double x, int k = 0) {
#if defined(__CUDA_ARCH__)
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
#else
  unsigned long long b;
  std::memcpy(&b, &x, sizeof b);
#endif
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const int e = (int)((b >> 52) & 0x7ff);
  const unsigned m = (unsigned)(b >> 29) & 0x7fffffu;
  const int fe = e - 1023 + 127 + k;
  unsigned r;
  if (e == 0x7ff) r = 0x7f800000u | (m ? 0x400000u : 0u);
  else if (e == 0 || fe <= 0) r = 0u;
  else if (fe >= 255) r = 0x7f800000u;
  else r = ((unsigned)fe << 23) | m;
  r |= sign;
#if defined(__CUDA_ARCH__)
  return __uint_as_float(r);
#else
  float f;
  std::memcpy(&f, &r, sizeof f);
  return f;
#endif
}

AD_HD double f64_of(float x, int k = 0) {
#if defined(__CUDA_ARCH__)
  const unsigned b = __float_as_uint(x);
#else
  unsigned b;
  std::memcpy(&b, &x, sizeof b);
#endif
  const unsigned long long sign = (unsigned long long)(b & 0x80000000u) << 32;
  const int e = (int)((b >> 23) & 0xff);
  const unsigned long long m = (unsigned long long)(b & 0x7fffffu) << 29;
  const int de = e - 127 + 1023 + k;
  unsigned long long r;
  if (e == 0xff) r = 0x7ff0000000000000ull | m;
  else if (e == 0 || de <= 0) r = 0ull;
  else if (de >= 2047) r = 0x7ff0000000000000ull;
  else r = ((unsigned long long)de << 52) | m;
  r |= sign;
#if defined(__CUDA_ARCH__)
  return __longlong_as_double((long long)r);
#else
  double d;
  std::memcpy(&d, &r, sizeof d);
  return d;
#endif
}

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

// psi_y and sigma = psi_eps in one first-order reverse sweep (strain and
// internal variables both active).
template <class Law, class T>
AD_HD void psi_y_and_stress(const LawParams<T>& p, const T (&eps)[6], const T (&y)[5], T (&g)[5], T (&sig)[6]) {
  ad::UniformPack<ad::Var<T>, 6> E;
  ad::For<0, 6>::run([&](auto kc) { ad::get_mut<decltype(kc)::value>(E).v = eps[decltype(kc)::value]; });
  ad::UniformPack<ad::Var<T>, 5> Y;
  ad::For<0, 5>::run([&](auto kc) { ad::get_mut<decltype(kc)::value>(Y).v = y[decltype(kc)::value]; });
  auto f = Law::psi(E, Y, p);
  f.fwd();
  f.back(T(1));
  ad::For<0, 6>::run([&](auto kc) { sig[decltype(kc)::value] = ad::get<decltype(kc)::value>(E).a; });
  ad::For<0, 5>::run([&](auto kc) { g[decltype(kc)::value] = ad::get<decltype(kc)::value>(Y).a; });
}

// Mixed block psi_ey (6x5): the change of sigma per change of y.
// Forward-over-reverse with unit seeds on y; the strain leaves carry no tangent.
template <class Law, class T>
AD_HD void psi_ey(const LawParams<T>& p, const T (&eps)[6], const T (&y)[5], T (&B)[6][5]) {
  using V0 = ad::Tan<T, 5, 0u>;
  ad::UniformPack<ad::Var<V0>, 6> E;
  ad::For<0, 6>::run([&](auto kc) {
    auto& l = ad::get_mut<decltype(kc)::value>(E);
    l.v.v = eps[decltype(kc)::value];
#pragma unroll
    for (int j = 0; j < 5; ++j) l.v.d[j] = T(0);
  });
  ad::SeededPack<ad::Var, T, 5, 0, 5> Y;
  ad::seed_unit<decltype(Y), T, 0, 5>(Y, y);
  auto f = Law::psi(E, Y, p);
  f.fwd();
  f.back(T(1));
  ad::For<0, 6>::run([&](auto kc) {
    constexpr int i = decltype(kc)::value;
#pragma unroll
    for (int j = 0; j < 5; ++j) B[i][j] = ad::get<i>(E).a.d[j];
  });
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

AD_HD bool any_lane(bool b) {
#if defined(__CUDA_ARCH__)
  return __any_sync(0xffffffffu, b);
#else
  return b;
#endif
}

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

// Time step and its reciprocal in both precisions, formed once per launch
// (a per-voxel FP64 division costs ~10 FP64-pipe slots).
struct Step {
  double h, inv_h;
  float hf, inv_hf;
};
AD_HD Step make_step(double h) { return Step{h, 1.0 / h, (float)h, (float)(1.0 / h)}; }
AD_HD void step_of(const Step& s, double& h, double& inv_h) { h = s.h; inv_h = s.inv_h; }
AD_HD void step_of(const Step& s, float& h, float& inv_h) { h = s.hf; inv_h = s.inv_hf; }

// FP64 finiteness from the exponent bits (integer pipe; an FP64 compare
// occupies the FP64 pipe).
AD_HD bool finite64(double x) {
#if defined(__CUDA_ARCH__)
  const unsigned hi = (unsigned)__double2hiint(x);
#else
  unsigned long long b;
  std::memcpy(&b, &x, sizeof b);
  const unsigned hi = (unsigned)(b >> 32);
#endif
  return (hi & 0x7ff00000u) != 0x7ff00000u;
}
AD_HD bool finite64(float x) { return std::isfinite(x); }

// 1/x for a positive normal FP64 x: Newton-Raphson reciprocal iteration
// r <- r (2 - x r) from an FP32 seed (two steps square the seed's 2^-22
// relative error twice; one more rounding), without the FP64 division
// sequence.  For scale factors, where a last-ulp difference is immaterial.
AD_HD double recip_pos(double x) {
#if defined(__CUDA_ARCH__)
  const int k = ((int)(((unsigned)__double2hiint(x) >> 20) & 0x7ffu)) - 1023;  // x = 2^k m, m in [1, 2)
  const float mf = f32_of(x, -k);
  double r = f64_of(__frcp_rn(mf), -k);
  double e = fma(-x, r, 1.0);
  r = fma(r, e, r);
  e = fma(-x, r, 1.0);
  return fma(r, e, r);
#else
  return 1.0 / x;
#endif
}

// Exact powers of two from the bit patterns (k in the normal range).
AD_HD float exp2i(int k, float) {
  const unsigned b = (unsigned)(k + 127) << 23;
#if defined(__CUDA_ARCH__)
  return __uint_as_float(b);
#else
  float f;
  std::memcpy(&f, &b, sizeof f);
  return f;
#endif
}
// floor(log2 max_i |a_i|) from the exponent fields (integer pipe); the
// smallest normal exponent when every entry is zero or subnormal.
AD_HD int ilog2_max(const double (&a)[6]) {
  int e = 0;
#pragma unroll
  for (int i = 0; i < 6; ++i) {
#if defined(__CUDA_ARCH__)
    const int ei = (int)(((unsigned)__double2hiint(a[i]) >> 20) & 0x7ffu);
#else
    unsigned long long b;
    std::memcpy(&b, &a[i], sizeof b);
    const int ei = (int)((b >> 52) & 0x7ff);
#endif
    e = ei > e ? ei : e;
  }
  return e == 0 ? -1022 : e - 1023;
}
AD_HD int ilog2_max(const float (&a)[6]) {
  int e = 0;
#pragma unroll
  for (int i = 0; i < 6; ++i) {
#if defined(__CUDA_ARCH__)
    const int ei = (int)((__float_as_uint(a[i]) >> 23) & 0xffu);
#else
    unsigned b;
    std::memcpy(&b, &a[i], sizeof b);
    const int ei = (int)((b >> 23) & 0xff);
#endif
    e = ei > e ? ei : e;
  }
  return e == 0 ? -126 : e - 127;
}

template <class T> AD_HD T absmax6(const T (&a)[6]) {
  T m = T(0);
#pragma unroll
  for (int i = 0; i < 6; ++i) m = fmax_(m, a[i] < T(0) ? -a[i] : a[i]);
  return m;
}

// One Newton step on R(w) = psi_y(e_s, w) + phi_v(w/h) = 0: w += dw with
// K dw = -R; the factor of K stays in `ch`.  Returns dw's largest entry, or
// -1 if K is not positive definite (w unchanged), +inf if dw is not finite.
template <class Law, class T>
AD_HD T newton_step(const LawParams<T>& p, const T (&es)[6], T inv_h, T (&w)[5], Chol5<T>& ch) {
  T v[5], R[5], K[5][5], gv[5], Hv[5][5];
#pragma unroll
  for (int a = 0; a < 5; ++a) v[a] = w[a] * inv_h;
  psi_y_yy<Law>(p, es, w, R, K);
  phi_v_vv<Law>(p, v, gv, Hv);
#pragma unroll
  for (int a = 0; a < 5; ++a) {
    R[a] = -(R[a] + gv[a]);
#pragma unroll
    for (int b = 0; b < 5; ++b) K[a][b] += Hv[a][b] * inv_h;
  }
  T dw[5];
  const bool spd = ch.factor(K);
  ch.solve(R, dw);
  if (!spd) return T(-1);
  const T dmax = absmax5(dw);
  if (!(dmax < T(sizeof(T) == 8 ? 1e300 : 1e37))) return T(INFINITY);
#pragma unroll
  for (int a = 0; a < 5; ++a) w[a] += dw[a];
  return dmax;
}

constexpr int kWarmIterMax = 4;

// Solve the implicit Euler step in precision T for the increment w, posed
// on the trial strain e_s (Law::trial_strain): R(w) = psi_y(e_s, w) +
// phi_v(w / h) = 0.  Returns the Cholesky factor of the last Newton matrix
// in `ch` (for the tangent or for an FP64 correction).  `active` = false for
// padding lanes: they take part in the warp votes only.
//
// Warm start (w0 != NULL, the basic scheme's later evaluations of a load
// step): Newton from w0, the previous evaluation's increment of the same
// voxel, which the scheme's strain update has moved only a little.  A lane
// whose warm Newton has not converged after kWarmIterMax steps, or meets a
// non-SPD or non-finite step, or starts from w0 = 0, takes the cold path
// (predictor, segment minimisation, Newton).  Pi is strictly convex, so both
// paths reach the same root.
//
// Rates below 1e-140 (FP64) or 1e-18 (FP32) of |d| / h, d the predictor,
// are not resolved (this keeps the dissipation's q = |v|^2 from
// underflowing), nor in FP32 roots where the dissipation Hessian overflows:
// the flow is then taken as zero.  Both happen only where the dissipation
// outweighs psi by many orders, i.e. for flows far below the resolution of
// the trial strain.
template <class Law, class T>
AD_HD unsigned solve_increment(const LawParams<T>& p, const T (&es)[6], const Step& hs, bool active, T newton_tol,
                               T (&w)[5], Chol5<T>& ch, const T* w0 = nullptr) {
  T h, inv_h;
  step_of(hs, h, inv_h);
  unsigned st = 0;
  int n_line = 0, n_newton = 0;
  bool warm = false;
  if (w0) {
    T wt[5];
#pragma unroll
    for (int a = 0; a < 5; ++a) wt[a] = w0[a];
    bool wdone = !(active && absmax5(wt) > T(0));
    for (int it = 0; it < kWarmIterMax; ++it) {
      if (all_done(wdone)) break;
      if (!wdone) {
        ++n_newton;
        const T dmax = newton_step<Law, T>(p, es, inv_h, wt, ch);
        if (!(dmax >= T(0) && dmax < T(INFINITY))) {
          wdone = true;  // not SPD or not finite: the cold path decides
        } else if (dmax <= newton_tol * fmax_(absmax5(wt), T(sizeof(T) == 8 ? 1e-300 : 1e-30))) {
          warm = true;
          wdone = true;
        }
      }
    }
    if (warm) {
#pragma unroll
      for (int a = 0; a < 5; ++a) w[a] = wt[a];
      st |= ST_CONVERGED;
    } else {
      n_newton = 0;
    }
  }
  const bool cold = active && !warm;
  if (!warm) {
#pragma unroll
    for (int a = 0; a < 5; ++a) w[a] = T(0);
  }
  if (all_done(!cold)) {  // every lane of the warp converged warm (or pads)
    if (!active) st |= ST_CONVERGED;
    st |= (unsigned)(n_newton & 0xff) << ST_NEWTON_SHIFT;
    return st;
  }

  // 1. predictor at w = 0.  In the trial frame psi_y(e_s, 0) vanishes only
  // for a zero deviatoric trial stress: then there is no flow.
  T d[5];
  bool flows;
  T A = T(0);  // -d . R(y_n): the segment function's value at theta = 0 is -A
  {
    T r0[5], Hp[5][5];
    const T zero[5] = {T(0), T(0), T(0), T(0), T(0)};
    psi_y_yy<Law>(p, es, zero, r0, Hp);
    const T r0max = absmax5(r0);
    flows = cold && r0max > T(0);
    if (cold && !(r0max == r0max)) { st |= ST_NONFINITE; flows = false; }
    Chol5<T> hp;
    const bool ok = hp.factor(Hp);
    if (flows && !ok) { st |= ST_NOT_SPD; flows = false; }
    T mr[5];
#pragma unroll
    for (int a = 0; a < 5; ++a) mr[a] = -r0[a];
    hp.solve(mr, d);
#pragma unroll
    for (int a = 0; a < 5; ++a) A += d[a] * mr[a];
  }
  int n_model = 0;
  const T th_min = T(sizeof(T) == 8 ? 1e-140 : 1e-18) * h / fmax_(absmax5(d), T(sizeof(T) == 8 ? 1e-300 : 1e-37));
  if (!(th_min < T(1))) flows = false;

  // 2. segment minimisation in u = ln(theta)
  T theta = T(1), lo = T(0), hi = T(1);
  bool done = !flows, below = false;
  for (int it = 0; it < kLineIterMax; ++it) {
    if (all_done(done)) break;
    if (!done) {
      ++n_line;
      T wt[5];
#pragma unroll
      for (int a = 0; a < 5; ++a) wt[a] = theta * d[a];
      T g, gp;
      line_eval<Law>(p, es, wt, wt, d, inv_h, g, gp);
      if (g >= T(0)) hi = theta; else lo = theta;
      // g' = d^T K d > 0; where the dissipation Hessian leaves the range of T
      // (FP32, rates near the floor) the step bisects instead, and a root
      // below such a point is not resolved
      const bool fin = gp > T(0) && gp < T(sizeof(T) == 8 ? 1e300 : 1e37);
      const T du = fin ? -g * ad::inv(theta * gp) : T(0);
      const bool small = fin && (du < T(0) ? -du : du) <= T(sizeof(T) == 8 ? 1e-12 : 1e-6);
      T tn = theta * fp64_exp_step(du);
      if (it == 0 && fin && !small && g > T(0) && gp > A && A > T(0)) {
        // after the evaluation at theta = 1: start from the root of the
        // segment model (a rounding of the model stays inside the bracket)
        const float pw = (float)((gp - A) / g);
        const float tm = segment_model_root((float)A, (float)g, pw, n_model);
        if (tm > 0.0f && tm < 1.0f) {
          tn = T(tm);
          if constexpr (sizeof(T) == 8) {
            // one FP64 Newton step of the model (table power), so that the
            // next evaluation of g already meets the FP64 step tolerance
            const T pwd = (gp - A) / g;
            const T e1 = fpow::pow_pos(tn, pwd);
            const T f = g * e1 - A * (T(1) - tn);
            const T fd = pwd * g * e1 + A * tn;
            const T tr = tn * fp64_exp_step(-f / fd);
            if (tr > T(0) && tr < T(1)) tn = tr;
          }
        }
      }
      // safeguard only steps that leave the bracket; a converged step may
      // round onto a bracket end and is kept
      if (!small && !(tn > lo && tn < hi)) tn = lo > T(0) ? sqrt_pos(lo * hi) : T(0.125) * hi;
      if (tn < th_min) tn = th_min;
      below = !(hi > th_min) || (!fin && g >= T(0));
      theta = tn;
      if (small || below || g == T(0) || !(g == g)) done = true;
    }
  }
  if (below || !(theta > T(0))) flows = false;
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
      const T dmax = newton_step<Law, T>(p, es, inv_h, w, ch);
      if (dmax < T(0)) {
        st |= ST_NOT_SPD;
        done = true;
      } else if (!(dmax < T(INFINITY))) {
        st |= ST_NONFINITE;  // w keeps the last finite iterate
        done = true;
      } else if (dmax <= newton_tol * fmax_(absmax5(w), T(sizeof(T) == 8 ? 1e-300 : 1e-30))) {
        conv = true;
        done = true;
      }
    }
  }
  if (active && !conv && !(st & (ST_NOT_SPD | ST_NONFINITE))) st |= ST_CAP;
  if (conv) st |= ST_CONVERGED;
  st |= (unsigned)(n_line & 0xff) << ST_LINE_SHIFT;
  st |= (unsigned)(n_newton & 0xff) << ST_NEWTON_SHIFT;
  st |= (unsigned)(n_model & 0xff) << ST_MODEL_SHIFT;
  return st;
}

}  // namespace gsm
