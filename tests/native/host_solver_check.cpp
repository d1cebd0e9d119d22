// Test-only host build of the device headers (AD, potentials, per-voxel
// solver), so the CPU suite can check the AD derivatives and the solve
// logic without a GPU.  Never part of the product library.
#include <cstdint>

#include "../../paper_2006_04391_gb300/csrc/common.cuh"
#include "../../paper_2006_04391_gb300/csrc/voxel.cuh"
#include "../../paper_2006_04391_gb300/csrc/ode23.cuh"
#include "../../paper_2006_04391_gb300/csrc/dpow.cuh"

using namespace gsm;

// ode23 update, kind 1 (Norton, params E, nu, sigma0, edot0, n) or 2
// (Michel-Suquet, params E, nu, sigma_Y, H, edot0, sigma_d, n); AoS eps_n,
// eps [n][6], z_n and z [n][nz] (nz = 6 or 7); tangent [n][36] or NULL.
template <class Law, int PAIR>
void run_ode23(const LawParams<double>& p, int64_t n, const double* eps_n, const double* eps, const double* zn,
               const Step& hs, const Ode23Ctl& ctl, double* sig, double* z, double* tan, int32_t* status) {
  constexpr int NZ = stored_nz<Law>();
  for (int64_t i = 0; i < n; ++i) {
    double e0[6], e1[6], zi[NZ], s[6], zo[NZ];
    for (int c = 0; c < 6; ++c) {
      e0[c] = eps_n[6 * i + c];
      e1[c] = eps[6 * i + c];
    }
    for (int c = 0; c < NZ; ++c) zi[c] = zn[NZ * i + c];
    unsigned st = tan ? voxel_ode23<Law, true, PAIR>(p, e0, e1, zi, hs, ctl, s, zo, tan + 36 * i)
                      : voxel_ode23<Law, false, PAIR>(p, e0, e1, zi, hs, ctl, s, zo, nullptr);
    for (int c = 0; c < 6; ++c) sig[6 * i + c] = s[c];
    for (int c = 0; c < NZ; ++c) z[NZ * i + c] = zo[c];
    status[i] = (int32_t)st;
  }
}

// psi's second-derivative blocks by one forward-over-reverse sweep at (eps, y)
// and at the origin (psi_const_blocks), and their structural pattern
// (PsiPattern): out = [Hye (NY x 6), Hyy (NY x NY), Cee (6 x 6), Cey (6 x NY)]
// twice (at the point, at the origin); rows[r] = pattern row r (leaves
// eps_0..5, then y_0..NY-1).
template <class Law>
void const_blocks_check(const LawParams<double>& p, const double* eps, const double* y, double* out, uint32_t* rows) {
  constexpr int NY = Law::NY;
  double e[6], yy[NY], g[NY], sig[6];
  for (int i = 0; i < 6; ++i) e[i] = eps[i];
  for (int a = 0; a < NY; ++a) yy[a] = y[a];
  PsiBlocks<NY> B, B0;
  ode_blocks<Law, true>(p, e, yy, g, B.Hye, B.Hyy, sig, B.Cee, B.Cey);
  psi_const_blocks<Law>(p, B0);
  const int m = NY * 6 + NY * NY + 36 + 6 * NY;
  const PsiBlocks<NY>* src[2] = {&B, &B0};
  for (int q = 0; q < 2; ++q) {
    double* o = out + q * m;
    for (int a = 0; a < NY; ++a)
      for (int k = 0; k < 6; ++k) *o++ = src[q]->Hye[a][k];
    for (int a = 0; a < NY; ++a)
      for (int b = 0; b < NY; ++b) *o++ = src[q]->Hyy[a][b];
    for (int i = 0; i < 6; ++i)
      for (int k = 0; k < 6; ++k) *o++ = src[q]->Cee[i][k];
    for (int i = 0; i < 6; ++i)
      for (int a = 0; a < NY; ++a) *o++ = src[q]->Cey[i][a];
  }
  ad::For<0, 6 + NY>::run([&](auto rc) {
    rows[decltype(rc)::value] = PsiPattern<Law>::template row<decltype(rc)::value>();
  });
}

extern "C" {

// params = {E, nu, sigma0, edot0, n}; fields AoS [n][6]; tangent [n][21] or NULL.
int host_update(int mode, const double* prm, int64_t n, const double* eps, const double* zn, double h,
                double* sig, double* z, double* tan, int32_t* status) {
  const LawParams<double> p = make_params(prm, 1);
  const LawParams<float> pf = to_float(p);
  for (int64_t i = 0; i < n; ++i) {
    double e[6], zi[6], s[6], zo[6];
    for (int c = 0; c < 6; ++c) { e[c] = eps[6 * i + c]; zi[c] = zn[6 * i + c]; }
    unsigned st;
    if (mode == 0) {
      st = voxel_fp64<NortonDev>(p, e, zi, make_step(h), true, s, zo, tan ? tan + 21 * i : nullptr);
    } else {
      st = voxel_fp32_fix<NortonDev>(p, pf, e, zi, make_step(h), true, s, zo, tan ? tan + 21 * i : nullptr);
    }
    for (int c = 0; c < 6; ++c) { sig[6 * i + c] = s[c]; z[6 * i + c] = zo[c]; }
    status[i] = (int32_t)st;
  }
  return 0;
}

int host_update_ode23(int kind, const double* prm, int64_t n, const double* eps_n, const double* eps,
                      const double* zn, double h, double rtol, double atol, int max_steps, double* sig, double* z,
                      double* tan, int32_t* status) {
  const LawParams<double> p = make_params(prm, kind);
  const Step hs = make_step(h);
  const Ode23Ctl ctl{rtol, atol, max_steps};
  if (kind == 1) run_ode23<NortonDev, ERK_BS23>(p, n, eps_n, eps, zn, hs, ctl, sig, z, tan, status);
  else run_ode23<MichelSuquet, ERK_BS23>(p, n, eps_n, eps, zn, hs, ctl, sig, z, tan, status);
  return 0;
}

// The same with the ode23s (Rosenbrock) triple.
int host_update_ode23s(int kind, const double* prm, int64_t n, const double* eps_n, const double* eps,
                       const double* zn, double h, double rtol, double atol, int max_steps, double* sig, double* z,
                       double* tan, int32_t* status) {
  const LawParams<double> p = make_params(prm, kind);
  const Step hs = make_step(h);
  const Ode23Ctl ctl{rtol, atol, max_steps};
  if (kind == 1) run_ode23<NortonDev, ROS_23S>(p, n, eps_n, eps, zn, hs, ctl, sig, z, tan, status);
  else run_ode23<MichelSuquet, ROS_23S>(p, n, eps_n, eps, zn, hs, ctl, sig, z, tan, status);
  return 0;
}

// W x = b by the register LU of the Rosenbrock stages (n = 5 or 6, W row-major).
int host_stage_solve(int n, const double* W, const double* b, double* x) {
  auto run = [&](auto tag) {
    constexpr int N = decltype(tag)::value;
    StageLU<N> lu;
    for (int i = 0; i < N; ++i)
      for (int j = 0; j < N; ++j) lu.w[i][j] = W[i * N + j];
    lu.factor();
    double bb[N], xx[N];
    for (int i = 0; i < N; ++i) bb[i] = b[i];
    lu.solve(bb, xx);
    for (int i = 0; i < N; ++i) x[i] = xx[i];
    return lu.ok ? 0 : -1;
  };
  if (n == 5) return run(std::integral_constant<int, 5>{});
  return run(std::integral_constant<int, 6>{});
}

// Psi_AAA[u, v] of the hand partial used by the ode23s tangent.
void host_force_aaa(int kind, const double* prm, const double* A, const double* u, const double* v, double* out) {
  const LawParams<double> p = make_params(prm, kind);
  if (kind == 1) {
    double a[5], uu[5], vv[5], o[5];
    for (int i = 0; i < 5; ++i) { a[i] = A[i]; uu[i] = u[i]; vv[i] = v[i]; }
    force_aaa<NortonDev>(p, a, uu, vv, o);
    for (int i = 0; i < 5; ++i) out[i] = o[i];
  } else {
    double a[6], uu[6], vv[6], o[6];
    for (int i = 0; i < 6; ++i) { a[i] = A[i]; uu[i] = u[i]; vv[i] = v[i]; }
    force_aaa<MichelSuquet>(p, a, uu, vv, o);
    for (int i = 0; i < 6; ++i) out[i] = o[i];
  }
}

// The same with the ode12 (explicit Euler / Heun) pair.
int host_update_ode12(int kind, const double* prm, int64_t n, const double* eps_n, const double* eps,
                      const double* zn, double h, double rtol, double atol, int max_steps, double* sig, double* z,
                      double* tan, int32_t* status) {
  const LawParams<double> p = make_params(prm, kind);
  const Step hs = make_step(h);
  const Ode23Ctl ctl{rtol, atol, max_steps};
  if (kind == 1) run_ode23<NortonDev, ERK_HEUN12>(p, n, eps_n, eps, zn, hs, ctl, sig, z, tan, status);
  else run_ode23<MichelSuquet, ERK_HEUN12>(p, n, eps_n, eps, zn, hs, ctl, sig, z, tan, status);
  return 0;
}

// AD derivatives of the shipped potentials at one point.
void host_psi_derivs(const double* prm, const double* eps, const double* y, double* g, double* H) {
  const LawParams<double> p = make_params(prm, 1);
  double e[6], yy[5], gg[5], HH[5][5];
  for (int c = 0; c < 6; ++c) e[c] = eps[c];
  for (int a = 0; a < 5; ++a) yy[a] = y[a];
  psi_y_yy<NortonDev>(p, e, yy, gg, HH);
  for (int a = 0; a < 5; ++a) { g[a] = gg[a]; for (int b = 0; b < 5; ++b) H[5 * a + b] = HH[a][b]; }
}

void host_phi_derivs(const double* prm, const double* v, double* g, double* H) {
  const LawParams<double> p = make_params(prm, 1);
  double vv[5], gg[5], HH[5][5];
  for (int a = 0; a < 5; ++a) vv[a] = v[a];
  phi_v_vv<NortonDev>(p, vv, gg, HH);
  for (int a = 0; a < 5; ++a) { g[a] = gg[a]; for (int b = 0; b < 5; ++b) H[5 * a + b] = HH[a][b]; }
}

void host_psi_blocks(const double* prm, const double* eps, const double* y, double* sig, double* Cee,
                     double* Cey) {
  const LawParams<double> p = make_params(prm, 1);
  double e[6], yy[5], s[6], A[6][6], B[6][5], Ct[5][6];
  for (int c = 0; c < 6; ++c) e[c] = eps[c];
  for (int a = 0; a < 5; ++a) yy[a] = y[a];
  psi_blocks<NortonDev>(p, e, yy, s, A, B, Ct);
  for (int i = 0; i < 6; ++i) {
    sig[i] = s[i];
    for (int j = 0; j < 6; ++j) Cee[6 * i + j] = A[i][j];
    for (int j = 0; j < 5; ++j) Cey[5 * i + j] = B[i][j];
  }
}

// kind 1 Norton (NY = 5), 2 Michel-Suquet (NY = 6); see const_blocks_check.
int host_const_blocks(int kind, const double* prm, const double* eps, const double* y, double* out, uint32_t* rows) {
  const LawParams<double> p = make_params(prm, kind);
  if (kind == 1) const_blocks_check<NortonDev>(p, eps, y, out, rows);
  else const_blocks_check<MichelSuquet>(p, eps, y, out, rows);
  return 0;
}

// Polynomial degree of psi read off its expression type (kind 1 Norton, 2 Michel-Suquet).
int host_psi_degree(int kind) {
  return kind == 1 ? ad::Degree<PsiPattern<NortonDev>::Expr>::value : ad::Degree<PsiPattern<MichelSuquet>::Expr>::value;
}

// The double-float power of the correction: F = ac (x 2^e)^a with x, a, ac
// given as doubles and rounded to pairs here; out = {x.hi, x.lo, F.hi, F.lo}
// (x the pair actually used).  Returns 1 on the fast path, 0 where the
// caller would take the FP64 power.
int host_dpow(double x, int e, double a, double ac, float* out) {
  const df xd = df_of(x), ad = df_of(a);
  const int ace = (int)((fpow::bits_of(ac) >> 52) & 0x7ff) - 1023;
  const df acm = df_of(ac, -ace);
  df F{0.0f, 0.0f};
  const bool ok = dpow::pow_scaled(xd, e, a, ad, acm, ace, F);
  out[0] = xd.hi;
  out[1] = xd.lo;
  out[2] = F.hi;
  out[3] = F.lo;
  return ok ? 1 : 0;
}

}  // extern "C"
