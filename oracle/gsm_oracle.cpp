// FP64 CPU oracle for the implicit-Euler update of a generalized standard
// material (GSM) -- TEST INFRASTRUCTURE ONLY.
//
// Only the test suite, the smoke check and the CPU-baseline leg of the
// benchmark may load this library.  It shares no code with the CUDA path: all
// derivatives below are derived by hand (no automatic differentiation), the
// linear algebra is written out, and the data layout is array-of-structs.
//
// What it computes (paper: AutoMat, Bluehdorn/Gauger/Kabel, arXiv 2006.04391):
//   * Sec. 2, Eq. (gsm_sigma): sigma = d psi / d eps.
//   * Sec. 4.1, Eq. (implicit_euler): one implicit Euler step for the internal
//     variables, solved by Newton.  We use the dissipation (dual) form of the
//     evolution law, d psi/dz (eps, z) + d phi/dzdot ((z - z_n)/h) = 0, which
//     for a convex dual pair (Psi = phi*) has the same solution as the force-
//     potential form of Eq. (gsm_internal).  Sec. 2 states that the dual
//     potential exists but is not used in the paper; the Norton phi below is
//     the exact dual of the paper's Psi of Eq. (michel_suquet_psi) with
//     sigma_Y = 0 and H = 0.
//   * Sec. 4.1, Eq. (tangent_formula): consistent tangent by the implicit
//     function theorem, C_t = psi_ee + psi_ey dy/deps, K dy/deps = -psi_ye.
//   * Sec. 4 (conventional strategy, Simo-Hughes radial return): an
//     independent scalar reduction used only as a pin of the generic solver.
//
// Conventions (Sec. 3 uses Voigt notation; H = diag(H,H,H,H/2,H/2,H/2) in
// Eq. (michel_suquet_omega) fixes engineering shears for strain vectors):
//   strain-like  (e11, e22, e33, g23, g13, g12), g_ij = 2 e_ij
//   stress-like  (s11, s22, s33, s23, s13, s12)
//   internal variable z = eps_vp, deviatoric (Sec. 6: one component is
//   eliminated), unknowns y = (z11, z22, g23, g13, g12), z33 = -z11 - z22,
//   i.e. z = P y with the 6x5 matrix P below.
//
// Parity with the paper's own numbers is unpinned: the paper prints no field
// values for a reproducible case.  Every function here is pinned in the tests
// against closed forms, finite differences, invariants and an independent
// radial return (see tests/test_oracle_material.py).

#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

// ---------------------------------------------------------------- constants

// z = P y: deviatoric viscoplastic strain from its 5 independent components.
const double P[6][5] = {
    {1, 0, 0, 0, 0},
    {0, 1, 0, 0, 0},
    {-1, -1, 0, 0, 0},
    {0, 0, 1, 0, 0},
    {0, 0, 0, 1, 0},
    {0, 0, 0, 0, 1},
};

// Equivalent strain rate |v|_eq^2 = (2/3) zdot:zdot written on the Voigt
// vector with engineering shears: weights 2/3 on normal, 1/3 on shear entries.
const double W[6] = {2.0 / 3.0, 2.0 / 3.0, 2.0 / 3.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 3.0};

struct Law {
  int kind;         // 0 = linear elastic, 1 = elastic + deviatoric Norton viscoplastic,
                    // 2 = Michel-Suquet (kinematic hardening H, yield sigma_Y; force-potential form)
  double lam, mu;   // Lame constants from (E, nu)
  double sigma0;    // drag stress (sigma_d for kind 2)
  double edot0;     // reference strain rate
  double n;         // rate sensitivity exponent
  double sigY;      // kind 2: yield stress (K(alpha) = sigma_Y)
  double Hkin;      // kind 2: kinematic hardening modulus H
  double C[6][6];   // isotropic stiffness in Voigt notation
  double G[5][5];   // P^T diag(W) P
};

void make_law(int kind, const double* prm, Law* L) {
  const double E = prm[0], nu = prm[1];
  L->kind = kind;
  L->lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  L->mu = E / (2.0 * (1.0 + nu));
  // kind 1: (E, nu, sigma0, edot0, n); kind 2: (E, nu, sigma_Y, H, edot0, sigma_d, n)
  L->sigma0 = kind == 1 ? prm[2] : kind == 2 ? prm[5] : 0.0;
  L->edot0 = kind == 1 ? prm[3] : kind == 2 ? prm[4] : 1.0;
  L->n = kind == 1 ? prm[4] : kind == 2 ? prm[6] : 1.0;
  L->sigY = kind == 2 ? prm[2] : 0.0;
  L->Hkin = kind == 2 ? prm[3] : 0.0;
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) L->C[i][j] = 0.0;
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j) L->C[i][j] = L->lam;
    L->C[i][i] = L->lam + 2.0 * L->mu;
    L->C[3 + i][3 + i] = L->mu;
  }
  for (int a = 0; a < 5; ++a)
    for (int b = 0; b < 5; ++b) {
      double s = 0.0;
      for (int i = 0; i < 6; ++i) s += P[i][a] * W[i] * P[i][b];
      L->G[a][b] = s;
    }
}

// ------------------------------------------------------------ free energy psi
// psi(eps, y) = 1/2 (eps - P y)^T C (eps - P y)   (Eq. michel_suquet_omega, H = 0)
//
// The helpers below are templates on the scalar type R: R = double is the
// oracle; R = Counted (further down) runs the same statements once to count
// the method's arithmetic (algorithmic flops per step of the update).

template <class R>
void elastic_strain(const R eps[6], const R y[5], R e[6]) {
  for (int i = 0; i < 6; ++i) {
    R pz = 0.0;
    for (int a = 0; a < 5; ++a) pz += P[i][a] * y[a];
    e[i] = eps[i] - pz;
  }
}

template <class R>
void stress(const Law& L, const R eps[6], const R y[5], R sig[6]) {
  R e[6];
  elastic_strain(eps, y, e);
  for (int i = 0; i < 6; ++i) {
    R s = 0.0;
    for (int j = 0; j < 6; ++j) s += L.C[i][j] * e[j];
    sig[i] = s;
  }
}

template <class R>
R psi(const Law& L, const R eps[6], const R y[5]) {
  R e[6], sig[6];
  elastic_strain(eps, y, e);
  stress(L, eps, y, sig);
  R s = 0.0;
  for (int i = 0; i < 6; ++i) s += e[i] * sig[i];
  return 0.5 * s;
}

// d psi / d y = -P^T C (eps - P y) = -P^T sigma
template <class R>
void psi_y(const Law& L, const R eps[6], const R y[5], R g[5]) {
  R sig[6];
  stress(L, eps, y, sig);
  for (int a = 0; a < 5; ++a) {
    R s = 0.0;
    for (int i = 0; i < 6; ++i) s += P[i][a] * sig[i];
    g[a] = -s;
  }
}

// d2 psi / dy2 = P^T C P (constant)
void psi_yy(const Law& L, double H[5][5]) {
  for (int a = 0; a < 5; ++a)
    for (int b = 0; b < 5; ++b) {
      double s = 0.0;
      for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) s += P[i][a] * L.C[i][j] * P[j][b];
      H[a][b] = s;
    }
}

// ------------------------------------------------------- dissipation phi (Norton)
// phi(v) = sigma0 edot0 n/(n+1) (s/edot0)^((n+1)/n),  s = sqrt(v^T G v)
// (convex dual of the paper's Psi, Eq. michel_suquet_psi, at sigma_Y = 0, H = 0)

template <class R>
R eqrate(const Law& L, const R v[5], R Gv[5]) {
  R q = 0.0;
  for (int a = 0; a < 5; ++a) {
    R s = 0.0;
    for (int b = 0; b < 5; ++b) s += L.G[a][b] * v[b];
    Gv[a] = s;
    q += v[a] * s;
  }
  using std::sqrt;
  return sqrt(q);
}

template <class R>
R phi(const Law& L, const R v[5]) {
  R Gv[5];
  const R s = eqrate(L, v, Gv);
  using std::pow;
  return L.sigma0 * L.edot0 * L.n / (L.n + 1.0) * pow(s / L.edot0, (L.n + 1.0) / L.n);
}

// phi_v = sigma0 edot0^(-1/n) s^(1/n - 1) G v   (= 0 at v = 0 by continuity)
template <class R>
void phi_v(const Law& L, const R v[5], R g[5]) {
  R Gv[5];
  const R s = eqrate(L, v, Gv);
  if (s == 0.0) {
    for (int a = 0; a < 5; ++a) g[a] = 0.0;
    return;
  }
  using std::pow;
  const R c = L.sigma0 * std::pow(L.edot0, -1.0 / L.n) * pow(s, 1.0 / L.n - 1.0);
  for (int a = 0; a < 5; ++a) g[a] = c * Gv[a];
}

// phi_vv = sigma0 edot0^(-1/n) [ s^(1/n-1) G + (1/n - 1) s^(1/n-3) (Gv)(Gv)^T ]
// At s = 0 it is finite only for n = 1; returns false otherwise.
template <class R>
bool phi_vv(const Law& L, const R v[5], R H[5][5]) {
  R Gv[5];
  const R s = eqrate(L, v, Gv);
  const double k = L.sigma0 * std::pow(L.edot0, -1.0 / L.n);
  if (s == 0.0) {
    if (L.n != 1.0) return false;
    for (int a = 0; a < 5; ++a)
      for (int b = 0; b < 5; ++b) H[a][b] = k * L.G[a][b];
    return true;
  }
  using std::pow;
  const R c1 = k * pow(s, 1.0 / L.n - 1.0);
  const R c2 = k * (1.0 / L.n - 1.0) * pow(s, 1.0 / L.n - 3.0);
  for (int a = 0; a < 5; ++a)
    for (int b = 0; b < 5; ++b) H[a][b] = c1 * L.G[a][b] + c2 * Gv[a] * Gv[b];
  return true;
}

// ------------------------------------------------- implicit Euler step pieces
// Incremental potential Pi(y) = psi(eps, y) + h phi((y - y_n)/h); its
// stationarity condition R(y) = psi_y + phi_v((y - y_n)/h) = 0 is the dual
// form of Eq. (implicit_euler); Newton matrix K = psi_yy + phi_vv / h.

template <class R>
void rate(const R y[5], const R yn[5], double h, R v[5]) {
  for (int a = 0; a < 5; ++a) v[a] = (y[a] - yn[a]) / h;
}

template <class R>
R Pi(const Law& L, const R eps[6], const R y[5], const R yn[5], double h) {
  R v[5];
  rate(y, yn, h, v);
  return psi(L, eps, y) + h * phi(L, v);
}

template <class R>
void residual(const Law& L, const R eps[6], const R y[5], const R yn[5], double h, R Rv[5]) {
  R v[5], g1[5], g2[5];
  rate(y, yn, h, v);
  psi_y(L, eps, y, g1);
  phi_v(L, v, g2);
  for (int a = 0; a < 5; ++a) Rv[a] = g1[a] + g2[a];
}

template <class R>
bool newton_matrix(const Law& L, const R y[5], const R yn[5], double h, R K[5][5]) {
  R v[5], H2[5][5];
  double H1[5][5];
  rate(y, yn, h, v);
  psi_yy(L, H1);
  if (!phi_vv(L, v, H2)) return false;
  for (int a = 0; a < 5; ++a)
    for (int b = 0; b < 5; ++b) K[a][b] = H1[a][b] + H2[a][b] / h;
  return true;
}

// Dense Cholesky solve of A x = b (A symmetric positive definite, n <= 6).
template <class RA, class R>
bool chol_solve(int n, const RA* A, const R* b, R* x) {
  RA Lm[36];
  using std::sqrt;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j <= i; ++j) {
      RA s = A[i * n + j];
      for (int k = 0; k < j; ++k) s -= Lm[i * n + k] * Lm[j * n + k];
      if (i == j) {
        if (!(s > 0.0)) return false;
        Lm[i * n + i] = sqrt(s);
      } else {
        Lm[i * n + j] = s / Lm[j * n + j];
      }
    }
  R t[6];
  for (int i = 0; i < n; ++i) {
    R s = b[i];
    for (int k = 0; k < i; ++k) s -= Lm[i * n + k] * t[k];
    t[i] = s / Lm[i * n + i];
  }
  for (int i = n - 1; i >= 0; --i) {
    R s = t[i];
    for (int k = i + 1; k < n; ++k) s -= Lm[k * n + i] * x[k];
    x[i] = s / Lm[i * n + i];
  }
  return true;
}

double maxabs(int n, const double* a) {
  double m = 0.0;
  for (int i = 0; i < n; ++i) m = std::fmax(m, std::fabs(a[i]));
  return m;
}

// Line-search function of step 3 of the update below: g(theta) = d . R(y_n +
// theta d) and its derivative g'(theta) = d^T K d.
template <class R>
R line_g(const Law& L, const R eps[6], const R yn[5], const R d[5], double h, R th, R* gp) {
  R yt[5], Rv[5], K[5][5];
  for (int a = 0; a < 5; ++a) yt[a] = yn[a] + th * d[a];
  residual(L, eps, yt, yn, h, Rv);
  newton_matrix(L, yt, yn, h, K);
  R g = 0.0, q = 0.0;
  for (int a = 0; a < 5; ++a) {
    g += d[a] * Rv[a];
    for (int b = 0; b < 5; ++b) q += d[a] * K[a][b] * d[b];
  }
  *gp = q;
  return g;
}

// Per-voxel diagnostics: line-search iterations, Newton iterations, flags.
enum { F_CONVERGED = 1, F_NONFINITE = 2, F_CAP = 4, F_NOT_SPD = 8 };
struct Info {
  int line_iters, newton_iters, flags;
};

// ------------------------------------------------ the implicit Euler update
// Newton start (reading of the singular dual form at y = y_n, where
// phi_vv ~ s^(1/n - 1) is unbounded for n > 1; the force-potential Newton of
// Sec. 4.1 starts at a_n and is regular there):
//   1. if psi_y(eps, y_n) = 0, then y = y_n solves R = 0;
//   2. psi-Newton predictor d = -psi_yy^{-1} psi_y(eps, y_n);
//   3. minimise Pi exactly on the segment y_n + theta d, theta in (0, 1]:
//      g(theta) = d.R(y_n + theta d) is increasing (Pi convex), g(0+) < 0,
//      g(1) > 0; safeguarded Newton on g with bisection fallback;
//   4. full Newton on R with Armijo backtracking on Pi until
//      |dy|_inf <= 1e-14 max(1, |y|_inf); at most 50 iterations.
void update_vp(const Law& L, const double eps[6], const double zn[6], double h, double sig[6],
               double z[6], double Ct[6][6], Info* info) {
  info->line_iters = 0;
  info->newton_iters = 0;
  info->flags = 0;
  double yn[5] = {zn[0], zn[1], zn[3], zn[4], zn[5]};
  double y[5];
  for (int a = 0; a < 5; ++a) y[a] = yn[a];

  double r0[5];
  psi_y(L, eps, yn, r0);
  bool relaxed = maxabs(5, r0) > 0.0;
  if (relaxed) {
    double H[5][5], d[5], mr0[5];
    psi_yy(L, H);
    for (int a = 0; a < 5; ++a) mr0[a] = -r0[a];
    if (!chol_solve(5, &H[0][0], mr0, d)) info->flags |= F_NOT_SPD;

    auto g_of = [&](double th, double* gp) { return line_g(L, eps, yn, d, h, th, gp); };
    double lo = 0.0, hi = 1.0, th = 1.0;
    for (int it = 0; it < 400; ++it) {
      ++info->line_iters;
      double gp;
      const double g = g_of(th, &gp);
      if (g == 0.0) break;
      if (g > 0.0) hi = th; else lo = th;
      double tn = th - g / gp;
      if (!(tn > lo && tn < hi)) tn = 0.5 * (lo + hi);
      if (tn == th || !(hi - lo > 4.0 * std::numeric_limits<double>::epsilon() * hi)) {
        th = tn;
        break;
      }
      th = tn;
    }
    for (int a = 0; a < 5; ++a) y[a] = yn[a] + th * d[a];

    for (int k = 0; k < 50; ++k) {
      ++info->newton_iters;
      double R[5], K[5][5], dy[5], mR[5];
      residual(L, eps, y, yn, h, R);
      if (!newton_matrix(L, y, yn, h, K)) { info->flags |= F_NOT_SPD; break; }
      for (int a = 0; a < 5; ++a) mR[a] = -R[a];
      if (!chol_solve(5, &K[0][0], mR, dy)) { info->flags |= F_NOT_SPD; break; }
      const bool small = maxabs(5, dy) <= 1e-14 * std::fmax(1.0, maxabs(5, y));
      double alpha = 1.0;
      if (!small) {
        const double P0 = Pi(L, eps, y, yn, h);
        double slope = 0.0;
        for (int a = 0; a < 5; ++a) slope += R[a] * dy[a];
        for (int ls = 0; ls < 40; ++ls) {
          double yt[5];
          for (int a = 0; a < 5; ++a) yt[a] = y[a] + alpha * dy[a];
          const double P1 = Pi(L, eps, yt, yn, h);
          if (P1 <= P0 + 1e-4 * alpha * slope + 8.0 * std::numeric_limits<double>::epsilon() * std::fabs(P0))
            break;
          alpha *= 0.5;
        }
      }
      for (int a = 0; a < 5; ++a) y[a] += alpha * dy[a];
      if (small) { info->flags |= F_CONVERGED; break; }
    }
    if (!(info->flags & F_CONVERGED) && !(info->flags & F_NOT_SPD)) info->flags |= F_CAP;
  } else {
    info->flags |= F_CONVERGED;
  }

  for (int i = 0; i < 6; ++i) {
    double s = 0.0;
    for (int a = 0; a < 5; ++a) s += P[i][a] * y[a];
    z[i] = s;
  }
  stress(L, eps, y, sig);

  if (Ct) {
    // C_t = C - C P K^{-1} P^T C  (Eq. tangent_formula with psi_ee = C,
    // psi_ey = -C P, K dy/deps = -psi_ye = P^T C).  Where K is unbounded
    // (y = y_n with n > 1) dy/deps = 0 and C_t = C.
    double K[5][5];
    const bool finite_K = newton_matrix(L, y, yn, h, K);
    for (int i = 0; i < 6; ++i)
      for (int j = 0; j < 6; ++j) Ct[i][j] = L.C[i][j];
    if (finite_K) {
      double PtC[5][6];
      for (int a = 0; a < 5; ++a)
        for (int j = 0; j < 6; ++j) {
          double s = 0.0;
          for (int i = 0; i < 6; ++i) s += P[i][a] * L.C[i][j];
          PtC[a][j] = s;
        }
      for (int j = 0; j < 6; ++j) {
        double col[5], dyde[5];
        for (int a = 0; a < 5; ++a) col[a] = PtC[a][j];
        if (!chol_solve(5, &K[0][0], col, dyde)) { info->flags |= F_NOT_SPD; continue; }
        for (int i = 0; i < 6; ++i) {
          double s = 0.0;
          for (int a = 0; a < 5; ++a) s += PtC[a][i] * dyde[a];  // (C P)_ia = (P^T C)_ai
          Ct[i][j] -= s;
        }
      }
    }
  }
  bool fin = true;
  for (int i = 0; i < 6; ++i) fin = fin && std::isfinite(sig[i]) && std::isfinite(z[i]);
  if (!fin) info->flags |= F_NONFINITE;
}

void update_elastic(const Law& L, const double eps[6], double sig[6], double Ct[6][6]) {
  for (int i = 0; i < 6; ++i) {
    double s = 0.0;
    for (int j = 0; j < 6; ++j) s += L.C[i][j] * eps[j];
    sig[i] = s;
  }
  if (Ct)
    for (int i = 0; i < 6; ++i)
      for (int j = 0; j < 6; ++j) Ct[i][j] = L.C[i][j];
}

// --------------------------------------------- independent radial return
// The paper's conventional strategy (Sec. 4, Simo-Hughes): with a deviatoric
// flow direction the implicit Euler step reduces to one scalar equation for
// the equivalent viscoplastic increment dp,
//   sigma_eq_trial - 3 mu dp = sigma0 (dp / (h edot0))^(1/n),
// after which z = z_n + 3/2 dp s_trial / sigma_eq_trial.  Written on 3x3
// tensors (not on the 5-vector y) so that it shares nothing with update_vp.
void voigt_to_tensor(const double v[6], double T[3][3], bool engineering) {
  const double f = engineering ? 0.5 : 1.0;
  T[0][0] = v[0]; T[1][1] = v[1]; T[2][2] = v[2];
  T[1][2] = T[2][1] = f * v[3];
  T[0][2] = T[2][0] = f * v[4];
  T[0][1] = T[1][0] = f * v[5];
}

void tensor_to_voigt(const double T[3][3], double v[6], bool engineering) {
  const double f = engineering ? 2.0 : 1.0;
  v[0] = T[0][0]; v[1] = T[1][1]; v[2] = T[2][2];
  v[3] = f * T[1][2]; v[4] = f * T[0][2]; v[5] = f * T[0][1];
}

void radial_return(const Law& L, const double eps[6], const double zn[6], double h, double sig[6],
                   double z[6]) {
  double Et[3][3], Zt[3][3], Ee[3][3], S[3][3], Sd[3][3];
  voigt_to_tensor(eps, Et, true);
  voigt_to_tensor(zn, Zt, true);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) Ee[i][j] = Et[i][j] - Zt[i][j];
  const double tr = Ee[0][0] + Ee[1][1] + Ee[2][2];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) S[i][j] = 2.0 * L.mu * Ee[i][j] + (i == j ? L.lam * tr : 0.0);
  const double p = (S[0][0] + S[1][1] + S[2][2]) / 3.0;
  double ss = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      Sd[i][j] = S[i][j] - (i == j ? p : 0.0);
      ss += Sd[i][j] * Sd[i][j];
    }
  const double seq = std::sqrt(1.5 * ss);
  double dp = 0.0;
  if (seq > 0.0) {
    // f(dp) = seq - 3 mu dp - sigma0 (dp/(h edot0))^(1/n): decreasing, f(0) > 0,
    // f(seq / 3mu) < 0.  Bracketed Newton with bisection fallback.
    auto f = [&](double x, double* fp) {
      const double r = std::pow(x / (h * L.edot0), 1.0 / L.n);
      *fp = -3.0 * L.mu - (x > 0.0 ? L.sigma0 * r / (L.n * x) : std::numeric_limits<double>::infinity());
      return seq - 3.0 * L.mu * x - L.sigma0 * r;
    };
    double lo = 0.0, hi = seq / (3.0 * L.mu), x = hi;
    for (int it = 0; it < 400; ++it) {
      double fp;
      const double fx = f(x, &fp);
      if (fx == 0.0) break;
      if (fx > 0.0) lo = x; else hi = x;
      double xn = x - fx / fp;
      if (!(xn > lo && xn < hi)) xn = 0.5 * (lo + hi);
      if (xn == x || !(hi - lo > 4.0 * std::numeric_limits<double>::epsilon() * hi)) { x = xn; break; }
      x = xn;
    }
    dp = x;
  }
  double Zn1[3][3], Sig[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      const double dz = seq > 0.0 ? 1.5 * dp * Sd[i][j] / seq : 0.0;
      Zn1[i][j] = Zt[i][j] + dz;
      Sig[i][j] = S[i][j] - 2.0 * L.mu * dz;
    }
  tensor_to_voigt(Zn1, z, true);
  tensor_to_voigt(Sig, sig, false);
}

// ================================================= force-potential form, ode23
// Sec. 2, Eq. (gsm_internal): adot = dPsi/dA (A) with A = -d omega/d a.
//
// Norton law (kind 1): a = y (the 5 unknowns of z = P y), A = -psi_y = P^T sigma,
// Psi of Eq. (michel_suquet_psi) at sigma_Y = 0, H = 0:
//   Psi(A) = sigma0 edot0 / (n+1) (s_A / sigma0)^(n+1),  s_A^2 = A^T G^{-1} A
// (G^{-1} is the dual metric of the rate norm; s_A is the von Mises stress).
//   Psi_A  = edot0 (s_A/sigma0)^n G^{-1}A / s_A
//   Psi_AA = edot0 sigma0^{-n} [ s_A^{n-1} G^{-1} + (n-1) s_A^{n-3} (G^{-1}A)(G^{-1}A)^T ]
// (at s_A = 0: Psi_A = 0; Psi_AA = edot0/sigma0 G^{-1} for n = 1 and 0 for n > 1).
//
// Michel-Suquet law (kind 2), Eq. (michel_suquet_omega) and (michel_suquet_psi)
// with K(alpha) = sigma_Y: a = (y, alpha),
//   omega = 1/2 (eps - P y)^T C (eps - P y) + 1/3 (P y)^T Hv (P y) + sigma_Y alpha,
//   Hv = diag(H, H, H, H/2, H/2, H/2),
//   A_y = P^T (sigma - X), X = 2/3 Hv P y (back stress),  A_alpha = -sigma_Y,
//   Psi = sigma_d edot0 / (n+1) ( (s + A_alpha)^+ / sigma_d )^(n+1),  s^2 = A_y^T G^{-1} A_y.
// With x = (s + A_alpha)^+, r = edot0 (x/sigma_d)^n, r' = n edot0/sigma_d (x/sigma_d)^(n-1):
//   Psi_{A_y} = r G^{-1}A_y / s,  Psi_{A_alpha} = r,
//   Psi_{A_y A_y} = r' (G^{-1}A_y)(G^{-1}A_y)^T / s^2 + r [ G^{-1}/s - (G^{-1}A_y)(G^{-1}A_y)^T / s^3 ],
//   Psi_{A_y A_alpha} = r' G^{-1}A_y / s,  Psi_{A_alpha A_alpha} = r'
// (all zero where x = 0, i.e. inside the elastic domain).
// The Norton law is kind 2 with sigma_Y = 0, H = 0 (alpha then only counts).
//
// Sec. 4.3 integrates the evolution equation over [t_n, t_{n+1}] with strain
// eps(t) interpolated linearly between eps_n and eps_{n+1}, by the embedded
// Runge-Kutta pair of Bogacki and Shampine (MATLAB's ode23) with automatic
// step size control after Hairer, Norsett, Wanner (Solving ODEs I, II.4).
// Corollary 1: the tangent dy/deps_{n+1} is the solution of the derivative
// ODE d/dt (da/de) = Psi_AA(A) dA/de, integrated together with a by the same
// steps, with the step sizes undifferentiated and the derivative in the error
// measure.  Sec. 4.5 (stress-driven error control): the error measure is taken
// on the pair of stresses (and of tangents) that the two embedded solutions
// give at the end of the substep.

struct Ode23Opts {
  double rtol, atol;
  int max_steps;
  bool tangent;
};

void g_inverse(const Law& L, double Gi[5][5]) {
  for (int c = 0; c < 5; ++c) {
    double e[5] = {0, 0, 0, 0, 0}, x[5];
    e[c] = 1.0;
    chol_solve(5, &L.G[0][0], e, x);
    for (int a = 0; a < 5; ++a) Gi[a][c] = x[a];
  }
}

// Psi_A(A) and (optionally) Psi_AA(A) of the Norton force potential.
void psi_force_a(const Law& L, const double Gi[5][5], const double A[5], double g[5], double H[5][5]) {
  double GA[5];
  double s2 = 0.0;
  for (int a = 0; a < 5; ++a) {
    double t = 0.0;
    for (int b = 0; b < 5; ++b) t += Gi[a][b] * A[b];
    GA[a] = t;
    s2 += A[a] * t;
  }
  const double s = std::sqrt(s2);
  const double n = L.n;
  if (s == 0.0) {
    for (int a = 0; a < 5; ++a) g[a] = 0.0;
    if (H)
      for (int a = 0; a < 5; ++a)
        for (int b = 0; b < 5; ++b) H[a][b] = n == 1.0 ? L.edot0 / L.sigma0 * Gi[a][b] : 0.0;
    return;
  }
  const double r = std::pow(s / L.sigma0, n);  // (s/sigma0)^n
  for (int a = 0; a < 5; ++a) g[a] = L.edot0 * r * GA[a] / s;
  if (H) {
    const double c1 = L.edot0 * r / s;                        // edot0 sigma0^-n s^(n-1)
    const double c2 = (n - 1.0) * L.edot0 * r / (s * s * s);  // (n-1) edot0 sigma0^-n s^(n-3)
    for (int a = 0; a < 5; ++a)
      for (int b = 0; b < 5; ++b) H[a][b] = c1 * Gi[a][b] + c2 * GA[a] * GA[b];
  }
}

// Psi of the Michel-Suquet law and its gradient / Hessian in (A_y, A_alpha).
double psi_force_ms(const Law& L, const double Gi[5][5], const double A[6], double g[6], double H[6][6]) {
  double GA[5];
  double s2 = 0.0;
  for (int a = 0; a < 5; ++a) {
    double t = 0.0;
    for (int b = 0; b < 5; ++b) t += Gi[a][b] * A[b];
    GA[a] = t;
    s2 += A[a] * t;
  }
  const double s = std::sqrt(s2);
  const double x = s + A[5];
  if (g)
    for (int a = 0; a < 6; ++a) g[a] = 0.0;
  if (H)
    for (int a = 0; a < 6; ++a)
      for (int b = 0; b < 6; ++b) H[a][b] = 0.0;
  if (!(x > 0.0) || s == 0.0) return 0.0;
  const double n = L.n, sd = L.sigma0, e0 = L.edot0;
  const double r = e0 * std::pow(x / sd, n);
  const double rp = n * e0 / sd * std::pow(x / sd, n - 1.0);
  if (g) {
    for (int a = 0; a < 5; ++a) g[a] = r * GA[a] / s;
    g[5] = r;
  }
  if (H) {
    for (int a = 0; a < 5; ++a) {
      for (int b = 0; b < 5; ++b)
        H[a][b] = rp * GA[a] * GA[b] / s2 + r * (Gi[a][b] / s - GA[a] * GA[b] / (s2 * s));
      H[a][5] = H[5][a] = rp * GA[a] / s;
    }
    H[5][5] = rp;
  }
  return sd * e0 / (n + 1.0) * std::pow(x / sd, n + 1.0);
}

// Generalized stress A (NY entries) at (eps(t), y): A_y = P^T (sigma - X),
// X = 2/3 Hv P y; A_alpha = -sigma_Y (kind 2).  Hv = 0 for the Norton law.
template <int NY>
void gen_stress(const Law& L, const double et[6], const double y[NY], double A[NY]) {
  double sig[6], z[6];
  stress(L, et, y, sig);
  for (int i = 0; i < 6; ++i) {
    double pz = 0.0;
    for (int a = 0; a < 5; ++a) pz += P[i][a] * y[a];
    z[i] = pz;
  }
  for (int a = 0; a < 5; ++a) {
    double t = 0.0;
    for (int i = 0; i < 6; ++i) {
      const double hv = i < 3 ? L.Hkin : 0.5 * L.Hkin;
      t += P[i][a] * (sig[i] - (2.0 / 3.0) * hv * z[i]);
    }
    A[a] = t;
  }
  if (NY == 6) A[NY - 1] = -L.sigY;
}

// Right-hand side at time t in [0, h] of the step: f = Psi_A(A) and, with
// Y = da/deps_{n+1} (NY x 6), F = Psi_AA(A) dA/deps_{n+1},
// dA_y/deps = P^T [C (theta I - P Y_y) - 2/3 Hv P Y_y], dA_alpha/deps = 0.
template <int NY>
void ode_rhs(const Law& L, const double Gi[5][5], const double epsn[6], const double eps1[6], double h, double t,
             const double y[NY], const double (*Y)[6], double f[NY], double (*F)[6]) {
  const double th = t / h;
  double et[6], A[NY];
  for (int i = 0; i < 6; ++i) et[i] = epsn[i] + th * (eps1[i] - epsn[i]);
  gen_stress<NY>(L, et, y, A);
  double H[6][6];
  if (NY == 5) {
    double H5[5][5];
    psi_force_a(L, Gi, A, f, F ? H5 : nullptr);
    if (F)
      for (int a = 0; a < 5; ++a)
        for (int b = 0; b < 5; ++b) H[a][b] = H5[a][b];
  } else {
    psi_force_ms(L, Gi, A, f, H);
  }
  if (!F) return;
  double D[6][6], dA[6][6];
  for (int i = 0; i < 6; ++i)
    for (int k = 0; k < 6; ++k) {
      double pz = 0.0;
      for (int a = 0; a < 5; ++a) pz += P[i][a] * Y[a][k];
      D[i][k] = (i == k ? th : 0.0) - pz;  // theta I - P Y_y
    }
  for (int a = 0; a < 5; ++a)
    for (int k = 0; k < 6; ++k) {
      double v = 0.0;
      for (int i = 0; i < 6; ++i) {
        double cd = 0.0;
        for (int j = 0; j < 6; ++j) cd += L.C[i][j] * D[j][k];
        double pz = 0.0;
        for (int b = 0; b < 5; ++b) pz += P[i][b] * Y[b][k];
        const double hv = i < 3 ? L.Hkin : 0.5 * L.Hkin;
        v += P[i][a] * (cd - (2.0 / 3.0) * hv * pz);
      }
      dA[a][k] = v;
    }
  if (NY == 6)
    for (int k = 0; k < 6; ++k) dA[5][k] = 0.0;
  for (int a = 0; a < NY; ++a)
    for (int k = 0; k < 6; ++k) {
      double v = 0.0;
      for (int b = 0; b < NY; ++b) v += H[a][b] * dA[b][k];
      F[a][k] = v;
    }
}

// Stress and tangent at the end of a substep: sigma = C (eps(t) - P y),
// Ct = C (theta I - P Y_y).
template <int NY>
void stress_tangent(const Law& L, const double epsn[6], const double eps1[6], double h, double t, const double y[NY],
                    const double (*Y)[6], double sig[6], double (*Ct)[6]) {
  const double th = t / h;
  double et[6];
  for (int i = 0; i < 6; ++i) et[i] = epsn[i] + th * (eps1[i] - epsn[i]);
  stress(L, et, y, sig);
  if (!Ct) return;
  for (int i = 0; i < 6; ++i)
    for (int k = 0; k < 6; ++k) {
      double v = 0.0;
      for (int j = 0; j < 6; ++j) {
        double pz = 0.0;
        for (int a = 0; a < 5; ++a) pz += P[j][a] * Y[a][k];
        v += L.C[i][j] * ((j == k ? th : 0.0) - pz);
      }
      Ct[i][k] = v;
    }
}

// Bogacki-Shampine 3(2): c = (0, 1/2, 3/4, 1); y_{+} = y + dt (2/9 k1 + 1/3 k2
// + 4/9 k3); the order-2 solution uses (7/24, 1/4, 1/3, 1/8) with k4 =
// f(t + dt, y_{+}), which is k1 of the next step (first same as last).
const double BS_A21 = 0.5, BS_A32 = 0.75;
const double BS_B[3] = {2.0 / 9.0, 1.0 / 3.0, 4.0 / 9.0};
const double BS_E[4] = {2.0 / 9.0 - 7.0 / 24.0, 1.0 / 3.0 - 1.0 / 4.0, 4.0 / 9.0 - 1.0 / 3.0, -1.0 / 8.0};

struct OdeInfo {
  int accepted, rejected, flags;
};

// One material update by ode23 over [t_n, t_{n+1}] (length h).  a_n: z_n (6)
// and, for NY = 6, alpha_n; a_out likewise.
template <int NY>
void update_ode23(const Law& L, const double epsn[6], const double eps1[6], const double zn[6], double alpha_n,
                  double h, const Ode23Opts& o, double sig_out[6], double z_out[6], double* alpha_out,
                  double (*Ct_out)[6], OdeInfo* info) {
  double Gi[5][5];
  g_inverse(L, Gi);
  double y[NY];
  y[0] = zn[0];
  y[1] = zn[1];
  y[2] = zn[3];
  y[3] = zn[4];
  y[4] = zn[5];
  if (NY == 6) y[NY - 1] = alpha_n;
  double Y[NY][6] = {};
  const bool tan = o.tangent;
  double k[4][NY], K[4][NY][6];
  double t = 0.0, dt = h;
  ode_rhs<NY>(L, Gi, epsn, eps1, h, 0.0, y, Y, k[0], tan ? K[0] : nullptr);
  double sig_old[6], C_old[6][6];
  stress_tangent<NY>(L, epsn, eps1, h, 0.0, y, Y, sig_old, tan ? C_old : nullptr);
  info->accepted = info->rejected = 0;
  info->flags = 0;
  bool last_rejected = false;
  while (t < h) {
    if (info->accepted + info->rejected >= o.max_steps) {
      info->flags |= F_CAP;
      break;
    }
    const bool clip = t + dt >= h;  // the substep that ends the interval ends at h exactly
    if (clip) dt = h - t;
    double ys[NY], Ys[NY][6];
    // stage 2
    for (int a = 0; a < NY; ++a) {
      ys[a] = y[a] + dt * BS_A21 * k[0][a];
      if (tan)
        for (int c = 0; c < 6; ++c) Ys[a][c] = Y[a][c] + dt * BS_A21 * K[0][a][c];
    }
    ode_rhs<NY>(L, Gi, epsn, eps1, h, t + 0.5 * dt, ys, Ys, k[1], tan ? K[1] : nullptr);
    // stage 3
    for (int a = 0; a < NY; ++a) {
      ys[a] = y[a] + dt * BS_A32 * k[1][a];
      if (tan)
        for (int c = 0; c < 6; ++c) Ys[a][c] = Y[a][c] + dt * BS_A32 * K[1][a][c];
    }
    ode_rhs<NY>(L, Gi, epsn, eps1, h, t + 0.75 * dt, ys, Ys, k[2], tan ? K[2] : nullptr);
    // order-3 solution and the last stage
    double yn1[NY], Yn1[NY][6];
    for (int a = 0; a < NY; ++a) {
      yn1[a] = y[a] + dt * (BS_B[0] * k[0][a] + BS_B[1] * k[1][a] + BS_B[2] * k[2][a]);
      if (tan)
        for (int c = 0; c < 6; ++c)
          Yn1[a][c] = Y[a][c] + dt * (BS_B[0] * K[0][a][c] + BS_B[1] * K[1][a][c] + BS_B[2] * K[2][a][c]);
    }
    const double tn1 = clip ? h : t + dt;
    ode_rhs<NY>(L, Gi, epsn, eps1, h, tn1, yn1, Yn1, k[3], tan ? K[3] : nullptr);
    // embedded difference (order 3 minus order 2) and the stress pair it gives
    double e[NY], E[NY][6];
    for (int a = 0; a < NY; ++a) {
      e[a] = dt * (BS_E[0] * k[0][a] + BS_E[1] * k[1][a] + BS_E[2] * k[2][a] + BS_E[3] * k[3][a]);
      if (tan)
        for (int c = 0; c < 6; ++c)
          E[a][c] = dt * (BS_E[0] * K[0][a][c] + BS_E[1] * K[1][a][c] + BS_E[2] * K[2][a][c] + BS_E[3] * K[3][a][c]);
    }
    double y2[NY], Y2[NY][6], s3[6], s2[6], C3[6][6], C2[6][6];
    for (int a = 0; a < NY; ++a) {
      y2[a] = yn1[a] - e[a];
      if (tan)
        for (int c = 0; c < 6; ++c) Y2[a][c] = Yn1[a][c] - E[a][c];
    }
    stress_tangent<NY>(L, epsn, eps1, h, tn1, yn1, Yn1, s3, tan ? C3 : nullptr);
    stress_tangent<NY>(L, epsn, eps1, h, tn1, y2, Y2, s2, tan ? C2 : nullptr);
    double sum = 0.0;
    int m = 0;
    // (a zero scale, atol = 0 at zero stress, counts a zero difference as no error)
    auto sq_scaled = [](double d, double sc) {
      const double q = sc > 0.0 ? d / sc : (d == 0.0 ? 0.0 : 1e300);
      return q * q;
    };
    for (int i = 0; i < 6; ++i, ++m)
      sum += sq_scaled(s3[i] - s2[i], o.atol + o.rtol * std::fmax(std::fabs(sig_old[i]), std::fabs(s3[i])));
    if (tan)
      for (int i = 0; i < 6; ++i)
        for (int c = 0; c < 6; ++c, ++m)
          sum += sq_scaled(C3[i][c] - C2[i][c], o.atol + o.rtol * std::fmax(std::fabs(C_old[i][c]), std::fabs(C3[i][c])));
    // a trial step that overflows is rejected like one with a large error
    const double err = std::isfinite(sum) ? std::sqrt(sum / m) : 1e300;
    // step size after Hairer II.4: fac = 0.9, facmin = 0.2, facmax = 5
    // (1 right after a rejection), exponent 1/(q+1) with q = 2
    const double facmax = last_rejected ? 1.0 : 5.0;
    const double grow = err == 0.0 ? facmax : std::fmin(facmax, std::fmax(0.2, 0.9 * std::pow(err, -1.0 / 3.0)));
    if (err <= 1.0) {
      t = tn1;
      for (int a = 0; a < NY; ++a) {
        y[a] = yn1[a];
        k[0][a] = k[3][a];
        if (tan)
          for (int c = 0; c < 6; ++c) {
            Y[a][c] = Yn1[a][c];
            K[0][a][c] = K[3][a][c];
          }
      }
      for (int i = 0; i < 6; ++i) {
        sig_old[i] = s3[i];
        if (tan)
          for (int c = 0; c < 6; ++c) C_old[i][c] = C3[i][c];
      }
      ++info->accepted;
      last_rejected = false;
    } else {
      ++info->rejected;
      last_rejected = true;
    }
    dt *= grow;
  }
  if (t >= h && !(info->flags & (F_NONFINITE | F_CAP))) info->flags |= F_CONVERGED;
  stress_tangent<NY>(L, epsn, eps1, h, h, y, Y, sig_out, Ct_out);
  z_out[0] = y[0];
  z_out[1] = y[1];
  z_out[2] = -(y[0] + y[1]);
  z_out[3] = y[2];
  z_out[4] = y[3];
  z_out[5] = y[4];
  if (alpha_out) *alpha_out = NY == 6 ? y[NY - 1] : 0.0;
}

// One material update by ode12, the pair of the explicit Euler scheme (order
// 1) and Heun's method (order 2), Sec. 4.3.  Per attempt of length dt from
// (t, y) with k1 = f(t, y):
//   y_E = y + dt k1,  k2 = f(t + dt, y_E),  y_H = y + dt/2 (k1 + k2);
// the substep continues with y_H (the higher order, as ode23 continues with
// its order-3 solution); the error compares the stresses of y_H and y_E at
// t + dt like ode23 compares those of its two solutions; the step control is
// ode23's with exponent 1/2 (1/(q+1), q = 1 the lower order).  k1 of the next
// substep is f(t + dt, y_H), evaluated after an acceptance.
template <int NY>
void update_ode12(const Law& L, const double epsn[6], const double eps1[6], const double zn[6], double alpha_n,
                  double h, const Ode23Opts& o, double sig_out[6], double z_out[6], double* alpha_out,
                  double (*Ct_out)[6], OdeInfo* info) {
  double Gi[5][5];
  g_inverse(L, Gi);
  double y[NY];
  y[0] = zn[0];
  y[1] = zn[1];
  y[2] = zn[3];
  y[3] = zn[4];
  y[4] = zn[5];
  if (NY == 6) y[NY - 1] = alpha_n;
  double Y[NY][6] = {};
  const bool tan = o.tangent;
  double k1[NY], K1[NY][6], k2[NY], K2[NY][6];
  double t = 0.0, dt = h;
  ode_rhs<NY>(L, Gi, epsn, eps1, h, 0.0, y, Y, k1, tan ? K1 : nullptr);
  double sig_old[6], C_old[6][6];
  stress_tangent<NY>(L, epsn, eps1, h, 0.0, y, Y, sig_old, tan ? C_old : nullptr);
  info->accepted = info->rejected = 0;
  info->flags = 0;
  bool last_rejected = false;
  while (t < h) {
    if (info->accepted + info->rejected >= o.max_steps) {
      info->flags |= F_CAP;
      break;
    }
    const bool clip = t + dt >= h;
    if (clip) dt = h - t;
    const double tn1 = clip ? h : t + dt;
    // Euler predictor and Heun corrector
    double yE[NY], YE[NY][6], yH[NY], YH[NY][6];
    for (int a = 0; a < NY; ++a) {
      yE[a] = y[a] + dt * k1[a];
      if (tan)
        for (int c = 0; c < 6; ++c) YE[a][c] = Y[a][c] + dt * K1[a][c];
    }
    ode_rhs<NY>(L, Gi, epsn, eps1, h, tn1, yE, YE, k2, tan ? K2 : nullptr);
    for (int a = 0; a < NY; ++a) {
      yH[a] = y[a] + 0.5 * dt * (k1[a] + k2[a]);
      if (tan)
        for (int c = 0; c < 6; ++c) YH[a][c] = Y[a][c] + 0.5 * dt * (K1[a][c] + K2[a][c]);
    }
    double sH[6], sE[6], CH[6][6], CE[6][6];
    stress_tangent<NY>(L, epsn, eps1, h, tn1, yH, YH, sH, tan ? CH : nullptr);
    stress_tangent<NY>(L, epsn, eps1, h, tn1, yE, YE, sE, tan ? CE : nullptr);
    double sum = 0.0;
    int m = 0;
    auto sq_scaled = [](double d, double sc) {
      const double q = sc > 0.0 ? d / sc : (d == 0.0 ? 0.0 : 1e300);
      return q * q;
    };
    for (int i = 0; i < 6; ++i, ++m)
      sum += sq_scaled(sH[i] - sE[i], o.atol + o.rtol * std::fmax(std::fabs(sig_old[i]), std::fabs(sH[i])));
    if (tan)
      for (int i = 0; i < 6; ++i)
        for (int c = 0; c < 6; ++c, ++m)
          sum += sq_scaled(CH[i][c] - CE[i][c], o.atol + o.rtol * std::fmax(std::fabs(C_old[i][c]), std::fabs(CH[i][c])));
    const double err = std::isfinite(sum) ? std::sqrt(sum / m) : 1e300;
    const double facmax = last_rejected ? 1.0 : 5.0;
    const double grow = err == 0.0 ? facmax : std::fmin(facmax, std::fmax(0.2, 0.9 / std::sqrt(err)));
    if (err <= 1.0) {
      t = tn1;
      for (int a = 0; a < NY; ++a) {
        y[a] = yH[a];
        if (tan)
          for (int c = 0; c < 6; ++c) Y[a][c] = YH[a][c];
      }
      for (int i = 0; i < 6; ++i) {
        sig_old[i] = sH[i];
        if (tan)
          for (int c = 0; c < 6; ++c) C_old[i][c] = CH[i][c];
      }
      ode_rhs<NY>(L, Gi, epsn, eps1, h, t, y, Y, k1, tan ? K1 : nullptr);
      ++info->accepted;
      last_rejected = false;
    } else {
      ++info->rejected;
      last_rejected = true;
    }
    dt *= grow;
  }
  if (t >= h && !(info->flags & (F_NONFINITE | F_CAP))) info->flags |= F_CONVERGED;
  stress_tangent<NY>(L, epsn, eps1, h, h, y, Y, sig_out, Ct_out);
  z_out[0] = y[0];
  z_out[1] = y[1];
  z_out[2] = -(y[0] + y[1]);
  z_out[3] = y[2];
  z_out[4] = y[3];
  z_out[5] = y[4];
  if (alpha_out) *alpha_out = NY == 6 ? y[NY - 1] : 0.0;
}

// Dense solve of W x = b (W general, n <= 6) by Gaussian elimination with
// partial pivoting; false if W is singular.
bool gauss_solve(int n, const double* W, const double* b, double* x) {
  double M[6][7];
  for (int i = 0; i < n; ++i) {
    for (int j = 0; j < n; ++j) M[i][j] = W[i * n + j];
    M[i][n] = b[i];
  }
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(M[r][c]) > std::fabs(M[piv][c])) piv = r;
    if (M[piv][c] == 0.0) return false;
    if (piv != c)
      for (int j = 0; j <= n; ++j) std::swap(M[c][j], M[piv][j]);
    for (int r = c + 1; r < n; ++r) {
      const double f = M[r][c] / M[c][c];
      for (int j = c; j <= n; ++j) M[r][j] -= f * M[c][j];
    }
  }
  for (int i = n - 1; i >= 0; --i) {
    double t = M[i][n];
    for (int j = i + 1; j < n; ++j) t -= M[i][j] * x[j];
    x[i] = t / M[i][i];
  }
  return true;
}

// Third derivative of the force potential contracted with two directions u,
// v (NY entries each): out = Psi_AAA[u, v].  Both laws have the form Psi =
// sigma0 edot0/(n+1) (x^+/sigma0)^(n+1) with x = s (Norton) or s + A_alpha
// (Michel-Suquet), s^2 = A_z^T G^-1 A_z.  With m = G^-1 A_z / s, Q = G^-1 - m
// m^T and r(x) = edot0 (x/sigma0)^n the Hessian is H_zz = r' m m^T + r Q/s,
// H_za = r' m, H_aa = r'; its derivative along u, with dx = m.u_z + u_a,
// ds = m.u_z, dm = Q u_z/s:
//   dH_zz = r'' dx m m^T + (r' - r/s)(dm m^T + m dm^T) + (r' dx - r ds/s) Q/s,
//   dH_za = r'' dx m + r' dm,  dH_aa = r'' dx.
// Zero where the potential is inactive (x <= 0) or s = 0.
template <int NY>
void psi_force_aaa(const Law& L, const double Gi[5][5], const double A[NY], const double u[NY], const double v[NY],
                   double out[NY]) {
  for (int a = 0; a < NY; ++a) out[a] = 0.0;
  double GA[5], s2 = 0.0;
  for (int a = 0; a < 5; ++a) {
    double t = 0.0;
    for (int b = 0; b < 5; ++b) t += Gi[a][b] * A[b];
    GA[a] = t;
    s2 += A[a] * t;
  }
  const double s = std::sqrt(s2);
  const double x = NY == 6 ? s + A[5] : s;
  if (!(x > 0.0) || s == 0.0) return;
  const double n = L.n, sg = L.sigma0, e0 = L.edot0;
  const double r = e0 * std::pow(x / sg, n);
  const double r1 = n * e0 / sg * std::pow(x / sg, n - 1.0);
  const double r2 = n * (n - 1.0) * e0 / (sg * sg) * std::pow(x / sg, n - 2.0);
  double m[5], Q[5][5], dm[5];
  for (int a = 0; a < 5; ++a) m[a] = GA[a] / s;
  for (int a = 0; a < 5; ++a)
    for (int b = 0; b < 5; ++b) Q[a][b] = Gi[a][b] - m[a] * m[b];
  double ds = 0.0;
  for (int a = 0; a < 5; ++a) ds += m[a] * u[a];
  const double dx = ds + (NY == 6 ? u[5] : 0.0);
  for (int a = 0; a < 5; ++a) {
    double t = 0.0;
    for (int b = 0; b < 5; ++b) t += Q[a][b] * u[b];
    dm[a] = t / s;
  }
  double mv = 0.0, dmv = 0.0;
  for (int a = 0; a < 5; ++a) {
    mv += m[a] * v[a];
    dmv += dm[a] * v[a];
  }
  const double va = NY == 6 ? v[5] : 0.0;
  for (int a = 0; a < 5; ++a) {
    double Qv = 0.0;
    for (int b = 0; b < 5; ++b) Qv += Q[a][b] * v[b];
    out[a] = r2 * dx * m[a] * mv + (r1 - r / s) * (dm[a] * mv + m[a] * dmv) + (r1 * dx - r * ds / s) * Qv / s +
             (r2 * dx * m[a] + r1 * dm[a]) * va;
  }
  if (NY == 6) out[5] = r2 * dx * mv + r1 * dmv + r2 * dx * va;
}

// Generalized-stress sensitivities of the force-potential ODE: dA/dy (NY x
// NY; dA_z/dz = -P^T (C + 2/3 Hv) P, zero for alpha) and dA/dt (NY; dA_z/dt
// = P^T C (eps_{n+1} - eps_n)/h).
template <int NY>
void gen_stress_sens(const Law& L, const double epsn[6], const double eps1[6], double h, double dAdy[NY][NY],
                     double dAdt[NY]) {
  for (int a = 0; a < NY; ++a) {
    dAdt[a] = 0.0;
    for (int b = 0; b < NY; ++b) dAdy[a][b] = 0.0;
  }
  for (int a = 0; a < 5; ++a) {
    for (int b = 0; b < 5; ++b) {
      double t = 0.0;
      for (int i = 0; i < 6; ++i) {
        const double hv = i < 3 ? L.Hkin : 0.5 * L.Hkin;
        for (int j = 0; j < 6; ++j) t += P[i][a] * (L.C[i][j] + (i == j ? (2.0 / 3.0) * hv : 0.0)) * P[j][b];
      }
      dAdy[a][b] = -t;
    }
    double t = 0.0;
    for (int i = 0; i < 6; ++i)
      for (int j = 0; j < 6; ++j) t += P[i][a] * L.C[i][j] * (eps1[j] - epsn[j]);
    dAdt[a] = t / h;
  }
}

// Psi_AA at the generalized stress of (t, y).
template <int NY>
void force_hessian_at(const Law& L, const double Gi[5][5], const double epsn[6], const double eps1[6], double h,
                      double t, const double y[NY], double A[NY], double H[NY][NY]) {
  const double th = t / h;
  double et[6];
  for (int i = 0; i < 6; ++i) et[i] = epsn[i] + th * (eps1[i] - epsn[i]);
  gen_stress<NY>(L, et, y, A);
  double g[6];
  if (NY == 5) {
    double H5[5][5];
    psi_force_a(L, Gi, A, g, H5);
    for (int a = 0; a < 5; ++a)
      for (int b = 0; b < 5; ++b) H[a][b] = H5[a][b];
  } else {
    double H6[6][6];
    psi_force_ms(L, Gi, A, g, H6);
    for (int a = 0; a < NY; ++a)
      for (int b = 0; b < NY; ++b) H[a][b] = H6[a][b];
  }
}

// One material update by ode23s, the modified Rosenbrock triple of Shampine
// and Reichelt (SIAM J. Sci. Comput. 18 (1997) 1-22; MATLAB's ode23s), Sec.
// 4.3.  With d = 1/(2 + sqrt 2), e32 = 6 + sqrt 2, J = df/dy and T = df/dt
// at the start (t, y) of a substep of length dt and W = I - dt d J:
//   k1 = W^-1 (F0 + dt d T),          F0 = f(t, y)
//   F1 = f(t + dt/2, y + dt/2 k1),   k2 = W^-1 (F1 - k1) + k1
//   y_new = y + dt k2,               F2 = f(t + dt, y_new)
//   k3 = W^-1 (F2 - e32 (k2 - F1) - 2 (k1 - F0) + dt d T)
//   error estimate dt/6 (k1 - 2 k2 + k3)
// The error compares the stresses of y_new and y_new minus the estimate (as
// ode23 compares its two solutions); step control as ode23's (exponent 1/3);
// F2 is F0 of the next substep, J and T are re-evaluated at the accepted point.
// Tangent (Corollary 1, the Rosenbrock form of the stage derivatives): for
// each column k of Y = dy/deps_{n+1}, with dA_k the total derivative of A,
//   J~_k w = Psi_AAA[dA_k, dA/dy w],  T~_k = Psi_AAA[dA_k, dA/dt] + Psi_AA d2A_k,
//   d2A_k = d(dA/dt)/deps_k = P^T C e_k / h,
//   k1~ = W^-1 (F0~ + dt d T~ + dt d J~ k1)
//   k2~ = k1~ + W^-1 (F1~ - k1~ + dt d J~ (k2 - k1))
//   k3~ = W^-1 (F2~ - e32 (k2~ - F1~) - 2 (k1~ - F0~) + dt d T~ + dt d J~ k3)
// with Fi~ the tangent right-hand sides (ode_rhs) at the stage states.
template <int NY>
void update_ode23s(const Law& L, const double epsn[6], const double eps1[6], const double zn[6], double alpha_n,
                   double h, const Ode23Opts& o, double sig_out[6], double z_out[6], double* alpha_out,
                   double (*Ct_out)[6], OdeInfo* info) {
  const double d = 1.0 / (2.0 + std::sqrt(2.0)), e32 = 6.0 + std::sqrt(2.0);
  double Gi[5][5];
  g_inverse(L, Gi);
  double dAdy[NY][NY], dAdt[NY];
  gen_stress_sens<NY>(L, epsn, eps1, h, dAdy, dAdt);
  double y[NY];
  y[0] = zn[0];
  y[1] = zn[1];
  y[2] = zn[3];
  y[3] = zn[4];
  y[4] = zn[5];
  if (NY == 6) y[NY - 1] = alpha_n;
  double Y[NY][6] = {};
  const bool tan = o.tangent;
  double F0[NY], G0[NY][6];
  ode_rhs<NY>(L, Gi, epsn, eps1, h, 0.0, y, Y, F0, tan ? G0 : nullptr);
  double sig_old[6], C_old[6][6];
  stress_tangent<NY>(L, epsn, eps1, h, 0.0, y, Y, sig_old, tan ? C_old : nullptr);
  // J, T (and Psi_AA, A for the tangent) at the start of the substep
  double A0[NY], H0[NY][NY], J[NY][NY], T[NY];
  auto refresh = [&](double t) {
    force_hessian_at<NY>(L, Gi, epsn, eps1, h, t, y, A0, H0);
    for (int a = 0; a < NY; ++a) {
      double tt = 0.0;
      for (int b = 0; b < NY; ++b) tt += H0[a][b] * dAdt[b];
      T[a] = tt;
      for (int b = 0; b < NY; ++b) {
        double jj = 0.0;
        for (int c = 0; c < NY; ++c) jj += H0[a][c] * dAdy[c][b];
        J[a][b] = jj;
      }
    }
  };
  refresh(0.0);
  info->accepted = info->rejected = 0;
  info->flags = 0;
  bool last_rejected = false;
  double t = 0.0, dt = h;
  while (t < h) {
    if (info->accepted + info->rejected >= o.max_steps) {
      info->flags |= F_CAP;
      break;
    }
    const bool clip = t + dt >= h;
    if (clip) dt = h - t;
    const double tn1 = clip ? h : t + dt;
    double W[NY * NY];
    for (int a = 0; a < NY; ++a)
      for (int b = 0; b < NY; ++b) W[a * NY + b] = (a == b ? 1.0 : 0.0) - dt * d * J[a][b];
    bool ok = true;
    double rhs[NY], k1[NY], k2[NY], k3[NY], F1[NY], F2[NY], ys[NY], yn1[NY], e[NY];
    for (int a = 0; a < NY; ++a) rhs[a] = F0[a] + dt * d * T[a];
    ok &= gauss_solve(NY, W, rhs, k1);
    for (int a = 0; a < NY; ++a) ys[a] = y[a] + 0.5 * dt * k1[a];
    double Ys[NY][6], G1[NY][6], G2[NY][6], K1[NY][6], K2[NY][6], K3[NY][6], Yn1[NY][6], E[NY][6];
    // the tangent stages need F1~ at y + dt/2 k1 with Y + dt/2 k1~: k1~ first
    double dA[6][NY];  // total dA/deps_k at (t, y, Y), column k
    if (tan) {
      for (int k = 0; k < 6; ++k) {
        double th = t / h;
        for (int a = 0; a < NY; ++a) {
          double v = 0.0;
          for (int b = 0; b < NY; ++b) v += dAdy[a][b] * Y[b][k];
          if (a < 5)
            for (int i = 0; i < 6; ++i) v += th * P[i][a] * L.C[i][k];
          dA[k][a] = v;
        }
      }
    }
    // J~_k w for the k-th column
    auto Jt = [&](int k, const double w[NY], double out[NY]) {
      double v[NY];
      for (int a = 0; a < NY; ++a) {
        double tt = 0.0;
        for (int b = 0; b < NY; ++b) tt += dAdy[a][b] * w[b];
        v[a] = tt;
      }
      psi_force_aaa<NY>(L, Gi, A0, dA[k], v, out);
    };
    double Tt[6][NY];
    if (tan)
      for (int k = 0; k < 6; ++k) {
        psi_force_aaa<NY>(L, Gi, A0, dA[k], dAdt, Tt[k]);
        for (int a = 0; a < NY; ++a) {
          double tt = 0.0;
          for (int b = 0; b < 5; ++b) {
            double d2 = 0.0;
            for (int i = 0; i < 6; ++i) d2 += P[i][b] * L.C[i][k];
            tt += H0[a][b] * d2 / h;
          }
          Tt[k][a] += tt;
        }
        double jk[NY], r2[NY], col[NY];
        Jt(k, k1, jk);
        for (int a = 0; a < NY; ++a) r2[a] = G0[a][k] + dt * d * Tt[k][a] + dt * d * jk[a];
        ok &= gauss_solve(NY, W, r2, col);
        for (int a = 0; a < NY; ++a) {
          K1[a][k] = col[a];
          Ys[a][k] = Y[a][k] + 0.5 * dt * col[a];
        }
      }
    ode_rhs<NY>(L, Gi, epsn, eps1, h, t + 0.5 * dt, ys, Ys, F1, tan ? G1 : nullptr);
    for (int a = 0; a < NY; ++a) rhs[a] = F1[a] - k1[a];
    double w2[NY];
    ok &= gauss_solve(NY, W, rhs, w2);
    for (int a = 0; a < NY; ++a) {
      k2[a] = w2[a] + k1[a];
      yn1[a] = y[a] + dt * k2[a];
    }
    if (tan)
      for (int k = 0; k < 6; ++k) {
        double dk[NY], jk[NY], r2[NY], col[NY];
        for (int a = 0; a < NY; ++a) dk[a] = k2[a] - k1[a];
        Jt(k, dk, jk);
        for (int a = 0; a < NY; ++a) r2[a] = G1[a][k] - K1[a][k] + dt * d * jk[a];
        ok &= gauss_solve(NY, W, r2, col);
        for (int a = 0; a < NY; ++a) {
          K2[a][k] = K1[a][k] + col[a];
          Yn1[a][k] = Y[a][k] + dt * K2[a][k];
        }
      }
    ode_rhs<NY>(L, Gi, epsn, eps1, h, tn1, yn1, Yn1, F2, tan ? G2 : nullptr);
    for (int a = 0; a < NY; ++a) rhs[a] = F2[a] - e32 * (k2[a] - F1[a]) - 2.0 * (k1[a] - F0[a]) + dt * d * T[a];
    ok &= gauss_solve(NY, W, rhs, k3);
    for (int a = 0; a < NY; ++a) e[a] = dt / 6.0 * (k1[a] - 2.0 * k2[a] + k3[a]);
    if (tan)
      for (int k = 0; k < 6; ++k) {
        double jk[NY], r2[NY], col[NY];
        Jt(k, k3, jk);
        for (int a = 0; a < NY; ++a)
          r2[a] = G2[a][k] - e32 * (K2[a][k] - G1[a][k]) - 2.0 * (K1[a][k] - G0[a][k]) + dt * d * Tt[k][a] +
                  dt * d * jk[a];
        ok &= gauss_solve(NY, W, r2, col);
        for (int a = 0; a < NY; ++a) {
          K3[a][k] = col[a];
          E[a][k] = dt / 6.0 * (K1[a][k] - 2.0 * K2[a][k] + K3[a][k]);
        }
      }
    double y2[NY], Y2[NY][6], s3[6], s2[6], C3[6][6], C2[6][6];
    for (int a = 0; a < NY; ++a) {
      y2[a] = yn1[a] - e[a];
      if (tan)
        for (int c = 0; c < 6; ++c) Y2[a][c] = Yn1[a][c] - E[a][c];
    }
    stress_tangent<NY>(L, epsn, eps1, h, tn1, yn1, Yn1, s3, tan ? C3 : nullptr);
    stress_tangent<NY>(L, epsn, eps1, h, tn1, y2, Y2, s2, tan ? C2 : nullptr);
    double sum = 0.0;
    int m = 0;
    auto sq_scaled = [](double dd, double sc) {
      const double q = sc > 0.0 ? dd / sc : (dd == 0.0 ? 0.0 : 1e300);
      return q * q;
    };
    for (int i = 0; i < 6; ++i, ++m)
      sum += sq_scaled(s3[i] - s2[i], o.atol + o.rtol * std::fmax(std::fabs(sig_old[i]), std::fabs(s3[i])));
    if (tan)
      for (int i = 0; i < 6; ++i)
        for (int c = 0; c < 6; ++c, ++m)
          sum += sq_scaled(C3[i][c] - C2[i][c], o.atol + o.rtol * std::fmax(std::fabs(C_old[i][c]), std::fabs(C3[i][c])));
    // a singular W or an overflow rejects the trial step
    const double err = ok && std::isfinite(sum) ? std::sqrt(sum / m) : 1e300;
    const double facmax = last_rejected ? 1.0 : 5.0;
    const double grow = err == 0.0 ? facmax : std::fmin(facmax, std::fmax(0.2, 0.9 * std::pow(err, -1.0 / 3.0)));
    if (err <= 1.0) {
      t = tn1;
      for (int a = 0; a < NY; ++a) {
        y[a] = yn1[a];
        F0[a] = F2[a];
        if (tan)
          for (int c = 0; c < 6; ++c) {
            Y[a][c] = Yn1[a][c];
            G0[a][c] = G2[a][c];
          }
      }
      for (int i = 0; i < 6; ++i) {
        sig_old[i] = s3[i];
        if (tan)
          for (int c = 0; c < 6; ++c) C_old[i][c] = C3[i][c];
      }
      refresh(t);
      ++info->accepted;
      last_rejected = false;
    } else {
      ++info->rejected;
      last_rejected = true;
    }
    dt *= grow;
  }
  if (t >= h && !(info->flags & (F_NONFINITE | F_CAP))) info->flags |= F_CONVERGED;
  stress_tangent<NY>(L, epsn, eps1, h, h, y, Y, sig_out, Ct_out);
  z_out[0] = y[0];
  z_out[1] = y[1];
  z_out[2] = -(y[0] + y[1]);
  z_out[3] = y[2];
  z_out[4] = y[3];
  z_out[5] = y[4];
  if (alpha_out) *alpha_out = NY == 6 ? y[NY - 1] : 0.0;
}

// ------------------------------------------------------ algorithmic flops
// A scalar that counts the arithmetic of the statements above when they run
// once on it (the algorithmic work of the method per step of the update; the
// benchmark multiplies it by the iteration counts a GPU run reports).
//   * Inputs of a voxel (eps, z_n, theta, ...) are "active"; law constants and
//     the constant matrices P, G, C are "passive" and cost nothing: an
//     implementation computes their products once per law.
//   * An operation with a passive 0 (x + 0, x * 0) or a passive +-1 factor or
//     divisor (P's entries) is structure, not work, and is not counted; nor is
//     a negation, a comparison or |x|.
//   * Every other add, sub, mul, div and sqrt counts as one flop; an FMA of a
//     hardware implementation is two.  pow(x, c) counts as one power (an
//     implementation spends tens of operations on it; reported apart).
struct FlopTally {
  int64_t add, mul, div, sqrt, pow;
};
FlopTally g_tally;  // ora_flop_pieces runs single-threaded

struct Counted {
  double v;
  bool active;
  Counted(double x = 0.0) : v(x), active(false) {}
  static Counted var(double x) {
    Counted c(x);
    c.active = true;
    return c;
  }
};
inline bool is_pm1(const Counted& a) { return !a.active && (a.v == 1.0 || a.v == -1.0); }
inline bool is_zero(const Counted& a) { return !a.active && a.v == 0.0; }
inline Counted act(double x) { return Counted::var(x); }
inline Counted operator-(const Counted& a) { Counted r(-a.v); r.active = a.active; return r; }
inline Counted operator+(const Counted& a, const Counted& b) {
  if (!a.active && !b.active) return Counted(a.v + b.v);
  if (is_zero(a)) return b;
  if (is_zero(b)) return a;
  ++g_tally.add;
  return act(a.v + b.v);
}
inline Counted operator-(const Counted& a, const Counted& b) { return a + (-b); }
inline Counted operator*(const Counted& a, const Counted& b) {
  if (!a.active && !b.active) return Counted(a.v * b.v);
  if (is_zero(a) || is_zero(b)) return Counted(0.0);
  if (is_pm1(a)) return a.v > 0 ? b : -b;
  if (is_pm1(b)) return b.v > 0 ? a : -a;
  ++g_tally.mul;
  return act(a.v * b.v);
}
inline Counted operator/(const Counted& a, const Counted& b) {
  if (!a.active && !b.active) return Counted(a.v / b.v);
  if (is_zero(a)) return Counted(0.0);
  if (is_pm1(b)) return b.v > 0 ? a : -a;
  ++g_tally.div;
  return act(a.v / b.v);
}
inline Counted& operator+=(Counted& a, const Counted& b) { return a = a + b; }
inline Counted& operator-=(Counted& a, const Counted& b) { return a = a - b; }
inline bool operator==(const Counted& a, double b) { return a.v == b; }
inline bool operator>(const Counted& a, double b) { return a.v > b; }
inline Counted sqrt(const Counted& a) {
  if (!a.active) return Counted(std::sqrt(a.v));
  ++g_tally.sqrt;
  return act(std::sqrt(a.v));
}
inline Counted pow(const Counted& a, double e) {
  if (!a.active) return Counted(std::pow(a.v, e));
  ++g_tally.pow;
  return act(std::pow(a.v, e));
}

}  // namespace

// ======================================================================= C ABI
// Field arrays are array-of-structs: eps[n][6], z_n[n][6], sigma[n][6], z[n][6],
// tangent[n][6][6] (may be NULL), info[n][3] (may be NULL).
// params = {E, nu, sigma0, edot0, n}; kind 0 = elastic, 1 = elastic-viscoplastic.

extern "C" {

int ora_max_threads() {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

int ora_update(int kind, const double* params, int64_t n, const double* eps, const double* zn,
               double h, double* sigma, double* z, double* tangent, int32_t* info) {
  if (kind != 0 && kind != 1) return -1;
  Law L;
  make_law(kind, params, &L);
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t i = 0; i < n; ++i) {
    double(*Ct)[6] = tangent ? reinterpret_cast<double(*)[6]>(tangent + 36 * i) : nullptr;
    if (kind == 0) {
      update_elastic(L, eps + 6 * i, sigma + 6 * i, Ct);
      for (int k = 0; k < 6; ++k) z[6 * i + k] = zn[6 * i + k];
      if (info) { info[3 * i] = 0; info[3 * i + 1] = 0; info[3 * i + 2] = F_CONVERGED; }
    } else {
      Info inf;
      update_vp(L, eps + 6 * i, zn + 6 * i, h, sigma + 6 * i, z + 6 * i, Ct, &inf);
      if (info) { info[3 * i] = inf.line_iters; info[3 * i + 1] = inf.newton_iters; info[3 * i + 2] = inf.flags; }
    }
  }
  return 0;
}

int ora_radial_return(const double* params, int64_t n, const double* eps, const double* zn, double h,
                      double* sigma, double* z) {
  Law L;
  make_law(1, params, &L);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) radial_return(L, eps + 6 * i, zn + 6 * i, h, sigma + 6 * i, z + 6 * i);
  return 0;
}

// Algorithmic flops of the pieces of the implicit-Euler update (Sec. 4.1) of
// the Norton law, counted by running the oracle's own statements once on the
// Counted scalar at a flowing state: voxel inputs eps, z_n [6], the converged
// y [5] (y != y_n) and h.  out[7][5]: per piece (add, mul, div, sqrt, pow):
//   0 predictor  psi_y(eps, y_n) and d = -psi_yy^{-1} psi_y (psi_yy and its
//                factor are law constants: only the substitutions count);
//   1 line       one step of the 1-D search on y_n + theta d: g, g' and the
//                Newton update of theta (a division and a subtraction);
//   2 newton     one Newton step: R, K, the 5x5 Cholesky factor and solve, y += dy;
//   3 residual   R = psi_y + phi_v alone (the residual sweep of a correction);
//   4 subst      forward and back substitution with a given Cholesky factor;
//   5 stress     z = P y and sigma = C (eps - P y);
//   6 tangent    C_t = C - C P K^{-1} P^T C at y (Eq. tangent_formula).
// Returns 0, or -1 if the state does not flow (s = 0).
int ora_flop_pieces(const double* params, const double* eps, const double* zn, const double* y, double h,
                    int64_t* out) {
  Law L;
  make_law(1, params, &L);
  Counted E[6], Yn[5], Y[5];
  for (int i = 0; i < 6; ++i) E[i] = Counted::var(eps[i]);
  const double yn5[5] = {zn[0], zn[1], zn[3], zn[4], zn[5]};
  for (int a = 0; a < 5; ++a) {
    Yn[a] = Counted::var(yn5[a]);
    Y[a] = Counted::var(y[a]);
  }
  bool flows = false;
  for (int a = 0; a < 5; ++a) flows = flows || y[a] != yn5[a];
  if (!flows) return -1;
  auto take = [&](int piece) {
    out[5 * piece + 0] = g_tally.add;
    out[5 * piece + 1] = g_tally.mul;
    out[5 * piece + 2] = g_tally.div;
    out[5 * piece + 3] = g_tally.sqrt;
    out[5 * piece + 4] = g_tally.pow;
    g_tally = FlopTally{0, 0, 0, 0, 0};
  };
  g_tally = FlopTally{0, 0, 0, 0, 0};
  double H[5][5];
  psi_yy(L, H);
  // 0 predictor
  Counted r0[5], mr0[5], d[5];
  psi_y(L, E, Yn, r0);
  for (int a = 0; a < 5; ++a) mr0[a] = -r0[a];
  chol_solve(5, &H[0][0], mr0, d);
  take(0);
  // 1 line: g, g' at theta = 1/2 and the Newton update of theta
  {
    Counted gp;
    const Counted th = Counted::var(0.5);
    const Counted g = line_g(L, E, Yn, d, h, th, &gp);
    const Counted tn = th - g / gp;
    (void)tn;
  }
  take(1);
  // 2 newton
  {
    Counted Rv[5], K[5][5], mR[5], dy[5], yy[5];
    residual(L, E, Y, Yn, h, Rv);
    newton_matrix(L, Y, Yn, h, K);
    for (int a = 0; a < 5; ++a) mR[a] = -Rv[a];
    chol_solve(5, &K[0][0], mR, dy);
    for (int a = 0; a < 5; ++a) yy[a] = Y[a] + dy[a];
  }
  take(2);
  // 3 residual
  {
    Counted Rv[5];
    residual(L, E, Y, Yn, h, Rv);
  }
  take(3);
  // the Cholesky factor alone: a solve with a zero right-hand side (0 / x and
  // x * 0 are not counted, so only the factorization remains)
  auto factor_count = [&](Counted (&K)[5][5]) {
    const FlopTally keep = g_tally;
    g_tally = FlopTally{0, 0, 0, 0, 0};
    Counted zero[5], x[5];
    chol_solve(5, &K[0][0], zero, x);
    const FlopTally f = g_tally;
    g_tally = keep;
    return f;
  };
  auto minus = [](FlopTally a, const FlopTally& b) {
    a.add -= b.add; a.mul -= b.mul; a.div -= b.div; a.sqrt -= b.sqrt; a.pow -= b.pow;
    return a;
  };
  // 4 substitutions with a given factor
  {
    Counted K[5][5], Rv[5], dy[5];
    newton_matrix(L, Y, Yn, h, K);
    residual(L, E, Y, Yn, h, Rv);
    const FlopTally fac = factor_count(K);
    g_tally = FlopTally{0, 0, 0, 0, 0};
    chol_solve(5, &K[0][0], Rv, dy);
    g_tally = minus(g_tally, fac);
  }
  take(4);
  // 5 stress and z
  {
    Counted z[6], sig[6];
    for (int i = 0; i < 6; ++i) {
      Counted t = 0.0;
      for (int a = 0; a < 5; ++a) t += P[i][a] * Y[a];
      z[i] = t;
    }
    stress(L, E, Y, sig);
  }
  take(5);
  // 6 tangent: K, one factor of K, then per column j of P^T C the solve
  // K dy/deps_j = (P^T C)_j and C_t(:, j) = C(:, j) - (C P) dy/deps_j
  // (update_vp's tangent block, with the factor counted once)
  {
    Counted K[5][5], Ct[6][6];
    newton_matrix(L, Y, Yn, h, K);
    const FlopTally fac = factor_count(K);
    const FlopTally before = g_tally;
    for (int i = 0; i < 6; ++i)
      for (int j = 0; j < 6; ++j) Ct[i][j] = L.C[i][j];
    double PtC[5][6];
    for (int a = 0; a < 5; ++a)
      for (int j = 0; j < 6; ++j) {
        double t = 0.0;
        for (int i = 0; i < 6; ++i) t += P[i][a] * L.C[i][j];
        PtC[a][j] = t;
      }
    FlopTally solves{0, 0, 0, 0, 0};
    for (int j = 0; j < 6; ++j) {
      Counted col[5], x[5];
      for (int a = 0; a < 5; ++a) col[a] = PtC[a][j];
      const FlopTally t0 = g_tally;
      chol_solve(5, &K[0][0], col, x);
      const FlopTally one = minus(minus(g_tally, t0), fac);  // substitutions of this column
      g_tally = t0;
      solves.add += one.add; solves.mul += one.mul; solves.div += one.div;
      for (int i = 0; i < 6; ++i) {
        Counted t = 0.0;
        for (int a = 0; a < 5; ++a) t += PtC[a][i] * x[a];
        Ct[i][j] -= t;
      }
    }
    g_tally.add += fac.add + solves.add;
    g_tally.mul += fac.mul + solves.mul;
    g_tally.div += fac.div + solves.div;
    g_tally.sqrt += fac.sqrt;
    (void)before;
  }
  take(6);
  return 0;
}

// Single-point accessors of the hand-derived potentials (used by the
// finite-difference and invariant pins).
double ora_psi(const double* params, const double* eps, const double* y) {
  Law L; make_law(1, params, &L); return psi(L, eps, y);
}
void ora_psi_y(const double* params, const double* eps, const double* y, double* g) {
  Law L; make_law(1, params, &L); psi_y(L, eps, y, g);
}
void ora_psi_yy(const double* params, double* H) {
  Law L; make_law(1, params, &L); psi_yy(L, reinterpret_cast<double(*)[5]>(H));
}
void ora_stress(const double* params, const double* eps, const double* y, double* sig) {
  Law L; make_law(1, params, &L); stress(L, eps, y, sig);
}
double ora_phi(const double* params, const double* v) {
  Law L; make_law(1, params, &L); return phi(L, v);
}
void ora_phi_v(const double* params, const double* v, double* g) {
  Law L; make_law(1, params, &L); phi_v(L, v, g);
}
int ora_phi_vv(const double* params, const double* v, double* H) {
  Law L; make_law(1, params, &L); return phi_vv(L, v, reinterpret_cast<double(*)[5]>(H)) ? 0 : -1;
}
void ora_residual(const double* params, const double* eps, const double* y, const double* yn, double h,
                  double* R) {
  Law L; make_law(1, params, &L); residual(L, eps, y, yn, h, R);
}
int ora_newton_matrix(const double* params, const double* y, const double* yn, double h, double* K) {
  Law L; make_law(1, params, &L); return newton_matrix(L, y, yn, h, reinterpret_cast<double(*)[5]>(K)) ? 0 : -1;
}
double ora_Pi(const double* params, const double* eps, const double* y, const double* yn, double h) {
  Law L; make_law(1, params, &L); return Pi(L, eps, y, yn, h);
}

// Batched Newton matrix K = psi_yy + phi_vv/h and dissipation Hessian phi_vv
// at converged states (n voxels, y and y_n [n][5]); for the adjoint.
// Voxels with y = y_n (no flow) get K = psi_yy + 0 and phi_vv = 0 when n > 1
// (the unbounded Hessian multiplies a zero adjoint there: dy/dy_n = 0).
void ora_newton_matrix_batch(const double* params, int64_t n, const double* y, const double* yn, double h,
                             double* K, double* Hphi) {
  Law L; make_law(1, params, &L);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double v[5], H1[5][5], H2[5][5];
    rate(y + 5 * i, yn + 5 * i, h, v);
    psi_yy(L, H1);
    const bool finite = phi_vv(L, v, H2);
    for (int a = 0; a < 5; ++a)
      for (int b = 0; b < 5; ++b) {
        const double hp = finite ? H2[a][b] : 0.0;
        Hphi[25 * i + 5 * a + b] = hp;
        K[25 * i + 5 * a + b] = H1[a][b] + hp / h;
      }
  }
}

// ode23 / ode12 update (Sec. 4.3 with the stress-driven error control of Sec. 4.5):
// kind 1 (Norton, params E, nu, sigma0, edot0, n) or 2 (Michel-Suquet, params
// E, nu, sigma_Y, H, edot0, sigma_d, n); eps_n, eps, z_n [n][6]; alpha_n,
// alpha [n] (kind 2; alpha_n may be NULL = 0); tangent [n][6][6] or NULL;
// info [n][3] = accepted, rejected substeps, flags (1 converged, 4 substep cap).
// method 0 = ode23 (Bogacki-Shampine 3(2)), 1 = ode12 (explicit Euler / Heun),
// 2 = ode23s (Shampine-Reichelt Rosenbrock triple).
int ora_update_ode(int kind, int method, const double* params, int64_t n, const double* eps_n, const double* eps,
                   const double* zn, const double* alpha_n, double h, double rtol, double atol, int max_steps,
                   double* sigma, double* z, double* alpha, double* tangent, int32_t* info) {
  if ((kind != 1 && kind != 2) || method < 0 || method > 2) return -1;
  Law L;
  make_law(kind, params, &L);
  Ode23Opts o{rtol, atol, max_steps, tangent != nullptr};
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t i = 0; i < n; ++i) {
    double(*Ct)[6] = tangent ? reinterpret_cast<double(*)[6]>(tangent + 36 * i) : nullptr;
    OdeInfo inf;
    double al = 0.0;
    const double a0 = alpha_n ? alpha_n[i] : 0.0;
    if (kind == 1 && method == 0)
      update_ode23<5>(L, eps_n + 6 * i, eps + 6 * i, zn + 6 * i, 0.0, h, o, sigma + 6 * i, z + 6 * i, nullptr, Ct,
                      &inf);
    else if (kind == 1 && method == 1)
      update_ode12<5>(L, eps_n + 6 * i, eps + 6 * i, zn + 6 * i, 0.0, h, o, sigma + 6 * i, z + 6 * i, nullptr, Ct,
                      &inf);
    else if (kind == 1)
      update_ode23s<5>(L, eps_n + 6 * i, eps + 6 * i, zn + 6 * i, 0.0, h, o, sigma + 6 * i, z + 6 * i, nullptr, Ct,
                       &inf);
    else if (method == 0)
      update_ode23<6>(L, eps_n + 6 * i, eps + 6 * i, zn + 6 * i, a0, h, o, sigma + 6 * i, z + 6 * i, &al, Ct, &inf);
    else if (method == 1)
      update_ode12<6>(L, eps_n + 6 * i, eps + 6 * i, zn + 6 * i, a0, h, o, sigma + 6 * i, z + 6 * i, &al, Ct, &inf);
    else
      update_ode23s<6>(L, eps_n + 6 * i, eps + 6 * i, zn + 6 * i, a0, h, o, sigma + 6 * i, z + 6 * i, &al, Ct, &inf);
    if (alpha) alpha[i] = al;
    if (info) {
      info[3 * i] = inf.accepted;
      info[3 * i + 1] = inf.rejected;
      info[3 * i + 2] = inf.flags;
    }
  }
  return 0;
}

// Psi_AAA[u, v] of the Norton (kind 1, NY = 5) or Michel-Suquet (kind 2, NY = 6) force potential.
void ora_psi_force_aaa(int kind, const double* params, const double* A, const double* u, const double* v,
                       double* out) {
  Law L;
  make_law(kind, params, &L);
  double Gi[5][5];
  g_inverse(L, Gi);
  if (kind == 1) psi_force_aaa<5>(L, Gi, A, u, v, out);
  else psi_force_aaa<6>(L, Gi, A, u, v, out);
}

// Michel-Suquet force potential Psi(A) at A [6] = (A_y, A_alpha); g [6], H [6][6] or NULL.
double ora_psi_force_ms(const double* params, const double* A, double* g, double* H) {
  Law L;
  make_law(2, params, &L);
  double Gi[5][5], gg[6], HH[6][6];
  g_inverse(L, Gi);
  const double v = psi_force_ms(L, Gi, A, gg, HH);
  if (g)
    for (int a = 0; a < 6; ++a) g[a] = gg[a];
  if (H)
    for (int a = 0; a < 6; ++a)
      for (int b = 0; b < 6; ++b) H[6 * a + b] = HH[a][b];
  return v;
}

// Generalized stress A of the Michel-Suquet law at (eps, y, alpha): [6].
void ora_gen_stress_ms(const double* params, const double* eps, const double* y6, double* A) {
  Law L;
  make_law(2, params, &L);
  gen_stress<6>(L, eps, y6, A);
}

// Psi_A (and Psi_AA when H != NULL) of the force potential at A [5].
void ora_psi_force_a(const double* params, const double* A, double* g, double* H) {
  Law L;
  make_law(1, params, &L);
  double Gi[5][5];
  g_inverse(L, Gi);
  double HH[5][5];
  psi_force_a(L, Gi, A, g, H ? HH : nullptr);
  if (H)
    for (int a = 0; a < 5; ++a)
      for (int b = 0; b < 5; ++b) H[5 * a + b] = HH[a][b];
}

}  // extern "C"
