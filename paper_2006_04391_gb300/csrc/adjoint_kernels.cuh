// Device kernels of the adjoint of the load history (basic scheme + implicit
// Euler material update).  The paper differentiates only locally, inside one
// material evaluation (Sec. 4.1, Eq. tangent_formula; Sec. 5); this is the
// discrete adjoint of a whole homogenization run, hand-written on top of the
// AD blocks of the law.  Included by ms_solve.cu only.
//
// For J = w . Sigma_K and step k with checkpoint (eps_k, z_{k-1}), given the
// adjoints g_sig (uniform w/N^3 at the last step, else 0) and g_z of
// (sigma_k, z_k):
//   prepare:  re-solve the update, K = psi_yy + phi_vv/h, C_t = psi_ee + psi_ey dy/deps,
//             a_u = C_t g_sig + (dz/deps)^T g_z = C_t g_sig - psi_ey K^-1 (P^T g_z)
//   solve:    compatible zero-mean lam with P_V(C_t lam) = P_V(a_u)     (host loop)
//   finish:   a = g_sig - lam,  b = K^-1 (P^T g_z + psi_ye a)   (psi_ye a = -P^T C a)
//             g_{z,k-1} = (phi_vv/h) b on (z11, z22, g23, g13, g12)  (= P^T g_z + psi_ye a
//             where the voxel does not flow, dy/dy_n = I there)
//             dJ/dtheta += a . dsigma/dtheta|_y - b . dR/dtheta  (Norton: theta = E, sigma0, n)
#pragma once

#include "ms_kernels.cuh"

namespace gsm {
namespace {

constexpr int kAdjBlock = 128;

struct NortonTheta {
  double E, sigma0, edot0, n;
};

// P^T g for a strain-adjoint 6-vector g (z = P y).
__device__ __forceinline__ void pt_of(const double (&g)[6], double (&gy)[5]) {
  gy[0] = g[0] - g[2];
  gy[1] = g[1] - g[2];
  gy[2] = g[3];
  gy[3] = g[4];
  gy[4] = g[5];
}

template <int MODE>
__global__ void __launch_bounds__(kAdjBlock) adj_prepare_kernel(int64_t nvox, const uint8_t* __restrict__ phase,
                                                                const PhaseTable* __restrict__ tab, double h,
                                                                const double* __restrict__ eps_k,
                                                                const double* __restrict__ zprev, double gs0,
                                                                double gs1, double gs2, double gs3, double gs4,
                                                                double gs5, const double* __restrict__ g_z,
                                                                double* __restrict__ Ct21, double* __restrict__ a_u,
                                                                double* __restrict__ yK) {
  const double gs[6] = {gs0, gs1, gs2, gs3, gs4, gs5};
  const Step hs = make_step(h);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < nvox; base += stride) {
    const int64_t i = base + threadIdx.x;
    const bool in = i < nvox;
    const int ph = in ? (int)phase[i] : 0;
    const bool vp = in && tab->kind[ph] == GSM_PSI_ELASTIC_VP_DEV;
    double e[6], zi[6], s[6], zo[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      e[c] = in ? eps_k[c * nvox + i] : 0.0;
      zi[c] = vp ? zprev[c * nvox + i] : 0.0;
    }
    if constexpr (MODE == MODE_FP64) voxel_fp64<NortonDev>(tab->p64[ph], e, zi, hs, vp, s, zo, nullptr);
    else voxel_fp32_fix<NortonDev>(tab->p64[ph], tab->p32[ph], e, zi, hs, vp, s, zo, nullptr);
    if (!in) continue;
    double C[6][6], au[6];
    if (vp) {
      const LawParams<double>& p = tab->p64[ph];
      const double y[5] = {zo[0], zo[1], zo[3], zo[4], zo[5]};
      const double yn[5] = {zi[0], zi[1], zi[3], zi[4], zi[5]};
      double sig[6], Cee[6][6], Cey[6][5], Cye[5][6], g[5], K[5][5];
      psi_blocks<NortonDev>(p, e, y, sig, Cee, Cey, Cye);
      psi_y_yy<NortonDev>(p, e, y, g, K);
      bool flow = false;
#pragma unroll
      for (int a = 0; a < 5; ++a) flow = flow || (y[a] != yn[a]);
      double gz[6], gy[5], t[5] = {0, 0, 0, 0, 0};
#pragma unroll
      for (int c = 0; c < 6; ++c) gz[c] = g_z[c * nvox + i];
      pt_of(gz, gy);
#pragma unroll
      for (int r = 0; r < 6; ++r)
#pragma unroll
        for (int c = 0; c < 6; ++c) C[r][c] = Cee[r][c];
      if (flow) {
        const double inv_h = 1.0 / h;
        double v[5], gv[5], Hv[5][5];
#pragma unroll
        for (int a = 0; a < 5; ++a) v[a] = (y[a] - yn[a]) * inv_h;
        phi_v_vv<NortonDev>(p, v, gv, Hv);
#pragma unroll
        for (int a = 0; a < 5; ++a)
#pragma unroll
          for (int b = 0; b < 5; ++b) K[a][b] += Hv[a][b] * inv_h;
        Chol5<double> ch;
        ch.factor(K);
        ch.solve(gy, t);
        // C_t = Cee + Cey dy/deps, dy/deps = -K^-1 Cye
#pragma unroll
        for (int c = 0; c < 6; ++c) {
          double rhs[5], dy[5];
#pragma unroll
          for (int a = 0; a < 5; ++a) rhs[a] = -Cye[a][c];
          ch.solve(rhs, dy);
#pragma unroll
          for (int r = 0; r < 6; ++r) {
            double acc = 0.0;
#pragma unroll
            for (int a = 0; a < 5; ++a) acc += Cey[r][a] * dy[a];
            C[r][c] += acc;
          }
        }
      }
#pragma unroll
      for (int r = 0; r < 6; ++r) {
        double acc = 0.0;
#pragma unroll
        for (int c = 0; c < 6; ++c) acc += C[c][r] * gs[c];
#pragma unroll
        for (int a = 0; a < 5; ++a) acc -= Cey[r][a] * t[a];
        au[r] = acc;
      }
#pragma unroll
      for (int a = 0; a < 5; ++a) yK[a * nvox + i] = y[a];
      int q = 5;
#pragma unroll
      for (int a = 0; a < 5; ++a)
#pragma unroll
        for (int b = a; b < 5; ++b) yK[(q++) * nvox + i] = K[a][b];
    } else {
      double C21[21];
      voxel_elastic<double>(tab->p64[ph], e, s, C21);
      int q = 0;
#pragma unroll
      for (int r = 0; r < 6; ++r)
#pragma unroll
        for (int c = r; c < 6; ++c) {
          C[r][c] = C21[q];
          C[c][r] = C21[q];
          ++q;
        }
#pragma unroll
      for (int r = 0; r < 6; ++r) {
        double acc = 0.0;
#pragma unroll
        for (int c = 0; c < 6; ++c) acc += C[c][r] * gs[c];
        au[r] = acc;
      }
    }
    int q = 0;
#pragma unroll
    for (int r = 0; r < 6; ++r)
#pragma unroll
      for (int c = r; c < 6; ++c) Ct21[(q++) * nvox + i] = 0.5 * (C[r][c] + C[c][r]);
#pragma unroll
    for (int c = 0; c < 6; ++c) a_u[c * nvox + i] = au[c];
  }
}

// tau = C_t lam - a_u, lam = lam_raw / N^3 (C2R output).
// Reference medium of a step's adjoint equilibrium from its tangent field
// (as the forward per-step reference, Sec. 3): per voxel the isotropic
// measures 3k = (1/3) sum_{i,j<3} C_ij and 10 mu = tr_Mandel C - 3k of C_t,
// per block their min and max -> part[q * gridDim.x + block], q = kmin,
// kmax, mumin, mumax.  Launch with kAdjBlock threads.
__global__ void __launch_bounds__(kAdjBlock) adj_reference_kernel(int64_t nvox, const double* __restrict__ Ct21,
                                                                  double* __restrict__ part) {
  double r[4] = {1e300, -1e300, 1e300, -1e300};
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nvox; i += stride) {
    // packed upper triangle: C11 0, C12 1, C13 2, C22 6, C23 7, C33 11, C44 15, C55 18, C66 20
    const double d0 = Ct21[i], d1 = Ct21[6 * nvox + i], d2 = Ct21[11 * nvox + i];
    const double tk = (d0 + d1 + d2 + 2.0 * (Ct21[nvox + i] + Ct21[2 * nvox + i] + Ct21[7 * nvox + i])) * (1.0 / 3.0);
    const double tr = d0 + d1 + d2 + 2.0 * (Ct21[15 * nvox + i] + Ct21[18 * nvox + i] + Ct21[20 * nvox + i]);
    const double k = tk * (1.0 / 3.0), mu = (tr - tk) * 0.1;
    r[0] = fmin(r[0], k);
    r[1] = fmax(r[1], k);
    r[2] = fmin(r[2], mu);
    r[3] = fmax(r[3], mu);
  }
  __shared__ double sh[4][kAdjBlock / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    double v = r[q];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const double o = __shfl_down_sync(0xffffffffu, v, off);
      v = (q & 1) ? fmax(v, o) : fmin(v, o);
    }
    if (lane == 0) sh[q][w] = v;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    const int q = threadIdx.x;
    double v = sh[q][0];
    for (int k = 1; k < kAdjBlock / 32; ++k) v = (q & 1) ? fmax(v, sh[q][k]) : fmin(v, sh[q][k]);
    part[q * gridDim.x + blockIdx.x] = v;
  }
}

__global__ void adj_tau_kernel(int64_t nvox, const double* __restrict__ Ct21, const double* __restrict__ a_u,
                               const double* __restrict__ lam_raw, double inv_n3, double* __restrict__ tau) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nvox; i += stride) {
    double l[6], C[6][6];
#pragma unroll
    for (int c = 0; c < 6; ++c) l[c] = lam_raw[c * nvox + i] * inv_n3;
    int q = 0;
#pragma unroll
    for (int r = 0; r < 6; ++r)
#pragma unroll
      for (int c = r; c < 6; ++c) {
        const double v = Ct21[(q++) * nvox + i];
        C[r][c] = v;
        C[c][r] = v;
      }
#pragma unroll
    for (int r = 0; r < 6; ++r) {
      double acc = -a_u[r * nvox + i];
#pragma unroll
      for (int c = 0; c < 6; ++c) acc += C[r][c] * l[c];
      tau[r * nvox + i] = acc;
    }
  }
}

__global__ void __launch_bounds__(kAdjBlock) adj_finish_kernel(
    int64_t nvox, const uint8_t* __restrict__ phase, const PhaseTable* __restrict__ tab, double h, int phase_id,
    NortonTheta th, const double* __restrict__ eps_k, const double* __restrict__ zprev, double gs0, double gs1,
    double gs2, double gs3, double gs4, double gs5, const double* __restrict__ g_z, const double* __restrict__ lam_raw,
    double inv_n3, const double* __restrict__ yK, double* __restrict__ g_z_prev, double* __restrict__ partials) {
  const double gs[6] = {gs0, gs1, gs2, gs3, gs4, gs5};
  double acc[3] = {0.0, 0.0, 0.0};
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nvox; i += stride) {
    const int ph = (int)phase[i];
    double out[6] = {0, 0, 0, 0, 0, 0};
    if (tab->kind[ph] == GSM_PSI_ELASTIC_VP_DEV) {
      const LawParams<double>& p = tab->p64[ph];
      double e[6], a[6], gz[6], gy[5], y[5], yn[5], K[5][5];
#pragma unroll
      for (int c = 0; c < 6; ++c) {
        e[c] = eps_k[c * nvox + i];
        a[c] = gs[c] - lam_raw[c * nvox + i] * inv_n3;
        gz[c] = g_z[c * nvox + i];
      }
      yn[0] = zprev[i];
      yn[1] = zprev[nvox + i];
      yn[2] = zprev[3 * nvox + i];
      yn[3] = zprev[4 * nvox + i];
      yn[4] = zprev[5 * nvox + i];
#pragma unroll
      for (int b = 0; b < 5; ++b) y[b] = yK[b * nvox + i];
      int q = 5;
#pragma unroll
      for (int r = 0; r < 5; ++r)
#pragma unroll
        for (int c = r; c < 5; ++c) {
          const double v = yK[(q++) * nvox + i];
          K[r][c] = v;
          K[c][r] = v;
        }
      pt_of(gz, gy);
      double sig[6], Cee[6][6], Cey[6][5], Cye[5][6], psy[5];
      psi_blocks<NortonDev>(p, e, y, sig, Cee, Cey, Cye);
      psi_y_and_stress<NortonDev>(p, e, y, psy, sig);
      double rhs[5];
#pragma unroll
      for (int r = 0; r < 5; ++r) {
        double s = gy[r];
#pragma unroll
        for (int c = 0; c < 6; ++c) s += Cye[r][c] * a[c];
        rhs[r] = s;
      }
      bool flow = false;
#pragma unroll
      for (int b = 0; b < 5; ++b) flow = flow || (y[b] != yn[b]);
      double b5[5] = {0, 0, 0, 0, 0}, gyn[5];
      double v[5];
      const double inv_h = 1.0 / h;
#pragma unroll
      for (int b = 0; b < 5; ++b) v[b] = (y[b] - yn[b]) * inv_h;
      if (flow) {
        Chol5<double> ch;
        ch.factor(K);
        ch.solve(rhs, b5);
        double gv[5], Hv[5][5];
        phi_v_vv<NortonDev>(p, v, gv, Hv);
#pragma unroll
        for (int r = 0; r < 5; ++r) {
          double s = 0.0;
#pragma unroll
          for (int c = 0; c < 5; ++c) s += Hv[r][c] * b5[c];
          gyn[r] = s * inv_h;
        }
      } else {
#pragma unroll
        for (int r = 0; r < 5; ++r) gyn[r] = rhs[r];
      }
      out[0] = gyn[0];
      out[1] = gyn[1];
      out[3] = gyn[2];
      out[4] = gyn[3];
      out[5] = gyn[4];
      if (ph == phase_id) {
        // P^T sigma = -psi_y; dR/dE = psi_y / E, dR/dsigma0 = phi_v / sigma0 = P^T sigma / sigma0,
        // dR/dn = P^T sigma (-ln(s/edot0) / n^2); dsigma/dE|_y = sigma / E
        double bP = 0.0, aS = 0.0;
#pragma unroll
        for (int r = 0; r < 5; ++r) bP -= b5[r] * psy[r];
#pragma unroll
        for (int c = 0; c < 6; ++c) aS += a[c] * sig[c];
        const double qv = (4.0 / 3.0) * (v[0] * v[0] + v[1] * v[1] + v[0] * v[1]) +
                          (1.0 / 3.0) * (v[2] * v[2] + v[3] * v[3] + v[4] * v[4]);
        const double logt = qv > 0.0 ? 0.5 * log(qv) - log(th.edot0) : 0.0;
        acc[0] += (aS + bP) / th.E;
        acc[1] += -bP / th.sigma0;
        acc[2] += bP * logt / (th.n * th.n);
      }
    }
#pragma unroll
    for (int c = 0; c < 6; ++c) g_z_prev[c * nvox + i] = out[c];
  }
  block_sum<3>(acc, partials, gridDim.x);
}

// ---------------------------------------------- conjugate gradients (adjoint)
// The adjoint equilibrium G (C_t lam) = G a_u on compatible zero-mean strain
// fields, with G the Green operator of the reference C0 = identity (lam0 =
// 0, mu0 = 1/2), which is the orthogonal projector onto those fields in the
// tensor inner product X : Y, is symmetric positive definite there (C_t is
// SPD, Theorem 1); conjugate gradients need about the square root of the
// basic scheme's iterations.  On strain-like Voigt vectors (engineering
// shears) X : Y = sum of the normal products + half the shear products.

// out = C_t x (stress-like, tensor shears) for a strain-like x.
__global__ void adj_ct_apply_kernel(int64_t nvox, const double* __restrict__ Ct21, const double* __restrict__ x,
                                    double* __restrict__ out) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nvox; i += stride) {
    double l[6], C[6][6];
#pragma unroll
    for (int c = 0; c < 6; ++c) l[c] = x[c * nvox + i];
    int q = 0;
#pragma unroll
    for (int r = 0; r < 6; ++r)
#pragma unroll
      for (int c = r; c < 6; ++c) {
        const double v = Ct21[(q++) * nvox + i];
        C[r][c] = v;
        C[c][r] = v;
      }
#pragma unroll
    for (int r = 0; r < 6; ++r) {
      double acc = 0.0;
#pragma unroll
      for (int c = 0; c < 6; ++c) acc += C[r][c] * l[c];
      out[r * nvox + i] = acc;
    }
  }
}

// Block-wide fixed-order sum; thread 0 writes part[blockIdx.x].
__device__ void cg_block_sum(double v, double* __restrict__ part) {
  __shared__ double sh[kAdjBlock / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kAdjBlock / 32; ++w) s += sh[w];
    part[blockIdx.x] = s;
  }
}

// part[block] = block's share of x : (ys y) for strain-like x, y.
__global__ void __launch_bounds__(kAdjBlock) cg_dot_kernel(int64_t nvox, const double* __restrict__ x,
                                                           const double* __restrict__ y, double ys,
                                                           double* __restrict__ part) {
  double acc = 0.0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nvox; i += stride) {
#pragma unroll
    for (int c = 0; c < 6; ++c) acc += (c < 3 ? 1.0 : 0.5) * x[c * nvox + i] * (ys * y[c * nvox + i]);
  }
  cg_block_sum(acc, part);
}

// lam += a p, r -= a (qs q); part[block] = block's share of r : r.
__global__ void __launch_bounds__(kAdjBlock) cg_update_kernel(int64_t nvox, double a, double qs,
                                                              const double* __restrict__ p,
                                                              const double* __restrict__ q, double* __restrict__ lam,
                                                              double* __restrict__ r, double* __restrict__ part) {
  double acc = 0.0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nvox; i += stride) {
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      const int64_t k = c * nvox + i;
      lam[k] += a * p[k];
      const double rn = r[k] - a * (qs * q[k]);
      r[k] = rn;
      acc += (c < 3 ? 1.0 : 0.5) * rn * rn;
    }
  }
  cg_block_sum(acc, part);
}

// p = r + b p.
__global__ void cg_direction_kernel(int64_t n, double b, const double* __restrict__ r, double* __restrict__ p) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) p[i] = r[i] + b * p[i];
}

__global__ void adj_sum_kernel(const double* __restrict__ partials, int n, double* __restrict__ out) {
  const int t = threadIdx.x;
  if (t < 3) {
    double s = 0.0;
    for (int b = 0; b < n; ++b) s += partials[t * n + b];
    out[t] = s;
  }
}

}  // namespace
}  // namespace gsm
