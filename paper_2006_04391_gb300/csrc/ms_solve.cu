// Moulinec-Suquet basic scheme driving the GSM update (AutoMat, arXiv
// 2006.04391: Sec. 1 and Sec. 3 "Material Law Evaluations" -- fixed reference
// stiffness, one material evaluation without tangent per voxel and
// iteration).  The paper ran this solver on the CPU; here every step runs on
// the GPU and the fields stay resident in HBM:
//
//   material kernel   sigma, z = law(eps_raw / N^3, z_n)   + FP64 partial sums of sigma
//   cuFFT R2C (x6)    sigma -> sig_hat
//   gamma kernel      per mode: q = sig_hat k, residual partial sums (FP64),
//                     eps_hat -= Gamma0(k) : sig_hat, and a copy of eps_hat
//                     into sig_hat's buffer for the inverse transform
//   finalize kernel   fixed-order sums -> e and <sigma> (FP64), 1 value to host
//   cuFFT C2R (x6)    eps_hat copy -> eps_raw (unnormalised: N^3 eps)
//
// The C2R output is never normalised in a separate pass: the material kernel
// scales it by 1/N^3 as it loads it.  cuFFT may overwrite the input of a
// multi-dimensional C2R, which is why the gamma kernel writes the updated
// eps_hat twice (state and transform input).
//
// Green operator of the isotropic reference medium (lambda0, mu0), applied to
// a symmetric tau with q = tau k (homogeneous of degree 0 in k):
//   (Gamma0 : tau)_ij = (k_j q_i + k_i q_j) / (2 mu0 |k|^2)
//                       - (lambda0 + mu0) / (mu0 (lambda0 + 2 mu0)) (k.q) k_i k_j / |k|^4.
// Even N: a mode with the Nyquist index N/2 together with any other nonzero
// index has no Hermitian-consistent Gamma0; it gets Gamma0 := 0 and is left
// out of the equilibrium error.  Pure-axis Nyquist modes keep the operator.
#include <cufft.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "common.cuh"
#include "voxel.cuh"

namespace gsm {

int material_update(const Material& m, int64_t n, const void* eps, const void* zn, int64_t ld, double h,
                    void* sig, void* z, void* tan, int32_t* status, cudaStream_t s);

namespace {

constexpr int kMaxPhases = 16;
constexpr int kMatBlock = 128;
constexpr int kGamBlock = 256;
constexpr double kTwoPi = 6.283185307179586476925286766559;

struct PhaseTable {
  int kind[kMaxPhases];  // GSM_PSI_* of each phase
  LawParams<double> p64[kMaxPhases];
  LawParams<float> p32[kMaxPhases];
};

template <class T> struct cplx;
template <> struct cplx<double> { using type = cufftDoubleComplex; };
template <> struct cplx<float> { using type = cufftComplex; };

// ------------------------------------------------------------------ kernels

// Block-wide deterministic sum of 6 FP64 values (fixed shuffle order).
template <int NV>
__device__ void block_sum(double (&v)[NV], double* out, int64_t out_stride) {
  __shared__ double sh[NV][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < NV; ++c)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[c] += __shfl_down_sync(0xffffffffu, v[c], o);
  if (lane == 0)
#pragma unroll
    for (int c = 0; c < NV; ++c) sh[c][warp] = v[c];
  __syncthreads();
  if (threadIdx.x == 0) {
    const int nw = blockDim.x >> 5;
#pragma unroll
    for (int c = 0; c < NV; ++c) {
      double s = 0.0;
      for (int w = 0; w < nw; ++w) s += sh[c][w];
      out[c * out_stride + blockIdx.x] = s;
    }
  }
}

// Material evaluation of every voxel.  T = field type; MODE = MODE_FP64 or MODE_FP32.
template <class T, int MODE>
__global__ void __launch_bounds__(kMatBlock) ms_material_kernel(int64_t nvox, const uint8_t* __restrict__ phase,
                                                                PhaseTable tab, double h, double inv_n3,
                                                                const T* __restrict__ eps_raw,
                                                                const T* __restrict__ zn, T* __restrict__ sig,
                                                                T* __restrict__ z, double* __restrict__ partials) {
  double acc[6] = {0, 0, 0, 0, 0, 0};
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < nvox; base += stride) {
    const int64_t i = base + threadIdx.x;
    const bool in = i < nvox;
    const int ph = in ? (int)phase[i] : 0;
    const bool vp = in && tab.kind[ph] == GSM_PSI_ELASTIC_VP_DEV;
    T e[6], zi[6], s[6], zo[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      e[c] = in ? (T)((double)__ldg(eps_raw + c * nvox + i) * inv_n3) : T(0);
      zi[c] = vp ? __ldg(zn + c * nvox + i) : T(0);
    }
    // every lane enters the solver so that the warp votes see all 32 lanes
    if constexpr (MODE == MODE_FP64) {
      voxel_fp64<NortonDev>(tab.p64[ph], e, zi, h, vp, s, zo, nullptr);
    } else {
      voxel_fp32<NortonDev>(tab.p32[ph], e, zi, (float)h, vp, s, zo, nullptr);
    }
    if (in && !vp) {
      if constexpr (MODE == MODE_FP64) voxel_elastic<double>(tab.p64[ph], e, s, nullptr);
      else voxel_elastic<float>(tab.p32[ph], e, s, nullptr);
#pragma unroll
      for (int c = 0; c < 6; ++c) zo[c] = T(0);
    }
    if (in) {
#pragma unroll
      for (int c = 0; c < 6; ++c) {
        sig[c * nvox + i] = s[c];
        z[c * nvox + i] = zo[c];
        acc[c] += (double)s[c];
      }
    }
  }
  block_sum<6>(acc, partials, gridDim.x);
}

// Mode (a, b, c) of the half spectrum -> signed integer frequency.
__device__ __forceinline__ int freq(int a, int N) { return a < (N + 1) / 2 ? a : a - N; }

// Fused Green-operator application, equilibrium-error partial sums and copy
// of the updated strain spectrum into the inverse-transform input.
template <class T>
__global__ void __launch_bounds__(kGamBlock) ms_gamma_kernel(int N, double lam0, double mu0,
                                                             typename cplx<T>::type* __restrict__ sig_hat,
                                                             typename cplx<T>::type* __restrict__ eps_hat,
                                                             int64_t nmodes, double* __restrict__ partials) {
  using C = typename cplx<T>::type;
  const int Nh = N / 2 + 1;
  const bool even = (N % 2) == 0;
  const double inv2mu = 1.0 / (2.0 * mu0);
  const double coef = (lam0 + mu0) / (mu0 * (lam0 + 2.0 * mu0));
  double res = 0.0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < nmodes; m += stride) {
    const int c = (int)(m % Nh);
    const int64_t ab = m / Nh;
    const int b = (int)(ab % N);
    const int a = (int)(ab / N);
    const int kx = freq(a, N), ky = freq(b, N), kz = c;
    const int nz = (kx != 0) + (ky != 0) + (kz != 0);
    const bool nyq = even && (a == N / 2 || b == N / 2 || c == N / 2);
    const bool skip = nz == 0 || (nyq && nz >= 2);
    C s[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) s[q] = sig_hat[q * nmodes + m];
    if (skip) {
      // Gamma0 = 0: eps_hat unchanged; the transform input gets eps_hat
#pragma unroll
      for (int q = 0; q < 6; ++q) sig_hat[q * nmodes + m] = eps_hat[q * nmodes + m];
      continue;
    }
    // Arithmetic in the field precision T; the error sum accumulates in FP64.
    const T k1 = (T)kx, k2 = (T)ky, k3 = (T)kz;
    // q = sigma k (Voigt 11,22,33,23,13,12; tensor shears)
    T qr[3], qi[3];
    qr[0] = s[0].x * k1 + s[5].x * k2 + s[4].x * k3;
    qi[0] = s[0].y * k1 + s[5].y * k2 + s[4].y * k3;
    qr[1] = s[5].x * k1 + s[1].x * k2 + s[3].x * k3;
    qi[1] = s[5].y * k1 + s[1].y * k2 + s[3].y * k3;
    qr[2] = s[4].x * k1 + s[3].x * k2 + s[2].x * k3;
    qi[2] = s[4].y * k1 + s[3].y * k2 + s[2].y * k3;
    const double w = (c == 0 || (even && c == N / 2)) ? 1.0 : 2.0;
    res += w * ((double)(qr[0] * qr[0] + qi[0] * qi[0]) + (double)(qr[1] * qr[1] + qi[1] * qi[1]) +
                (double)(qr[2] * qr[2] + qi[2] * qi[2]));
    const T kk = k1 * k1 + k2 * k2 + k3 * k3;
    const T ik2 = T(1) / kk;
    const T a1 = (T)inv2mu * ik2;
    const T a2 = (T)coef * ik2 * ik2;
    const T kqr = k1 * qr[0] + k2 * qr[1] + k3 * qr[2];
    const T kqi = k1 * qi[0] + k2 * qi[1] + k3 * qi[2];
    const T kv[3] = {k1, k2, k3};
    const int ii[6] = {0, 1, 2, 1, 0, 0}, jj[6] = {0, 1, 2, 2, 2, 1};
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      const int i = ii[q], j = jj[q];
      const T f = q < 3 ? T(1) : T(2);  // engineering shears for strain
      const T dr = f * (a1 * (kv[j] * qr[i] + kv[i] * qr[j]) - a2 * kqr * kv[i] * kv[j]);
      const T di = f * (a1 * (kv[j] * qi[i] + kv[i] * qi[j]) - a2 * kqi * kv[i] * kv[j]);
      C e = eps_hat[q * nmodes + m];
      e.x -= dr;
      e.y -= di;
      eps_hat[q * nmodes + m] = e;
      sig_hat[q * nmodes + m] = e;
    }
  }
  double v[1] = {res};
  block_sum<1>(v, partials, gridDim.x);
}

struct Reduced {
  double e;        // equilibrium error
  double mean[6];  // <sigma>
  double res;      // sum |xi . c|^2
};

// Fixed-order final sums of the block partials.
__global__ void ms_finalize_kernel(const double* __restrict__ mat_part, int n_mat, const double* __restrict__ gam_part,
                                   int n_gam, double inv_n3, double floor_, Reduced* __restrict__ out) {
  __shared__ double sh[7];
  const int t = threadIdx.x;
  if (t < 7) {
    double s = 0.0;
    if (t < 6)
      for (int b = 0; b < n_mat; ++b) s += mat_part[t * n_mat + b];
    else
      for (int b = 0; b < n_gam; ++b) s += gam_part[b];
    sh[t] = s;
  }
  __syncthreads();
  if (t == 0) {
    double m[6];
    for (int c = 0; c < 6; ++c) m[c] = sh[c] * inv_n3;
    // sum |xi . c|^2 with xi = 2 pi k and c = sigma^ / N^3
    const double num = sqrt(sh[6]) * kTwoPi * inv_n3;
    const double fro = sqrt(m[0] * m[0] + m[1] * m[1] + m[2] * m[2] + 2.0 * (m[3] * m[3] + m[4] * m[4] + m[5] * m[5]));
    out->e = num / fmax(fro, floor_);
    for (int c = 0; c < 6; ++c) out->mean[c] = m[c];
    out->res = sh[6];
  }
}

// eps_raw += N^3 dE (uniform macro-strain increment at a step start).
template <class T>
__global__ void ms_add_uniform_kernel(int64_t nvox, T* __restrict__ eps_raw, double d0, double d1, double d2,
                                      double d3, double d4, double d5) {
  const double d[6] = {d0, d1, d2, d3, d4, d5};
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nvox; i += stride)
#pragma unroll
    for (int c = 0; c < 6; ++c) eps_raw[c * nvox + i] = (T)((double)eps_raw[c * nvox + i] + d[c]);
}

// eps_hat = R2C(eps_raw) / N^3 with the mean mode set to N^3 E exactly.
template <class T>
__global__ void ms_spectrum_init_kernel(int64_t nmodes, const typename cplx<T>::type* __restrict__ raw_hat,
                                        typename cplx<T>::type* __restrict__ eps_hat, double inv_n3, double n3,
                                        double E0, double E1, double E2, double E3, double E4, double E5) {
  const double E[6] = {E0, E1, E2, E3, E4, E5};
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < nmodes; m += stride) {
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      typename cplx<T>::type v = raw_hat[q * nmodes + m];
      if (m == 0) {
        v.x = (T)(n3 * E[q]);
        v.y = T(0);
      } else {
        v.x = (T)((double)v.x * inv_n3);
        v.y = (T)((double)v.y * inv_n3);
      }
      eps_hat[q * nmodes + m] = v;
    }
  }
}

// Precision conversion / scaling: dst = src * scale.
template <class S, class D>
__global__ void ms_convert_kernel(int64_t n, const S* __restrict__ src, D* __restrict__ dst, double scale) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    dst[i] = (D)((double)src[i] * scale);
}

int grid_cap(int64_t n, int block, int per_sm) {
  const int64_t need = (n + block - 1) / block;
  const int64_t cap = (int64_t)sm_count() * per_sm;
  return (int)std::max<int64_t>(1, std::min(need, cap));
}

// ---------------------------------------------------------- field buffers

template <class T> struct Fields {
  using C = typename cplx<T>::type;
  T* eps_raw = nullptr;  // [6][nvox] unnormalised strain (C2R output)
  T* zn = nullptr;       // [6][nvox] internal variables at t_n (FP32 copy in bulk mode)
  T* sig = nullptr;      // [6][nvox]
  T* z = nullptr;        // [6][nvox]
  C* sig_hat = nullptr;  // [6][nmodes] (also the C2R input)
  C* eps_hat = nullptr;  // [6][nmodes]
  cufftHandle r2c = 0, c2r = 0;
  bool planned = false;
};

template <class T> size_t field_bytes(int64_t nvox, int64_t nmodes) {
  return 4 * 6 * nvox * sizeof(T) + 2 * 6 * nmodes * sizeof(typename cplx<T>::type);
}

}  // namespace

struct MsContext {
  int N = 0;
  int64_t nvox = 0, nmodes = 0;
  int precision = MS_PREC_FP64;
  const uint8_t* phase = nullptr;
  int n_phases = 0;
  PhaseTable tab;
  double lam0 = 0, mu0 = 0;
  cudaStream_t stream = nullptr;
  Fields<double> f64;
  Fields<float> f32;
  double* mat_part = nullptr;
  double* gam_part = nullptr;
  Reduced* red_dev = nullptr;
  Reduced* red_host = nullptr;
  int mat_grid64 = 0, mat_grid32 = 0, gam_grid = 0, elt_grid = 0;
  double E_prev[6] = {0, 0, 0, 0, 0, 0};
  bool have_state = false;
};

namespace {

template <class T> cufftType r2c_type();
template <> cufftType r2c_type<double>() { return CUFFT_D2Z; }
template <> cufftType r2c_type<float>() { return CUFFT_R2C; }
template <class T> cufftType c2r_type();
template <> cufftType c2r_type<double>() { return CUFFT_Z2D; }
template <> cufftType c2r_type<float>() { return CUFFT_C2R; }

template <class T> int plan_fields(MsContext& c, Fields<T>& f) {
  int n[3] = {c.N, c.N, c.N};
  const int64_t nv = c.nvox, nm = c.nmodes;
  if (cufftPlanMany(&f.r2c, 3, n, nullptr, 1, (int)nv, nullptr, 1, (int)nm, r2c_type<T>(), 6) != CUFFT_SUCCESS)
    return GSM_ECUDA;
  if (cufftPlanMany(&f.c2r, 3, n, nullptr, 1, (int)nm, nullptr, 1, (int)nv, c2r_type<T>(), 6) != CUFFT_SUCCESS)
    return GSM_ECUDA;
  cufftSetStream(f.r2c, c.stream);
  cufftSetStream(f.c2r, c.stream);
  f.planned = true;
  auto alloc = [](void** p, size_t b) { return cudaMalloc(p, b) == cudaSuccess; };
  bool ok = alloc((void**)&f.eps_raw, 6 * nv * sizeof(T)) && alloc((void**)&f.zn, 6 * nv * sizeof(T)) &&
            alloc((void**)&f.sig, 6 * nv * sizeof(T)) && alloc((void**)&f.z, 6 * nv * sizeof(T)) &&
            alloc((void**)&f.sig_hat, 6 * nm * sizeof(typename Fields<T>::C)) &&
            alloc((void**)&f.eps_hat, 6 * nm * sizeof(typename Fields<T>::C));
  return ok ? GSM_OK : GSM_ENOMEM;
}

template <class T> void free_fields(Fields<T>& f) {
  cudaFree(f.eps_raw);
  cudaFree(f.zn);
  cudaFree(f.sig);
  cudaFree(f.z);
  cudaFree(f.sig_hat);
  cudaFree(f.eps_hat);
  if (f.planned) {
    cufftDestroy(f.r2c);
    cufftDestroy(f.c2r);
  }
  f = Fields<T>();
}

cufftResult exec_r2c(Fields<double>& f, double* in, cufftDoubleComplex* out) { return cufftExecD2Z(f.r2c, in, out); }
cufftResult exec_r2c(Fields<float>& f, float* in, cufftComplex* out) { return cufftExecR2C(f.r2c, in, out); }
cufftResult exec_c2r(Fields<double>& f, cufftDoubleComplex* in, double* out) { return cufftExecZ2D(f.c2r, in, out); }
cufftResult exec_c2r(Fields<float>& f, cufftComplex* in, float* out) { return cufftExecC2R(f.c2r, in, out); }

template <class T> Fields<T>& fields(MsContext& c);
template <> Fields<double>& fields<double>(MsContext& c) { return c.f64; }
template <> Fields<float>& fields<float>(MsContext& c) { return c.f32; }

// Step start in precision T: eps_raw += N^3 (E - E_prev); eps_hat = spectrum of eps with mean N^3 E.
template <class T> int step_start(MsContext& c, const double* E, const double* E_prev) {
  Fields<T>& f = fields<T>(c);
  const double n3 = (double)c.nvox;
  double d[6];
  for (int q = 0; q < 6; ++q) d[q] = n3 * (E[q] - E_prev[q]);
  ms_add_uniform_kernel<T><<<c.elt_grid, 256, 0, c.stream>>>(c.nvox, f.eps_raw, d[0], d[1], d[2], d[3], d[4], d[5]);
  count_launch();
  if (exec_r2c(f, f.eps_raw, f.sig_hat) != CUFFT_SUCCESS) return GSM_ECUDA;
  ms_spectrum_init_kernel<T><<<c.elt_grid, 256, 0, c.stream>>>(c.nmodes, f.sig_hat, f.eps_hat, 1.0 / n3, n3, E[0],
                                                                E[1], E[2], E[3], E[4], E[5]);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? GSM_OK : GSM_ECUDA;
}

// One iteration's evaluation half: material, forward FFT, gamma + residual, finalize.
template <class T> int evaluate(MsContext& c, double h) {
  Fields<T>& f = fields<T>(c);
  const double inv_n3 = 1.0 / (double)c.nvox;
  constexpr bool d = sizeof(T) == 8;
  if constexpr (d)
    ms_material_kernel<T, MODE_FP64><<<c.mat_grid64, kMatBlock, 0, c.stream>>>(
        c.nvox, c.phase, c.tab, h, inv_n3, f.eps_raw, f.zn, f.sig, f.z, c.mat_part);
  else
    ms_material_kernel<T, MODE_FP32><<<c.mat_grid32, kMatBlock, 0, c.stream>>>(
        c.nvox, c.phase, c.tab, h, inv_n3, f.eps_raw, f.zn, f.sig, f.z, c.mat_part);
  count_launch();
  if (exec_r2c(f, f.sig, f.sig_hat) != CUFFT_SUCCESS) return GSM_ECUDA;
  ms_gamma_kernel<T><<<c.gam_grid, kGamBlock, 0, c.stream>>>(c.N, c.lam0, c.mu0, f.sig_hat, f.eps_hat, c.nmodes,
                                                             c.gam_part);
  count_launch();
  ms_finalize_kernel<<<1, 32, 0, c.stream>>>(c.mat_part, d ? c.mat_grid64 : c.mat_grid32, c.gam_part, c.gam_grid,
                                             inv_n3, c.mu0 * 1e-6, c.red_dev);
  count_launch();
  cudaMemcpyAsync(c.red_host, c.red_dev, sizeof(Reduced), cudaMemcpyDeviceToHost, c.stream);
  if (cudaStreamSynchronize(c.stream) != cudaSuccess) return GSM_ECUDA;
  return cudaGetLastError() == cudaSuccess ? GSM_OK : GSM_ECUDA;
}

template <class T> int inverse(MsContext& c) {
  Fields<T>& f = fields<T>(c);
  return exec_c2r(f, f.sig_hat, f.eps_raw) == CUFFT_SUCCESS ? GSM_OK : GSM_ECUDA;
}

template <class S, class D> void convert(MsContext& c, const S* src, D* dst, int64_t n, double scale) {
  ms_convert_kernel<S, D><<<c.elt_grid, 256, 0, c.stream>>>(n, src, dst, scale);
  count_launch();
}

size_t plan_bytes(int N, bool fp32) {
  size_t total = 0;
  int n[3] = {N, N, N};
  const long long nv = (long long)N * N * N, nm = (long long)N * N * (N / 2 + 1);
  size_t ws = 0;
  if (cufftEstimateMany(3, n, nullptr, 1, (int)nv, nullptr, 1, (int)nm, CUFFT_D2Z, 6, &ws) == CUFFT_SUCCESS) total += ws;
  if (cufftEstimateMany(3, n, nullptr, 1, (int)nm, nullptr, 1, (int)nv, CUFFT_Z2D, 6, &ws) == CUFFT_SUCCESS) total += ws;
  if (fp32) {
    if (cufftEstimateMany(3, n, nullptr, 1, (int)nv, nullptr, 1, (int)nm, CUFFT_R2C, 6, &ws) == CUFFT_SUCCESS) total += ws;
    if (cufftEstimateMany(3, n, nullptr, 1, (int)nm, nullptr, 1, (int)nv, CUFFT_C2R, 6, &ws) == CUFFT_SUCCESS) total += ws;
  }
  return total;
}

void destroy(MsContext* c) {
  if (!c) return;
  free_fields(c->f64);
  free_fields(c->f32);
  cudaFree(c->mat_part);
  cudaFree(c->gam_part);
  cudaFree(c->red_dev);
  cudaFreeHost(c->red_host);
  delete c;
}

}  // namespace
}  // namespace gsm

using namespace gsm;

extern "C" {

size_t ms_workspace_bytes(const ms_problem* prob) {
  if (!prob || prob->N < 2 || prob->N > 1024) return 0;
  const int N = prob->N;
  const int64_t nv = (int64_t)N * N * N, nm = (int64_t)N * N * (N / 2 + 1);
  const bool fp32 = prob->precision == MS_PREC_FP32_BULK;
  size_t b = field_bytes<double>(nv, nm) + (fp32 ? field_bytes<float>(nv, nm) : 0);
  b += plan_bytes(N, fp32);
  b += (size_t)(6 + 1) * 4096 * sizeof(double) + sizeof(Reduced);
  return b;
}

int ms_create(ms_handle* out, const ms_problem* prob, void* stream) {
  if (!out || !prob) return GSM_EINVAL;
  *out = nullptr;
  if (prob->N < 2 || prob->N > 1024 || !prob->phase || prob->n_phases < 1 || prob->n_phases > kMaxPhases ||
      !prob->laws || (prob->precision != MS_PREC_FP64 && prob->precision != MS_PREC_FP32_BULK))
    return GSM_EINVAL;
  const int64_t N = prob->N;
  if (N * N * N > (int64_t)INT32_MAX / 6) return GSM_EINVAL;  // cuFFT batch distances are int
  MsContext* c = new (std::nothrow) MsContext;
  if (!c) return GSM_ENOMEM;
  c->N = prob->N;
  c->nvox = N * N * N;
  c->nmodes = N * N * (N / 2 + 1);
  c->precision = prob->precision;
  c->phase = prob->phase;
  c->n_phases = prob->n_phases;
  c->stream = static_cast<cudaStream_t>(stream);
  std::memset(&c->tab, 0, sizeof(c->tab));
  double lam_min = 1e300, lam_max = -1e300, mu_min = 1e300, mu_max = -1e300;
  for (int p = 0; p < prob->n_phases; ++p) {
    const Material* m = reinterpret_cast<const Material*>(prob->laws[p]);
    if (!m) { delete c; return GSM_EINVAL; }
    c->tab.kind[p] = m->psi_kind;
    c->tab.p64[p] = m->p64;
    c->tab.p32[p] = m->p32;
    lam_min = std::min(lam_min, m->p64.lam);
    lam_max = std::max(lam_max, m->p64.lam);
    mu_min = std::min(mu_min, m->p64.mu);
    mu_max = std::max(mu_max, m->p64.mu);
  }
  c->lam0 = 0.5 * (lam_min + lam_max);
  c->mu0 = 0.5 * (mu_min + mu_max);

  int per = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, ms_material_kernel<double, MODE_FP64>, kMatBlock, 0);
  c->mat_grid64 = std::min(grid_cap(c->nvox, kMatBlock, std::max(per, 1)), 4096);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, ms_material_kernel<float, MODE_FP32>, kMatBlock, 0);
  c->mat_grid32 = std::min(grid_cap(c->nvox, kMatBlock, std::max(per, 1)), 4096);
  c->gam_grid = std::min(grid_cap(c->nmodes, kGamBlock, 8), 4096);
  c->elt_grid = grid_cap(c->nvox, 256, 8);

  int rc = plan_fields<double>(*c, c->f64);
  if (rc == GSM_OK && c->precision == MS_PREC_FP32_BULK) rc = plan_fields<float>(*c, c->f32);
  if (rc == GSM_OK) {
    bool ok = cudaMalloc((void**)&c->mat_part, 6 * 4096 * sizeof(double)) == cudaSuccess &&
              cudaMalloc((void**)&c->gam_part, 4096 * sizeof(double)) == cudaSuccess &&
              cudaMalloc((void**)&c->red_dev, sizeof(Reduced)) == cudaSuccess &&
              cudaMallocHost((void**)&c->red_host, sizeof(Reduced)) == cudaSuccess;
    if (!ok) rc = GSM_ENOMEM;
  }
  if (rc != GSM_OK) {
    cudaGetLastError();
    destroy(c);
    return rc;
  }
  *out = reinterpret_cast<ms_handle>(c);
  return GSM_OK;
}

int ms_destroy(ms_handle h) {
  if (h) {
    MsContext* c = reinterpret_cast<MsContext*>(h);
    cudaStreamSynchronize(c->stream);
    destroy(c);
  }
  return GSM_OK;
}

int ms_run(ms_handle h, const ms_load* load, ms_state* state, ms_result* result) {
  if (!h || !load || !result || load->n_steps < 1 || !load->E || !load->h || load->max_iter < 1 ||
      !result->Sigma || !result->iters || !result->final_error)
    return GSM_EINVAL;
  for (int k = 0; k < load->n_steps; ++k)
    if (!(std::isfinite(load->h[k]) && load->h[k] > 0.0)) return GSM_EINVAL;
  if (load->forced_iters)
    for (int k = 0; k < load->n_steps; ++k)
      if (load->forced_iters[k] < 1) return GSM_EINVAL;
  MsContext& c = *reinterpret_cast<MsContext*>(h);
  const int64_t n6 = 6 * c.nvox;
  const double n3 = (double)c.nvox;
  Fields<double>& F = c.f64;
  Fields<float>& H = c.f32;
  const bool bulk32 = c.precision == MS_PREC_FP32_BULK;
  const double switch_tol = load->switch_tol > 0.0 ? load->switch_tol : 1e-5;

  // initial state
  double E_prev[6] = {0, 0, 0, 0, 0, 0};
  if (state && state->resume) {
    if (!state->eps || !state->z) return GSM_EINVAL;
    convert<double, double>(c, state->eps, F.eps_raw, n6, n3);
    cudaMemcpyAsync(F.zn, state->z, n6 * sizeof(double), cudaMemcpyDeviceToDevice, c.stream);
    for (int q = 0; q < 6; ++q) E_prev[q] = state->E_prev[q];
  } else {
    cudaMemsetAsync(F.eps_raw, 0, n6 * sizeof(double), c.stream);
    cudaMemsetAsync(F.zn, 0, n6 * sizeof(double), c.stream);
  }
  int rc_all = GSM_OK;
  result->total_iters = 0;
  for (int k = 0; k < load->n_steps; ++k) {
    const double* E = load->E + 6 * k;
    const double hk = load->h[k];
    const int forced = load->forced_iters ? load->forced_iters[k] : 0;
    const int cap = forced ? forced : load->max_iter;
    int n_eval = 0, n32 = 0;
    bool converged = false;
    int rc = GSM_OK;

    if (bulk32) {
      // FP32 phase from the FP64 state
      convert<double, float>(c, F.eps_raw, H.eps_raw, n6, 1.0);
      convert<double, float>(c, F.zn, H.zn, n6, 1.0);
      rc = step_start<float>(c, E, E_prev);
      double best = 1e300;
      int since_best = 0;
      // leave at least one evaluation for the FP64 phase
      while (rc == GSM_OK && n_eval < cap - 1) {
        rc = evaluate<float>(c, hk);
        if (rc != GSM_OK) break;
        ++n_eval;
        ++n32;
        const double e = c.red_host->e;
        if (e < best * 0.999) { best = e; since_best = 0; } else { ++since_best; }
        if (e < std::max(switch_tol, load->tol) || since_best >= 20 || n_eval >= cap - 1) break;
        rc = inverse<float>(c);
      }
      // hand the FP32 strain (eps_raw of the last evaluation) to FP64
      if (rc == GSM_OK) {
        convert<float, double>(c, H.eps_raw, F.eps_raw, n6, 1.0);
        rc = step_start<double>(c, E, E);  // no increment: already at E_k
        // resynthesise the FP64 strain from the spectrum so that its mean is E_k exactly
        if (rc == GSM_OK) {
          cudaMemcpyAsync(F.sig_hat, F.eps_hat, 6 * c.nmodes * sizeof(cufftDoubleComplex), cudaMemcpyDeviceToDevice,
                          c.stream);
          rc = inverse<double>(c);
        }
      }
    } else {
      rc = step_start<double>(c, E, E_prev);
    }
    while (rc == GSM_OK && n_eval < cap) {
      rc = evaluate<double>(c, hk);
      if (rc != GSM_OK) break;
      ++n_eval;
      const double e = c.red_host->e;
      if (forced) {
        if (n_eval >= forced) { converged = true; break; }
      } else if (e < load->tol) {
        converged = true;
        break;
      }
      if (n_eval >= cap) break;
      rc = inverse<double>(c);
    }
    if (rc != GSM_OK) return rc;
    if (!converged) rc_all = GSM_ENOTCONV;
    // step end: z_n <- z (swap), Sigma_k = <sigma>
    std::swap(F.zn, F.z);
    for (int q = 0; q < 6; ++q) {
      result->Sigma[6 * k + q] = c.red_host->mean[q];
      E_prev[q] = E[q];
    }
    result->iters[k] = n_eval;
    result->final_error[k] = c.red_host->e;
    if (result->fp32_iters) result->fp32_iters[k] = n32;
    result->total_iters += n_eval;
  }
  if (state && state->eps && state->z) {
    convert<double, double>(c, F.eps_raw, state->eps, n6, 1.0 / n3);
    cudaMemcpyAsync(state->z, F.zn, n6 * sizeof(double), cudaMemcpyDeviceToDevice, c.stream);
    for (int q = 0; q < 6; ++q) state->E_prev[q] = E_prev[q];
  }
  if (cudaStreamSynchronize(c.stream) != cudaSuccess) return GSM_ECUDA;
  return rc_all;
}

int ms_solve(const ms_problem* prob, const ms_load* load, ms_state* state, ms_result* result, void* stream) {
  ms_handle h = nullptr;
  int rc = ms_create(&h, prob, stream);
  if (rc != GSM_OK) return rc;
  rc = ms_run(h, load, state, result);
  ms_destroy(h);
  return rc;
}

}  // extern "C"

// ===================================================== allocation-free variant
// ms_evaluate_noalloc: one material evaluation of a microstructure plus its
// FP64 mean stress, for callers that cannot allocate device memory (a process
// whose device memory is owned by another allocator, or code running where a
// cudaMalloc would be illegal or would synchronise).  It runs the same kernel
// as the basic scheme's material step (ms_material_kernel, FP64) and the same
// fixed-order reduction, but its block partial sums live in the file-scope
// array below instead of a context's workspace.
//
// The array is part of the library's device image: every GPU that loads the
// library holds it (48 KB + 64 B) until the process exits.  In host code its
// name is only a stand-in, so its device address is fetched once per device
// with cudaGetSymbolAddress and passed to the kernels.  All calls share the
// array: two calls whose work overlaps on the GPU (different streams, or
// different host threads) race on it.  Each block writes its own partial sum
// before the reduction reads it, so nothing has to be cleared between calls.
static constexpr int kNoAllocMaxBlocks = 1024;
static __device__ __align__(256) double g_ms_eval_scratch[6 * kNoAllocMaxBlocks + 8];

namespace gsm {
namespace {

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
double* g_noalloc_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (set up on the
// first call per device).
int noalloc_scratch(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return GSM_ECUDA;
  if (dev < 0 || dev >= kMaxDevices) return GSM_ENOTSUP;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_ms_eval_scratch) != cudaSuccess || !p) return GSM_ECUDA;
    g_noalloc_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return GSM_OK;
}

}  // namespace
}  // namespace gsm

extern "C" int ms_evaluate_noalloc(int N, const uint8_t* phase, int n_phases, const gsm_handle* laws, double step_h,
                                   const double* eps, const double* z_n, double* sigma, double* z, double* mean,
                                   void* stream) {
  using namespace gsm;
  if (N < 2 || N > 1024 || !phase || n_phases < 1 || n_phases > kMaxPhases || !laws || !eps || !z_n || !sigma ||
      !z || !mean || !(std::isfinite(step_h) && step_h > 0.0))
    return GSM_EINVAL;
  PhaseTable tab;
  std::memset(&tab, 0, sizeof(tab));
  for (int p = 0; p < n_phases; ++p) {
    const Material* m = reinterpret_cast<const Material*>(laws[p]);
    if (!m) return GSM_EINVAL;
    tab.kind[p] = m->psi_kind;
    tab.p64[p] = m->p64;
    tab.p32[p] = m->p32;
  }
  double* scratch = nullptr;
  int rc = noalloc_scratch(&scratch);
  if (rc != GSM_OK) return rc;
  const int64_t nvox = (int64_t)N * N * N;
  static int per_sm = 0;
  if (per_sm == 0) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, ms_material_kernel<double, MODE_FP64>, kMatBlock, 0) !=
            cudaSuccess ||
        b <= 0)
      b = 1;
    per_sm = b;
  }
  const int grid = std::min(grid_cap(nvox, kMatBlock, per_sm), kNoAllocMaxBlocks);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double* partials = scratch;                                    // [6][grid]
  Reduced* red = reinterpret_cast<Reduced*>(scratch + 6 * kNoAllocMaxBlocks);
  ms_material_kernel<double, MODE_FP64><<<grid, kMatBlock, 0, s>>>(nvox, phase, tab, step_h, 1.0, eps, z_n, sigma, z,
                                                                   partials);
  ms_finalize_kernel<<<1, 32, 0, s>>>(partials, grid, nullptr, 0, 1.0 / (double)nvox, 1.0, red);
  count_launch(2);
  if (cudaGetLastError() != cudaSuccess) return GSM_ECUDA;
  if (cudaMemcpyAsync(mean, red->mean, 6 * sizeof(double), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return GSM_ECUDA;
  return GSM_OK;
}
