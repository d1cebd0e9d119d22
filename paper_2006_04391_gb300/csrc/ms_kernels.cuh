// Device kernels of the Moulinec-Suquet basic scheme (AutoMat, arXiv
// 2006.04391: Sec. 1 and Sec. 3 "Material Law Evaluations").  Included by
// ms_solve.cu and (for the job views and block reductions) ms_ode.cu.
//
// Every kernel works on a batch of independent problems ("jobs") at once: a
// job's voxels (modes) are cut into fixed chunks of kVChunk (kMChunk), the
// chunks of all jobs in a launch are numbered consecutively, and each block
// walks the global chunk list.  Partial sums are written per chunk and summed
// per job in chunk order, so a job's results are bit-identical whether it
// runs alone or in a batch.  A single basic-scheme solve is a batch of one.
//
// Green operator of the isotropic reference medium (lambda0, mu0), applied to
// a symmetric tau with q = tau k (homogeneous of degree 0 in k):
//   (Gamma0 : tau)_ij = (k_j q_i + k_i q_j) / (2 mu0 |k|^2)
//                       - (lambda0 + mu0) / (mu0 (lambda0 + 2 mu0)) (k.q) k_i k_j / |k|^4.
// Even N: a mode with the Nyquist index N/2 together with any other nonzero
// index has no Hermitian-consistent Gamma0; it gets Gamma0 := 0 and is left
// out of the equilibrium error.  Pure-axis Nyquist modes keep the operator.
#pragma once

#include <cufft.h>

#include "common.cuh"
#include "voxel.cuh"

namespace gsm {
namespace {

constexpr int kMaxPhases = 16;
constexpr int kMatBlock = 128;
constexpr int kGamBlock = 256;
constexpr int kVChunk = 1024;  // voxels per chunk (8 sweeps of a material block)
constexpr int kMChunk = 2048;  // modes per chunk (8 sweeps of a gamma block)
constexpr int kMaxBatch = 256; // jobs per launch
constexpr double kTwoPi = 6.283185307179586476925286766559;

struct PhaseTable {
  int kind[kMaxPhases];  // GSM_PSI_* of each phase
  LawParams<double> p64[kMaxPhases];
  LawParams<float> p32[kMaxPhases];
};

template <class T> struct cplx;
template <> struct cplx<double> { using type = cufftDoubleComplex; };
template <> struct cplx<float> { using type = cufftComplex; };

struct Reduced {
  double e;        // equilibrium error
  double mean[6];  // <sigma>
  double res;      // sum |xi . c|^2
};

// One job of a batched launch (device copy, rebuilt by the host every tick).
struct JobView {
  const uint8_t* phase;
  const void* eps_raw;   // [6][nvox] N^3 * strain (C2R output)
  const void* zn;        // [6][nvox]
  void* sig;             // [6][nvox]
  void* z;               // [6][nvox]
  void* sig_hat;         // [6][nmodes]
  void* eps_hat;         // [6][nmodes]
  double* mat_part;      // [6][n_vch]
  double* gam_part;      // [n_mch]
  const PhaseTable* tab;
  int64_t nvox, nmodes;
  int64_t vchunk0, mchunk0;  // first chunk of this job in its launch
  int n_vch, n_mch;
  int N;
  int warm;              // 1: z holds this job's previous evaluation of the current step (warm start)
  double h, inv_h, inv_n3, lam0, mu0;
  // ode23 laws (Sec. 4.3): strain at t_n, the Michel-Suquet alpha, tolerances
  const double* eps_prev;  // [6][nvox]
  const double* alpha_n;   // [nvox] or NULL
  double* alpha;           // [nvox] or NULL
  double ode_rtol, ode_atol;
  int ode_max, pad2;
};

// ------------------------------------------------------------------ helpers

// Block-wide deterministic sum of NV FP64 values (fixed shuffle order);
// thread 0 writes out[c * stride + index].  Ends with a barrier so the
// shared buffer can be reused by the next call.
template <int NV>
__device__ void block_sum_at(double (&v)[NV], double* out, int64_t stride, int64_t index) {
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
      out[c * stride + index] = s;
    }
  }
  __syncthreads();
}

template <int NV> __device__ void block_sum(double (&v)[NV], double* out, int64_t stride) {
  block_sum_at<NV>(v, out, stride, blockIdx.x);
}

// Material evaluation of voxel i.  Every lane of a warp must call this (the
// Newton loops vote warp-wide); lanes with in = false only vote.  The field
// precision T is also that of the 1/N^3 scaling and of the lane's partial
// stress sums (FP32 fields: no FP64 work, a sixty-fourth of the FP32 rate on
// GB300, outside the law; the block sums are FP64).
template <class T, int MODE>
__device__ __forceinline__ void material_voxel(int64_t i, bool in, int64_t nvox, const uint8_t* __restrict__ phase,
                                               const PhaseTable& tab, const Step& hs, T inv_n3,
                                               const T* __restrict__ eps_raw, const T* __restrict__ zn,
                                               T* __restrict__ sig, T* __restrict__ z, T (&acc)[6],
                                               bool warm = false) {
  const int ph = in ? (int)phase[i] : 0;
  const bool vp = in && tab.kind[ph] == GSM_PSI_ELASTIC_VP_DEV;
  T e[6], zi[6], s[6], zo[6], zp[6];
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    e[c] = in ? __ldg(eps_raw + c * nvox + i) * inv_n3 : T(0);
    zi[c] = vp ? __ldg(zn + c * nvox + i) : T(0);
    // warm start: this voxel's z from the previous evaluation of the step
    // (read before this evaluation overwrites it)
    zp[c] = (warm && vp) ? z[c * nvox + i] : zi[c];
  }
  const T* zprev = warm ? zp : nullptr;
  if constexpr (MODE == MODE_FP64) {
    voxel_fp64<NortonDev>(tab.p64[ph], e, zi, hs, vp, s, zo, nullptr, zprev);
  } else if constexpr (MODE == MODE_FP32_FIX) {
    voxel_fp32_fix<NortonDev>(tab.p64[ph], tab.p32[ph], e, zi, hs, vp, s, zo, nullptr, zprev);
  } else {
    voxel_fp32<NortonDev>(tab.p32[ph], e, zi, hs, vp, s, zo, nullptr, zprev);
  }
  if (in && !vp) {
    if constexpr (sizeof(T) == 8) voxel_elastic<double>(tab.p64[ph], e, s, nullptr);
    else voxel_elastic<float>(tab.p32[ph], e, s, nullptr);
#pragma unroll
    for (int c = 0; c < 6; ++c) zo[c] = T(0);
  }
  if (in) {
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      sig[c * nvox + i] = s[c];
      z[c * nvox + i] = zo[c];
      acc[c] += s[c];
    }
  }
}

// Mode (a, b, c) of the half spectrum -> signed integer frequency.
__device__ __forceinline__ int freq(int a, int N) { return a < (N + 1) / 2 ? a : a - N; }

// Green-operator update of mode m: eps_hat -= Gamma0 : sig_hat, the updated
// eps_hat copied into sig_hat (the inverse-transform input); adds the mode's
// |k . sig_hat|^2 (Hermitian weight 1 or 2) to res.  Arithmetic in the field
// precision T, the error sum in FP64.
template <class T>
__device__ __forceinline__ void gamma_mode(int N, double inv2mu, double coef, typename cplx<T>::type* __restrict__ sig_hat,
                                           typename cplx<T>::type* __restrict__ eps_hat, int64_t nmodes, int64_t m,
                                           double& res) {
  using C = typename cplx<T>::type;
  const int Nh = N / 2 + 1;
  const bool even = (N % 2) == 0;
  const int c = (int)(m % Nh);
  const int64_t ab = m / Nh;
  const int b = (int)(ab % N);
  const int a = (int)(ab / N);
  const int kx = freq(a, N), ky = freq(b, N), kz = c;
  const int nz = (kx != 0) + (ky != 0) + (kz != 0);
  const bool nyq = even && (a == N / 2 || b == N / 2 || c == N / 2);
  const bool skip = nz == 0 || (nyq && nz >= 2);
  if (skip) {
    // Gamma0 = 0: eps_hat unchanged; the transform input gets eps_hat
#pragma unroll
    for (int q = 0; q < 6; ++q) sig_hat[q * nmodes + m] = eps_hat[q * nmodes + m];
    return;
  }
  C s[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) s[q] = sig_hat[q * nmodes + m];
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

// The Green-operator update of one FP32 mode on registers: s = sig_hat, e =
// eps_hat (in/out, the updated strain spectrum); (a, b, c) its half-spectrum
// index.  Same arithmetic as gamma_mode.
__device__ __forceinline__ void gamma_mode_f32_regs(int N, int a, int b, int c, float inv2mu, float coef,
                                                    const float2 (&s)[6], float2 (&e)[6], double& res) {
  const int Nh = N / 2 + 1;
  (void)Nh;
  const bool even = (N % 2) == 0;
  const int kx = freq(a, N), ky = freq(b, N), kz = c;
  const int nz = (kx != 0) + (ky != 0) + (kz != 0);
  const bool nyq = even && (a == N / 2 || b == N / 2 || c == N / 2);
  if (nz == 0 || (nyq && nz >= 2)) return;  // Gamma0 = 0: eps_hat unchanged
  const float k1 = (float)kx, k2 = (float)ky, k3 = (float)kz;
  float qr[3], qi[3];
  qr[0] = s[0].x * k1 + s[5].x * k2 + s[4].x * k3;
  qi[0] = s[0].y * k1 + s[5].y * k2 + s[4].y * k3;
  qr[1] = s[5].x * k1 + s[1].x * k2 + s[3].x * k3;
  qi[1] = s[5].y * k1 + s[1].y * k2 + s[3].y * k3;
  qr[2] = s[4].x * k1 + s[3].x * k2 + s[2].x * k3;
  qi[2] = s[4].y * k1 + s[3].y * k2 + s[2].y * k3;
  const double w = (c == 0 || (even && c == N / 2)) ? 1.0 : 2.0;
  res += w * ((double)(qr[0] * qr[0] + qi[0] * qi[0]) + (double)(qr[1] * qr[1] + qi[1] * qi[1]) +
              (double)(qr[2] * qr[2] + qi[2] * qi[2]));
  const float kk = k1 * k1 + k2 * k2 + k3 * k3;
  const float ik2 = 1.0f / kk;
  const float a1 = inv2mu * ik2;
  const float a2 = coef * ik2 * ik2;
  const float kqr = k1 * qr[0] + k2 * qr[1] + k3 * qr[2];
  const float kqi = k1 * qi[0] + k2 * qi[1] + k3 * qi[2];
  const float kv[3] = {k1, k2, k3};
  const int ii[6] = {0, 1, 2, 1, 0, 0}, jj[6] = {0, 1, 2, 2, 2, 1};
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    const int i = ii[q], j = jj[q];
    const float f = q < 3 ? 1.0f : 2.0f;
    e[q].x -= f * (a1 * (kv[j] * qr[i] + kv[i] * qr[j]) - a2 * kqr * kv[i] * kv[j]);
    e[q].y -= f * (a1 * (kv[j] * qi[i] + kv[i] * qi[j]) - a2 * kqi * kv[i] * kv[j]);
  }
}

// Two consecutive FP32 modes m0 (even) and m0 + 1 with 16-byte loads and
// stores (nmodes even, so every component's base is 16-byte aligned); the
// index (a, b, c) of m0 by 32-bit division (nmodes < 2^31), that of m0 + 1 by
// a carry.
__device__ __forceinline__ void gamma_pair_f32(int N, float inv2mu, float coef, float4* __restrict__ sig_hat,
                                               float4* __restrict__ eps_hat, int64_t nmodes, unsigned m0,
                                               double& res) {
  const unsigned Nh = (unsigned)(N / 2 + 1);
  const size_t st = (size_t)nmodes / 2, p = m0 / 2;
  float4 S[6], E[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) S[q] = sig_hat[q * st + p];
#pragma unroll
  for (int q = 0; q < 6; ++q) E[q] = eps_hat[q * st + p];
  const unsigned ab = m0 / Nh;
  int c = (int)(m0 - ab * Nh);
  int a = (int)(ab / (unsigned)N);
  int b = (int)(ab - (unsigned)a * (unsigned)N);
  float2 s0[6], e0[6], s1[6], e1[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    s0[q] = make_float2(S[q].x, S[q].y);
    s1[q] = make_float2(S[q].z, S[q].w);
    e0[q] = make_float2(E[q].x, E[q].y);
    e1[q] = make_float2(E[q].z, E[q].w);
  }
  gamma_mode_f32_regs(N, a, b, c, inv2mu, coef, s0, e0, res);
  if (++c == (int)Nh) {
    c = 0;
    if (++b == N) {
      b = 0;
      ++a;
    }
  }
  gamma_mode_f32_regs(N, a, b, c, inv2mu, coef, s1, e1, res);
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    const float4 o = make_float4(e0[q].x, e0[q].y, e1[q].x, e1[q].y);
    eps_hat[q * st + p] = o;
    sig_hat[q * st + p] = o;
  }
}

// ------------------------------------------------------------------ kernels

// Single-problem material evaluation (grid-stride over voxels; one partial
// sum per block).  Used by the allocation-free entry point.
template <class T, int MODE>
__global__ void __launch_bounds__(kMatBlock) ms_material_kernel(int64_t nvox, const uint8_t* __restrict__ phase,
                                                                PhaseTable tab, Step hs, double inv_n3,
                                                                const T* __restrict__ eps_raw,
                                                                const T* __restrict__ zn, T* __restrict__ sig,
                                                                T* __restrict__ z, double* __restrict__ partials) {
  T acc[6] = {0, 0, 0, 0, 0, 0};
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < nvox; base += stride) {
    const int64_t i = base + threadIdx.x;
    material_voxel<T, MODE>(i, i < nvox, nvox, phase, tab, hs, (T)inv_n3, eps_raw, zn, sig, z, acc);
  }
  double accd[6];
#pragma unroll
  for (int c = 0; c < 6; ++c) accd[c] = (double)acc[c];
  block_sum<6>(accd, partials, gridDim.x);
}

// Index of the job owning global chunk c (starts ascending, starts[0] = 0).
__device__ __forceinline__ int owner(const int64_t* starts, int n, int64_t c) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (starts[mid] <= c) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Batched material evaluation: all jobs of the launch, chunk by chunk.
template <class T, int MODE>
__global__ void __launch_bounds__(kMatBlock) ms_material_batch_kernel(const JobView* __restrict__ views, int n_jobs,
                                                                      int64_t total_chunks) {
  __shared__ int64_t starts[kMaxBatch];
  for (int j = threadIdx.x; j < n_jobs; j += blockDim.x) starts[j] = views[j].vchunk0;
  __syncthreads();
  for (int64_t gc = blockIdx.x; gc < total_chunks; gc += gridDim.x) {
    const JobView& v = views[owner(starts, n_jobs, gc)];
    const int64_t lc = gc - v.vchunk0;
    const Step hs{v.h, v.inv_h, (float)v.h, (float)v.inv_h};
    T acc[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll 1
    for (int sweep = 0; sweep < kVChunk / kMatBlock; ++sweep) {
      const int64_t i = lc * kVChunk + sweep * kMatBlock + threadIdx.x;
      material_voxel<T, MODE>(i, i < v.nvox, v.nvox, v.phase, *v.tab, hs, (T)v.inv_n3,
                              static_cast<const T*>(v.eps_raw), static_cast<const T*>(v.zn),
                              static_cast<T*>(v.sig), static_cast<T*>(v.z), acc, v.warm != 0);
    }
    double accd[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) accd[c] = (double)acc[c];
    block_sum_at<6>(accd, v.mat_part, v.n_vch, lc);
  }
}

// Batched Green-operator update and error partial sums.
template <class T>
__global__ void __launch_bounds__(kGamBlock) ms_gamma_batch_kernel(const JobView* __restrict__ views, int n_jobs,
                                                                   int64_t total_chunks) {
  __shared__ int64_t starts[kMaxBatch];
  for (int j = threadIdx.x; j < n_jobs; j += blockDim.x) starts[j] = views[j].mchunk0;
  __syncthreads();
  for (int64_t gc = blockIdx.x; gc < total_chunks; gc += gridDim.x) {
    const JobView& v = views[owner(starts, n_jobs, gc)];
    const int64_t lc = gc - v.mchunk0;
    const double inv2mu = 1.0 / (2.0 * v.mu0);
    const double coef = (v.lam0 + v.mu0) / (v.mu0 * (v.lam0 + 2.0 * v.mu0));
    double res[1] = {0.0};
    if (sizeof(T) == 4 && v.nmodes % 2 == 0) {
      // FP32 fields: pairs of modes per thread, 16-byte accesses
#pragma unroll 1
      for (int sweep = 0; sweep < kMChunk / (2 * kGamBlock); ++sweep) {
        const int64_t m = lc * kMChunk + sweep * 2 * kGamBlock + 2 * threadIdx.x;
        if (m < v.nmodes)
          gamma_pair_f32(v.N, (float)inv2mu, (float)coef, static_cast<float4*>(v.sig_hat),
                         static_cast<float4*>(v.eps_hat), v.nmodes, (unsigned)m, res[0]);
      }
    } else {
#pragma unroll 1
      for (int sweep = 0; sweep < kMChunk / kGamBlock; ++sweep) {
        const int64_t m = lc * kMChunk + sweep * kGamBlock + threadIdx.x;
        if (m < v.nmodes)
          gamma_mode<T>(v.N, inv2mu, coef, static_cast<typename cplx<T>::type*>(v.sig_hat),
                        static_cast<typename cplx<T>::type*>(v.eps_hat), v.nmodes, m, res[0]);
      }
    }
    block_sum_at<1>(res, v.gam_part, v.n_mch, lc);
  }
}

// Final sums of one problem's partials: warp c (c < 6) sums component c of
// the material partials, warp 6 the error partials; lane l takes partials
// l, l + 32, ... and the lanes combine in a fixed shuffle tree, so the order
// depends only on the partial count (never on other problems in a batch).
// Launch with kFinBlock threads.
constexpr int kFinBlock = 224;
__device__ void finalize_sums(const double* __restrict__ mat_part, int n_mat, const double* __restrict__ gam_part,
                              int n_gam, double inv_n3, double floor_, Reduced* __restrict__ out) {
  __shared__ double sh[7];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double s = 0.0;
  if (w < 6) {
    for (int b = lane; b < n_mat; b += 32) s += mat_part[w * n_mat + b];
  } else if (w == 6) {
    for (int b = lane; b < n_gam; b += 32) s += gam_part[b];
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  if (lane == 0 && w < 7) sh[w] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
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

// Fixed-order final sums of one problem's partials (single-problem path).
__global__ void ms_finalize_kernel(const double* __restrict__ mat_part, int n_mat, const double* __restrict__ gam_part,
                                   int n_gam, double inv_n3, double floor_, Reduced* __restrict__ out) {
  finalize_sums(mat_part, n_mat, gam_part, n_gam, inv_n3, floor_, out);
}

// One block per job.
__global__ void ms_finalize_batch_kernel(const JobView* __restrict__ views, Reduced* __restrict__ out) {
  const JobView& v = views[blockIdx.x];
  finalize_sums(v.mat_part, v.n_vch, v.gam_part, v.n_mch, v.inv_n3, v.mu0 * 1e-6, out + blockIdx.x);
}

// Mean mode of the strain spectrum and of the inverse-transform input:
// m = N^3 E (mixed boundary conditions move E during a load step).  One warp.
template <class T>
__global__ void ms_set_mean_kernel(typename cplx<T>::type* __restrict__ eps_hat, typename cplx<T>::type* __restrict__ sig_hat,
                                   int64_t nmodes, double m0, double m1, double m2, double m3, double m4, double m5) {
  const double m[6] = {m0, m1, m2, m3, m4, m5};
  const int q = threadIdx.x;
  if (q < 6) {
    typename cplx<T>::type v;
    v.x = (T)m[q];
    v.y = T(0);
    eps_hat[q * nmodes] = v;
    sig_hat[q * nmodes] = v;
  }
}

// Reference medium from tangents (Sec. 3: adjusted per load step to the
// current tangential stiffness): the law with tangent at the predicted strain
// eps_raw / N^3 + dE and z_n; per voxel the isotropic measures
// 3k = J::C = (1/3) sum_{i,j<3} C_ij and 10 mu = tr_Mandel C - 3k; per block
// their min and max -> part[q * gridDim.x + block], q = kmin, kmax, mumin, mumax.
template <int MODE>
__global__ void __launch_bounds__(kMatBlock) ms_reference_kernel(int64_t nvox, const uint8_t* __restrict__ phase,
                                                                 const PhaseTable* __restrict__ tab, Step hs,
                                                                 const double* __restrict__ eps_raw,
                                                                 const double* __restrict__ zn, double inv_n3,
                                                                 double d0, double d1, double d2, double d3, double d4,
                                                                 double d5, double* __restrict__ part) {
  const double d[6] = {d0, d1, d2, d3, d4, d5};
  double r[4] = {1e300, -1e300, 1e300, -1e300};
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < nvox; base += stride) {
    const int64_t i = base + threadIdx.x;
    const bool in = i < nvox;
    const int ph = in ? (int)phase[i] : 0;
    const bool vp = in && tab->kind[ph] == GSM_PSI_ELASTIC_VP_DEV;
    double e[6], zi[6], s[6], zo[6], t[21];
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      e[c] = in ? fma(eps_raw[c * nvox + i], inv_n3, d[c]) : 0.0;
      zi[c] = vp ? zn[c * nvox + i] : 0.0;
    }
    if constexpr (MODE == MODE_FP64) voxel_fp64<NortonDev>(tab->p64[ph], e, zi, hs, vp, s, zo, t);
    else voxel_fp32_fix<NortonDev>(tab->p64[ph], tab->p32[ph], e, zi, hs, vp, s, zo, t);
    if (in && !vp) voxel_elastic<double>(tab->p64[ph], e, s, t);
    if (in) {
      // packed upper triangle: C11 0, C12 1, C13 2, C22 6, C23 7, C33 11, C44 15, C55 18, C66 20
      const double tk = (t[0] + t[6] + t[11] + 2.0 * (t[1] + t[2] + t[7])) * (1.0 / 3.0);
      const double tr = t[0] + t[6] + t[11] + 2.0 * (t[15] + t[18] + t[20]);
      const double k = tk * (1.0 / 3.0), mu = (tr - tk) * 0.1;
      r[0] = fmin(r[0], k);
      r[1] = fmax(r[1], k);
      r[2] = fmin(r[2], mu);
      r[3] = fmax(r[3], mu);
    }
  }
  __shared__ double sh[4][kMatBlock / 32];
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
    for (int k = 1; k < kMatBlock / 32; ++k) v = (q & 1) ? fmax(v, sh[q][k]) : fmin(v, sh[q][k]);
    part[q * gridDim.x + blockIdx.x] = v;
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

}  // namespace
}  // namespace gsm
