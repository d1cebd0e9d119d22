// Basic-scheme kernels for laws integrated over the load step by an ODE
// integrator (AutoMat, arXiv 2006.04391, Sec. 4.3: ode23, ode12 or ode23s;
// tangent ODE of Corollary 1) and their host launchers, instantiated per
// integrator in ms_ode{23,12,23s}.cu (material kernels) and
// ms_ode{23,12,23s}_ref.cu (reference kernels, with the tangent): the
// integrator instantiations dominate the compile time, one unit each.
#pragma once

#include "ms_kernels.cuh"
#include "ms_ode.h"
#include "ode23.cuh"

namespace gsm {
namespace {


// Material evaluation of voxel i with the ode23 laws (Sec. 4.3): Norton and
// Michel-Suquet voxels integrate the force-potential form from the strain of
// the previous step, elastic voxels are direct.  All lanes of a warp call
// this; each law runs its own warp-voted substep loop (lanes of other laws
// skip it), so the two integrator states do not live at the same time.
template <int PAIR>
__device__ __forceinline__ void material_voxel_ode(int64_t i, bool in, const JobView& v, const Step& hs,
                                                   const Ode23Ctl& ctl, double (&acc)[6]) {
  const int64_t nvox = v.nvox;
  const int ph = in ? (int)v.phase[i] : 0;
  const int kind = in ? v.tab->kind[ph] : GSM_PSI_ELASTIC;
  const LawParams<double>& p = v.tab->p64[ph];
  const double* eps_raw = static_cast<const double*>(v.eps_raw);
  const double* zn = static_cast<const double*>(v.zn);
  double* sig = static_cast<double*>(v.sig);
  double* z = static_cast<double*>(v.z);
  double e[6], e0[6], s[6], zo[7];
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    e[c] = in ? __ldg(eps_raw + c * nvox + i) * v.inv_n3 : 0.0;
    e0[c] = in ? __ldg(v.eps_prev + c * nvox + i) : 0.0;
    s[c] = 0.0;
  }
#pragma unroll
  for (int c = 0; c < 7; ++c) zo[c] = 0.0;
  const bool nor = in && kind == GSM_PSI_ELASTIC_VP_DEV;
  if (any_lane(nor)) {
    OdeVoxel<NortonDev, false, PAIR> w;
    double zi[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) zi[c] = nor ? __ldg(zn + c * nvox + i) : 0.0;
    if (nor) w.init(p, e0, e, zi, hs.h);
    else w.done = true;
    for (;;) {
      if (all_done(w.done)) break;
      if (!w.done) w.attempt(p, hs, ctl);
    }
    if (nor) {
      double z6[6];
      w.finish(hs.h, s, z6, nullptr);
#pragma unroll
      for (int c = 0; c < 6; ++c) zo[c] = z6[c];
    }
  }
  const bool kin = in && kind == GSM_PSI_ELASTIC_VP_KIN;
  if (any_lane(kin)) {
    OdeVoxel<MichelSuquet, false, PAIR> w;
    double zi[7];
#pragma unroll
    for (int c = 0; c < 6; ++c) zi[c] = kin ? __ldg(zn + c * nvox + i) : 0.0;
    zi[6] = kin ? __ldg(v.alpha_n + i) : 0.0;
    if (kin) w.init(p, e0, e, zi, hs.h);
    else w.done = true;
    for (;;) {
      if (all_done(w.done)) break;
      if (!w.done) w.attempt(p, hs, ctl);
    }
    if (kin) w.finish(hs.h, s, zo, nullptr);
  }
  if (in && kind == GSM_PSI_ELASTIC) voxel_elastic<double>(p, e, s, nullptr);
  if (in) {
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      sig[c * nvox + i] = s[c];
      z[c * nvox + i] = zo[c];
      acc[c] += s[c];
    }
    if (v.alpha) v.alpha[i] = zo[6];
  }
}

// Batched material evaluation of jobs whose laws integrate by the pair PAIR (FP64).
template <int PAIR>
__global__ void __launch_bounds__(kMatBlock) ms_material_ode_kernel(const JobView* __restrict__ views, int n_jobs,
                                                                    int64_t total_chunks) {
  __shared__ int64_t starts[kMaxBatch];
  for (int j = threadIdx.x; j < n_jobs; j += blockDim.x) starts[j] = views[j].vchunk0;
  __syncthreads();
  for (int64_t gc = blockIdx.x; gc < total_chunks; gc += gridDim.x) {
    const JobView& v = views[owner(starts, n_jobs, gc)];
    const int64_t lc = gc - v.vchunk0;
    const Step hs{v.h, v.inv_h, (float)v.h, (float)v.inv_h};
    const Ode23Ctl ctl{v.ode_rtol, v.ode_atol, v.ode_max};
    double acc[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll 1
    for (int sweep = 0; sweep < kVChunk / kMatBlock; ++sweep) {
      const int64_t i = lc * kVChunk + sweep * kMatBlock + threadIdx.x;
      material_voxel_ode<PAIR>(i, i < v.nvox, v, hs, ctl, acc);
    }
    block_sum_at<6>(acc, v.mat_part, v.n_vch, lc);
  }
}

// Isotropic measures (k, mu) of a full 6x6 tangent (row-major, stress-like
// rows, engineering-shear columns): 3k = (1/3) sum_{i,j<3} C_ij, 10 mu =
// tr_Mandel C - 3k.
__device__ __forceinline__ void iso_measures36(const double (&C)[36], double& k, double& mu) {
  double tk = 0.0;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) tk += C[6 * a + b];
  tk *= 1.0 / 3.0;
  const double tr = C[0] + C[7] + C[14] + 2.0 * (C[21] + C[28] + C[35]);
  k = tk * (1.0 / 3.0);
  mu = (tr - tk) * 0.1;
}

// Reference medium from the tangents of the ode laws (tangent ODE of
// Corollary 1) at the predicted strain; partials as ms_reference_kernel.
template <int PAIR>
__global__ void __launch_bounds__(kMatBlock) ms_reference_ode_kernel(int64_t nvox, const uint8_t* __restrict__ phase,
                                                                     const PhaseTable* __restrict__ tab, Step hs,
                                                                     Ode23Ctl ctl, const double* __restrict__ eps_raw,
                                                                     const double* __restrict__ eps_prev,
                                                                     const double* __restrict__ zn,
                                                                     const double* __restrict__ alpha_n, double inv_n3,
                                                                     double d0, double d1, double d2, double d3,
                                                                     double d4, double d5, double* __restrict__ part) {
  const double d[6] = {d0, d1, d2, d3, d4, d5};
  double r[4] = {1e300, -1e300, 1e300, -1e300};
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < nvox; base += stride) {
    const int64_t i = base + threadIdx.x;
    const bool in = i < nvox;
    const int ph = in ? (int)phase[i] : 0;
    const int kind = in ? tab->kind[ph] : GSM_PSI_ELASTIC;
    const LawParams<double>& p = tab->p64[ph];
    double e[6], e0[6], s[6], C[36];
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      e[c] = in ? fma(eps_raw[c * nvox + i], inv_n3, d[c]) : 0.0;
      e0[c] = in ? eps_prev[c * nvox + i] : 0.0;
    }
#pragma unroll
    for (int c = 0; c < 36; ++c) C[c] = 0.0;
    if (in && kind == GSM_PSI_ELASTIC_VP_DEV) {
      double zi[6], zo[6];
#pragma unroll
      for (int c = 0; c < 6; ++c) zi[c] = zn[c * nvox + i];
      voxel_ode23<NortonDev, true, PAIR>(p, e0, e, zi, hs, ctl, s, zo, C);
    } else if (in && kind == GSM_PSI_ELASTIC_VP_KIN) {
      double zi[7], zo[7];
#pragma unroll
      for (int c = 0; c < 6; ++c) zi[c] = zn[c * nvox + i];
      zi[6] = alpha_n[i];
      voxel_ode23<MichelSuquet, true, PAIR>(p, e0, e, zi, hs, ctl, s, zo, C);
    } else if (in) {
      double t[21];
      voxel_elastic<double>(p, e, s, t);
      int c = 0;
      for (int a = 0; a < 6; ++a)
        for (int b = a; b < 6; ++b, ++c) C[6 * a + b] = C[6 * b + a] = t[c];
    }
    if (in) {
      double k, mu;
      iso_measures36(C, k, mu);
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

}  // namespace

template <int PAIR> int ms_ode_blocks_per_sm_p() {
  int b = 0;
  const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, ms_material_ode_kernel<PAIR>, kMatBlock, 0);
  return e == cudaSuccess && b > 0 ? b : 1;
}

template <int PAIR>
void ms_launch_material_ode_p(int grid, cudaStream_t s, const void* views, int n_jobs, int64_t total_chunks) {
  ms_material_ode_kernel<PAIR><<<grid, kMatBlock, 0, s>>>(static_cast<const JobView*>(views), n_jobs, total_chunks);
}

template <int PAIR>
void ms_launch_reference_ode_p(int grid, cudaStream_t s, int64_t nvox, const uint8_t* phase, const void* tab, double h,
                               double rtol, double atol, int max_steps, const double* eps_raw, const double* eps_prev,
                               const double* zn, const double* alpha_n, double inv_n3, const double (&dE)[6],
                               double* part) {
  ms_reference_ode_kernel<PAIR><<<grid, kMatBlock, 0, s>>>(
      nvox, phase, static_cast<const PhaseTable*>(tab), make_step(h), Ode23Ctl{rtol, atol, max_steps}, eps_raw,
      eps_prev, zn, alpha_n, inv_n3, dE[0], dE[1], dE[2], dE[3], dE[4], dE[5], part);
}

// explicit instantiations: the material kernel and the (tangent-heavy)
// reference kernel of an integrator go to separate translation units
#define GSM_MS_ODE_INSTANTIATE_MATERIAL(PAIR)                                                                    \
  template int ms_ode_blocks_per_sm_p<PAIR>();                                                                \
  template void ms_launch_material_ode_p<PAIR>(int, cudaStream_t, const void*, int, int64_t);
#define GSM_MS_ODE_INSTANTIATE_REFERENCE(PAIR)                                                                   \
  template void ms_launch_reference_ode_p<PAIR>(int, cudaStream_t, int64_t, const uint8_t*, const void*, double, \
                                                double, double, int, const double*, const double*,          \
                                                const double*, const double*, double, const double (&)[6],  \
                                                double*);

}  // namespace gsm
