// Moulinec-Suquet basic scheme driving the GSM update (AutoMat, arXiv
// 2006.04391: Sec. 1 and Sec. 3 "Material Law Evaluations" -- fixed reference
// stiffness, one material evaluation without tangent per voxel and
// iteration), and the serving loop that runs many such solves at once.  The
// paper ran this solver on the CPU; here every step runs on the GPU and the
// fields stay resident in HBM.  One iteration ("tick") of every active job:
//
//   material kernel   sigma, z = law(eps_raw / N^3, z_n)   + FP64 partial sums of sigma
//   cuFFT R2C (x6)    sigma -> sig_hat                      (per job)
//   gamma kernel      per mode: error partial sums (FP64), eps_hat -= Gamma0 : sig_hat,
//                     and a copy of eps_hat into sig_hat's buffer for the inverse
//   finalize kernel   fixed-order sums -> e and <sigma> (FP64) per job, one copy to host
//   cuFFT C2R (x6)    eps_hat copy -> eps_raw (unnormalised: N^3 eps)   (per job)
//
// The material, gamma and finalize kernels take every job of the tick in one
// launch (ms_kernels.cuh); ms_run is a tick loop over a single job, the
// serve_* API a tick loop over a job table with admission by an HBM budget.
// The C2R output is never normalised in a separate pass: the material kernel
// scales it by 1/N^3 as it loads it.  cuFFT may overwrite the input of a
// multi-dimensional C2R, which is why the gamma kernel writes the updated
// eps_hat twice (state and transform input).
#include <cufft.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <vector>

#include "adjoint_kernels.cuh"
#include "common.cuh"
#include "ms_kernels.cuh"
#include "ms_ode.h"

namespace gsm {
namespace {

int grid_cap(int64_t n, int block, int per_sm) {
  const int64_t need = (n + block - 1) / block;
  const int64_t cap = (int64_t)sm_count() * per_sm;
  return (int)std::max<int64_t>(1, std::min(need, cap));
}

template <class T> struct Fields {
  using C = typename cplx<T>::type;
  T* eps_raw = nullptr;  // [6][nvox] unnormalised strain (C2R output)
  T* zn = nullptr;       // [6][nvox] internal variables at t_n (FP32 copy in bulk mode)
  T* sig = nullptr;      // [6][nvox]
  T* z = nullptr;        // [6][nvox]
  C* sig_hat = nullptr;  // [6][nmodes] (also the C2R input)
  C* eps_hat = nullptr;  // [6][nmodes]
};

template <class T> size_t field_bytes(int64_t nvox, int64_t nmodes) {
  return 4 * 6 * nvox * sizeof(T) + 2 * 6 * nmodes * sizeof(typename cplx<T>::type);
}

int64_t n_vchunks(int64_t nvox) { return (nvox + kVChunk - 1) / kVChunk; }
int64_t n_mchunks(int64_t nmodes) { return (nmodes + kMChunk - 1) / kMChunk; }

size_t job_bytes(int N, int precision) {
  const int64_t nv = (int64_t)N * N * N, nm = (int64_t)N * N * (N / 2 + 1);
  size_t b = field_bytes<double>(nv, nm) + (precision == MS_PREC_FP32_BULK ? field_bytes<float>(nv, nm) : 0);
  b += (6 * n_vchunks(nv) + n_mchunks(nm)) * sizeof(double) + sizeof(PhaseTable) + (size_t)nv;  // + phase copy
  return b;
}

size_t plan_bytes_one(int N, bool fp32) {
  int n[3] = {N, N, N};
  const long long nv = (long long)N * N * N, nm = (long long)N * N * (N / 2 + 1);
  size_t total = 0, ws = 0;
  if (cufftEstimateMany(3, n, nullptr, 1, (int)nv, nullptr, 1, (int)nm, fp32 ? CUFFT_R2C : CUFFT_D2Z, 6, &ws) ==
      CUFFT_SUCCESS)
    total += ws;
  if (cufftEstimateMany(3, n, nullptr, 1, (int)nm, nullptr, 1, (int)nv, fp32 ? CUFFT_C2R : CUFFT_Z2D, 6, &ws) ==
      CUFFT_SUCCESS)
    total += ws;
  return total;
}

size_t plan_bytes(int N, int precision) {
  return plan_bytes_one(N, false) + (precision == MS_PREC_FP32_BULK ? plan_bytes_one(N, true) : 0);
}

// ------------------------------------------------------------------- engine

struct Plans {
  cufftHandle r2c = 0, c2r = 0;
};

// Stream, cuFFT plan cache and the per-tick job table shared by all jobs.
struct Engine {
  cudaStream_t stream = nullptr;
  std::map<std::pair<int, int>, Plans> plans;  // (N, fp32) -> plans
  JobView* views_dev = nullptr;                // scratch: the tick's job table
  JobView* views_host = nullptr;               // pinned staging
  Reduced* red_dev = nullptr;
  Reduced* red_host = nullptr;
  int cap = 0;
  bool inited = false;
  int per_sm_mat[6] = {1, 1, 1, 1, 1, 1};  // FP64, FP32-fix, FP32 laws; ode23, ode12, ode23s laws
  int per_sm_gam[2] = {1, 1};

  int init(cudaStream_t s, int capacity) {
    stream = s;
    cap = capacity;
    inited = true;
    if (cudaMalloc((void**)&views_dev, cap * sizeof(JobView)) != cudaSuccess ||
        cudaMallocHost((void**)&views_host, cap * sizeof(JobView)) != cudaSuccess ||
        cudaMalloc((void**)&red_dev, cap * sizeof(Reduced)) != cudaSuccess ||
        cudaMallocHost((void**)&red_host, cap * sizeof(Reduced)) != cudaSuccess) {
      cudaGetLastError();
      return GSM_ENOMEM;
    }
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, ms_material_batch_kernel<double, MODE_FP64>, kMatBlock, 0) ==
        cudaSuccess)
      per_sm_mat[0] = std::max(b, 1);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, ms_material_batch_kernel<double, MODE_FP32_FIX>, kMatBlock,
                                                      0) == cudaSuccess)
      per_sm_mat[1] = std::max(b, 1);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, ms_material_batch_kernel<float, MODE_FP32>, kMatBlock, 0) ==
        cudaSuccess)
      per_sm_mat[2] = std::max(b, 1);
    for (int q = 0; q < 3; ++q) per_sm_mat[3 + q] = ms_ode_blocks_per_sm(q);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, ms_gamma_batch_kernel<double>, kGamBlock, 0) == cudaSuccess)
      per_sm_gam[0] = std::max(b, 1);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, ms_gamma_batch_kernel<float>, kGamBlock, 0) == cudaSuccess)
      per_sm_gam[1] = std::max(b, 1);
    return GSM_OK;
  }

  int get_plans(int N, bool fp32, Plans** out) {
    auto key = std::make_pair(N, fp32 ? 1 : 0);
    auto it = plans.find(key);
    if (it == plans.end()) {
      Plans p;
      int n[3] = {N, N, N};
      const int nv = N * N * N, nm = N * N * (N / 2 + 1);
      if (cufftPlanMany(&p.r2c, 3, n, nullptr, 1, nv, nullptr, 1, nm, fp32 ? CUFFT_R2C : CUFFT_D2Z, 6) !=
          CUFFT_SUCCESS)
        return GSM_ECUDA;
      if (cufftPlanMany(&p.c2r, 3, n, nullptr, 1, nm, nullptr, 1, nv, fp32 ? CUFFT_C2R : CUFFT_Z2D, 6) !=
          CUFFT_SUCCESS) {
        cufftDestroy(p.r2c);
        return GSM_ECUDA;
      }
      cufftSetStream(p.r2c, stream);
      cufftSetStream(p.c2r, stream);
      it = plans.emplace(key, p).first;
    }
    *out = &it->second;
    return GSM_OK;
  }

  ~Engine() {
    if (inited) cudaStreamSynchronize(stream);
    for (auto& kv : plans) {
      cufftDestroy(kv.second.r2c);
      cufftDestroy(kv.second.c2r);
    }
    cudaFree(views_dev);
    cudaFreeHost(views_host);
    cudaFree(red_dev);
    cudaFreeHost(red_host);
  }
};

// --------------------------------------------------------------------- jobs

struct Job {
  int64_t id = 0;
  int N = 0;
  int64_t nvox = 0, nmodes = 0;
  int n_vch = 0, n_mch = 0;
  int precision = MS_PREC_FP64;
  int law_mode = MODE_FP64;  // arithmetic of the laws on FP64 fields
  uint8_t* phase_owned = nullptr;
  const uint8_t* phase = nullptr;
  PhaseTable tab_host;
  PhaseTable* tab_dev = nullptr;
  double lam0 = 0, mu0 = 0;          // reference medium of the current step
  double lam0_el = 0, mu0_el = 0;    // the fixed elastic reference
  double theta[kMaxPhases][3] = {};  // (sigma0, edot0, n) of Norton phases
  Fields<double> f64;
  Fields<float> f32;
  double* mat_part = nullptr;
  double* gam_part = nullptr;
  size_t bytes = 0;
  bool allocated = false;
  // load
  std::vector<double> E, h;
  std::vector<int32_t> forced;
  double tol = 1e-8, switch_tol = 1e-5;
  int max_iter = 10000;
  int stress_mask = 0;               // mixed boundary conditions: prescribed-stress components
  std::vector<double> S_target;      // [n_steps][6]
  bool ref_update = false;           // per-step reference medium from tangents
  int integrator = 0;                // 0 implicit Euler, 1 ode23, 2 ode12, 3 ode23s (Sec. 4.3)
  double ode_rtol = 1e-3, ode_atol = 1e-6;
  int ode_max = 100000;
  bool has_kin = false;              // a Michel-Suquet phase: alpha, and an explicit pair only
  double* eps_prev = nullptr;        // [6][nvox] strain at t_n (ode23, ode12)
  double* alpha_n = nullptr;         // [nvox] Michel-Suquet alpha at t_n
  double* alpha = nullptr;           // [nvox] and at t_{n+1}
  double C0ss_inv[36] = {};          // (C0 on the prescribed-stress components)^-1, n_s x n_s
  int n_s = 0, s_idx[6] = {};
  // state
  int step = 0, n_eval = 0, n32 = 0, since_best = 0;
  bool fp32_phase = false, need_start = true, done = false, notconv = false;
  bool warm = false;  // z holds the previous evaluation of this step, in the current field precision
  double best = 1e300;
  double E_prev[6] = {0, 0, 0, 0, 0, 0};  // macroscopic strain at the end of the previous step
  double E_cur[6] = {0, 0, 0, 0, 0, 0};   // macroscopic strain of the current iterate
  // results
  std::vector<double> Sigma, final_error, E_out, ref_out;
  std::vector<int32_t> iters, fp32_iters;
  int64_t total_iters = 0;
  double vt = 0.0;  // serving: virtual time, the GPU work this job has received (voxel-iteration units)
  // optional per-step checkpoints for the adjoint: [n_steps][6][nvox] each
  double* tape_eps = nullptr;   // converged strain eps_k
  double* tape_zprev = nullptr; // internal variables z_{k-1} entering step k
};

int job_setup(Job& j, int N, const uint8_t* phase_dev, int n_phases, const gsm_handle* laws, int precision) {
  if (N < 2 || N > 1024 || n_phases < 1 || n_phases > kMaxPhases || !laws ||
      (precision != MS_PREC_FP64 && precision != MS_PREC_FP32_BULK))
    return GSM_EINVAL;
  const int64_t n = N;
  if (n * n * n > (int64_t)INT32_MAX / 6) return GSM_EINVAL;  // cuFFT batch distances are int
  j.N = N;
  j.nvox = n * n * n;
  j.nmodes = n * n * (n / 2 + 1);
  j.n_vch = (int)n_vchunks(j.nvox);
  j.n_mch = (int)n_mchunks(j.nmodes);
  j.precision = precision;
  j.phase = phase_dev;
  std::memset(&j.tab_host, 0, sizeof(j.tab_host));
  double lam_min = 1e300, lam_max = -1e300, mu_min = 1e300, mu_max = -1e300;
  j.law_mode = MODE_FP64;
  for (int p = 0; p < n_phases; ++p) {
    const Material* m = reinterpret_cast<const Material*>(laws[p]);
    if (!m) return GSM_EINVAL;
    if (m->psi_kind == GSM_PSI_ELASTIC_VP_KIN) j.has_kin = true;  // runs with ode23 or ode12 only
    j.tab_host.kind[p] = m->psi_kind;
    j.tab_host.p64[p] = m->p64;
    j.tab_host.p32[p] = m->p32;
    if (m->psi_kind == GSM_PSI_ELASTIC_VP_DEV && m->precision != GSM_FP64) j.law_mode = MODE_FP32_FIX;
    if (m->psi_kind == GSM_PSI_ELASTIC_VP_DEV) {
      j.theta[p][0] = m->params[2];
      j.theta[p][1] = m->params[3];
      j.theta[p][2] = m->params[4];
    }
    lam_min = std::min(lam_min, m->p64.lam);
    lam_max = std::max(lam_max, m->p64.lam);
    mu_min = std::min(mu_min, m->p64.mu);
    mu_max = std::max(mu_max, m->p64.mu);
  }
  j.lam0 = j.lam0_el = 0.5 * (lam_min + lam_max);
  j.mu0 = j.mu0_el = 0.5 * (mu_min + mu_max);
  j.bytes = job_bytes(N, precision);
  return GSM_OK;
}

template <class T> bool alloc_fields(Fields<T>& f, int64_t nv, int64_t nm, cudaStream_t s) {
  using C = typename cplx<T>::type;
  return cudaMallocAsync((void**)&f.eps_raw, 6 * nv * sizeof(T), s) == cudaSuccess &&
         cudaMallocAsync((void**)&f.zn, 6 * nv * sizeof(T), s) == cudaSuccess &&
         cudaMallocAsync((void**)&f.sig, 6 * nv * sizeof(T), s) == cudaSuccess &&
         cudaMallocAsync((void**)&f.z, 6 * nv * sizeof(T), s) == cudaSuccess &&
         cudaMallocAsync((void**)&f.sig_hat, 6 * nm * sizeof(C), s) == cudaSuccess &&
         cudaMallocAsync((void**)&f.eps_hat, 6 * nm * sizeof(C), s) == cudaSuccess;
}

template <class T> void free_fields(Fields<T>& f, cudaStream_t s) {
  void* ptrs[6] = {f.eps_raw, f.zn, f.sig, f.z, f.sig_hat, f.eps_hat};
  for (void* p : ptrs)
    if (p) cudaFreeAsync(p, s);
  f = Fields<T>();
}

void job_free(Job& j, cudaStream_t s) {
  if (!j.allocated) return;
  free_fields(j.f64, s);
  free_fields(j.f32, s);
  if (j.mat_part) cudaFreeAsync(j.mat_part, s);
  if (j.gam_part) cudaFreeAsync(j.gam_part, s);
  if (j.tab_dev) cudaFreeAsync(j.tab_dev, s);
  if (j.phase_owned) cudaFreeAsync(j.phase_owned, s);
  if (j.eps_prev) cudaFreeAsync(j.eps_prev, s);
  if (j.alpha_n) cudaFreeAsync(j.alpha_n, s);
  if (j.alpha) cudaFreeAsync(j.alpha, s);
  j.eps_prev = j.alpha_n = j.alpha = nullptr;
  j.mat_part = j.gam_part = nullptr;
  j.tab_dev = nullptr;
  j.phase_owned = nullptr;
  j.allocated = false;
}

// Device memory of a job (stream-ordered allocations).  `phase_host` (may be
// NULL) is copied into a job-owned device array.
int job_alloc(Job& j, cudaStream_t s, const uint8_t* phase_host) {
  bool ok = alloc_fields(j.f64, j.nvox, j.nmodes, s);
  if (ok && j.precision == MS_PREC_FP32_BULK) ok = alloc_fields(j.f32, j.nvox, j.nmodes, s);
  ok = ok && cudaMallocAsync((void**)&j.mat_part, 6 * (size_t)j.n_vch * sizeof(double), s) == cudaSuccess &&
       cudaMallocAsync((void**)&j.gam_part, (size_t)j.n_mch * sizeof(double), s) == cudaSuccess &&
       cudaMallocAsync((void**)&j.tab_dev, sizeof(PhaseTable), s) == cudaSuccess;
  if (ok && phase_host) {
    ok = cudaMallocAsync((void**)&j.phase_owned, (size_t)j.nvox, s) == cudaSuccess &&
         cudaMemcpyAsync(j.phase_owned, phase_host, (size_t)j.nvox, cudaMemcpyHostToDevice, s) == cudaSuccess;
    j.phase = j.phase_owned;
  }
  j.allocated = true;
  if (!ok) {
    cudaGetLastError();
    job_free(j, s);
    return GSM_ENOMEM;
  }
  cudaMemcpyAsync(j.tab_dev, &j.tab_host, sizeof(PhaseTable), cudaMemcpyHostToDevice, s);
  cudaMemsetAsync(j.f64.eps_raw, 0, 6 * j.nvox * sizeof(double), s);
  cudaMemsetAsync(j.f64.zn, 0, 6 * j.nvox * sizeof(double), s);
  // the host sources of the copies above must outlive them
  if (cudaStreamSynchronize(s) != cudaSuccess) return GSM_ECUDA;
  return GSM_OK;
}

// Work arrays of the ODE integrators (the strain at t_n and, for Michel-Suquet
// phases, alpha double-buffered), allocated once; alpha_n starts at 0.
int job_alloc_ode(Job& j, cudaStream_t s) {
  const size_t n6 = 6 * (size_t)j.nvox * sizeof(double), n1 = (size_t)j.nvox * sizeof(double);
  if (j.integrator >= 1 && !j.eps_prev && cudaMallocAsync(&j.eps_prev, n6, s) != cudaSuccess) return GSM_ENOMEM;
  if (j.has_kin) {
    if (!j.alpha_n && cudaMallocAsync(&j.alpha_n, n1, s) != cudaSuccess) return GSM_ENOMEM;
    if (!j.alpha && cudaMallocAsync(&j.alpha, n1, s) != cudaSuccess) return GSM_ENOMEM;
    cudaMemsetAsync(j.alpha_n, 0, n1, s);
  }
  return GSM_OK;
}

// Device bytes of the ODE work arrays of a loaded job.
size_t ode_bytes(const Job& j) {
  size_t b = 0;
  if (j.integrator >= 1) b += 6 * (size_t)j.nvox * sizeof(double);
  if (j.has_kin) b += 2 * (size_t)j.nvox * sizeof(double);
  return b;
}

int job_load(Job& j, const ms_load* load) {
  if (!load || load->n_steps < 1 || !load->E || !load->h || load->max_iter < 1) return GSM_EINVAL;
  for (int k = 0; k < load->n_steps; ++k)
    if (!(std::isfinite(load->h[k]) && load->h[k] > 0.0)) return GSM_EINVAL;
  if (load->forced_iters)
    for (int k = 0; k < load->n_steps; ++k)
      if (load->forced_iters[k] < 1) return GSM_EINVAL;
  if (load->stress_mask < 0 || load->stress_mask > 63 || (load->ref_update != 0 && load->ref_update != 1))
    return GSM_EINVAL;
  if (load->integrator < 0 || load->integrator > 3) return GSM_EINVAL;
  if (load->integrator >= 1 && (!(load->ode_rtol > 0.0) || !(load->ode_atol >= 0.0) || load->ode_max_substeps < 1))
    return GSM_EINVAL;
  // the Michel-Suquet law integrates by an explicit pair only; those run in FP64
  if (j.has_kin && load->integrator == 0) return GSM_ENOTSUP;
  if (load->integrator >= 1 && j.precision != MS_PREC_FP64) return GSM_ENOTSUP;
  j.integrator = load->integrator;
  if (j.integrator >= 1) {
    j.ode_rtol = load->ode_rtol;
    j.ode_atol = load->ode_atol;
    j.ode_max = load->ode_max_substeps;
  }
  const int n = load->n_steps;
  j.stress_mask = load->stress_mask;
  j.S_target.assign(6 * n, 0.0);
  if (load->Sigma) j.S_target.assign(load->Sigma, load->Sigma + 6 * n);
  j.ref_update = load->ref_update == 1;
  j.lam0 = j.lam0_el;
  j.mu0 = j.mu0_el;
  j.E_out.assign(6 * n, 0.0);
  j.ref_out.assign(2 * n, 0.0);
  j.E.assign(load->E, load->E + 6 * n);
  j.h.assign(load->h, load->h + n);
  j.forced.clear();
  if (load->forced_iters) j.forced.assign(load->forced_iters, load->forced_iters + n);
  j.tol = load->tol;
  j.max_iter = load->max_iter;
  j.switch_tol = load->switch_tol > 0.0 ? load->switch_tol : 1e-5;
  j.Sigma.assign(6 * n, 0.0);
  j.final_error.assign(n, 0.0);
  j.iters.assign(n, 0);
  j.fp32_iters.assign(n, 0);
  j.total_iters = 0;
  j.step = 0;
  j.need_start = true;
  j.done = false;
  j.notconv = false;
  return GSM_OK;
}

template <class T> Fields<T>& fields(Job& j);
template <> Fields<double>& fields<double>(Job& j) { return j.f64; }
template <> Fields<float>& fields<float>(Job& j) { return j.f32; }

cufftResult exec_r2c(const Plans& p, double* in, cufftDoubleComplex* out) { return cufftExecD2Z(p.r2c, in, out); }
cufftResult exec_r2c(const Plans& p, float* in, cufftComplex* out) { return cufftExecR2C(p.r2c, in, out); }
cufftResult exec_c2r(const Plans& p, cufftDoubleComplex* in, double* out) { return cufftExecZ2D(p.c2r, in, out); }
cufftResult exec_c2r(const Plans& p, cufftComplex* in, float* out) { return cufftExecC2R(p.c2r, in, out); }

int elt_grid(int64_t n) { return grid_cap(n, 256, 8); }

template <class S, class D> void convert(cudaStream_t s, const S* src, D* dst, int64_t n, double scale) {
  ms_convert_kernel<S, D><<<elt_grid(n), 256, 0, s>>>(n, src, dst, scale);
  count_launch();
}

// eps_raw += N^3 (E - E_prev); eps_hat = spectrum of eps with mean N^3 E.
template <class T> int spectrum_start(Engine& g, Job& j, const double* E, const double* E_prev) {
  Fields<T>& f = fields<T>(j);
  Plans* p = nullptr;
  int rc = g.get_plans(j.N, sizeof(T) == 4, &p);
  if (rc != GSM_OK) return rc;
  const double n3 = (double)j.nvox;
  double d[6];
  for (int q = 0; q < 6; ++q) d[q] = n3 * (E[q] - E_prev[q]);
  ms_add_uniform_kernel<T><<<elt_grid(j.nvox), 256, 0, g.stream>>>(j.nvox, f.eps_raw, d[0], d[1], d[2], d[3], d[4],
                                                                     d[5]);
  if (exec_r2c(*p, f.eps_raw, f.sig_hat) != CUFFT_SUCCESS) return GSM_ECUDA;
  ms_spectrum_init_kernel<T><<<elt_grid(j.nmodes), 256, 0, g.stream>>>(j.nmodes, f.sig_hat, f.eps_hat, 1.0 / n3, n3,
                                                                         E[0], E[1], E[2], E[3], E[4], E[5]);
  count_launch(2);
  return cudaGetLastError() == cudaSuccess ? GSM_OK : GSM_ECUDA;
}

template <class T> int inverse(Engine& g, Job& j) {
  Fields<T>& f = fields<T>(j);
  Plans* p = nullptr;
  int rc = g.get_plans(j.N, sizeof(T) == 4, &p);
  if (rc != GSM_OK) return rc;
  return exec_c2r(*p, f.sig_hat, f.eps_raw) == CUFFT_SUCCESS ? GSM_OK : GSM_ECUDA;
}

int cap_of(const Job& j) { return j.forced.empty() ? j.max_iter : j.forced[j.step]; }

// (C0 restricted to the prescribed-stress components)^-1 for the mixed
// boundary conditions; C0 isotropic (Voigt, engineering shears).
void mixed_setup(Job& j) {
  j.n_s = 0;
  for (int q = 0; q < 6; ++q)
    if ((j.stress_mask >> q) & 1) j.s_idx[j.n_s++] = q;
  const int m = j.n_s;
  if (m == 0) return;
  double A[6][12];
  for (int a = 0; a < m; ++a)
    for (int b = 0; b < m; ++b) {
      const int p = j.s_idx[a], q = j.s_idx[b];
      double c = 0.0;
      if (p < 3 && q < 3) c = j.lam0 + (p == q ? 2.0 * j.mu0 : 0.0);
      else if (p == q) c = j.mu0;
      A[a][b] = c;
      A[a][m + b] = a == b ? 1.0 : 0.0;
    }
  // Gauss-Jordan (C0_ss is symmetric positive definite)
  for (int c = 0; c < m; ++c) {
    const double inv = 1.0 / A[c][c];
    for (int k = 0; k < 2 * m; ++k) A[c][k] *= inv;
    for (int r = 0; r < m; ++r)
      if (r != c) {
        const double f = A[r][c];
        for (int k = 0; k < 2 * m; ++k) A[r][k] -= f * A[c][k];
      }
  }
  for (int a = 0; a < m; ++a)
    for (int b = 0; b < m; ++b) j.C0ss_inv[a * m + b] = A[a][m + b];
}

// Reference medium of the step from the tangents at the predicted strain
// (eps of the previous step + the uniform increment dE, z_n): (k0, mu0) the
// midpoints of the per-voxel isotropic measures, lambda0 = k0 - 2 mu0 / 3.
int reference_update(Engine& g, Job& j, const double (&dE)[6]) {
  const int grid = (int)std::min<int64_t>(j.n_vch, (int64_t)sm_count() * 2);
  const double inv_n3 = 1.0 / (double)j.nvox;
  const Step hs = make_step(j.h[j.step]);
  if (j.integrator >= 1)
    ms_launch_reference_ode(j.integrator - 1, grid, g.stream, j.nvox, j.phase, j.tab_dev, hs.h, j.ode_rtol, j.ode_atol,
                            j.ode_max, j.f64.eps_raw, j.eps_prev, j.f64.zn, j.alpha_n, inv_n3, dE, j.mat_part);
  else if (j.law_mode == MODE_FP64)
    ms_reference_kernel<MODE_FP64><<<grid, kMatBlock, 0, g.stream>>>(j.nvox, j.phase, j.tab_dev, hs, j.f64.eps_raw,
                                                                    j.f64.zn, inv_n3, dE[0], dE[1], dE[2], dE[3],
                                                                    dE[4], dE[5], j.mat_part);
  else
    ms_reference_kernel<MODE_FP32_FIX><<<grid, kMatBlock, 0, g.stream>>>(j.nvox, j.phase, j.tab_dev, hs,
                                                                        j.f64.eps_raw, j.f64.zn, inv_n3, dE[0], dE[1],
                                                                        dE[2], dE[3], dE[4], dE[5], j.mat_part);
  count_launch();
  std::vector<double> part(4 * (size_t)grid);
  if (cudaMemcpyAsync(part.data(), j.mat_part, part.size() * sizeof(double), cudaMemcpyDeviceToHost, g.stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(g.stream) != cudaSuccess)
    return GSM_ECUDA;
  double r[4] = {1e300, -1e300, 1e300, -1e300};
  for (int b = 0; b < grid; ++b) {
    r[0] = std::min(r[0], part[b]);
    r[1] = std::max(r[1], part[grid + b]);
    r[2] = std::min(r[2], part[2 * grid + b]);
    r[3] = std::max(r[3], part[3 * grid + b]);
  }
  const double k0 = 0.5 * (r[0] + r[1]), mu0 = 0.5 * (r[2] + r[3]);
  if (!(mu0 > 0.0) || !(k0 > 0.0) || !std::isfinite(k0 + mu0)) return GSM_ENOTCONV;
  j.mu0 = mu0;
  j.lam0 = k0 - 2.0 * mu0 / 3.0;
  return GSM_OK;
}

// Start load step j.step: macro-strain increment (prescribed-stress
// components keep the previous step's strain as their start), the reference
// medium and, in FP32-bulk mode, the FP32 copies of the FP64 state.
int step_start(Engine& g, Job& j) {
  double E[6], dE[6];
  for (int q = 0; q < 6; ++q) {
    E[q] = ((j.stress_mask >> q) & 1) ? j.E_prev[q] : j.E[6 * j.step + q];
    dE[q] = E[q] - j.E_prev[q];
    j.E_cur[q] = E[q];
  }
  // ODE-integrated laws integrate over the step from each voxel's strain at t_n
  if (j.integrator >= 1) convert<double, double>(g.stream, j.f64.eps_raw, j.eps_prev, 6 * j.nvox, 1.0 / (double)j.nvox);
  if (j.ref_update) {
    const int rc = reference_update(g, j, dE);
    if (rc != GSM_OK) return rc;
  }
  mixed_setup(j);
  j.warm = false;
  j.n_eval = 0;
  j.n32 = 0;
  j.best = 1e300;
  j.since_best = 0;
  j.fp32_phase = j.precision == MS_PREC_FP32_BULK && cap_of(j) > 1;
  if (j.fp32_phase) {
    convert<double, float>(g.stream, j.f64.eps_raw, j.f32.eps_raw, 6 * j.nvox, 1.0);
    convert<double, float>(g.stream, j.f64.zn, j.f32.zn, 6 * j.nvox, 1.0);
    return spectrum_start<float>(g, j, E, j.E_prev);
  }
  return spectrum_start<double>(g, j, E, j.E_prev);
}

// Mixed boundary conditions: dE_s = (C0_ss)^-1 (Sigma_s - <sigma>_s) on the
// prescribed-stress components, written into the mean mode of the strain
// spectrum and of the inverse-transform input.
template <class T> void move_mean(Engine& g, Job& j, const double (&dS)[6]) {
  for (int a = 0; a < j.n_s; ++a) {
    double d = 0.0;
    for (int b = 0; b < j.n_s; ++b) d += j.C0ss_inv[a * j.n_s + b] * dS[j.s_idx[b]];
    j.E_cur[j.s_idx[a]] += d;
  }
  const double n3 = (double)j.nvox;
  Fields<T>& f = fields<T>(j);
  ms_set_mean_kernel<T><<<1, 32, 0, g.stream>>>(f.eps_hat, f.sig_hat, j.nmodes, n3 * j.E_cur[0], n3 * j.E_cur[1],
                                                n3 * j.E_cur[2], n3 * j.E_cur[3], n3 * j.E_cur[4], n3 * j.E_cur[5]);
  count_launch();
}

// FP32 -> FP64 hand-over within a step: the FP32 strain of the last
// evaluation becomes the FP64 strain, resynthesised from its spectrum so that
// its mean is E_k exactly.
int switch_to_fp64(Engine& g, Job& j) {
  j.warm = false;  // the FP64 z is not this step's
  convert<float, double>(g.stream, j.f32.eps_raw, j.f64.eps_raw, 6 * j.nvox, 1.0);
  int rc = spectrum_start<double>(g, j, j.E_cur, j.E_cur);
  if (rc != GSM_OK) return rc;
  cudaMemcpyAsync(j.f64.sig_hat, j.f64.eps_hat, 6 * j.nmodes * sizeof(cufftDoubleComplex), cudaMemcpyDeviceToDevice,
                  g.stream);
  j.fp32_phase = false;
  return inverse<double>(g, j);
}

// After the tick's evaluation: convergence, precision switch, step end.
int post_eval(Engine& g, Job& j, const Reduced& r) {
  ++j.n_eval;
  j.warm = true;  // z now holds this evaluation (step_start and the precision switch clear it)
  double e = r.e;
  double dS[6] = {0, 0, 0, 0, 0, 0};
  if (j.stress_mask) {
    // residual of the prescribed stresses (tensor Frobenius weights), in the error
    const double* St = j.S_target.data() + 6 * j.step;
    double num = 0.0, den = 0.0;
    for (int q = 0; q < 6; ++q) {
      const double w = q < 3 ? 1.0 : 2.0;
      den += w * r.mean[q] * r.mean[q];
      if ((j.stress_mask >> q) & 1) {
        dS[q] = St[q] - r.mean[q];
        num += w * dS[q] * dS[q];
      }
    }
    e = std::max(e, std::sqrt(num) / std::max(std::sqrt(den), j.mu0 * 1e-6));
  }
  const int cap = cap_of(j);
  if (j.fp32_phase) {
    ++j.n32;
    if (e < j.best * 0.999) {
      j.best = e;
      j.since_best = 0;
    } else {
      ++j.since_best;
    }
    if (e < std::max(j.switch_tol, j.tol) || j.since_best >= 20 || j.n_eval >= cap - 1) return switch_to_fp64(g, j);
    if (j.stress_mask) move_mean<float>(g, j, dS);
    return inverse<float>(g, j);
  }
  bool end = false, conv = false;
  if (!j.forced.empty()) {
    end = conv = j.n_eval >= cap;
  } else if (e < j.tol) {
    end = conv = true;
  } else if (j.n_eval >= cap) {
    end = true;
  }
  if (!end) {
    if (j.stress_mask) move_mean<double>(g, j, dS);
    return inverse<double>(g, j);
  }
  if (!conv) j.notconv = true;
  if (j.tape_eps) {
    const int64_t n6 = 6 * j.nvox;
    convert<double, double>(g.stream, j.f64.eps_raw, j.tape_eps + j.step * n6, n6, 1.0 / (double)j.nvox);
    cudaMemcpyAsync(j.tape_zprev + j.step * n6, j.f64.zn, n6 * sizeof(double), cudaMemcpyDeviceToDevice, g.stream);
  }
  std::swap(j.f64.zn, j.f64.z);  // z_n <- z
  if (j.alpha) std::swap(j.alpha_n, j.alpha);
  for (int q = 0; q < 6; ++q) {
    j.Sigma[6 * j.step + q] = r.mean[q];
    j.E_prev[q] = j.E_cur[q];
    j.E_out[6 * j.step + q] = j.E_cur[q];
  }
  j.ref_out[2 * j.step] = j.lam0;
  j.ref_out[2 * j.step + 1] = j.mu0;
  j.iters[j.step] = j.n_eval;
  j.final_error[j.step] = e;
  j.fp32_iters[j.step] = j.n32;
  j.total_iters += j.n_eval;
  ++j.step;
  if (j.step >= (int)j.h.size()) j.done = true;
  else j.need_start = true;
  return GSM_OK;
}

// One iteration of every job in `jobs` (none may be done).
int tick(Engine& g, const std::vector<Job*>& jobs) {
  const int n = (int)jobs.size();
  if (n == 0) return GSM_OK;
  if (n > g.cap || n > kMaxBatch) return GSM_EINVAL;
  for (Job* j : jobs)
    if (j->need_start) {
      int rc = step_start(g, *j);
      if (rc != GSM_OK) return rc;
      j->need_start = false;
    }
  // launch groups: FP64 fields + FP64 laws, FP64 fields + FP32-fix laws,
  // FP64 fields + ode23 / ode12 / ode23s laws, FP32 fields (FP64 groups
  // first: one Green launch)
  constexpr int kGroups = 6, kF32 = 5;
  auto key = [](const Job* j) {
    if (j->fp32_phase) return kF32;
    if (j->integrator >= 1) return 1 + j->integrator;
    return j->law_mode == MODE_FP32_FIX ? 1 : 0;
  };
  std::vector<Job*> order;
  order.reserve(n);
  int gstart[kGroups + 1] = {0, 0, 0, 0, 0, 0, 0};
  for (int k = 0; k < kGroups; ++k) {
    for (Job* j : jobs)
      if (key(j) == k) order.push_back(j);
    gstart[k + 1] = (int)order.size();
  }
  int64_t vtot[kGroups] = {0, 0, 0, 0, 0, 0}, mtot[2] = {0, 0};
  for (int i = 0; i < n; ++i) {
    Job& j = *order[i];
    const int k = key(&j);
    const int pk = k == kF32 ? 1 : 0;
    const bool f = j.fp32_phase;
    JobView& v = g.views_host[i];
    v.phase = j.phase;
    v.eps_raw = f ? (const void*)j.f32.eps_raw : (const void*)j.f64.eps_raw;
    v.zn = f ? (const void*)j.f32.zn : (const void*)j.f64.zn;
    v.sig = f ? (void*)j.f32.sig : (void*)j.f64.sig;
    v.z = f ? (void*)j.f32.z : (void*)j.f64.z;
    v.sig_hat = f ? (void*)j.f32.sig_hat : (void*)j.f64.sig_hat;
    v.eps_hat = f ? (void*)j.f32.eps_hat : (void*)j.f64.eps_hat;
    v.mat_part = j.mat_part;
    v.gam_part = j.gam_part;
    v.tab = j.tab_dev;
    v.nvox = j.nvox;
    v.nmodes = j.nmodes;
    v.vchunk0 = vtot[k];
    v.mchunk0 = mtot[pk];
    v.n_vch = j.n_vch;
    v.n_mch = j.n_mch;
    v.N = j.N;
    v.warm = (j.warm && j.integrator == 0) ? 1 : 0;
    v.h = j.h[j.step];
    v.inv_h = 1.0 / v.h;
    v.inv_n3 = 1.0 / (double)j.nvox;
    v.lam0 = j.lam0;
    v.mu0 = j.mu0;
    v.eps_prev = j.eps_prev;
    v.alpha_n = j.alpha_n;
    v.alpha = j.alpha;
    v.ode_rtol = j.ode_rtol;
    v.ode_atol = j.ode_atol;
    v.ode_max = j.ode_max;
    v.pad2 = 0;
    vtot[k] += j.n_vch;
    mtot[pk] += j.n_mch;
  }
  cudaStream_t s = g.stream;
  cudaMemcpyAsync(g.views_dev, g.views_host, n * sizeof(JobView), cudaMemcpyHostToDevice, s);
  const int64_t sms = sm_count();
  if (gstart[1] > gstart[0]) {
    const int grid = (int)std::min<int64_t>(vtot[0], sms * g.per_sm_mat[0]);
    ms_material_batch_kernel<double, MODE_FP64><<<grid, kMatBlock, 0, s>>>(g.views_dev + gstart[0],
                                                                          gstart[1] - gstart[0], vtot[0]);
    count_launch();
  }
  if (gstart[2] > gstart[1]) {
    const int grid = (int)std::min<int64_t>(vtot[1], sms * g.per_sm_mat[1]);
    ms_material_batch_kernel<double, MODE_FP32_FIX><<<grid, kMatBlock, 0, s>>>(g.views_dev + gstart[1],
                                                                              gstart[2] - gstart[1], vtot[1]);
    count_launch();
  }
  for (int k = 2; k <= 4; ++k)
    if (gstart[k + 1] > gstart[k]) {
      const int grid = (int)std::min<int64_t>(vtot[k], sms * g.per_sm_mat[k + 1]);
      ms_launch_material_ode(k - 2, grid, s, g.views_dev + gstart[k], gstart[k + 1] - gstart[k], vtot[k]);
      count_launch();
    }
  if (gstart[kF32 + 1] > gstart[kF32]) {
    const int grid = (int)std::min<int64_t>(vtot[kF32], sms * g.per_sm_mat[2]);
    ms_material_batch_kernel<float, MODE_FP32><<<grid, kMatBlock, 0, s>>>(g.views_dev + gstart[kF32],
                                                                         gstart[kF32 + 1] - gstart[kF32], vtot[kF32]);
    count_launch();
  }
  for (Job* j : order) {
    Plans* p = nullptr;
    int rc = g.get_plans(j->N, j->fp32_phase, &p);
    if (rc != GSM_OK) return rc;
    const cufftResult fr =
        j->fp32_phase ? exec_r2c(*p, j->f32.sig, j->f32.sig_hat) : exec_r2c(*p, j->f64.sig, j->f64.sig_hat);
    if (fr != CUFFT_SUCCESS) return GSM_ECUDA;
  }
  if (gstart[kF32] > gstart[0]) {
    const int grid = (int)std::min<int64_t>(mtot[0], sms * g.per_sm_gam[0]);
    ms_gamma_batch_kernel<double><<<grid, kGamBlock, 0, s>>>(g.views_dev + gstart[0], gstart[kF32] - gstart[0],
                                                             mtot[0]);
    count_launch();
  }
  if (gstart[kF32 + 1] > gstart[kF32]) {
    const int grid = (int)std::min<int64_t>(mtot[1], sms * g.per_sm_gam[1]);
    ms_gamma_batch_kernel<float><<<grid, kGamBlock, 0, s>>>(g.views_dev + gstart[kF32],
                                                            gstart[kF32 + 1] - gstart[kF32], mtot[1]);
    count_launch();
  }
  ms_finalize_batch_kernel<<<n, kFinBlock, 0, s>>>(g.views_dev, g.red_dev);
  count_launch();
  cudaMemcpyAsync(g.red_host, g.red_dev, n * sizeof(Reduced), cudaMemcpyDeviceToHost, s);
  if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess) return GSM_ECUDA;
  for (int i = 0; i < n; ++i) {
    int rc = post_eval(g, *order[i], g.red_host[i]);
    if (rc != GSM_OK) return rc;
  }
  return GSM_OK;
}

// ------------------------------------------------------------ single solve

struct Ctx {
  Engine eng;
  Job job;
};

// ------------------------------------------------------------------ serving

struct Pending {
  std::unique_ptr<Job> job;
  std::vector<uint8_t> phase;
};

// GPU work of one iteration of a job, in FP32-voxel units: an FP64 iteration
// (FP64 fields, FFTs and law) costs several FP32 ones.
double serve_cost(const Job& j) { return (double)j.nvox * (j.fp32_phase ? 1.0 : 8.0); }

struct Server {
  Engine eng;
  size_t budget = 0, used = 0;
  int max_active = 0;
  int64_t next_id = 1;
  std::deque<Pending> queue;
  std::vector<std::unique_ptr<Job>> active;
  std::map<int64_t, std::unique_ptr<Job>> finished;
  std::map<int64_t, int> state;  // 0 queued, 1 active, 2 done, 3 done without convergence
  std::map<std::pair<int, int>, size_t> plan_cost;
};

}  // namespace
}  // namespace gsm

using namespace gsm;

extern "C" {

size_t ms_workspace_bytes(const ms_problem* prob) {
  if (!prob || prob->N < 2 || prob->N > 1024) return 0;
  return job_bytes(prob->N, prob->precision) + plan_bytes(prob->N, prob->precision) +
         2 * (sizeof(JobView) + sizeof(Reduced));
}

int ms_create(ms_handle* out, const ms_problem* prob, void* stream) {
  if (!out || !prob) return GSM_EINVAL;
  *out = nullptr;
  if (!prob->phase) return GSM_EINVAL;
  Ctx* c = new (std::nothrow) Ctx;
  if (!c) return GSM_ENOMEM;
  int rc = job_setup(c->job, prob->N, prob->phase, prob->n_phases, prob->laws, prob->precision);
  if (rc == GSM_OK) rc = c->eng.init(static_cast<cudaStream_t>(stream), 1);
  if (rc == GSM_OK) rc = job_alloc(c->job, c->eng.stream, nullptr);
  Plans* p = nullptr;
  if (rc == GSM_OK) rc = c->eng.get_plans(c->job.N, false, &p);
  if (rc == GSM_OK && c->job.precision == MS_PREC_FP32_BULK) rc = c->eng.get_plans(c->job.N, true, &p);
  if (rc != GSM_OK) {
    job_free(c->job, c->eng.stream);
    delete c;
    return rc;
  }
  *out = reinterpret_cast<ms_handle>(c);
  return GSM_OK;
}

int ms_destroy(ms_handle h) {
  if (h) {
    Ctx* c = reinterpret_cast<Ctx*>(h);
    job_free(c->job, c->eng.stream);
    delete c;  // the engine synchronises its stream
  }
  return GSM_OK;
}

int ms_run(ms_handle h, const ms_load* load, ms_state* state, ms_result* result) {
  if (!h || !result || !result->Sigma || !result->iters || !result->final_error) return GSM_EINVAL;
  Ctx& c = *reinterpret_cast<Ctx*>(h);
  Job& j = c.job;
  int rc = job_load(j, load);
  if (rc != GSM_OK) return rc;
  const int64_t n6 = 6 * j.nvox;
  const double n3 = (double)j.nvox;
  cudaStream_t s = c.eng.stream;
  for (int q = 0; q < 6; ++q) j.E_prev[q] = 0.0;
  // alpha (the Michel-Suquet law's seventh internal variable) lives in the context only
  if (j.has_kin && state && state->resume) return GSM_ENOTSUP;
  rc = job_alloc_ode(j, s);
  if (rc != GSM_OK) return rc;
  if (state && state->resume) {
    if (!state->eps || !state->z) return GSM_EINVAL;
    convert<double, double>(s, state->eps, j.f64.eps_raw, n6, n3);
    cudaMemcpyAsync(j.f64.zn, state->z, n6 * sizeof(double), cudaMemcpyDeviceToDevice, s);
    for (int q = 0; q < 6; ++q) j.E_prev[q] = state->E_prev[q];
  } else {
    cudaMemsetAsync(j.f64.eps_raw, 0, n6 * sizeof(double), s);
    cudaMemsetAsync(j.f64.zn, 0, n6 * sizeof(double), s);
  }
  const std::vector<Job*> batch{&j};
  while (!j.done) {
    rc = tick(c.eng, batch);
    if (rc != GSM_OK) return rc;
  }
  const int n = (int)j.h.size();
  std::memcpy(result->Sigma, j.Sigma.data(), 6 * n * sizeof(double));
  std::memcpy(result->iters, j.iters.data(), n * sizeof(int32_t));
  std::memcpy(result->final_error, j.final_error.data(), n * sizeof(double));
  if (result->fp32_iters) std::memcpy(result->fp32_iters, j.fp32_iters.data(), n * sizeof(int32_t));
  if (result->E) std::memcpy(result->E, j.E_out.data(), 6 * n * sizeof(double));
  if (result->reference) std::memcpy(result->reference, j.ref_out.data(), 2 * n * sizeof(double));
  result->total_iters = j.total_iters;
  if (state && state->eps && state->z) {
    convert<double, double>(s, j.f64.eps_raw, state->eps, n6, 1.0 / n3);
    cudaMemcpyAsync(state->z, j.f64.zn, n6 * sizeof(double), cudaMemcpyDeviceToDevice, s);
    for (int q = 0; q < 6; ++q) state->E_prev[q] = j.E_prev[q];
  }
  if (cudaStreamSynchronize(s) != cudaSuccess) return GSM_ECUDA;
  return j.notconv ? GSM_ENOTCONV : GSM_OK;
}

int ms_solve(const ms_problem* prob, const ms_load* load, ms_state* state, ms_result* result, void* stream) {
  ms_handle h = nullptr;
  int rc = ms_create(&h, prob, stream);
  if (rc != GSM_OK) return rc;
  rc = ms_run(h, load, state, result);
  ms_destroy(h);
  return rc;
}

// ------------------------------------------------------------------ serving

int serve_create(serve_handle* out, size_t hbm_budget_bytes, int max_active, void* stream) {
  if (!out || max_active < 1 || max_active > kMaxBatch || hbm_budget_bytes == 0) return GSM_EINVAL;
  *out = nullptr;
  Server* sv = new (std::nothrow) Server;
  if (!sv) return GSM_ENOMEM;
  int rc = sv->eng.init(static_cast<cudaStream_t>(stream), max_active);
  if (rc != GSM_OK) {
    delete sv;
    return rc;
  }
  sv->budget = hbm_budget_bytes;
  sv->max_active = max_active;
  *out = reinterpret_cast<serve_handle>(sv);
  return GSM_OK;
}

int serve_destroy(serve_handle h) {
  if (!h) return GSM_OK;
  Server* sv = reinterpret_cast<Server*>(h);
  for (auto& j : sv->active) job_free(*j, sv->eng.stream);
  delete sv;  // the engine synchronises its stream
  return GSM_OK;
}

int serve_submit(serve_handle h, const serve_job* desc, int64_t* id) {
  if (!h || !desc || !id || !desc->phase || !desc->laws) return GSM_EINVAL;
  if (desc->n_phases < 1 || desc->n_phases > kMaxPhases) return GSM_EINVAL;
  Server* sv = reinterpret_cast<Server*>(h);
  Pending p;
  p.job.reset(new (std::nothrow) Job);
  if (!p.job) return GSM_ENOMEM;
  int rc = job_setup(*p.job, desc->N, nullptr, desc->n_phases, desc->laws, desc->precision);
  if (rc != GSM_OK) return rc;
  for (int64_t i = 0; i < p.job->nvox; ++i)
    if (desc->phase[i] >= desc->n_phases) return GSM_EINVAL;
  ms_load ld;
  ld.n_steps = desc->n_steps;
  ld.E = desc->E;
  ld.h = desc->h;
  ld.tol = desc->tol;
  ld.max_iter = desc->max_iter;
  ld.forced_iters = nullptr;
  ld.switch_tol = desc->switch_tol;
  ld.stress_mask = 0;
  ld.Sigma = nullptr;
  ld.ref_update = 0;
  ld.integrator = desc->integrator;
  ld.ode_rtol = desc->ode_rtol;
  ld.ode_atol = desc->ode_atol;
  ld.ode_max_substeps = desc->ode_max_substeps;
  rc = job_load(*p.job, &ld);
  if (rc != GSM_OK) return rc;
  p.job->bytes += ode_bytes(*p.job);
  if (p.job->bytes + plan_bytes(desc->N, desc->precision) > sv->budget) return GSM_ENOMEM;  // never admissible
  p.phase.assign(desc->phase, desc->phase + p.job->nvox);
  p.job->id = sv->next_id++;
  *id = p.job->id;
  sv->state[p.job->id] = 0;
  sv->queue.push_back(std::move(p));
  return GSM_OK;
}

int serve_tick(serve_handle h, int32_t* n_active, int32_t* n_queued, int32_t* n_finished) {
  if (!h) return GSM_EINVAL;
  Server* sv = reinterpret_cast<Server*>(h);
  Engine& g = sv->eng;
  // admission: first come first served while a slot and the HBM budget allow;
  // an admitted job starts at the smallest virtual time of the active jobs
  double vt_min = 0.0;
  for (size_t i = 0; i < sv->active.size(); ++i) vt_min = i ? std::min(vt_min, sv->active[i]->vt) : sv->active[i]->vt;
  while (!sv->queue.empty() && (int)sv->active.size() < sv->max_active) {
    Pending& p = sv->queue.front();
    Job& j = *p.job;
    const int n_prec = j.precision == MS_PREC_FP32_BULK ? 2 : 1;
    size_t extra = j.bytes;
    for (int f = 0; f < n_prec; ++f)
      if (!sv->plan_cost.count(std::make_pair(j.N, f))) extra += plan_bytes_one(j.N, f == 1);
    if (sv->used + extra > sv->budget) break;
    int rc = job_alloc(j, g.stream, p.phase.data());
    if (rc == GSM_OK) rc = job_alloc_ode(j, g.stream);
    if (rc != GSM_OK) return rc;
    Plans* pl = nullptr;
    for (int f = 0; f < n_prec; ++f) {
      const auto key = std::make_pair(j.N, f);
      if (!sv->plan_cost.count(key)) sv->plan_cost[key] = plan_bytes_one(j.N, f == 1);
      rc = g.get_plans(j.N, f == 1, &pl);
      if (rc != GSM_OK) return rc;
    }
    sv->used += extra;
    sv->state[j.id] = 1;
    j.vt = vt_min;
    sv->active.push_back(std::move(p.job));
    sv->queue.pop_front();
  }
  // fair share: the tick takes the jobs whose virtual time is within one
  // iteration of the largest job of the least-served job, so each active job
  // receives about the same GPU work per unit of time (a small grid runs many
  // iterations while a large one runs one) instead of one iteration each
  std::vector<Job*> batch;
  if (!sv->active.empty()) {
    double lo = sv->active[0]->vt, quantum = 0.0;
    for (auto& j : sv->active) {
      lo = std::min(lo, j->vt);
      quantum = std::max(quantum, serve_cost(*j));
    }
    for (auto& j : sv->active)
      if (j->vt <= lo + quantum) batch.push_back(j.get());
  }
  int rc = tick(g, batch);
  if (rc != GSM_OK) return rc;
  for (Job* j : batch) j->vt += serve_cost(*j);
  for (size_t i = 0; i < sv->active.size();) {
    if (sv->active[i]->done) {
      std::unique_ptr<Job> j = std::move(sv->active[i]);
      sv->active.erase(sv->active.begin() + i);
      job_free(*j, g.stream);
      sv->used -= j->bytes;
      sv->state[j->id] = j->notconv ? 3 : 2;
      sv->finished[j->id] = std::move(j);
    } else {
      ++i;
    }
  }
  if (n_active) *n_active = (int32_t)sv->active.size();
  if (n_queued) *n_queued = (int32_t)sv->queue.size();
  if (n_finished) *n_finished = (int32_t)sv->finished.size();
  return GSM_OK;
}

int serve_job_state(serve_handle h, int64_t id, int32_t* state, int32_t* step, int64_t* total_iters) {
  if (!h || !state) return GSM_EINVAL;
  Server* sv = reinterpret_cast<Server*>(h);
  auto it = sv->state.find(id);
  if (it == sv->state.end()) return GSM_EINVAL;
  *state = it->second;
  const Job* j = nullptr;
  for (auto& a : sv->active)
    if (a->id == id) j = a.get();
  if (!j) {
    auto f = sv->finished.find(id);
    if (f != sv->finished.end()) j = f->second.get();
  }
  if (step) *step = j ? j->step : 0;
  if (total_iters) *total_iters = j ? j->total_iters : 0;
  return GSM_OK;
}

int serve_fetch(serve_handle h, int64_t id, double* Sigma, int32_t* iters, double* final_error) {
  if (!h || !Sigma || !iters || !final_error) return GSM_EINVAL;
  Server* sv = reinterpret_cast<Server*>(h);
  auto it = sv->finished.find(id);
  if (it == sv->finished.end()) return GSM_EINVAL;
  const Job& j = *it->second;
  const int n = (int)j.h.size();
  std::memcpy(Sigma, j.Sigma.data(), 6 * n * sizeof(double));
  std::memcpy(iters, j.iters.data(), n * sizeof(int32_t));
  std::memcpy(final_error, j.final_error.data(), n * sizeof(double));
  const int rc = j.notconv ? GSM_ENOTCONV : GSM_OK;
  sv->finished.erase(it);
  sv->state.erase(id);
  return rc;
}

size_t serve_job_bytes(int N, int precision) {
  if (N < 2 || N > 1024) return 0;
  return job_bytes(N, precision) + plan_bytes(N, precision);
}

}  // extern "C"

// ============================================================= adjoint (tape)
// ms_run_taped keeps the per-step checkpoints (eps_k, z_{k-1}) of a load
// history; ms_adjoint runs the backward sweep over them (kernels and
// equations in adjoint_kernels.cuh).  The adjoint equilibrium of each step is
// solved by the basic-scheme fixed point lam <- lam - Gamma0 (C_t lam - a_u)
// with the context's FFT plans, Green-operator kernel and reductions.

struct Tape {
  Ctx* ctx = nullptr;
  int n_steps = 0;
  std::vector<double> E, h;
  double* ckpt = nullptr;  // [2][n_steps][6][nvox]: eps_k, then z_{k-1}
  double* Ct21 = nullptr;  // [21][nvox]
  double* a_u = nullptr;   // [6][nvox]
  double* yK = nullptr;    // [20][nvox]: y (5) and K upper triangle (15)
  double* gz = nullptr;    // [6][nvox]
  double* gz_prev = nullptr;
  double* cg_lam = nullptr;  // [6][nvox] conjugate gradients: lam, residual, direction
  double* cg_r = nullptr;
  double* cg_p = nullptr;
  double* part = nullptr;  // [3][grid]
  double* out_dev = nullptr;
  double* out_host = nullptr;
};

extern "C" {

int ms_run_taped(ms_handle h, const ms_load* load, ms_result* result, ms_tape_handle* tape_out) {
  if (!h || !load || !result || !tape_out) return GSM_EINVAL;
  *tape_out = nullptr;
  Ctx& c = *reinterpret_cast<Ctx*>(h);
  Job& j = c.job;
  if (load->n_steps < 1) return GSM_EINVAL;
  // the adjoint assumes prescribed macroscopic strains and the implicit-Euler
  // update; the reference medium of the forward run (fixed or per step) does
  // not enter the converged states the adjoint linearises
  if (load->stress_mask != 0 || load->integrator != 0) return GSM_ENOTSUP;
  Tape* t = new (std::nothrow) Tape;
  if (!t) return GSM_ENOMEM;
  t->ctx = &c;
  t->n_steps = load->n_steps;
  const int64_t n6 = 6 * j.nvox;
  const size_t ck = (size_t)2 * load->n_steps * n6 * sizeof(double);
  bool ok = cudaMalloc((void**)&t->ckpt, ck) == cudaSuccess &&
            cudaMalloc((void**)&t->Ct21, 21 * j.nvox * sizeof(double)) == cudaSuccess &&
            cudaMalloc((void**)&t->a_u, n6 * sizeof(double)) == cudaSuccess &&
            cudaMalloc((void**)&t->yK, 20 * j.nvox * sizeof(double)) == cudaSuccess &&
            cudaMalloc((void**)&t->gz, n6 * sizeof(double)) == cudaSuccess &&
            cudaMalloc((void**)&t->gz_prev, n6 * sizeof(double)) == cudaSuccess &&
            cudaMalloc((void**)&t->cg_lam, n6 * sizeof(double)) == cudaSuccess &&
            cudaMalloc((void**)&t->cg_r, n6 * sizeof(double)) == cudaSuccess &&
            cudaMalloc((void**)&t->cg_p, n6 * sizeof(double)) == cudaSuccess &&
            cudaMalloc((void**)&t->part, 3 * 4096 * sizeof(double)) == cudaSuccess &&
            cudaMalloc((void**)&t->out_dev, 4 * sizeof(double)) == cudaSuccess &&
            cudaMallocHost((void**)&t->out_host, 4 * sizeof(double)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    ms_tape_destroy(reinterpret_cast<ms_tape_handle>(t));
    return GSM_ENOMEM;
  }
  j.tape_eps = t->ckpt;
  j.tape_zprev = t->ckpt + (size_t)load->n_steps * n6;
  const int rc = ms_run(h, load, nullptr, result);
  j.tape_eps = j.tape_zprev = nullptr;
  if (rc != GSM_OK && rc != GSM_ENOTCONV) {
    ms_tape_destroy(reinterpret_cast<ms_tape_handle>(t));
    return rc;
  }
  t->E.assign(load->E, load->E + 6 * load->n_steps);
  t->h.assign(load->h, load->h + load->n_steps);
  *tape_out = reinterpret_cast<ms_tape_handle>(t);
  return rc;
}

int ms_adjoint(ms_tape_handle th, const double* w, int phase_id, double tol, int max_iter, double* grad,
               int32_t* lam_iters) {
  if (!th || !w || !grad || max_iter < 1 || !(tol > 0.0)) return GSM_EINVAL;
  Tape& t = *reinterpret_cast<Tape*>(th);
  Ctx& c = *t.ctx;
  Job& j = c.job;
  Engine& g = c.eng;
  if (phase_id < 0 || phase_id >= kMaxPhases || j.tab_host.kind[phase_id] != GSM_PSI_ELASTIC_VP_DEV)
    return GSM_EINVAL;
  cudaStream_t s = g.stream;
  const int64_t nv = j.nvox, n6 = 6 * nv;
  const double n3 = (double)nv, inv_n3 = 1.0 / n3;
  // parameters of the differentiated phase (E, sigma0, edot0, n)
  NortonTheta nt;
  {
    const LawParams<double>& p = j.tab_host.p64[phase_id];
    // E from the Lame constants: E = mu (3 lam + 2 mu) / (lam + mu)
    nt.E = p.mu * (3.0 * p.lam + 2.0 * p.mu) / (p.lam + p.mu);
  }
  nt.sigma0 = j.theta[phase_id][0];
  nt.edot0 = j.theta[phase_id][1];
  nt.n = j.theta[phase_id][2];
  Plans* pl = nullptr;
  int rc = g.get_plans(j.N, false, &pl);
  if (rc != GSM_OK) return rc;
  const int grid_prep = grid_cap(nv, kAdjBlock, 4);
  const int grid_fin = std::min(grid_cap(nv, kAdjBlock, 8), 4096);
  double total[3] = {0.0, 0.0, 0.0};
  bool capped = false;
  cudaMemsetAsync(t.gz, 0, n6 * sizeof(double), s);
  for (int k = t.n_steps - 1; k >= 0; --k) {
    const double* eps_k = t.ckpt + (size_t)k * n6;
    const double* zprev = t.ckpt + (size_t)(t.n_steps + k) * n6;
    const double hk = t.h[k];
    double gs[6] = {0, 0, 0, 0, 0, 0};
    if (k == t.n_steps - 1)
      for (int q = 0; q < 6; ++q) gs[q] = w[q] * inv_n3;
    if (j.law_mode == MODE_FP64)
      adj_prepare_kernel<MODE_FP64><<<grid_prep, kAdjBlock, 0, s>>>(nv, j.phase, j.tab_dev, hk, eps_k, zprev, gs[0],
                                                                     gs[1], gs[2], gs[3], gs[4], gs[5], t.gz, t.Ct21,
                                                                     t.a_u, t.yK);
    else
      adj_prepare_kernel<MODE_FP32_FIX><<<grid_prep, kAdjBlock, 0, s>>>(nv, j.phase, j.tab_dev, hk, eps_k, zprev,
                                                                         gs[0], gs[1], gs[2], gs[3], gs[4], gs[5],
                                                                         t.gz, t.Ct21, t.a_u, t.yK);
    count_launch();
    // adjoint equilibrium by conjugate gradients on G (C_t lam) = G a_u, G the
    // Green operator of C0 = identity (lam0 = 0, mu0 = 1/2): lam, r, p
    // normalised in the tape's CG arrays, C_t p in sig, G (.) through sig_hat /
    // eps_hat into eps_raw as -N^3 G (.)
    JobView& v = g.views_host[0];
    std::memset(&v, 0, sizeof v);
    v.sig_hat = j.f64.sig_hat;
    v.eps_hat = j.f64.eps_hat;
    v.mat_part = j.mat_part;
    v.gam_part = j.gam_part;
    v.nvox = nv;
    v.nmodes = j.nmodes;
    v.n_vch = 0;
    v.n_mch = j.n_mch;
    v.N = j.N;
    v.inv_n3 = inv_n3;
    v.lam0 = 0.0;
    v.mu0 = 0.5;
    cudaMemcpyAsync(g.views_dev, g.views_host, sizeof(JobView), cudaMemcpyHostToDevice, s);
    const int gam_grid = (int)std::min<int64_t>(j.n_mch, (int64_t)sm_count() * g.per_sm_gam[0]);
    auto apply_G = [&](const double* tau) -> int {
      if (cufftExecD2Z(pl->r2c, const_cast<double*>(tau), j.f64.sig_hat) != CUFFT_SUCCESS) return GSM_ECUDA;
      cudaMemsetAsync(j.f64.eps_hat, 0, 6 * j.nmodes * sizeof(cufftDoubleComplex), s);
      ms_gamma_batch_kernel<double><<<gam_grid, kGamBlock, 0, s>>>(g.views_dev, 1, j.n_mch);
      count_launch();
      if (cufftExecZ2D(pl->c2r, j.f64.sig_hat, j.f64.eps_raw) != CUFFT_SUCCESS) return GSM_ECUDA;
      return GSM_OK;
    };
    std::vector<double> part_h(grid_fin);
    auto reduce = [&](double* out) -> int {  // fixed-order sum of the block partials
      if (cudaMemcpyAsync(part_h.data(), t.part, grid_fin * sizeof(double), cudaMemcpyDeviceToHost, s) !=
              cudaSuccess ||
          cudaStreamSynchronize(s) != cudaSuccess)
        return GSM_ECUDA;
      double acc = 0.0;
      for (int b = 0; b < grid_fin; ++b) acc += part_h[b];
      *out = acc;
      return GSM_OK;
    };
    int it = 0;
    bool conv = false, cg_ok = true;
    {
      if ((rc = apply_G(t.a_u)) != GSM_OK) return rc;
      convert<double, double>(s, j.f64.eps_raw, t.cg_r, n6, -inv_n3);
      cudaMemcpyAsync(t.cg_p, t.cg_r, n6 * sizeof(double), cudaMemcpyDeviceToDevice, s);
      cudaMemsetAsync(t.cg_lam, 0, n6 * sizeof(double), s);
      double rr = 0.0;
      cg_dot_kernel<<<grid_fin, kAdjBlock, 0, s>>>(nv, t.cg_r, t.cg_r, 1.0, t.part);
      count_launch();
      if ((rc = reduce(&rr)) != GSM_OK) return rc;
      const double rr0 = rr;
      if (!(rr0 > 0.0)) conv = true;
      while (!conv && it < max_iter) {
        adj_ct_apply_kernel<<<elt_grid(nv), 256, 0, s>>>(nv, t.Ct21, t.cg_p, j.f64.sig);
        count_launch();
        if ((rc = apply_G(j.f64.sig)) != GSM_OK) return rc;
        double pq = 0.0;
        cg_dot_kernel<<<grid_fin, kAdjBlock, 0, s>>>(nv, t.cg_p, j.f64.eps_raw, -inv_n3, t.part);
        count_launch();
        if ((rc = reduce(&pq)) != GSM_OK) return rc;
        if (!(pq > 0.0) || !std::isfinite(pq)) {  // not positive definite: the fixed point below
          cg_ok = false;
          break;
        }
        const double a = rr / pq;
        double rr_new = 0.0;
        cg_update_kernel<<<grid_fin, kAdjBlock, 0, s>>>(nv, a, -inv_n3, t.cg_p, j.f64.eps_raw, t.cg_lam, t.cg_r,
                                                         t.part);
        count_launch();
        if ((rc = reduce(&rr_new)) != GSM_OK) return rc;
        ++it;
        if (std::sqrt(rr_new) <= tol * std::sqrt(rr0)) {
          conv = true;
          break;
        }
        cg_direction_kernel<<<elt_grid(n6), 256, 0, s>>>(n6, rr_new / rr, t.cg_r, t.cg_p);
        count_launch();
        rr = rr_new;
      }
      if (cg_ok) convert<double, double>(s, t.cg_lam, j.f64.eps_raw, n6, n3);  // N^3 lam for the finish kernel
    }
    if (!cg_ok) {
      it = 0;
      conv = false;
      // the step's reference medium for the adjoint equilibrium: midpoints of the
      // tangent field's isotropic measures
      double lam0 = j.lam0_el, mu0 = j.mu0_el;
      {
        const int rg = std::min(grid_cap(nv, kAdjBlock, 4), 1024);
        adj_reference_kernel<<<rg, kAdjBlock, 0, s>>>(nv, t.Ct21, t.part);
        count_launch();
        std::vector<double> part(4 * (size_t)rg);
        if (cudaMemcpyAsync(part.data(), t.part, part.size() * sizeof(double), cudaMemcpyDeviceToHost, s) !=
                cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
          return GSM_ECUDA;
        double r[4] = {1e300, -1e300, 1e300, -1e300};
        for (int b = 0; b < rg; ++b) {
          r[0] = std::min(r[0], part[b]);
          r[1] = std::max(r[1], part[rg + b]);
          r[2] = std::min(r[2], part[2 * rg + b]);
          r[3] = std::max(r[3], part[3 * rg + b]);
        }
        const double k0 = 0.5 * (r[0] + r[1]), m0 = 0.5 * (r[2] + r[3]);
        if (m0 > 0.0 && k0 > 0.0 && std::isfinite(k0 + m0)) {
          mu0 = m0;
          lam0 = k0 - 2.0 * m0 / 3.0;
        }
      }
      // adjoint equilibrium: lam in eps_raw (N^3 lam), lam^ in eps_hat
      cudaMemsetAsync(j.f64.eps_raw, 0, n6 * sizeof(double), s);
      cudaMemsetAsync(j.f64.eps_hat, 0, 6 * j.nmodes * sizeof(cufftDoubleComplex), s);
      std::memset(&v, 0, sizeof v);
      v.sig_hat = j.f64.sig_hat;
      v.eps_hat = j.f64.eps_hat;
      v.mat_part = j.mat_part;
      v.gam_part = j.gam_part;
      v.nvox = nv;
      v.nmodes = j.nmodes;
      v.n_vch = 0;
      v.n_mch = j.n_mch;
      v.N = j.N;
      v.inv_n3 = inv_n3;
      v.lam0 = lam0;
      v.mu0 = mu0;
      cudaMemcpyAsync(g.views_dev, g.views_host, sizeof(JobView), cudaMemcpyHostToDevice, s);
      double first = -1.0;
      for (; it < max_iter; ++it) {
        adj_tau_kernel<<<elt_grid(nv), 256, 0, s>>>(nv, t.Ct21, t.a_u, j.f64.eps_raw, inv_n3, j.f64.sig);
        if (cufftExecD2Z(pl->r2c, j.f64.sig, j.f64.sig_hat) != CUFFT_SUCCESS) return GSM_ECUDA;
        ms_gamma_batch_kernel<double><<<gam_grid, kGamBlock, 0, s>>>(g.views_dev, 1, j.n_mch);
        ms_finalize_batch_kernel<<<1, kFinBlock, 0, s>>>(g.views_dev, g.red_dev);
        count_launch(3);
        cudaMemcpyAsync(g.red_host, g.red_dev, sizeof(Reduced), cudaMemcpyDeviceToHost, s);
        if (cudaStreamSynchronize(s) != cudaSuccess) return GSM_ECUDA;
        const double r = std::sqrt(g.red_host->res);
        if (first < 0.0) first = r;
        if (r <= tol * first || first == 0.0) {
          conv = true;
          break;
        }
        if (cufftExecZ2D(pl->c2r, j.f64.sig_hat, j.f64.eps_raw) != CUFFT_SUCCESS) return GSM_ECUDA;
      }
      if (conv) ++it;  // the evaluation that met the tolerance
    }
    if (lam_iters) lam_iters[k] = it;
    capped = capped || !conv;
    adj_finish_kernel<<<grid_fin, kAdjBlock, 0, s>>>(nv, j.phase, j.tab_dev, hk, phase_id, nt, eps_k, zprev, gs[0],
                                                     gs[1], gs[2], gs[3], gs[4], gs[5], t.gz, j.f64.eps_raw, inv_n3,
                                                     t.yK, t.gz_prev, t.part);
    adj_sum_kernel<<<1, 32, 0, s>>>(t.part, grid_fin, t.out_dev);
    count_launch(2);
    cudaMemcpyAsync(t.out_host, t.out_dev, 3 * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess) return GSM_ECUDA;
    for (int q = 0; q < 3; ++q) total[q] += t.out_host[q];
    std::swap(t.gz, t.gz_prev);
  }
  for (int q = 0; q < 3; ++q) grad[q] = total[q];
  return capped ? GSM_ENOTCONV : GSM_OK;
}

int ms_tape_destroy(ms_tape_handle th) {
  if (!th) return GSM_OK;
  Tape* t = reinterpret_cast<Tape*>(th);
  if (t->ctx) cudaStreamSynchronize(t->ctx->eng.stream);
  cudaFree(t->ckpt);
  cudaFree(t->Ct21);
  cudaFree(t->a_u);
  cudaFree(t->yK);
  cudaFree(t->gz);
  cudaFree(t->gz_prev);
  cudaFree(t->cg_lam);
  cudaFree(t->cg_r);
  cudaFree(t->cg_p);
  cudaFree(t->part);
  cudaFree(t->out_dev);
  cudaFreeHost(t->out_host);
  delete t;
  return GSM_OK;
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
int g_noalloc_per_sm[kMaxDevices] = {};

// Device address of the scratch array on the current device and the material
// kernel's resident blocks per SM there (both set up on the first call per
// device, under the mutex).
int noalloc_scratch(double** out, int* per_sm) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return GSM_ECUDA;
  if (dev < 0 || dev >= kMaxDevices) return GSM_ENOTSUP;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_ms_eval_scratch) != cudaSuccess || !p) return GSM_ECUDA;
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, ms_material_kernel<double, MODE_FP64>, kMatBlock, 0) !=
            cudaSuccess ||
        b <= 0)
      b = 1;
    g_noalloc_per_sm[dev] = b;
    g_noalloc_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_noalloc_ptr[dev];
  *per_sm = g_noalloc_per_sm[dev];
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
    if (m->psi_kind == GSM_PSI_ELASTIC_VP_KIN) return GSM_ENOTSUP;  // implicit-Euler laws only
    tab.kind[p] = m->psi_kind;
    tab.p64[p] = m->p64;
    tab.p32[p] = m->p32;
  }
  double* scratch = nullptr;
  int per_sm = 1;
  int rc = noalloc_scratch(&scratch, &per_sm);
  if (rc != GSM_OK) return rc;
  const int64_t nvox = (int64_t)N * N * N;
  const int grid = std::min(grid_cap(nvox, kMatBlock, per_sm), kNoAllocMaxBlocks);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double* partials = scratch;                                    // [6][grid]
  Reduced* red = reinterpret_cast<Reduced*>(scratch + 6 * kNoAllocMaxBlocks);
  ms_material_kernel<double, MODE_FP64><<<grid, kMatBlock, 0, s>>>(nvox, phase, tab, make_step(step_h), 1.0, eps, z_n, sigma, z,
                                                                   partials);
  ms_finalize_kernel<<<1, kFinBlock, 0, s>>>(partials, grid, nullptr, 0, 1.0 / (double)nvox, 1.0, red);
  count_launch(2);
  if (cudaGetLastError() != cudaSuccess) return GSM_ECUDA;
  if (cudaMemcpyAsync(mean, red->mean, 6 * sizeof(double), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return GSM_ECUDA;
  return GSM_OK;
}
