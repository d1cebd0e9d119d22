// gsm_create / gsm_update / gsm_destroy: the batched per-voxel material
// update (AutoMat, arXiv 2006.04391, Sec. 4.1 and Sec. 6) on sm_103a.
//
// One thread per voxel, as in the paper (Sec. 6), but with the fields
// resident in HBM in structure-of-arrays layout (the paper staged chunks
// through pinned host memory over PCIe): every component load and store of a
// warp is one coalesced 256-byte (FP64) transaction.  The grid is a
// persistent grid-stride loop sized from the occupancy of the instantiation;
// the loop bound is uniform per block so every lane of a warp takes part in
// the Newton convergence votes (padding lanes are inactive).
#include <cstdio>
#include <mutex>

#include <algorithm>

#include "common.cuh"
#include "voxel.cuh"

namespace gsm {

std::atomic<int64_t> g_launches{0};

namespace {

constexpr int kBlock = 128;

template <class T> __device__ __forceinline__ T ldg(const T* p) { return __ldg(p); }

// Viscoplastic (Norton) voxels.  The FP32-bulk update without tangent is
// held to kFixBlocks blocks of 128 threads per SM (128 registers at 4): its
// FP64 and double-float correction needs the warps to hide the FP64 pipe's
// latency.
#ifndef GSM_FIX_BLOCKS
#define GSM_FIX_BLOCKS 4
#endif
constexpr int kFixBlocks = GSM_FIX_BLOCKS;
template <int MODE, bool TAN>
__global__ void __launch_bounds__(kBlock, (MODE == MODE_FP32_FIX && !TAN) ? kFixBlocks : 1) norton_kernel(int64_t n, int64_t ld, LawParams<double> p,
                                                        LawParams<float> pf, Step hs,
                                                        const void* __restrict__ eps_,
                                                        const void* __restrict__ zn_, void* __restrict__ sig_,
                                                        void* __restrict__ z_, void* __restrict__ tan_,
                                                        int32_t* __restrict__ status) {
  using IO = std::conditional_t<MODE == MODE_FP32, float, double>;
  const IO* eps = static_cast<const IO*>(eps_);
  const IO* zn = static_cast<const IO*>(zn_);
  IO* sig = static_cast<IO*>(sig_);
  IO* z = static_cast<IO*>(z_);
  IO* tan = static_cast<IO*>(tan_);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const NortonDf cdf = norton_df(p, hs.inv_h);  // formed once per thread (FP32_FIX)
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
    const int64_t i = base + threadIdx.x;
    const bool active = i < n;
    IO e[6], zi[6], s[6], zo[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      e[c] = active ? ldg(eps + c * ld + i) : IO(0);
      zi[c] = active ? ldg(zn + c * ld + i) : IO(0);
    }
    IO t[21];
    unsigned st;
    if constexpr (MODE == MODE_FP64) {
      st = voxel_fp64<NortonDev>(p, e, zi, hs, active, s, zo, TAN ? t : nullptr);
    } else if constexpr (MODE == MODE_FP32_FIX) {
      st = voxel_fp32_fix<NortonDev>(p, pf, e, zi, hs, active, s, zo, TAN ? t : nullptr, nullptr, &cdf);
    } else {
      st = voxel_fp32<NortonDev>(pf, e, zi, hs, active, s, zo, TAN ? t : nullptr);
    }
    bool fin = true;
#pragma unroll
    for (int c = 0; c < 6; ++c) fin = fin && finite64(s[c]) && finite64(zo[c]);
    if (!fin) st |= ST_NONFINITE;
    if (active) {
#pragma unroll
      for (int c = 0; c < 6; ++c) {
        sig[c * ld + i] = s[c];
        z[c * ld + i] = zo[c];
      }
      if (TAN) {
#pragma unroll
        for (int c = 0; c < 21; ++c) tan[c * ld + i] = t[c];
      }
      if (status) status[i] = (int32_t)st;
    }
  }
}

// Linear-elastic voxels.
template <class IO, bool TAN>
__global__ void __launch_bounds__(kBlock) elastic_kernel(int64_t n, int64_t ld, LawParams<IO> p,
                                                         const IO* __restrict__ eps, const IO* __restrict__ zn,
                                                         IO* __restrict__ sig, IO* __restrict__ z,
                                                         IO* __restrict__ tan, int32_t* __restrict__ status) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    IO e[6], s[6], t[21];
#pragma unroll
    for (int c = 0; c < 6; ++c) e[c] = ldg(eps + c * ld + i);
    voxel_elastic<IO>(p, e, s, TAN ? t : nullptr);
    bool fin = true;
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      sig[c * ld + i] = s[c];
      fin = fin && isfinite(s[c]);
    }
    if (z) {
#pragma unroll
      for (int c = 0; c < 6; ++c) z[c * ld + i] = zn ? ldg(zn + c * ld + i) : IO(0);
    }
    if (TAN) {
#pragma unroll
      for (int c = 0; c < 21; ++c) tan[c * ld + i] = t[c];
    }
    if (status) status[i] = (int32_t)(ST_CONVERGED | (fin ? 0u : ST_NONFINITE));
  }
}

// Persistent grid: SMs x resident blocks of this instantiation (one cached
// occupancy per kernel: the template parameter is the kernel itself).
template <auto Kernel> int grid_for(int64_t n) {
  static const int per_sm = [] {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, Kernel, kBlock, 0) != cudaSuccess || b <= 0) b = 1;
    return b;
  }();
  const int64_t need = (n + kBlock - 1) / kBlock;
  const int64_t cap = (int64_t)sm_count() * per_sm;
  return (int)(need < cap ? need : cap);
}

template <int MODE, bool TAN>
cudaError_t launch_norton(const Material& m, int64_t n, int64_t ld, double h, const void* eps, const void* zn,
                          void* sig, void* z, void* tan, int32_t* status, cudaStream_t s) {
  norton_kernel<MODE, TAN><<<grid_for<norton_kernel<MODE, TAN>>(n), kBlock, 0, s>>>(n, ld, m.p64, m.p32, make_step(h), eps, zn, sig, z, tan, status);
  count_launch();
  return cudaGetLastError();
}

template <class IO, bool TAN>
cudaError_t launch_elastic(const LawParams<IO>& p, int64_t n, int64_t ld, const void* eps, const void* zn,
                           void* sig, void* z, void* tan, int32_t* status, cudaStream_t s) {
  elastic_kernel<IO, TAN><<<grid_for<elastic_kernel<IO, TAN>>(n), kBlock, 0, s>>>(
      n, ld, p, static_cast<const IO*>(eps), static_cast<const IO*>(zn), static_cast<IO*>(sig),
      static_cast<IO*>(z), static_cast<IO*>(tan), status);
  count_launch();
  return cudaGetLastError();
}

bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

}  // namespace

// Launch the update of one material on n voxels (also used by the basic scheme).
int material_update(const Material& m, int64_t n, const void* eps, const void* zn, int64_t ld, double h,
                    void* sig, void* z, void* tan, int32_t* status, cudaStream_t s) {
  cudaError_t err;
  const bool t = tan != nullptr;
  if (m.psi_kind == GSM_PSI_ELASTIC) {
    if (m.precision == GSM_FP32)
      err = t ? launch_elastic<float, true>(m.p32, n, ld, eps, zn, sig, z, tan, status, s)
              : launch_elastic<float, false>(m.p32, n, ld, eps, zn, sig, z, tan, status, s);
    else
      err = t ? launch_elastic<double, true>(m.p64, n, ld, eps, zn, sig, z, tan, status, s)
              : launch_elastic<double, false>(m.p64, n, ld, eps, zn, sig, z, tan, status, s);
  } else {
    switch (m.precision) {
      case GSM_FP64:
        err = t ? launch_norton<MODE_FP64, true>(m, n, ld, h, eps, zn, sig, z, tan, status, s)
                : launch_norton<MODE_FP64, false>(m, n, ld, h, eps, zn, sig, z, tan, status, s);
        break;
      case GSM_FP32_FP64FIX:
        err = t ? launch_norton<MODE_FP32_FIX, true>(m, n, ld, h, eps, zn, sig, z, tan, status, s)
                : launch_norton<MODE_FP32_FIX, false>(m, n, ld, h, eps, zn, sig, z, tan, status, s);
        break;
      default:
        err = t ? launch_norton<MODE_FP32, true>(m, n, ld, h, eps, zn, sig, z, tan, status, s)
                : launch_norton<MODE_FP32, false>(m, n, ld, h, eps, zn, sig, z, tan, status, s);
        break;
    }
  }
  return err == cudaSuccess ? GSM_OK : GSM_ECUDA;
}

// The address under which the current device reaches p: p itself for device
// and managed memory, the mapped address for page-locked host memory; false
// for memory the device cannot reach.  NULL maps to NULL.
bool device_address(const void* p, const void** out) {
  *out = p;
  if (!p) return true;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  switch (a.type) {
    case cudaMemoryTypeDevice:
    case cudaMemoryTypeManaged:
      return true;
    case cudaMemoryTypeHost:
      if (!a.devicePointer) return false;
      *out = a.devicePointer;
      return true;
    default:
      return false;
  }
}

int validate_material(int psi_kind, int phi_kind, const double* prm, int n_params, int precision) {
  if (!prm) return GSM_EINVAL;
  if (precision < GSM_FP64 || precision > GSM_FP32) return GSM_EINVAL;
  if (psi_kind == GSM_PSI_ELASTIC && phi_kind == GSM_PHI_NONE) {
    if (n_params != 2) return GSM_EINVAL;
  } else if (psi_kind == GSM_PSI_ELASTIC_VP_DEV && phi_kind == GSM_PHI_NORTON) {
    if (n_params != 5) return GSM_EINVAL;
    if (!finite_pos(prm[2]) || !finite_pos(prm[3]) || !finite_pos(prm[4])) return GSM_EINVAL;
  } else if (psi_kind == GSM_PSI_ELASTIC_VP_KIN && phi_kind == GSM_PHI_MS_FORCE) {
    if (n_params != 7) return GSM_EINVAL;
    if (!(std::isfinite(prm[2]) && prm[2] >= 0.0) || !(std::isfinite(prm[3]) && prm[3] >= 0.0) ||
        !finite_pos(prm[4]) || !finite_pos(prm[5]) || !(std::isfinite(prm[6]) && prm[6] >= 1.0))
      return GSM_EINVAL;
  } else {
    return GSM_EINVAL;
  }
  if (!finite_pos(prm[0]) || !std::isfinite(prm[1]) || !(prm[1] > -1.0 && prm[1] < 0.5)) return GSM_EINVAL;
  return GSM_OK;
}

}  // namespace gsm

using namespace gsm;

extern "C" {

int gsm_create(gsm_handle* out, int psi_kind, int phi_kind, const double* params, int n_params, int precision) {
  if (!out) return GSM_EINVAL;
  *out = nullptr;
  const int rc = validate_material(psi_kind, phi_kind, params, n_params, precision);
  if (rc != GSM_OK) return rc;
  Material* m = new (std::nothrow) Material;
  if (!m) return GSM_ENOMEM;
  m->psi_kind = psi_kind;
  m->phi_kind = phi_kind;
  m->precision = precision;
  for (int i = 0; i < 8; ++i) m->params[i] = i < n_params ? params[i] : 0.0;
  m->p64 = make_params(params, psi_kind);
  m->p32 = to_float(m->p64);
  *out = reinterpret_cast<gsm_handle>(m);
  return GSM_OK;
}

int gsm_destroy(gsm_handle h) {
  delete reinterpret_cast<Material*>(h);
  return GSM_OK;
}

int gsm_update(gsm_handle h, int64_t n_vox, const void* eps, const void* z_n, int64_t ld, double step_h,
               void* sigma, void* z, void* tangent, int32_t* status, void* stream) {
  if (!h || n_vox < 0 || ld < n_vox) return GSM_EINVAL;
  if (n_vox == 0) return GSM_OK;
  const Material& m = *reinterpret_cast<const Material*>(h);
  if (!eps || !sigma) return GSM_EINVAL;
  if (m.psi_kind == GSM_PSI_ELASTIC_VP_KIN) return GSM_ENOTSUP;  // force-potential form: gsm_update_ode23
  if (m.psi_kind == GSM_PSI_ELASTIC_VP_DEV && (!z_n || !z)) return GSM_EINVAL;
  if (!(std::isfinite(step_h) && step_h > 0.0)) return GSM_EINVAL;
  // every array may be device memory or page-locked host memory (read and
  // written by the kernel over the host link); unregistered host memory is
  // refused rather than faulted on
  const void* in[2] = {eps, z_n};
  void* out[4] = {sigma, z, tangent, status};
  for (auto& p : in)
    if (!device_address(p, &p)) return GSM_EINVAL;
  for (auto& p : out) {
    const void* q = p;
    if (!device_address(q, &q)) return GSM_EINVAL;
    p = const_cast<void*>(q);
  }
  return material_update(m, n_vox, in[0], in[1], ld, step_h, out[0], out[1], out[2], static_cast<int32_t*>(out[3]),
                         static_cast<cudaStream_t>(stream));
}

// Chunked host <-> device streaming of gsm_update: three slots of device
// staging buffers; host->device copies on one stream, the updates on the
// caller's stream, device->host copies on a third, ordered by events so that
// the copies of chunks i + 1 and i - 1 overlap the update of chunk i.
int gsm_update_host(gsm_handle h, int64_t n_vox, const void* eps, const void* z_n, int64_t ld, double step_h,
                    void* sigma, void* z, void* tangent, int32_t* status, int64_t chunk, void* stream) {
  if (!h || n_vox < 0 || ld < n_vox || chunk < 0) return GSM_EINVAL;
  if (n_vox == 0) return GSM_OK;
  const Material& m = *reinterpret_cast<const Material*>(h);
  if (!eps || !sigma) return GSM_EINVAL;
  if (m.psi_kind == GSM_PSI_ELASTIC_VP_KIN) return GSM_ENOTSUP;
  const bool vp = m.psi_kind == GSM_PSI_ELASTIC_VP_DEV;
  if (vp && (!z_n || !z)) return GSM_EINVAL;
  if (!(std::isfinite(step_h) && step_h > 0.0)) return GSM_EINVAL;
  // every array must be page-locked host memory (the copy engines read and write it)
  const void* all[6] = {eps, z_n, sigma, z, tangent, status};
  for (const void* p : all) {
    if (!p) continue;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
      cudaGetLastError();
      return GSM_EINVAL;
    }
    if (a.type != cudaMemoryTypeHost) return GSM_EINVAL;
  }
  const int64_t C = std::min<int64_t>(chunk > 0 ? chunk : (int64_t)1 << 20, n_vox);
  const size_t es = m.precision == GSM_FP32 ? sizeof(float) : sizeof(double);
  const bool use_z = z_n && z;  // (the elastic law copies z_n into z when both are given)
  // per slot: eps, z_n, sigma, z [6][C]; tangent [21][C]; status [C]
  const size_t f6 = 6 * C * es, f21 = tangent ? 21 * C * es : 0, fst = status ? C * sizeof(int32_t) : 0;
  const size_t slot = 2 * f6 + (use_z ? 2 * f6 : 0) + f21 + fst;
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  constexpr int kSlots = 3;
  char* buf = nullptr;
  if (cudaMallocAsync((void**)&buf, kSlots * slot, cs) != cudaSuccess) {
    cudaGetLastError();
    return GSM_ENOMEM;
  }
  cudaStream_t in_s = nullptr, out_s = nullptr;
  cudaEvent_t start = nullptr, end = nullptr, in_done[kSlots] = {}, comp_done[kSlots] = {}, out_done[kSlots] = {};
  bool ok = cudaStreamCreateWithFlags(&in_s, cudaStreamNonBlocking) == cudaSuccess &&
            cudaStreamCreateWithFlags(&out_s, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&start, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&end, cudaEventDisableTiming) == cudaSuccess;
  for (int k = 0; ok && k < kSlots; ++k)
    ok = cudaEventCreateWithFlags(&in_done[k], cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&comp_done[k], cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&out_done[k], cudaEventDisableTiming) == cudaSuccess;
  int rc = ok ? GSM_OK : GSM_ECUDA;
  if (ok) {
    // the copies start after the work already queued on the caller's stream
    ok = cudaEventRecord(start, cs) == cudaSuccess && cudaStreamWaitEvent(in_s, start, 0) == cudaSuccess;
    const size_t hp = ld * es;  // host row pitch
    const int64_t n_chunks = (n_vox + C - 1) / C;
    for (int64_t i = 0; ok && i < n_chunks; ++i) {
      const int k = (int)(i % kSlots);
      const int64_t c0 = i * C, len = std::min<int64_t>(C, n_vox - c0);
      char* sb = buf + k * slot;
      char* d_eps = sb;
      char* d_zn = use_z ? sb + f6 : nullptr;
      char* d_sig = sb + (use_z ? 2 * f6 : f6);
      char* d_z = use_z ? sb + 3 * f6 : nullptr;
      char* d_tan = tangent ? sb + (use_z ? 4 * f6 : 2 * f6) : nullptr;
      int32_t* d_st = status ? reinterpret_cast<int32_t*>(sb + (use_z ? 4 * f6 : 2 * f6) + f21) : nullptr;
      const size_t dp = C * es, w = len * es, off = c0 * es;
      // host -> device, once the update of the slot's previous chunk has read its inputs
      if (i >= kSlots) ok = ok && cudaStreamWaitEvent(in_s, comp_done[k], 0) == cudaSuccess;
      ok = ok && cudaMemcpy2DAsync(d_eps, dp, static_cast<const char*>(eps) + off, hp, w, 6,
                                   cudaMemcpyHostToDevice, in_s) == cudaSuccess;
      if (use_z)
        ok = ok && cudaMemcpy2DAsync(d_zn, dp, static_cast<const char*>(z_n) + off, hp, w, 6,
                                     cudaMemcpyHostToDevice, in_s) == cudaSuccess;
      ok = ok && cudaEventRecord(in_done[k], in_s) == cudaSuccess;
      // the update, once the inputs are in and the slot's previous outputs are out
      ok = ok && cudaStreamWaitEvent(cs, in_done[k], 0) == cudaSuccess;
      if (i >= kSlots) ok = ok && cudaStreamWaitEvent(cs, out_done[k], 0) == cudaSuccess;
      if (ok) {
        const int r = material_update(m, len, d_eps, d_zn, C, step_h, d_sig, d_z, d_tan, d_st, cs);
        if (r != GSM_OK) {
          rc = r;
          ok = false;
        }
      }
      ok = ok && cudaEventRecord(comp_done[k], cs) == cudaSuccess;
      // device -> host
      ok = ok && cudaStreamWaitEvent(out_s, comp_done[k], 0) == cudaSuccess;
      ok = ok && cudaMemcpy2DAsync(static_cast<char*>(sigma) + off, hp, d_sig, dp, w, 6, cudaMemcpyDeviceToHost,
                                   out_s) == cudaSuccess;
      if (use_z)
        ok = ok && cudaMemcpy2DAsync(static_cast<char*>(z) + off, hp, d_z, dp, w, 6, cudaMemcpyDeviceToHost,
                                     out_s) == cudaSuccess;
      if (tangent)
        ok = ok && cudaMemcpy2DAsync(static_cast<char*>(tangent) + off, hp, d_tan, dp, w, 21,
                                     cudaMemcpyDeviceToHost, out_s) == cudaSuccess;
      if (status)
        ok = ok && cudaMemcpyAsync(status + c0, d_st, len * sizeof(int32_t), cudaMemcpyDeviceToHost, out_s) ==
                       cudaSuccess;
      ok = ok && cudaEventRecord(out_done[k], out_s) == cudaSuccess;
    }
    // the caller's stream continues once every result is in host memory
    ok = ok && cudaEventRecord(end, out_s) == cudaSuccess && cudaStreamWaitEvent(cs, end, 0) == cudaSuccess;
    if (!ok && rc == GSM_OK) rc = GSM_ECUDA;
    if (!ok) {
      // make sure nothing queued still uses the buffers before they go back
      cudaStreamSynchronize(in_s);
      cudaStreamSynchronize(out_s);
      cudaStreamSynchronize(cs);
    }
  }
  cudaFreeAsync(buf, cs);
  // (streams and events are released once their queued work has completed)
  for (int k = 0; k < kSlots; ++k) {
    if (in_done[k]) cudaEventDestroy(in_done[k]);
    if (comp_done[k]) cudaEventDestroy(comp_done[k]);
    if (out_done[k]) cudaEventDestroy(out_done[k]);
  }
  if (start) cudaEventDestroy(start);
  if (end) cudaEventDestroy(end);
  if (in_s) cudaStreamDestroy(in_s);
  if (out_s) cudaStreamDestroy(out_s);
  if (rc != GSM_OK) cudaGetLastError();
  return rc;
}

const char* gsm_strerror(int code) {
  switch (code) {
    case GSM_OK: return "ok";
    case GSM_EINVAL: return "invalid argument";
    case GSM_ENOMEM: return "out of memory";
    case GSM_ECUDA: return "CUDA or cuFFT error";
    case GSM_ENOTCONV: return "iteration cap reached";
    case GSM_ENOTSUP: return "not supported";
    default: return "unknown error";
  }
}

int64_t gsm_kernel_launches(void) { return g_launches.load(); }

}  // extern "C"
