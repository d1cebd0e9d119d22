// Double-float power for the double-float residual of the FP32-bulk
// correction: F = c (x 2^e)^a with x a positive double-float and 2^e an exact
// scaling, in FP32 pairs except three FP64 operations.
//
// The residual's power was ~26 of the correction's ~75 FP64 operations per
// voxel; on GB300 an FP32 instruction issues at 64 times the FP64 rate.  The
// method is that of fpow.cuh (Tang's table-driven log2 and exp2, ACM TOMS 15
// (1989) 144-157 and 16 (1990) 378-400) carried out in double-float
// arithmetic (dfloat.cuh), with the tables of gen_pow_tables.py split into
// FP32 pairs (within 2^-48 of their definitions):
//
//   x = 2^E2 m (m in [1, 2)), c_i = 1 + i/128 nearest to m (i = 0..128),
//   t = (m - c_i)/c_i with |t| <= 2^-8,
//   log2 m = log2 c_i + (t - t^2/2 + t^3/3 - t^4/4 + t^5/5 - t^6/6)/ln 2
//            (t - t^2/2 in pairs, the rest in FP32; remainder < 2^-56);
//   y = a (e + E2) + a log2 m: the first product can be large (e carries the
//   scaling of the residual, |a e| up to ~50) and a pair would lose 2^-48 of
//   it, so it is formed in FP64 and reduced there by its nearest multiple of
//   1/128 (one multiplication, one exact subtraction, one conversion);
//   y = N/128 + r, |r| <= 1/256 + 2^-20, 2^y = 2^(N >> 7) 2^((N & 127)/128) e^(r ln 2),
//   e^z - 1 = z + z^2/2 (pairs) + z^3/6 + z^4/24 + z^5/120 (FP32; |z| < 2^-8.4,
//   remainder < 2^-59).
//
// Relative error below 2^-45 (host test against a 40-digit reference; the
// pairs' own rounding, 2^-48 per operation, sets it).
// Inputs outside the fast path -- x not a positive normal pair, |a (e + E2)|
// >= 4096, a result exponent outside [-100, 100] -- report false; the caller
// takes the FP64 power there.
#pragma once

#include <cmath>
#include <cstring>

#include "dfloat.cuh"

namespace gsm {
namespace dpow {

#if defined(__CUDACC__)
#define GSM_DPOW_TABLE(name, n, ...)                  \
  __device__ const float name##_d[n] = __VA_ARGS__; \
  static const float name##_h[n] = __VA_ARGS__;
#else
#define GSM_DPOW_TABLE(name, n, ...) static const float name##_h[n] = __VA_ARGS__;
#endif
#include "dpow_tables.inc"
#undef GSM_DPOW_TABLE

#if defined(__CUDA_ARCH__)
#define GSM_DPOW_TAB(name, i) __ldg(&name##_d[i])
#else
#define GSM_DPOW_TAB(name, i) name##_h[i]
#endif

AD_HD unsigned fbits(float x) {
#if defined(__CUDA_ARCH__)
  return __float_as_uint(x);
#else
  unsigned b;
  std::memcpy(&b, &x, sizeof b);
  return b;
#endif
}

AD_HD float fof(unsigned b) {
#if defined(__CUDA_ARCH__)
  return __uint_as_float(b);
#else
  float x;
  std::memcpy(&x, &b, sizeof x);
  return x;
#endif
}

#define GSM_DPOW_PAIR(name, i) df{GSM_DPOW_TAB(name, 2 * (i)), GSM_DPOW_TAB(name, 2 * (i) + 1)}

// F = (acm 2^ace) (x 2^e)^a for a positive pair x, an integer scaling e, the
// exponent a as FP64 (a64) and as a pair (ad, the pair nearest to a64), and
// the constant factor as a pair mantissa acm in [1, 2) with its exponent ace.
// Returns false (F untouched) outside the fast path.
AD_HD bool pow_scaled(const df& x, int e, double a64, const df& ad, const df& acm, int ace, df& F) {
  const unsigned b = fbits(x.hi);
  const int ex = (int)((b >> 23) & 0xffu);
  if ((b >> 31) != 0u || ex < 2 || ex > 252) return false;
  const int E2 = ex - 127;
  // x 2^-E2 = m = mh + ml, mh in [1, 2) (exact scalings)
  const float mh = fof((b & 0x7fffffu) | 0x3f800000u);
  const float ml = x.lo * fof((unsigned)(127 - E2) << 23);
  // c_i = 1 + i/128 nearest to m; m - c_i exact in FP32
  const int i = (int)(((b & 0x7fffffu) + 0x8000u) >> 16);
  const float ci = 1.0f + (float)i * 0.0078125f;
  const df f = dfo::two_sum(dfo::sub_rn(mh, ci), ml);
  const df t = f * GSM_DPOW_PAIR(kDpRcp, i);
  // ln(1 + t): t - t^2/2 in pairs, t^3/3 - t^4/4 + t^5/5 - t^6/6 in FP32
  const df t2 = t * t;
  // (the FP32 tails by explicit round-to-nearest operations, so that device
  // and host builds give the same pairs)
  const float th = t.hi;
  const float pt = dfo::fma_rn(-th, dfo::fma_rn(-th, dfo::fma_rn(-th, 0.166666667f, 0.2f), 0.25f), 0.333333333f);
  const float tail = dfo::mul_rn(dfo::mul_rn(dfo::mul_rn(th, th), th), pt);
  const df ln1p = (t - df{0.5f * t2.hi, 0.5f * t2.lo}) + tail;
  const df lgm = GSM_DPOW_PAIR(kDpLog2, i) + ln1p * GSM_DPOW_PAIR(kDpConst, 0);
  // a (e + E2) in FP64, less its nearest multiple of 1/128 (n1 / 128)
#if defined(__CUDA_ARCH__)
  const double ae = __dmul_rn(a64, f64_of((float)(e + E2)));  // rounded, never contracted
#else
  const double ae = a64 * f64_of((float)(e + E2));
#endif
  const float aef = f32_of(ae);
  if (!(fabsf(aef) < 4096.0f)) return false;
  const float n1 = rintf(aef * 128.0f);
  const double r1 = ae - f64_of(n1 * 0.0078125f);
  // y = r1 + a log2 m = n2/128 + r
  const df y = df_of(r1) + ad * lgm;
  const float n2 = rintf(y.hi * 128.0f);
  const float u = dfo::fma_rn(y.hi, 128.0f, -n2);
  const df r128 = dfo::two_sum(u, y.lo * 128.0f);
  const df r = df{r128.hi * 0.0078125f, r128.lo * 0.0078125f};
  // e^z - 1, z = r ln 2: z + z^2/2 in pairs, z^3/6 + z^4/24 + z^5/120 in FP32
  const df z = r * GSM_DPOW_PAIR(kDpConst, 1);
  const df z2 = z * z;
  const float zh = z.hi;
  const float pz = dfo::fma_rn(zh, dfo::fma_rn(zh, 0.00833333333f, 0.0416666667f), 0.166666667f);
  const float tz = dfo::mul_rn(dfo::mul_rn(dfo::mul_rn(zh, zh), zh), pz);
  const df em1 = (z + df{0.5f * z2.hi, 0.5f * z2.lo}) + tz;
  const int N = (int)n1 + (int)n2;
  const int j = N & 127;
  const int M = (N - j) / 128;
  const df T = GSM_DPOW_PAIR(kDpExp2, j);
  const df P = acm * (T + T * em1);
  const int s = M + ace;
  if (s < -100 || s > 100) return false;
  const float sc = fof((unsigned)(s + 127) << 23);
  F = df{P.hi * sc, P.lo * sc};
  return true;
}

}  // namespace dpow
}  // namespace gsm
