// Table-driven FP64 power x^p = 2^(p log2 x) for x > 0.
//
// The dissipation potential needs q^(a-1) in FP64 once per FP64 residual,
// and the FP64-pipe cost of exp(p log x) (~54 FMA slots on GB300, measured)
// dominates the FP64 correction of the FP32-bulk update.  This follows
// Tang's table-driven logarithm and exponential (P. T. P. Tang, ACM TOMS 15
// (1989) 144-157; ACM TOMS 16 (1990) 378-400), with 128-entry tables:
//
//   x = 2^j m, m in [1, 2);  m_i = 1 + i/128 (top 7 mantissa bits),
//   t = (m - m_i)/m_i in [0, 1/128),  log2 m = log2 m_i + log2(1 + t),
//   log2(1 + t) by its Taylor series to t^7 (remainder < 2^-59);
//   y = p (j + log2 m) carried as a two-term sum (the FMA gives p*j exactly),
//   n = round(128 y),  r = y - n/128 in [-1/256, 1/256] (+ rounding),
//   2^y = 2^(n >> 7) * 2^((n & 127)/128) * 2^r, 2^r by its Taylor series in
//   r ln 2 to degree 6 (remainder < 2^-60).
//
// About 26 FP64 operations and three L1-resident table loads; the result is
// within a few ulp of x^p (checked against a 50-digit reference on the host
// and against CUDA's pow on the GPU).  Zero, subnormal, negative and
// non-finite x, and |p log2 x| >= 1000, take CUDA's pow.
#pragma once

#include <cmath>
#include <cstdint>
#include <cstring>

#ifndef AD_HD
#if defined(__CUDACC__)
#define AD_HD __host__ __device__ __forceinline__
#else
#define AD_HD inline
#endif
#endif

namespace gsm {
namespace fpow {

#if defined(__CUDACC__)
#define GSM_POW_TABLE(name, n, ...)                     \
  __device__ const double name##_d[n] = __VA_ARGS__; \
  static const double name##_h[n] = __VA_ARGS__;
#else
#define GSM_POW_TABLE(name, n, ...) static const double name##_h[n] = __VA_ARGS__;
#endif
#include "pow_tables.inc"
#undef GSM_POW_TABLE

#if defined(__CUDA_ARCH__)
#define GSM_POW_TAB(name, i) __ldg(&name##_d[i])
#else
#define GSM_POW_TAB(name, i) name##_h[i]
#endif

AD_HD uint64_t bits_of(double x) {
#if defined(__CUDA_ARCH__)
  return (uint64_t)__double_as_longlong(x);
#else
  uint64_t b;
  std::memcpy(&b, &x, sizeof b);
  return b;
#endif
}

AD_HD double double_of(uint64_t b) {
#if defined(__CUDA_ARCH__)
  return __longlong_as_double((long long)b);
#else
  double x;
  std::memcpy(&x, &b, sizeof x);
  return x;
#endif
}

AD_HD double pow_pos(double x, double p) {
  const uint64_t b = bits_of(x);
  const int e = (int)((b >> 52) & 0x7ff);
  if (e == 0 || e == 0x7ff || (b >> 63)) return ::pow(x, p);
  const int j = e - 1023;
  const int i = (int)((b >> 45) & 0x7f);
  const double m = double_of((b & 0x000fffffffffffffull) | 0x3ff0000000000000ull);
  const double mi = double_of(0x3ff0000000000000ull | ((uint64_t)i << 45));
  const double t = (m - mi) * GSM_POW_TAB(kPowRcp, i);  // m - m_i is exact
  double s = GSM_POW_TAB(kPowLnC, 6);
#pragma unroll
  for (int k = 5; k >= 0; --k) s = fma(s, t, GSM_POW_TAB(kPowLnC, k));
  const double l = fma(s, t, GSM_POW_TAB(kPowLog2, i));  // log2 m in [0, 1)
  const double jd = (double)j;
  const double yj = p * jd;
  const double yl = fma(p, l, fma(p, jd, -yj));  // y = yj + yl
  if (!(yj < 1000.0 && yj > -1000.0)) return ::pow(x, p);
  const double magic = 6755399441055744.0;  // 1.5 * 2^52: rounds to an integer
  const double sh = fma(yj + yl, 128.0, magic);
  const int64_t n = (int64_t)(bits_of(sh) - bits_of(magic));
  const double r = fma(sh - magic, -1.0 / 128.0, yj) + yl;
  double q = GSM_POW_TAB(kPowExpC, 6);
#pragma unroll
  for (int k = 5; k >= 0; --k) q = fma(q, r, GSM_POW_TAB(kPowExpC, k));
  const double f = GSM_POW_TAB(kPowExp2, (int)(n & 127)) * q;  // in [1, 2) up to rounding
  const int64_t k2 = n >> 7;                                  // floor(n / 128)
  return double_of(bits_of(f) + ((uint64_t)k2 << 52));
}

#undef GSM_POW_TAB

}  // namespace fpow
}  // namespace gsm
