// Double-float numbers: x = hi + lo held in two FP32 values, ~47 significant
// bits.  On GB300 an FP32 instruction issues at 64 times the FP64 rate, so a
// double-float addition (11 FP32 instructions) or multiplication (6) costs a
// fraction of one FP64 operation; the FP64 correction of the FP32-bulk
// material update evaluates its residual in this arithmetic.
//
// Algorithms: Knuth's two-sum and Dekker's fast two-sum; the product's
// rounding error by an FMA (Dekker's two-product); the addition is the two-sum
// of the high parts plus the sum of the low parts, renormalised, whose error
// is below ~2^-46 (|a| + |b|) -- relative to the operands, which is what a
// residual that cancels to ~0 needs.  Device code uses the _rn intrinsics, so
// no contraction into FMAs can change the error-free transformations; a host
// build must not contract either (g++ -ffp-contract=off: on aarch64 g++
// fuses a*b + c by default in C++).
//
// Conversions from and to FP64 go through the integer-pipe helpers f32_of /
// f64_of of solver.cuh (an F2F conversion occupies the FP64 pipe on GB300).
#pragma once

#include <cmath>

#include "solver.cuh"

namespace gsm {

struct df {
  float hi, lo;
};

namespace dfo {

AD_HD float add_rn(float a, float b) {
#if defined(__CUDA_ARCH__)
  return __fadd_rn(a, b);
#else
  return a + b;
#endif
}
AD_HD float sub_rn(float a, float b) {
#if defined(__CUDA_ARCH__)
  return __fsub_rn(a, b);
#else
  return a - b;
#endif
}
AD_HD float mul_rn(float a, float b) {
#if defined(__CUDA_ARCH__)
  return __fmul_rn(a, b);
#else
  return a * b;
#endif
}
AD_HD float fma_rn(float a, float b, float c) {
#if defined(__CUDA_ARCH__)
  return __fmaf_rn(a, b, c);
#else
  return std::fma(a, b, c);
#endif
}

// s + e = a + b exactly, |a| >= |b| or a = 0
AD_HD df fast_two_sum(float a, float b) {
  const float s = add_rn(a, b);
  const float e = sub_rn(b, sub_rn(s, a));
  return df{s, e};
}
// s + e = a + b exactly
AD_HD df two_sum(float a, float b) {
  const float s = add_rn(a, b);
  const float bb = sub_rn(s, a);
  const float e = add_rn(sub_rn(a, sub_rn(s, bb)), sub_rn(b, bb));
  return df{s, e};
}

}  // namespace dfo

AD_HD df operator+(const df& a, const df& b) {
  const df s = dfo::two_sum(a.hi, b.hi);
  const float e = dfo::add_rn(s.lo, dfo::add_rn(a.lo, b.lo));
  return dfo::fast_two_sum(s.hi, e);
}
AD_HD df operator-(const df& a) { return df{-a.hi, -a.lo}; }
AD_HD df operator-(const df& a, const df& b) { return a + (-b); }
AD_HD df operator+(const df& a, float b) {
  const df s = dfo::two_sum(a.hi, b);
  return dfo::fast_two_sum(s.hi, dfo::add_rn(s.lo, a.lo));
}
AD_HD df operator*(const df& a, const df& b) {
  const float p = dfo::mul_rn(a.hi, b.hi);
  float e = dfo::fma_rn(a.hi, b.hi, -p);
  e = dfo::fma_rn(a.hi, b.lo, e);
  e = dfo::fma_rn(a.lo, b.hi, e);
  return dfo::fast_two_sum(p, e);
}
AD_HD df operator*(const df& a, float b) {
  const float p = dfo::mul_rn(a.hi, b);
  float e = dfo::fma_rn(a.hi, b, -p);
  e = dfo::fma_rn(a.lo, b, e);
  return dfo::fast_two_sum(p, e);
}

// FP64 -> double-float: hi is x truncated to FP32, lo the (exact) FP64
// remainder truncated to FP32; relative error < 2^-46.  An exact scaling by
// 2^k is folded into both exponents (as in f32_of); |x 2^k| must lie in the
// FP32 normal range, else the parts flush to zero.
AD_HD df df_of(double x, int k = 0) {
  const float hi = f32_of(x, k);
  const double r = x - f64_of(hi, -k);
  return df{hi, f32_of(r, k)};
}
// double-float -> FP64 (one FP64 addition), with an exact scaling by 2^k.
AD_HD double f64_of(const df& a, int k = 0) { return f64_of(a.hi, k) + f64_of(a.lo, k); }

}  // namespace gsm
