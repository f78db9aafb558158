// frg_split.cuh -- FP64 <-> FP32 conversions on the integer pipe and float-float
// (double-single) arithmetic used by the split-precision paths.
//
// GB300 issues FP64 instructions (arithmetic and F2F conversions) at 1/58 of the
// FP32 rate, so the split paths convert with integer bit operations (exact
// widening; round-to-nearest-even narrowing) and accumulate sums of FP32 terms
// as unevaluated float pairs hi + lo (about 48 significant bits).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace frg {

__device__ __forceinline__ float2 round_c64(double2 z) {
  return make_float2(__double2float_rn(z.x), __double2float_rn(z.y));
}

// Exact float -> double on the integer pipe (subnormal floats flush to 0).
__device__ __forceinline__ double f2d(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint64_t sgn = (uint64_t)(u & 0x80000000u) << 32;
  const uint32_t e = (u >> 23) & 0xFFu, m = u & 0x7FFFFFu;
  uint64_t b;
  if (e == 0)
    b = sgn;
  else if (e == 255)
    b = sgn | (0x7FFull << 52) | ((uint64_t)m << 29);
  else
    b = sgn | ((uint64_t)(e + 896u) << 52) | ((uint64_t)m << 29);
  return __longlong_as_double((long long)b);
}

// double -> float, round to nearest even, on the integer pipe (results below
// the smallest normal float flush to 0; overflow gives infinity).
__device__ __forceinline__ float d2f(double d) {
  const uint64_t b = (uint64_t)__double_as_longlong(d);
  const uint32_t sgn = (uint32_t)(b >> 32) & 0x80000000u;
  const int e = (int)((b >> 52) & 0x7FF);
  const uint64_t m = b & 0xFFFFFFFFFFFFFull;
  if (e == 0x7FF) return __uint_as_float(sgn | 0x7F800000u | (m ? 0x400000u : 0u));
  const int fe = e - 1023 + 127;
  if (fe >= 255) return __uint_as_float(sgn | 0x7F800000u);
  if (fe <= 0) return __uint_as_float(sgn);
  uint32_t mant = (uint32_t)(m >> 29);
  const uint32_t rem = (uint32_t)(m & 0x1FFFFFFFull);
  if (rem > 0x10000000u || (rem == 0x10000000u && (mant & 1u))) ++mant;
  return __uint_as_float(sgn | (((uint32_t)fe << 23) + mant));
}

// ---------------------------------------------------------- float-float ----
// s + e = a + b exactly (Knuth's two-sum).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// (hi, lo) += (ah + al) * k, k a float.
__device__ __forceinline__ void ff_mac(float &hi, float &lo, float ah, float al, float k) {
  const float p = __fmul_rn(ah, k);
  const float pe = __fmaf_rn(ah, k, -p);
  float s, e;
  two_sum(hi, p, s, e);
  lo = __fadd_rn(lo, __fadd_rn(__fadd_rn(e, pe), __fmul_rn(al, k)));
  hi = s;
}

}  // namespace frg
