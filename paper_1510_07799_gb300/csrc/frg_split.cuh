// frg_split.cuh -- conversions between FP64 values and their float-pair form.
#pragma once
#include <cuda_runtime.h>

namespace frg {

// x ~ hi + lo with hi = RN_f32(x), lo = RN_f32(x - hi): 48 significant bits.
__device__ __forceinline__ float2 split_f64(double x) {
  const float hi = __double2float_rn(x);
  const float lo = __double2float_rn(x - (double)hi);
  return make_float2(hi, lo);
}

__device__ __forceinline__ float4 split_c128(double2 z) {
  const float2 a = split_f64(z.x), b = split_f64(z.y);
  return make_float4(a.x, a.y, b.x, b.y);
}

__device__ __forceinline__ double2 join_c128(float4 v) {
  return make_double2((double)v.x + (double)v.y, (double)v.z + (double)v.w);
}

}  // namespace frg
