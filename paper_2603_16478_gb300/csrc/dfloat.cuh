// Double-float arithmetic on the FP32 pipes.
//
// A value is carried as the unevaluated sum hi + lo of two floats, about 48 significant bits.
// This part's FP64 pipe issues about 1.6 FMA per clock per SM against about 116 for FP32, and
// its F64 <-> F32 conversions run at the FP64 rate too (both measured on the GB300), so
// accumulating FP32 data to FP64-class accuracy is several times cheaper in double-float than
// in double.  The building blocks are the error-free transformations: Knuth's TwoSum
// (s + e = a + b exactly) and TwoProd by FMA (p + e = a b exactly, e = fma(a, b, -p)).  The
// _rn intrinsics keep the compiler from contracting or reassociating them.
#pragma once

#include <cuda_runtime.h>

namespace ncpadj {

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// (h, l) += a * (xh + xl): the product's rounding error and a * xl go to the low part
__device__ __forceinline__ void df_fma(float a, float xh, float xl, float& h, float& l) {
  const float p = __fmul_rn(a, xh);
  const float pe = __fmaf_rn(a, xl, __fmaf_rn(a, xh, -p));
  float s, se;
  two_sum(h, p, s, se);
  h = s;
  l = __fadd_rn(l, __fadd_rn(se, pe));
}

// (h, l) += (h2, l2)
__device__ __forceinline__ void df_add(float& h, float& l, float h2, float l2) {
  float s, e;
  two_sum(h, h2, s, e);
  h = s;
  l = __fadd_rn(l, __fadd_rn(e, l2));
}

// x as (hi, lo): hi = fl32(x), lo = fl32(x - hi)
__device__ __forceinline__ float2 df_split(double x) {
  const float h = __double2float_rn(x);
  return make_float2(h, __double2float_rn(x - (double)h));
}

__device__ __forceinline__ double df_to_double(float h, float l) { return (double)h + (double)l; }

}  // namespace ncpadj
