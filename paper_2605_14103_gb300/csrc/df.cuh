// Double-float arithmetic: a value is the unevaluated sum hi + lo of two
// FP32 numbers (about 48 significant bits).  Built from the error-free
// transformations of Knuth (two-sum) and Dekker (two-product via FMA), so it
// runs on the FP32 pipes, which on this GPU are ~64x faster than FP64.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace zbus {

// s + e == a + b exactly, s = fl(a + b).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Same for |a| >= |b| (or a == 0).
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

// (sh, sl) += (ah + al) * (bh + bl), dropping al * bl; sl is left unnormalised.
__device__ __forceinline__ void df_mac(float& sh, float& sl, float ah, float al, float bh,
                                       float bl) {
  const float p = __fmul_rn(ah, bh);
  float e = __fmaf_rn(ah, bh, -p);
  e = __fmaf_rn(ah, bl, e);
  e = __fmaf_rn(al, bh, e);
  float s, t;
  two_sum(sh, p, s, t);
  sh = s;
  sl = __fadd_rn(sl, __fadd_rn(t, e));
}

// (dh, dl) = (bh + bl) - (ah + al), unnormalised (|dl| small against |dh|).
__device__ __forceinline__ void df_sub(float bh, float bl, float ah, float al, float& dh,
                                       float& dl) {
  float s, e;
  two_sum(bh, -ah, s, e);
  dh = s;
  dl = __fadd_rn(e, __fsub_rn(bl, al));
}

// float -> double, exact, by moving the bits (integer instructions): the
// conversion instruction runs on this GPU's FP64 units, which also do the
// FP64 arithmetic.  Zeros, subnormals, infinities and NaNs take the
// conversion instruction.
__device__ __forceinline__ double f2d_exact(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t e = (u >> 23) & 0xFFu;
  if (e == 0u || e == 0xFFu) return (double)f;
  const uint64_t d = ((uint64_t)(u & 0x80000000u) << 32) | ((uint64_t)(e + 896u) << 52) |
                     ((uint64_t)(u & 0x7FFFFFu) << 29);
  return __longlong_as_double((long long)d);
}

// Split a double into hi + lo floats.
__device__ __forceinline__ float2 df_split(double x) {
  const float h = __double2float_rn(x);
  return make_float2(h, __double2float_rn(x - (double)h));
}

}  // namespace zbus
