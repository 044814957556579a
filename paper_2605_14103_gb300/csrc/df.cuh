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

// float -> double, exact, by moving the bits with integer instructions only:
// the conversion instruction runs on this GPU's FP64 units, which also do
// the FP64 arithmetic (a merge kernel that converted through it, even only
// on a select, kept them 84 % busy).  Normal floats rebias the exponent;
// zeros keep their sign; subnormal floats (m 2^-149) become normal doubles;
// infinities and NaNs keep their payload (a quiet NaN stays quiet).
__device__ __forceinline__ double f2d_exact(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint64_t sign = (uint64_t)(u & 0x80000000u) << 32;
  const uint32_t e = (u >> 23) & 0xFFu;
  const uint32_t m = u & 0x7FFFFFu;
  uint64_t d;
  if (e == 0xFFu) {
    d = sign | (0x7FFull << 52) | ((uint64_t)m << 29);
  } else if (e != 0u) {
    d = sign | ((uint64_t)(e + 896u) << 52) | ((uint64_t)m << 29);
  } else if (m == 0u) {
    d = sign;
  } else {
    const int p = 31 - __clz((int)m);   // leading bit of m, 0..22
    d = sign | ((uint64_t)(p + 874) << 52) | (((uint64_t)m << (52 - p)) & 0xFFFFFFFFFFFFFull);
  }
  return __longlong_as_double((long long)d);
}

// double -> float, rounded to nearest even, with integer instructions only
// (the conversion instruction, like f2d_exact's, runs on the FP64 units).
// The 53-bit significand is shifted right to the float's precision (24
// bits, fewer for a subnormal result) and rounded on the bits shifted out; a
// carry out of the significand moves into the exponent, past the largest
// finite float to infinity.  Zeros, double subnormals and magnitudes below
// half the least float subnormal give a signed zero; NaNs stay (quiet) NaNs.
__device__ __forceinline__ float d2f_rn(double x) {
  const uint64_t u = (uint64_t)__double_as_longlong(x);
  const uint32_t sign = (uint32_t)(u >> 32) & 0x80000000u;
  const int ed = (int)((u >> 52) & 0x7FF);
  const uint64_t mant = u & 0xFFFFFFFFFFFFFull;
  uint32_t r;
  if (ed == 0x7FF) {
    r = 0x7F800000u | (mant ? (0x400000u | (uint32_t)(mant >> 29)) : 0u);
  } else if (ed == 0 || ed - 1023 < -150) {
    r = 0u;
  } else {
    const int E = ed - 1023;
    const uint64_t m = mant | (1ull << 52);
    const int sh = E >= -126 ? 29 : 29 + (-126 - E);   // 29 .. 53
    uint64_t q = m >> sh;
    const uint64_t rem = m & ((1ull << sh) - 1), half = 1ull << (sh - 1);
    if (rem > half || (rem == half && (q & 1ull))) ++q;
    if (E > 127) {
      r = 0x7F800000u;
    } else if (E >= -126) {
      r = ((uint32_t)(E + 126) << 23) + (uint32_t)q;   // q's leading bit adds 1 to the exponent
    } else {
      r = (uint32_t)q;                                  // subnormal (a carry gives the least normal)
    }
  }
  return __uint_as_float(sign | r);
}

// Split a double into hi + lo floats (integer conversions, one FP64 subtraction).
__device__ __forceinline__ float2 df_split(double x) {
  const float h = d2f_rn(x);
  return make_float2(h, d2f_rn(x - f2d_exact(h)));
}

}  // namespace zbus
