// Double-float ("df64") arithmetic: an FP64-range value carried as an
// unevaluated sum hi + lo of two FP32 numbers, ~2^-47 relative precision,
// every operation on the FP32 units (the FP64 pipe is 1/64 of the FP32 rate on
// GB300). Error-free transformations after Dekker (1971) and Knuth (TAOCP
// vol. 2): TwoSum, FastTwoSum, and the FMA residual of a product.
#pragma once

#include "common.cuh"

namespace dq {

// ----------------------------------------------------------------- FP64 <-> FP32 pairs
// Split x into hi + lo (FP32) with integer operations only (the FP64 pipe is
// 1/64 of the FP32 rate on GB300): hi carries the top 24 significand bits of
// x (truncated), lo the next 24 of the remaining 29 (rounded by the integer
// to FP32 conversion): |x - hi - lo| <= 2^-47 |x|. Values outside the FP32
// normal range map to 0 (|x| < 2^-126) or +-inf.
__device__ __forceinline__ float2 split_df_bits(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned int sign = (unsigned int)(b >> 63) << 31;
  const int e = (int)((b >> 52) & 0x7ff);
  const unsigned long long mant = b & 0xFFFFFFFFFFFFFull;
  const int e32 = e - 1023 + 127;
  if (e32 <= 0) return make_float2(0.f, 0.f);
  if (e32 >= 255) return make_float2(__int_as_float(sign | 0x7f800000u), 0.f);
  const float hi = __int_as_float(sign | ((unsigned int)e32 << 23) | (unsigned int)(mant >> 29));
  const unsigned int rem = (unsigned int)(mant & 0x1FFFFFFFull);  // 29 bits, weight 2^(e-1075)
  const int el = e - 1075 + 127;                                 // FP32 exponent of 2^(e-1075)
  float lo = 0.f;
  if (rem != 0u && el > 0) {
    lo = __uint2float_rn(rem) * __int_as_float((unsigned int)el << 23);
    if (sign) lo = -lo;
  }
  return make_float2(hi, lo);
}

// FP32 -> FP64 by re-biasing the exponent (integer operations only); FP32
// subnormals map to 0.
__device__ __forceinline__ double f2d_bits(float f) {
  const unsigned int b = (unsigned int)__float_as_int(f);
  const unsigned long long sign = (unsigned long long)(b >> 31) << 63;
  const unsigned int e = (b >> 23) & 0xff;
  if (e == 0) return __longlong_as_double((long long)sign);
  const unsigned long long e11 = (e == 255) ? 2047ull : (unsigned long long)(e + 896);
  const unsigned long long mant = (unsigned long long)(b & 0x7fffff) << 29;
  return __longlong_as_double((long long)(sign | (e11 << 52) | mant));
}

// ----------------------------------------------------------------- df64 type
struct df64 {
  float hi, lo;
  df64() = default;
  __host__ __device__ constexpr df64(float h, float l) : hi(h), lo(l) {}
  // from a compile-time or host constant (FP64 arithmetic, folded by the compiler)
  __host__ __device__ constexpr explicit df64(double x)
      : hi((float)x), lo((float)(x - (double)(float)x)) {}
  __host__ __device__ constexpr explicit df64(int x) : hi((float)x), lo(0.f) {}
};

// from an FP64 value at run time: integer operations only
__device__ __forceinline__ df64 df_from(double x) {
  const float2 p = split_df_bits(x);
  return df64(p.x, p.y);
}
// to FP64: one FP64 add
__device__ __forceinline__ double df_to(df64 a) { return f2d_bits(a.hi) + f2d_bits(a.lo); }

__device__ __forceinline__ df64 fast_two_sum(float a, float b) {
  const float s = a + b;
  return df64(s, b - (s - a));
}
__device__ __forceinline__ df64 two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return df64(s, (a - (s - bb)) + (b - bb));
}

// a + b with absolute error ~2^-47 (|a| + |b|)
__device__ __forceinline__ df64 operator+(df64 a, df64 b) {
  const df64 s = two_sum(a.hi, b.hi);
  return fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
}
__device__ __forceinline__ df64 operator-(df64 a) { return df64(-a.hi, -a.lo); }
__device__ __forceinline__ df64 operator-(df64 a, df64 b) { return a + (-b); }
// a * b with relative error ~2^-47
__device__ __forceinline__ df64 operator*(df64 a, df64 b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return fast_two_sum(p, e);
}
__device__ __forceinline__ df64 &operator+=(df64 &a, df64 b) { return a = a + b; }
__device__ __forceinline__ df64 &operator-=(df64 &a, df64 b) { return a = a - b; }
__device__ __forceinline__ df64 &operator*=(df64 &a, df64 b) { return a = a * b; }

}  // namespace dq
