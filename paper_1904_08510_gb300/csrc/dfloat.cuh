// Double-float ("float-float", double-word FP32) arithmetic for the
// preconditioner of the mixed mode SDCEF_MIXED_DF.
//
// A value is the unevaluated sum hi + lo of two FP32 numbers with
// |lo| <= ulp(hi): about 48 significant bits and the FP32 exponent range. The
// operations are built from error-free transformations:
//   TwoSum       (Knuth, TAOCP vol. 2, 4.2.2): s + e = a + b exactly, 6 adds;
//   Fast2Sum     (Dekker 1971):                 s + e = a + b exactly if |a| >= |b|;
//   TwoProduct   with FMA:                      p + e = a * b exactly, e = fma(a, b, -p);
// and the products and sums follow the double-word algorithms analysed by
// Joldes, Muller and Popescu ("Tight and rigorous error bounds for basic
// building blocks of double-word arithmetic", ACM TOMS 44, 2017): relative
// error of a product or multiply-add below ~2^-44.
//
// Why: on this part a warp FP64 instruction holds the FP64 pipe for 16 SM
// cycles while the four schedulers issue one FP32 warp instruction per cycle
// each, so a double-float multiply-add (about 15 FP32 instructions) costs
// about a fifth of a DFMA. The preconditioner only has to approximate J^-1
// (the paper applies it through multigrid cycles to a tolerance); with
// cond(J) ~ 1e8 the 48-bit arithmetic keeps its forward error near 1e-6,
// where plain FP32 (24 bits) loses it entirely.
//
// Conversions to and from FP64 use integer operations on the bit patterns
// (plus one FP64 add when returning to FP64), not FP64 conversion
// instructions. Values below 2^-126 (the FP32 normal range) convert to zero.
#pragma once
#include <cuda_runtime.h>

namespace sdcef {

struct __align__(8) dfloat {
  float hi, lo;
  dfloat() = default;
  __host__ __device__ constexpr dfloat(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ constexpr explicit dfloat(int v) : hi((float)v), lo(0.0f) {}
};

__device__ __forceinline__ dfloat df_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  const float e = (a - (s - bb)) + (b - bb);
  return dfloat(s, e);
}
__device__ __forceinline__ dfloat df_fast_two_sum(float a, float b) {
  const float s = a + b;
  return dfloat(s, b - (s - a));
}

__device__ __forceinline__ dfloat operator-(dfloat x) { return dfloat(-x.hi, -x.lo); }

// x * y: TwoProduct of the high parts plus the two cross terms (the lo*lo
// term is below the error bound), renormalised.
__device__ __forceinline__ dfloat operator*(dfloat x, dfloat y) {
  const float p = x.hi * y.hi;
  float e = fmaf(x.hi, y.hi, -p);
  e = fmaf(x.hi, y.lo, e);
  e = fmaf(x.lo, y.hi, e);
  return df_fast_two_sum(p, e);
}

// x * y + c with one final renormalisation: TwoProduct of the high parts,
// TwoSum with c.hi, and the low-order terms added in FP32.
__device__ __forceinline__ dfloat fma(dfloat x, dfloat y, dfloat c) {
  const float p = x.hi * y.hi;
  float e = fmaf(x.hi, y.hi, -p);
  e = fmaf(x.hi, y.lo, e);
  e = fmaf(x.lo, y.hi, e);
  const dfloat s = df_two_sum(c.hi, p);
  return df_fast_two_sum(s.hi, s.lo + (c.lo + e));
}

__device__ __forceinline__ dfloat operator+(dfloat x, dfloat y) {
  const dfloat s = df_two_sum(x.hi, y.hi);
  return df_fast_two_sum(s.hi, s.lo + (x.lo + y.lo));
}

// 1/d: the correctly rounded FP32 reciprocal y of d.hi refined by one Newton
// step y + y (1 - d y), where 1 - d y is formed with TwoProduct (d.hi y = 1
// up to 2^-24, so 1 - p is exact by Sterbenz's lemma).
__device__ __forceinline__ dfloat df_rcp(dfloat d) {
  const float y = __frcp_rn(d.hi);
  const float p = d.hi * y;
  const float pe = fmaf(d.hi, y, -p);
  const float r = ((1.0f - p) - pe) - d.lo * y;
  return df_fast_two_sum(y, y * r);
}
__device__ __forceinline__ dfloat operator/(dfloat x, dfloat y) { return x * df_rcp(y); }

// Pivot check on the high part: zero, or a non-finite inverse.
__device__ __forceinline__ bool bad_pivot(dfloat det, dfloat inv) {
  const int d = __float_as_int(det.hi), v = __float_as_int(inv.hi);
  return (d & 0x7FFFFFFF) == 0 || (v & 0x7F800000) == 0x7F800000;
}

// FP64 -> double-float: hi takes the leading 24 significant bits (truncated),
// lo the FP32 rounding of the remaining 29 bits; then renormalised.
__device__ __forceinline__ dfloat df_from_double(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const int e = (int)((b >> 52) & 0x7FF);
  const unsigned long long m = b & 0xFFFFFFFFFFFFFULL;
  const int ef = e - 1023 + 127;
  if (ef <= 0) return dfloat(__int_as_float((int)sign), 0.0f);
  if (ef >= 255) {
    const unsigned nan = (e == 0x7FF && m != 0) ? 0x400000u : 0u;
    return dfloat(__int_as_float((int)(sign | 0x7F800000u | nan)), 0.0f);
  }
  const float hi = __int_as_float((int)(sign | ((unsigned)ef << 23) | (unsigned)(m >> 29)));
  const unsigned m29 = (unsigned)(m & 0x1FFFFFFFu);
  const int es = e - 1075 + 127;   // biased FP32 exponent of 2^(e - 1075), the weight of bit 0
  float lo = 0.0f;
  if (m29 != 0u && es > 0) {
    lo = __uint2float_rn(m29) * __int_as_float(es << 23);
    lo = sign ? -lo : lo;
  }
  return df_fast_two_sum(hi, lo);
}

// FP32 -> FP64 on the bit pattern (FP32 subnormals convert to zero).
__device__ __forceinline__ double f32_bits_to_double(float f) {
  const unsigned u = (unsigned)__float_as_int(f);
  const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
  const unsigned e = (u >> 23) & 0xFFu;
  const unsigned long long frac = (unsigned long long)(u & 0x7FFFFFu) << 29;
  if (e == 0u) return __longlong_as_double((long long)sign);
  if (e == 0xFFu) return __longlong_as_double((long long)(sign | 0x7FF0000000000000ULL | frac));
  return __longlong_as_double((long long)(sign | ((unsigned long long)(e - 127 + 1023) << 52) | frac));
}
__device__ __forceinline__ double df_to_double(dfloat v) {
  return f32_bits_to_double(v.hi) + f32_bits_to_double(v.lo);
}

// Type conversions used by the templated block solver and the kernel.
template <typename To, typename From> struct Conv;
template <typename T> struct Conv<T, T> {
  static __device__ __forceinline__ T f(T x) { return x; }
};
template <> struct Conv<float, double> {
  static __device__ __forceinline__ float f(double x) { return (float)x; }
};
template <> struct Conv<double, float> {
  static __device__ __forceinline__ double f(float x) { return (double)x; }
};
template <> struct Conv<dfloat, double> {
  static __device__ __forceinline__ dfloat f(double x) { return df_from_double(x); }
};
template <> struct Conv<double, dfloat> {
  static __device__ __forceinline__ double f(dfloat x) { return df_to_double(x); }
};
template <typename To, typename From>
__device__ __forceinline__ To conv(From x) {
  return Conv<To, From>::f(x);
}

// Warp shuffles of one value.
__device__ __forceinline__ double shfl_up_v(double x, int s) { return __shfl_up_sync(0xffffffffu, x, s); }
__device__ __forceinline__ double shfl_down_v(double x, int s) { return __shfl_down_sync(0xffffffffu, x, s); }
__device__ __forceinline__ float shfl_up_v(float x, int s) { return __shfl_up_sync(0xffffffffu, x, s); }
__device__ __forceinline__ float shfl_down_v(float x, int s) { return __shfl_down_sync(0xffffffffu, x, s); }
__device__ __forceinline__ dfloat shfl_up_v(dfloat x, int s) {
  return dfloat(__shfl_up_sync(0xffffffffu, x.hi, s), __shfl_up_sync(0xffffffffu, x.lo, s));
}
__device__ __forceinline__ dfloat shfl_down_v(dfloat x, int s) {
  return dfloat(__shfl_down_sync(0xffffffffu, x.hi, s), __shfl_down_sync(0xffffffffu, x.lo, s));
}

}  // namespace sdcef
