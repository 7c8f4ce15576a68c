// Double-float arithmetic on the FP32 units: a value is the unevaluated sum hi + lo of two FP32
// numbers with |lo| <= ulp(hi) / 2, about 48 significant bits. GB300 issues FP32 fused
// multiply-adds at 64 times its FP64 rate, so an operator evaluated with these error-free
// transformations (about fifteen FP32 instructions per multiply-add) runs faster than native FP64
// while its rounding error (a few 2^-48 relative to the magnitude of the summed terms per
// operation) stays far below the 1e-12 bar of the FP64 applies.
//
// The building blocks are the classical error-free transformations: Knuth's two-sum (the exact
// rounding error of a + b from six additions), the fast two-sum for |a| >= |b| (three), and the
// exact product error fma(a, b, -a b). Every step uses the round-to-nearest intrinsics, which the
// compiler neither contracts into fused operations nor reorders.
#pragma once

#include <cuda_runtime.h>

namespace dgw {

struct df64 {
  float hi, lo;
};

__device__ __forceinline__ float ef_two_sum(float a, float b, float &err) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  err = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return s;
}

// requires |a| >= |b| (or a == 0)
__device__ __forceinline__ float ef_quick_two_sum(float a, float b, float &err) {
  const float s = __fadd_rn(a, b);
  err = __fsub_rn(b, __fsub_rn(s, a));
  return s;
}

__device__ __forceinline__ float ef_two_prod(float a, float b, float &err) {
  const float p = __fmul_rn(a, b);
  err = __fmaf_rn(a, b, -p);
  return p;
}

__device__ __forceinline__ df64 df_make(float h) { return df64{h, 0.0f}; }

// nearest double-float to a double (the split is exact up to the 48-bit precision)
__device__ __forceinline__ df64 df_from(double x) {
  const float h = __double2float_rn(x);
  return df64{h, __double2float_rn(x - (double)h)};
}

__device__ __forceinline__ double df_to(df64 a) { return (double)a.hi + (double)a.lo; }

// The same split with integer instructions only (the conversion instructions run on the FP64
// unit): hi keeps the sign, the exponent and the top 23 fraction bits of x, lo the remaining 29
// fraction bits truncated to 24 significant bits, so |lo| < ulp(hi) and hi + lo matches x to
// about 2^-47 relative. Zero, |x| < 2^-74 and |x| >= 2^127 take the conversion instructions.
__device__ __forceinline__ df64 df_split(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned int h = (unsigned int)(b >> 32);
  const int e = (int)((h >> 20) & 0x7ffu) - 1023;   // unbiased exponent
  if (e < -74 || e > 126) return df_from(x);
  const unsigned int sign = h & 0x80000000u;
  const unsigned int top = (unsigned int)((b >> 29) & 0x7fffffu);
  const unsigned int rest = (unsigned int)(b & 0x1fffffffu);
  df64 r;
  r.hi = __uint_as_float(sign | ((unsigned int)(e + 127) << 23) | top);
  if (rest == 0u) {
    r.lo = 0.0f;
  } else {
    const int lz = __clz((int)rest);                  // >= 3: rest < 2^29
    const int p = 31 - lz;                            // leading bit of rest
    const unsigned int frac = (rest << (lz + 1)) >> 9;   // 23 bits after the leading one
    r.lo = __uint_as_float(sign | ((unsigned int)(p + e - 52 + 127) << 23) | frac);
  }
  return r;
}

__device__ __forceinline__ df64 df_neg(df64 a) { return df64{-a.hi, -a.lo}; }

__device__ __forceinline__ df64 df_add(df64 a, df64 b) {
  float e;
  const float s = ef_two_sum(a.hi, b.hi, e);
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  df64 r;
  r.hi = ef_quick_two_sum(s, e, r.lo);
  return r;
}

__device__ __forceinline__ df64 df_mul(df64 a, df64 b) {
  float e;
  const float p = ef_two_prod(a.hi, b.hi, e);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  df64 r;
  r.hi = ef_quick_two_sum(p, e, r.lo);
  return r;
}

// a * b + c with one renormalisation
__device__ __forceinline__ df64 df_fma(df64 a, df64 b, df64 c) {
  float e, e2;
  const float p = ef_two_prod(a.hi, b.hi, e);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  const float s = ef_two_sum(p, c.hi, e2);
  e = __fadd_rn(e, __fadd_rn(e2, c.lo));
  df64 r;
  r.hi = ef_quick_two_sum(s, e, r.lo);
  return r;
}

__device__ __forceinline__ df64 operator+(df64 a, df64 b) { return df_add(a, b); }
__device__ __forceinline__ df64 operator-(df64 a, df64 b) { return df_add(a, df_neg(b)); }
__device__ __forceinline__ df64 operator-(df64 a) { return df_neg(a); }
__device__ __forceinline__ df64 operator*(df64 a, df64 b) { return df_mul(a, b); }
__device__ __forceinline__ df64 &operator+=(df64 &a, df64 b) { a = df_add(a, b); return a; }
__device__ __forceinline__ df64 &operator-=(df64 &a, df64 b) { a = df_add(a, df_neg(b)); return a; }

// Arithmetic helpers that templated kernels use for every compute type R (double, float, df64).
template <typename R>
__device__ __forceinline__ R r_zero();
template <>
__device__ __forceinline__ double r_zero<double>() { return 0.0; }
template <>
__device__ __forceinline__ float r_zero<float>() { return 0.0f; }
template <>
__device__ __forceinline__ df64 r_zero<df64>() { return df64{0.0f, 0.0f}; }

// a * b + c
__device__ __forceinline__ double r_fma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float r_fma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ df64 r_fma(df64 a, df64 b, df64 c) { return df_fma(a, b, c); }

// |x|, and whether |a| >= |b| (double-float: by the sign of the difference, exact for the
// normalised pairs the arithmetic produces)
__device__ __forceinline__ double r_abs(double x) { return fabs(x); }
__device__ __forceinline__ float r_abs(float x) { return fabsf(x); }
__device__ __forceinline__ df64 r_abs(df64 x) { return x.hi < 0.0f ? df_neg(x) : x; }
__device__ __forceinline__ bool r_abs_ge(double a, double b) { return fabs(a) >= fabs(b); }
__device__ __forceinline__ bool r_abs_ge(float a, float b) { return fabsf(a) >= fabsf(b); }
__device__ __forceinline__ bool r_abs_ge(df64 a, df64 b) { return df_add(r_abs(a), df_neg(r_abs(b))).hi >= 0.0f; }

// 1/2 in every compute type (exact)
template <typename R>
__device__ __forceinline__ R r_half();
template <>
__device__ __forceinline__ double r_half<double>() { return 0.5; }
template <>
__device__ __forceinline__ float r_half<float>() { return 0.5f; }
template <>
__device__ __forceinline__ df64 r_half<df64>() { return df64{0.5f, 0.0f}; }

// conversions between the storage type T of a vector and the compute type R
template <typename R, typename T>
__device__ __forceinline__ R r_load(T x) { return (R)x; }
template <>
__device__ __forceinline__ df64 r_load<df64, double>(double x) { return df_split(x); }
template <typename T, typename R>
__device__ __forceinline__ T r_store(R x) { return (T)x; }
template <>
__device__ __forceinline__ double r_store<double, df64>(df64 x) { return df_to(x); }

}  // namespace dgw
