// Double-float ("df64") arithmetic: a value is the unevaluated sum hi + lo of two FP32 numbers,
// about 48 significant bits. GB300 executes FP32 FMAs ~60x faster than FP64 ones, so kernels that
// need ~1e-13 relative accuracy (the FP64 residuals of the iterative refinement, right-hand
// sides and density response) run faster in df64 than in native FP64.
//
// The operations are the classical error-free transformations, written from their published
// definitions:
//   TwoSum (Knuth, TAOCP vol. 2):  s = a + b, e = (a - (s - (s - a))) + (b - (s - a)), a + b = s + e
//   FastTwoSum (Dekker 1971), |a| >= |b|:  s = a + b, e = b - (s - a)
//   TwoProd with a fused multiply-add: p = a b, e = fma(a, b, -p), a b = p + e
// Addition adds the two high parts exactly, the low parts approximately, and renormalises
// ("sloppy" addition: relative error ~ 2^-47 of |a| + |b|, enough for sums whose terms do not
// cancel catastrophically, such as FFT butterflies and dot products). Multiplication keeps the
// exact product of the high parts plus the two cross terms.
#pragma once

#include <cuda_runtime.h>

namespace wdf {

struct df64 {
  float hi, lo;
  df64() = default;
  __host__ __device__ constexpr df64(float h, float l) : hi(h), lo(l) {}
  // exact split of a double whose value fits (the low part is the rounded remainder)
  __host__ __device__ df64(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
  __host__ __device__ df64(float f) : hi(f), lo(0.0f) {}
  __host__ __device__ df64(int i) : df64((double)i) {}
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
  __host__ __device__ explicit operator float() const { return hi + lo; }
};

__device__ __forceinline__ df64 df_fast_two_sum(float a, float b) {
  const float s = a + b;
  return df64(s, b - (s - a));
}

__device__ __forceinline__ df64 operator+(df64 a, df64 b) {
  const float s = a.hi + b.hi;
  const float bb = s - a.hi;
  float e = (a.hi - (s - bb)) + (b.hi - bb);
  e += a.lo + b.lo;
  return df_fast_two_sum(s, e);
}
__device__ __forceinline__ df64 operator-(df64 a) { return df64(-a.hi, -a.lo); }
__device__ __forceinline__ df64 operator-(df64 a, df64 b) { return a + (-b); }
__device__ __forceinline__ df64 operator*(df64 a, df64 b) {
  const float p = a.hi * b.hi;
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_fast_two_sum(p, e);
}
__device__ __forceinline__ df64 &operator+=(df64 &a, df64 b) { return a = a + b; }
__device__ __forceinline__ df64 &operator-=(df64 &a, df64 b) { return a = a - b; }
__device__ __forceinline__ df64 &operator*=(df64 &a, df64 b) { return a = a * b; }

}  // namespace wdf
