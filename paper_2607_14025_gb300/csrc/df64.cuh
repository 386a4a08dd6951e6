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

// The error-free steps use the round-to-nearest intrinsics, which the compiler never contracts
// into fused multiply-adds (a contraction would break the exactness the transformations rely on).
__device__ __forceinline__ df64 df_fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return df64(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ df64 df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return df64(s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb)));
}

__device__ __forceinline__ df64 operator+(df64 a, df64 b) {
  const df64 s = df_two_sum(a.hi, b.hi);
  const float e = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return df_fast_two_sum(s.hi, e);
}
__device__ __forceinline__ df64 operator-(df64 a) { return df64(-a.hi, -a.lo); }
// the sum without its final renormalisation: TwoSum of the leading parts, the rest added in FP32
// (8 FP32 operations instead of 11). The low part may grow to a few ulp of the high part, which
// the next TwoSum of leading parts absorbs exactly; df_norm renormalises.
__device__ __forceinline__ df64 df_add_lazy(df64 a, df64 b) {
  const df64 s = df_two_sum(a.hi, b.hi);
  return df64(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ df64 df_norm(df64 a) { return df_fast_two_sum(a.hi, a.lo); }
__device__ __forceinline__ df64 operator-(df64 a, df64 b) { return a + (-b); }
__device__ __forceinline__ df64 operator*(df64 a, df64 b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_fast_two_sum(p, e);
}
__device__ __forceinline__ df64 &operator+=(df64 &a, df64 b) { return a = a + b; }
__device__ __forceinline__ df64 &operator-=(df64 &a, df64 b) { return a = a - b; }
__device__ __forceinline__ df64 &operator*=(df64 &a, df64 b) { return a = a * b; }

// a1 b1 + a2 b2 with one renormalisation: the exact leading products with their errors (TwoProd
// and the cross terms), TwoSum of the leading products, FastTwoSum at the end; 19 FP32
// operations instead of 25 for two double-float products and a double-float sum.
__device__ __forceinline__ df64 df_dot2(df64 a1, df64 b1, df64 a2, df64 b2) {
  const float p1 = __fmul_rn(a1.hi, b1.hi);
  float e1 = __fmaf_rn(a1.hi, b1.hi, -p1);
  e1 = __fmaf_rn(a1.hi, b1.lo, e1);
  e1 = __fmaf_rn(a1.lo, b1.hi, e1);
  const float p2 = __fmul_rn(a2.hi, b2.hi);
  float e2 = __fmaf_rn(a2.hi, b2.hi, -p2);
  e2 = __fmaf_rn(a2.hi, b2.lo, e2);
  e2 = __fmaf_rn(a2.lo, b2.hi, e2);
  const df64 s = df_two_sum(p1, p2);
  return df_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(e1, e2)));
}

// Lazy accumulation of double-float products, sum_k a_k b_k: the compensated dot product of
// Ogita, Rump and Oishi (SIAM J. Sci. Comput. 26, 2005) with FP32 as the working precision. s is
// the FP32 sum of the leading products; c collects, in FP32, every rounding error: TwoSum of s and
// each product, TwoProd of the leading parts and the two cross terms of the low parts. Each term
// costs 12 FP32 operations instead of 18 for a double-float multiply and add. Without
// renormalisation c would grow like sqrt(k) u |s| and its own rounding with it; df_acc_renorm
// (TwoSum of s and c) every few terms keeps |c| <= ulp(s), so the result stays within a small
// multiple of the error of double-float accumulation (~2^-47 per term of the running sum).
struct DfAcc {
  float s, c;
};
__device__ __forceinline__ void df_acc_fma(DfAcc &acc, df64 a, df64 b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float ep = __fmaf_rn(a.hi, b.hi, -p);
  ep = __fmaf_rn(a.hi, b.lo, ep);
  ep = __fmaf_rn(a.lo, b.hi, ep);
  const df64 t = df_two_sum(acc.s, p);
  acc.s = t.hi;
  acc.c = __fadd_rn(acc.c, __fadd_rn(t.lo, ep));
}
__device__ __forceinline__ void df_acc_renorm(DfAcc &acc) {
  const df64 t = df_two_sum(acc.s, acc.c);
  acc.s = t.hi;
  acc.c = t.lo;
}
__device__ __forceinline__ df64 df_acc_value(DfAcc acc) { return df_two_sum(acc.s, acc.c); }

}  // namespace wdf
