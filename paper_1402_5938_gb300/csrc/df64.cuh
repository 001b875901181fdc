// Double-float arithmetic for the FP64-accuracy operator of the finest level on a GPU whose FP64
// units run at a small fraction of its FP32 rate: a value is the unevaluated sum hi + lo of two
// FP32 numbers (|lo| <= ulp(hi) / 2, about 48 significant bits). The operations are built from
// error-free transformations: Knuth's two-sum (a + b = s + e exactly) and the FMA two-product
// (a b = p + e exactly, e = fma(a, b, -p)), composed as in Dekker (1971) and in the double-double
// library of Hida, Li and Bailey (2001) ("sloppy" addition: the error of a sum is a few u^2
// (|a| + |b|), u = 2^-24, the same form as an FP64 rounding bound with a 2^-46 unit). Every step
// uses the round-to-nearest intrinsics, which the compiler neither contracts into FMAs nor reorders.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

namespace hmg {

struct __align__(8) df64 {
  float hi, lo;
  df64() = default;
  __host__ __device__ constexpr df64(float h, float l) : hi(h), lo(l) {}
  // nearest FP32 to d, then the nearest FP32 to the remainder (exact for |d| in FP32's range up to
  // the 48th bit)
  __host__ __device__ df64(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

// s + e = a + b exactly (any magnitudes)
__device__ __forceinline__ df64 df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return df64(s, e);
}
// s + e = a + b exactly when |a| >= |b| (or a = 0)
__device__ __forceinline__ df64 df_fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return df64(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ df64 operator-(df64 a) { return df64(-a.hi, -a.lo); }

__device__ __forceinline__ df64 operator+(df64 a, df64 b) {
  df64 s = df_two_sum(a.hi, b.hi);
  s.lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return df_fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ df64 operator-(df64 a, df64 b) { return a + (-b); }

// a b: the exact product of the high parts plus the cross terms (lo * lo is below u^2 |a b|)
__device__ __forceinline__ df64 operator*(df64 a, df64 b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_fast_two_sum(p, e);
}

// a b + c in the arithmetic of the operands' type (templates over FP32, FP64 and double-float call
// this one name)
__host__ __device__ __forceinline__ float fmadd(float a, float b, float c) { return fmaf(a, b, c); }
__host__ __device__ __forceinline__ double fmadd(double a, double b, double c) { return fma(a, b, c); }
// double-float: the product's high part is added to c exactly, its error terms and c's low part are
// collected in the low word, then renormalized once
__device__ __forceinline__ df64 fmadd(df64 a, df64 b, df64 c) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  df64 s = df_two_sum(p, c.hi);
  s.lo = __fadd_rn(s.lo, __fadd_rn(e, c.lo));
  return df_fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ df64& operator+=(df64& a, df64 b) { return a = a + b; }

}  // namespace hmg
