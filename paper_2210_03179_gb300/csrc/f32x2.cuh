// FP64-class arithmetic on pairs of FP32 values (value = hi + lo, |lo| <= ulp(hi) / 2, about
// 48 significant bits), for operators that need FP64 accuracy on a GPU whose FP32 rate is a
// large multiple of its FP64 rate.  Built from two error-free transformations:
//   TwoSum (Knuth, The Art of Computer Programming vol. 2, 4.2.2):  s + e = a + b exactly;
//   TwoProduct with a fused multiply-add:                          p + e = a * b exactly.
// Every FP32 operation is an explicit round-to-nearest intrinsic, so the compiler can neither
// contract nor reorder them.  Range is FP32's: magnitudes must stay well inside 1e-30 .. 1e30.
#pragma once
#include <cuda_runtime.h>

namespace chebmg {

struct f32x2 {
  float hi, lo;
};

__device__ __forceinline__ f32x2 x2_zero() { return {0.f, 0.f}; }

__device__ __forceinline__ f32x2 x2_from(double v) {
  const float h = __double2float_rn(v);
  return {h, __double2float_rn(v - (double)h)};
}

__device__ __forceinline__ double x2_to_double(f32x2 a) { return (double)a.hi + (double)a.lo; }

// s = fl(a + b), e = (a + b) - s exactly
__device__ __forceinline__ float x2_two_sum(float a, float b, float& e) {
  const float s = __fadd_rn(a, b);
  const float bv = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bv)), __fsub_rn(b, bv));
  return s;
}

// the same when |a| >= |b| (or a == 0)
__device__ __forceinline__ float x2_quick_two_sum(float a, float b, float& e) {
  const float s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
  return s;
}

// a + b: the high parts' sum is exact (TwoSum), the low parts are added in FP32.  The error
// is a few units of 2^-48 of max(|a|, |b|) -- the behaviour of FP64 addition scaled by 2^5,
// since the operands themselves carry relative errors of 2^-48 (a version that also carries
// the low parts' rounding error is exact to 2^-48 of the result, at twice the cost).
__device__ __forceinline__ f32x2 x2_add(f32x2 a, f32x2 b) {
  float e;
  const float s = x2_two_sum(a.hi, b.hi, e);
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  float l;
  const float h = x2_quick_two_sum(s, e, l);
  return {h, l};
}

__device__ __forceinline__ f32x2 x2_neg(f32x2 a) { return {-a.hi, -a.lo}; }

__device__ __forceinline__ f32x2 x2_sub(f32x2 a, f32x2 b) { return x2_add(a, x2_neg(b)); }

// a * b: exact product of the high parts plus the cross terms (the lo * lo term is below the
// format's precision)
__device__ __forceinline__ f32x2 x2_mul(f32x2 a, f32x2 b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  float l;
  const float h = x2_quick_two_sum(p, e, l);
  return {h, l};
}

// a * b + c with the product's error terms folded into the low part of the sum (one
// normalisation instead of two)
__device__ __forceinline__ f32x2 x2_fma(f32x2 a, f32x2 b, f32x2 c) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  float t;
  const float s = x2_two_sum(p, c.hi, t);
  t = __fadd_rn(t, __fadd_rn(e, c.lo));
  float l;
  const float h = x2_quick_two_sum(s, t, l);
  return {h, l};
}

}  // namespace chebmg
