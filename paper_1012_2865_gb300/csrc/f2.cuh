// f2.cuh -- double-float arithmetic: a value carried as an unevaluated sum
// of two FP32 numbers (hi, lo) with |lo| <= ulp(hi)/2, about 48 significant
// bits.  Error-free transformations after Knuth (two_sum), Dekker
// (fast_two_sum, |a| >= |b|) and the FMA product error (two-product).
#pragma once
#include <cuda_runtime.h>
#include <math.h>

namespace rtg {

struct F2 {
  float hi, lo;
};
__device__ __forceinline__ F2 two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float err = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, err};
}
__device__ __forceinline__ F2 fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ F2 f2_mul(F2 a, F2 b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
  return fast_two_sum(p, e);
}
__device__ __forceinline__ F2 f2_add(F2 a, F2 b) {
  F2 s = two_sum(a.hi, b.hi);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
// a - b as FP32 (both pairs), accurate to ~2^-44 |a|
__device__ __forceinline__ float f2_diff(F2 a, F2 b) {
  const F2 d = two_sum(a.hi, -b.hi);
  return __fadd_rn(d.hi, __fadd_rn(d.lo, __fsub_rn(a.lo, b.lo)));
}
__device__ __forceinline__ bool f2_less(F2 a, F2 b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ bool f2_eq(F2 a, F2 b) { return a.hi == b.hi && a.lo == b.lo; }
// 1 / (n.hi + n.lo) as a pair (one Newton correction)
__device__ __forceinline__ F2 f2_recip(F2 n) {
  const float q = __frcp_rn(n.hi);
  float e = fmaf(-n.hi, q, 1.0f);
  e = fmaf(-n.lo, q, e);
  return fast_two_sum(q, __fmul_rn(e, q));
}
__device__ __forceinline__ int f2_floor(F2 u) {
  const float f = floorf(u.hi);
  if (u.hi == f && u.lo < 0.0f) return (int)f - 1;
  return (int)f;
}

// a - b as a pair
__device__ __forceinline__ F2 f2_sub(F2 a, F2 b) { return f2_add(a, F2{-b.hi, -b.lo}); }
// pair times an FP32 number
__device__ __forceinline__ F2 f2_mul_f(F2 a, float b) {
  const float p = __fmul_rn(a.hi, b);
  const float e = fmaf(a.lo, b, fmaf(a.hi, b, -p));
  return fast_two_sum(p, e);
}
// nearest pair to an FP64 value (v - hi is exact in FP64)
__device__ __forceinline__ F2 f2_from_double(double v) {
  const float hi = __double2float_rn(v);
  return {hi, __double2float_rn(__dsub_rn(v, (double)hi))};
}
__device__ __forceinline__ double f2_to_double(F2 a) { return __dadd_rn((double)a.hi, (double)a.lo); }
__device__ __forceinline__ float f2_to_float(F2 a) { return __fadd_rn(a.hi, a.lo); }

}  // namespace rtg
