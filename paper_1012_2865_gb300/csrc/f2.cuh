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

// The same two conversions with the format changes done in integer
// arithmetic (IEEE-754 binary64 / binary32 fields), for kernels where the
// FP64 pipe, a small fraction of the FP32 one, would otherwise bound them.
//
// Nearest pair to v: hi = v rounded to 24 bits (ties to even) by adding the
// rounding bias to the binary64 pattern (a carry moves into the exponent as
// it should); v - hi is then the difference of the two patterns, an integer
// of at most 2^28 units of v's last place, and lo its FP32 rounding.  Equal
// to f2_from_double for zeros and 2^-74 <= |v| < 2^125, which it handles
// this way (hi and lo stay normal FP32 numbers); other values take
// f2_from_double.
// The rare operands of these conversions go through functions that are
// never inlined, so the compiler cannot predicate their FP64 instructions
// into the common path.
static __device__ __noinline__ F2 f2_from_double_call(double v) { return f2_from_double(v); }
static __device__ __noinline__ double f32_widen_call(float f) { return (double)f; }
__device__ __forceinline__ F2 f2_from_double_bits(double v) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(v);
  const unsigned uh = (unsigned)(u >> 32);
  const unsigned long long mag = u & 0x7fffffffffffffffULL;
  if (mag == 0ULL) return {__uint_as_float(uh & 0x80000000u), 0.0f};  // signed zero
  const int e = (int)((uh >> 20) & 0x7ffu);  // biased binary64 exponent
  if (e < 949 || e > 1147) return f2_from_double_call(v);
  const unsigned long long r = (mag + 0x0fffffffULL + ((mag >> 29) & 1ULL)) & ~0x1fffffffULL;
  const long long d = (long long)(mag - r);  // |v| - |hi|, units of 2^(e - 1075)
  const unsigned rh = (unsigned)(r >> 32), rl = (unsigned)r;
  const unsigned sign = uh & 0x80000000u;
  const unsigned hb = sign | ((((rh >> 20) & 0x7ffu) - 896u) << 23) | ((rh & 0xfffffu) << 3) | (rl >> 29);
  const float scale = __uint_as_float((unsigned)(e - 948) << 23);  // 2^(e - 1075)
  const float lo = __fmul_rn(__int2float_rn((int)d), scale);  // |d| <= 2^28
  return {__uint_as_float(hb), sign ? -lo : lo};
}
// An FP32 number widened to binary64 exactly by moving its fields (normal
// numbers and zeros; others take the conversion instruction).
__device__ __forceinline__ double f32_widen_bits(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned ex = (b >> 23) & 0xffu;
  if (ex == 0u || ex == 0xffu) {
    if ((b << 1) == 0u) return __longlong_as_double((long long)((unsigned long long)b << 32));
    return f32_widen_call(f);
  }
  const unsigned hi = (b & 0x80000000u) | ((ex + 896u) << 20) | ((b & 0x7fffffu) >> 3);
  return __hiloint2double((int)hi, (int)(b << 29));
}
// hi + lo rounded to binary64 with one FP64 addition.
__device__ __forceinline__ double f2_to_double_bits(F2 a) { return __dadd_rn(f32_widen_bits(a.hi), f32_widen_bits(a.lo)); }
__device__ __forceinline__ float f2_to_float(F2 a) { return __fadd_rn(a.hi, a.lo); }
// a + b rounded to FP32: f2_to_float(f2_add(a, b)) without the final
// renormalisation (the same value)
__device__ __forceinline__ float f2_sum_float(F2 a, F2 b) {
  const F2 s = two_sum(a.hi, b.hi);
  return __fadd_rn(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}

}  // namespace rtg
