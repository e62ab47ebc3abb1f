// Unevaluated float pairs ("float-float"): a value a = hi + lo with |lo| <=
// ulp(hi)/2, about 48 significant bits, built only from FP32 operations.
// Error-free transformations: two_sum (Knuth 1969), fast_two_sum (Dekker
// 1971) and two_prod with a fused multiply-add.  Every operation is written
// with explicitly rounded intrinsics, so no compiler contraction changes a
// result between the kernels that must agree bit for bit.
#pragma once

#include <cuda_runtime.h>

namespace pic {

struct ff {
  float hi, lo;
};

__device__ __forceinline__ ff two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}

// requires |a| >= |b| (or a == 0)
__device__ __forceinline__ ff fast_two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float e = __fsub_rn(b, __fsub_rn(s, a));
  return {s, e};
}

__device__ __forceinline__ ff two_prod(float a, float b) {
  float p = __fmul_rn(a, b);
  float e = __fmaf_rn(a, b, -p);
  return {p, e};
}

__device__ __forceinline__ ff ff_add(ff a, ff b) {
  ff s = two_sum(a.hi, b.hi);
  float e = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return fast_two_sum(s.hi, e);
}

__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, {-b.hi, -b.lo}); }

__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  ff p = two_prod(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo));
  return fast_two_sum(p.hi, e);
}

// a * f with a float factor f
__device__ __forceinline__ ff ff_mul_f(ff a, float f) {
  ff p = two_prod(a.hi, f);
  float e = __fmaf_rn(a.lo, f, p.lo);
  return fast_two_sum(p.hi, e);
}

// Two float pairs side by side, lane x for one marker and lane y for
// another, with the packed two-lane FP32 add / multiply / FMA of sm_100 and
// later: each lane rounds as the scalar instruction does, and every function
// below performs, lane by lane, the operations of its scalar namesake above.
// a - b is the add of -b (the IEEE definition of subtraction).
struct ff2 {
  float2 hi, lo;
};

__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, neg2(b)); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 splat2(float a) { return make_float2(a, a); }

__device__ __forceinline__ ff2 two_sum2(float2 a, float2 b) {
  const float2 s = add2(a, b);
  const float2 bb = sub2(s, a);
  return {s, add2(sub2(a, sub2(s, bb)), sub2(b, bb))};
}

// requires |a| >= |b| (or a == 0) in each lane
__device__ __forceinline__ ff2 fast_two_sum2(float2 a, float2 b) {
  const float2 s = add2(a, b);
  return {s, sub2(b, sub2(s, a))};
}

__device__ __forceinline__ ff2 two_prod2(float2 a, float2 b) {
  const float2 p = mul2(a, b);
  return {p, fma2(a, b, neg2(p))};
}

__device__ __forceinline__ ff2 ff_add2(ff2 a, ff2 b) {
  const ff2 s = two_sum2(a.hi, b.hi);
  return fast_two_sum2(s.hi, add2(s.lo, add2(a.lo, b.lo)));
}

__host__ __device__ inline ff ff_from_double(double x) {
  float h = (float)x;
  float l = (float)(x - (double)h);
  return {h, l};
}

}  // namespace pic
