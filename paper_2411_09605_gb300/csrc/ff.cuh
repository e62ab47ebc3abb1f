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

__host__ __device__ inline ff ff_from_double(double x) {
  float h = (float)x;
  float l = (float)(x - (double)h);
  return {h, l};
}

}  // namespace pic
