// Helpers of the mixed-precision forms: velocities are float pairs in "V
// units" (an integer V moves a marker a fixed number of position units), v* is
// an integer V*, and divisions use one residual-corrected reciprocal.
#pragma once

#include <cuda_runtime.h>

#include "ff.cuh"
#include "pic_internal.cuh"

namespace pic {
namespace {

// rint(y) with a range flag: |y| must stay below the largest float under 2^31
__device__ __forceinline__ int to_fixed(float y, unsigned &bad) {
  if (!(fabsf(y) < 2147483520.0f)) bad |= kErrVelocityRange;
  return __float2int_rn(y);
}

// V* = rint(v + e) to one V unit for the float pair v = (vh, vl) and a float
// e: above 2^24 a float cannot hold every integer, so the sum is split into an
// integer part and an exact remainder, and only the remainder is rounded.
__device__ __forceinline__ int vstar_fixed(float vh, float vl, float e, unsigned &bad) {
  const ff s = two_sum(vh, e);
  const int vi = to_fixed(s.hi, bad);
  const float rem = __fadd_rn(__fadd_rn(__fsub_rn(s.hi, (float)vi), s.lo), vl);
  return vi + __float2int_rn(rem);
}

// vstar_fixed for two markers (lanes x, y), the float work in packed FP32
// with the same operations lane by lane.
__device__ __forceinline__ void vstar_fixed2(float2 vh, float2 vl, float2 e, unsigned &bad,
                                             int (&out)[2]) {
  const ff2 s = two_sum2(vh, e);
  const int v0 = to_fixed(s.hi.x, bad), v1 = to_fixed(s.hi.y, bad);
  const float2 rem =
      add2(add2(sub2(s.hi, make_float2((float)v0, (float)v1)), s.lo), vl);
  out[0] = v0 + __float2int_rn(rem.x);
  out[1] = v1 + __float2int_rn(rem.y);
}

// a / b by one correction of the hardware reciprocal estimate r with the
// exact FMA residual (Markstein's FMA division): q0 = a r, e = a - q0 b,
// q = q0 + e r.  Before its final rounding q is within about 2^-44 |a/b| of
// the quotient, so q is the correctly rounded quotient except next to a tie
// (then one ulp off, either way).  b = 0 or a subnormal b give a non-finite or
// huge q.
__device__ __forceinline__ float div_rcp_residual(float a, float b) {
  float r;
  asm("rcp.approx.f32 %0, %1;" : "=f"(r) : "f"(b));
  const float q0 = __fmul_rn(a, r);
  const float e = __fmaf_rn(-q0, b, a);
  return __fmaf_rn(e, r, q0);
}

}  // namespace
}  // namespace pic
