// Helpers of the mixed-precision forms: velocities are float pairs in "V
// units" (an integer V moves a marker a fixed number of position units), v* is
// an integer V*, and divisions use one residual-corrected reciprocal.
#pragma once

#include <cuda_runtime.h>

#include "debug_bounds.cuh"
#include "ff.cuh"
#include "pic_internal.cuh"

namespace pic {
namespace {

// Padded node indices.  The shared-memory field tables and current tiles carry
// ghost nodes so that the nodes of a marker's shape are consecutive with no
// periodic wrap: nc + 3 padded nodes, padded node q standing for grid node
// (q - kPad) mod nc with kPad = 1 for order 2 (nodes i0 - 1 .. i0 + 1, i0 in
// [0, nc]) and 0 for order 1 (nodes i, i + 1, i in [0, nc)).
template <int ORDER>
struct Pad {
  static constexpr int kPad = ORDER == 2 ? 1 : 0;
};
__device__ __forceinline__ int npad_of(int nc) { return nc + 3; }
__device__ __forceinline__ int wrap_node(int i, int nc) {
  return i < 0 ? i + nc : (i >= nc ? i - nc : i);
}

// Shape of a marker at X: first padded node p (in [0, nc + ORDER - 1) for
// any 32-bit X) and the weights.  The weights
// are quantised B-spline values, multiples of 2^-23, available both as floats
// (w, for the gathers) and as integers (s = w 2^23, for the deposits); gather
// and deposit at the same X therefore use exactly the same numbers and sum to
// 1 exactly.  Order 1: w = (1 - f, f).  Order 2: with f = xi - i0 + 1/2 in
// [0, 1), w = (1/2 (1 - f)^2, 1 - w0 - w2, 1/2 f^2) at nodes i0 - 1, i0, i0 + 1.
template <int ORDER>
struct ShapeMix {
  int p;
  float w[ORDER + 1];
  int s[ORDER + 1];
  ShapeMix() = default;
  __device__ __forceinline__ ShapeMix(uint32_t X, int nc) {
    // xi (+ 1/2 for order 2) in 32.32 fixed point
    const uint64_t P = (uint64_t)X * (uint32_t)nc + (ORDER == 2 ? 0x80000000ull : 0ull);
    p = PIC_INDEX((int)(P >> 32), nc + ORDER - 1);
    const uint32_t f23 = (uint32_t)P >> 9;
    const float f = __fsub_rn(__uint_as_float(0x3F800000u | f23), 1.0f);  // exact
    if (ORDER == 1) {
      w[0] = __fsub_rn(1.0f, f);
      w[1] = f;
      s[0] = (1 << 23) - (int)f23;
      s[1] = (int)f23;
    } else {
      const float a = __fsub_rn(1.0f, f);
      // 1 + w0 and 1 + w2 in [1, 1.5]: rounding to float puts w on the 2^-23 grid
      const float q0 = __fmaf_rn(__fmul_rn(0.5f, a), a, 1.0f);
      const float q2 = __fmaf_rn(__fmul_rn(0.5f, f), f, 1.0f);
      w[0] = __fsub_rn(q0, 1.0f);
      w[ORDER] = __fsub_rn(q2, 1.0f);
      w[1] = __fsub_rn(__fsub_rn(1.0f, w[0]), w[ORDER]);
      s[0] = __float_as_int(q0) & 0x7FFFFF;
      s[ORDER] = __float_as_int(q2) & 0x7FFFFF;
      s[1] = (1 << 23) - s[0] - s[ORDER];
    }
  }
};

// The shapes of two markers at once: the integer parts per marker, the float
// weights in packed FP32 with the constructor's operations, lane by lane (the
// same bits).
template <int ORDER>
__device__ __forceinline__ void shape_mix_pair(uint32_t X0, uint32_t X1, int nc,
                                               ShapeMix<ORDER> &S0, ShapeMix<ORDER> &S1) {
  const uint64_t P0 = (uint64_t)X0 * (uint32_t)nc + (ORDER == 2 ? 0x80000000ull : 0ull);
  const uint64_t P1 = (uint64_t)X1 * (uint32_t)nc + (ORDER == 2 ? 0x80000000ull : 0ull);
  S0.p = PIC_INDEX((int)(P0 >> 32), nc + ORDER - 1);
  S1.p = PIC_INDEX((int)(P1 >> 32), nc + ORDER - 1);
  const uint32_t g0 = (uint32_t)P0 >> 9, g1 = (uint32_t)P1 >> 9;
  const float2 one = splat2(1.0f);
  const float2 f = sub2(make_float2(__uint_as_float(0x3F800000u | g0),
                                    __uint_as_float(0x3F800000u | g1)), one);
  if (ORDER == 1) {
    const float2 w0 = sub2(one, f);
    S0.w[0] = w0.x;
    S1.w[0] = w0.y;
    S0.w[1] = f.x;
    S1.w[1] = f.y;
    S0.s[0] = (1 << 23) - (int)g0;
    S1.s[0] = (1 << 23) - (int)g1;
    S0.s[1] = (int)g0;
    S1.s[1] = (int)g1;
  } else {
    const float2 a = sub2(one, f);
    const float2 q0 = fma2(mul2(splat2(0.5f), a), a, one);
    const float2 q2 = fma2(mul2(splat2(0.5f), f), f, one);
    const float2 w0 = sub2(q0, one), w2 = sub2(q2, one);
    const float2 w1 = sub2(sub2(one, w0), w2);
    S0.w[0] = w0.x;
    S1.w[0] = w0.y;
    S0.w[1] = w1.x;
    S1.w[1] = w1.y;
    S0.w[ORDER] = w2.x;
    S1.w[ORDER] = w2.y;
    S0.s[0] = __float_as_int(q0.x) & 0x7FFFFF;
    S1.s[0] = __float_as_int(q0.y) & 0x7FFFFF;
    S0.s[ORDER] = __float_as_int(q2.x) & 0x7FFFFF;
    S1.s[ORDER] = __float_as_int(q2.y) & 0x7FFFFF;
    S0.s[1] = (1 << 23) - S0.s[0] - S0.s[ORDER];
    S1.s[1] = (1 << 23) - S1.s[0] - S1.s[ORDER];
  }
}

// The two tile counters' shares of round(V s / 2^r) (rnd = 2^(r-1)) with a
// low counter of b bits: bits [r, r + b) of P = V s + rnd (unsigned) and
// P >> (r + b) (signed); a node's value is (signed share) 2^b + (unsigned
// share).  Needs r <= 31 and r + b >= 32 (the signed share comes from the high
// word of P alone).
struct SplitTerm {
  unsigned lo;
  int hi;
};
__device__ __forceinline__ SplitTerm split_term(int V, int s, int rshift, long long rnd,
                                                unsigned lomask, int hishift) {
  // lomask = 2^b - 1, hishift = r + b - 32
  const long long P = (long long)V * (long long)s + rnd;
  const unsigned plo = (unsigned)P, phi = (unsigned)(P >> 32);
  return {__funnelshift_r(plo, phi, rshift) & lomask, (int)phi >> hishift};
}

// 16-byte asynchronous global -> shared copy (L2 only), its commit and the
// wait for all of this thread's copies: the passes stage a thread's next
// marker words in shared-memory slots of its own while it works on the
// current ones.
__device__ __forceinline__ void cp_async16(unsigned dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_group 0;" ::: "memory");
}
__device__ __forceinline__ float4 uint_as_float4(uint4 u) {
  return make_float4(__uint_as_float(u.x), __uint_as_float(u.y), __uint_as_float(u.z),
                     __uint_as_float(u.w));
}

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

// The correction of Eq. opt_solution in FP64, shared by the mixed forms.  With
// R = |v^n|^2 + 2 v* . (v^dag - v^n) and Delta = v^dag - v^n, R - |v^dag|^2 =
// 2a, a = sum_i Delta_i b_i, b_i = V*_i - v^n_i - Delta_i / 2.  bracket_fp64
// forms b_i from its exact pieces (V*_i - ih an integer, fr = vh - ih, vl, and
// the float pair Delta_i), so a and t = 2a / |v^dag|^2 keep FP64's relative
// precision however small they are.
__device__ __forceinline__ double bracket_fp64(float vh, float vl, int Vs, ff D) {
  const int ih = __float2int_rn(vh);
  const double fr = (double)__fsub_rn(vh, __int2float_rn(ih));
  return (((double)(Vs - ih) - 0.5 * (double)D.hi) - fr) - (double)vl - 0.5 * (double)D.lo;
}
__device__ __forceinline__ double ff_to_double(ff a) { return (double)a.hi + (double)a.lo; }

// Gamma - 1 = sqrt(1 + t) - 1, t = 2a / v2 (v2 = |v^dag|^2), in FP64 (one
// quotient, one root).  Its absolute error is about 2^-53, and v^{n+1} =
// v^dag + (Gamma - 1) v^dag needs no more: the float-pair velocity holds 48
// bits.  Returns false for the fallback of Sec. 3.2: R < 0 (t < -1) or v^dag =
// 0 (t not finite); R = 0 gives Gamma = 0.
__device__ __forceinline__ bool gamma_minus_one_fp64(double a, double v2, double &g) {
  const double t = 2.0 * a / v2;
  if (!(t >= -1.0 && t < 1e300)) return false;
  g = sqrt(1.0 + t) - 1.0;
  return true;
}

// v^dag_i + g v^dag_i: the product rounded once in FP64, added as a float pair
__device__ __forceinline__ ff scale_by_gamma_fp64(ff vd, double g) {
  return ff_add(vd, ff_from_double(g * ff_to_double(vd)));
}

}  // namespace
}  // namespace pic
