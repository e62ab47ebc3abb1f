// 2D3V electromagnetic step with the leapfrog / Yee field update (Sec. 4.1,
// Eq. EMleapfrog), mixed-precision form.
//
// The FP64 form of this step is bound by the FP64 pipe (a per-marker v* solve,
// two gathers of six components and Gamma).  This form keeps FP64 on the grid
// only (the field update, K5 and the energy sums are those of the FP64 form)
// and runs the per-marker work in FP32, float pairs and integers, with the
// energy still conserved to the FP64 bound:
//   * positions X, Y: 32-bit fixed point, x = X L / 2^32 (Lx = Ly = L); the
//     cell and in-cell fraction come from X n as a 32.32 number and the
//     periodic wrap is the integer overflow.
//   * velocities: float pairs (vh, vl) in V units, v cxk with cxk =
//     (dt 2^31 / L) 2^kv for all three components; v* is the integer V*, so
//     x^{n+1/2} = X + [V*_x]_kv and x^{n+1} = X + 2 [V*_x]_kv are exact.
//   * weights: quantised B-spline values (multiples of 2^-23) per axis; the
//     gather of E^{n+1/2} and the deposit of j^{*,n+1/2} use the same
//     integers s_x s_y, as Eq. exp_econs_simple requires.
//   * current: each marker adds floor(V*_c s_x s_y / 2^r + 1/2) (r >= 32, so
//     no node sum overflows) to the int64 node sums with global atomics: exact
//     integer sums, independent of the marker order.  With sort_period P the
//     markers are kept in quarter-cell order (written so by pass E every P
//     steps), and the terms of a thread's consecutive markers in one quarter
//     cell are summed in registers and then over the warp before the atomics.
//   * gather #1 (E*, B at x*) only shapes v*: FP32 tables and FP32 weights;
//     v* = (u + u x t + (u.t) t) / (1 + |t|^2) as u plus an FP32 correction.
//   * gather #2: kick E^{n+1/2} as float pairs with error-free products, so
//     the kick d is the grid's E^{n+1/2} to about 2^-46.
//   * the magnetic term mu = dt (q/m) V* x B is formed in float pairs from the
//     exact V*: V* . mu is zero to the pairs' precision, so B does no work
//     (whatever rounding the B table had).
//   * Gamma (Eq. opt_solution): with Delta = v^dag - v^n = d + mu,
//     |v^{n+1}|^2 - |v^dag|^2 = 2 Delta . (V* - v^n - Delta/2), the bracket
//     from the exact difference V* - v^n per component, t = 2a / |v^dag|^2,
//     and Gamma - 1 = sqrt(1 + t) - 1: a 4-term FP32 series for |t| < 2^-8,
//     FP64 otherwise (every candidate for the fallback among them).
#include <cuda_runtime.h>
#include <stdint.h>

#include "em2d_common.cuh"
#include "ff.cuh"
#include "mixed_common.cuh"
#include "pdl.cuh"
#include "pic_internal.cuh"

namespace pic {
namespace {

// Quantised B-spline weights of one axis.  X is the position as a 32-bit
// fraction of the box, n the cells of the axis; half = the component sits on
// the half nodes (i + 1/2).  i0 is the first node, k[] the periodic node
// indices, w[] the weights as floats and s[] = w 2^23 as integers (sum 2^23).
// Order 1: w = (1 - f, f) at floor(xi), floor(xi) + 1.  Order 2: with
// f = frac(xi + 1/2), w = (1/2 (1 - f)^2, 1 - w0 - w2, 1/2 f^2) at
// floor(xi + 1/2) - 1 .. + 1.  xi is in cells, less 1/2 for half nodes.
template <int ORDER>
struct AxisMix {
  int k[ORDER + 1];
  float w[ORDER + 1];
  uint32_t s[ORDER + 1];
  __device__ __forceinline__ AxisMix(uint32_t X, int n, bool half) {
    // xi (+ 1/2 for order 2, - 1/2 for half nodes) + n as a 32.32 number,
    // kept positive by the offset of n cells
    const uint64_t P = (uint64_t)X * (uint32_t)n + ((uint64_t)(uint32_t)n << 32) +
                       (ORDER == 2 ? 0x80000000ull : 0ull) - (half ? 0x80000000ull : 0ull);
    const int i0 = (int)(P >> 32) - n - (ORDER == 2 ? 1 : 0);
    // i0 lies in [0, n - 1] (order 1, integer nodes), [-1, n - 2] (order 2,
    // half nodes) or [-1, n - 1]: node i0 + a can fall below 0 only for a = 0
    // and i0 < 0 possible, and reach n only for a >= 1 (a = 2 when i0 <= n - 2)
#pragma unroll
    for (int a = 0; a <= ORDER; a++) {
      const int i = i0 + a;
      const bool low = a == 0 && (half || ORDER == 2);
      const bool high = a >= ((half && ORDER == 2) ? 2 : 1);
      k[a] = PIC_INDEX(low ? (i < 0 ? i + n : i) : (high ? (i >= n ? i - n : i) : i), n);
    }
    const uint32_t f23 = (uint32_t)P >> 9;
    const float f = __fsub_rn(__uint_as_float(0x3F800000u | f23), 1.0f);  // exact
    if (ORDER == 1) {
      w[0] = __fsub_rn(1.0f, f);
      w[1] = f;
      s[0] = (1u << 23) - f23;
      s[1] = f23;
    } else {
      const float a = __fsub_rn(1.0f, f);
      // 1 + w0 and 1 + w2 in [1, 1.5]: rounding to float puts w on the 2^-23 grid
      const float q0 = __fmaf_rn(__fmul_rn(0.5f, a), a, 1.0f);
      const float q2 = __fmaf_rn(__fmul_rn(0.5f, f), f, 1.0f);
      w[0] = __fsub_rn(q0, 1.0f);
      w[ORDER] = __fsub_rn(q2, 1.0f);
      w[1] = __fsub_rn(__fsub_rn(1.0f, w[0]), w[ORDER]);
      s[0] = (uint32_t)__float_as_int(q0) & 0x7FFFFFu;
      s[ORDER] = (uint32_t)__float_as_int(q2) & 0x7FFFFFu;
      s[1] = (1u << 23) - s[0] - s[ORDER];
    }
  }
};

// Weights of a point for integer-node (I) and half-node (H) components.
template <int ORDER>
struct Shape2Mix {
  AxisMix<ORDER> xI, xH, yI, yH;
  __device__ __forceinline__ Shape2Mix(uint32_t X, uint32_t Y, int nx, int ny)
      : xI(X, nx, false), xH(X, nx, true), yI(Y, ny, false), yH(Y, ny, true) {}
};

// V units -> position units for half a step (kv >= 1)
__device__ __forceinline__ uint32_t half_shift(int V, const Em2dMixConst &c) {
  return (uint32_t)((V + c.hround) >> c.kv);
}

template <int ORDER>
__device__ __forceinline__ float gather_f(const float *T, int nx, const AxisMix<ORDER> &ax,
                                          const AxisMix<ORDER> &ay) {
  float s = 0.0f;
#pragma unroll
  for (int b = 0; b <= ORDER; b++) {
    const float *row = T + ay.k[b] * nx;
    float r = 0.0f;
#pragma unroll
    for (int a = 0; a <= ORDER; a++) r = __fmaf_rn(__ldg(row + ax.k[a]), ax.w[a], r);
    s = __fmaf_rn(r, ay.w[b], s);
  }
  return s;
}

// sum_b w_y[b] sum_a w_x[a] T[b][a] of a float-pair table: error-free
// products with the quantised weights, the large parts summed by two-sums
template <int ORDER>
__device__ __forceinline__ ff gather_ff(const float2 *T, int nx, const AxisMix<ORDER> &ax,
                                        const AxisMix<ORDER> &ay) {
  ff acc{0.0f, 0.0f};
#pragma unroll
  for (int b = 0; b <= ORDER; b++) {
    const float2 *row = T + ay.k[b] * nx;
    float ph[ORDER + 1], pl = 0.0f;
#pragma unroll
    for (int a = 0; a <= ORDER; a++) {
      const float2 e = __ldg(row + ax.k[a]);
      const ff p = two_prod(e.x, ax.w[a]);
      ph[a] = p.hi;
      pl = __fadd_rn(pl, __fmaf_rn(e.y, ax.w[a], p.lo));
    }
    ff r = two_sum(ph[0], ph[1]);
    pl = __fadd_rn(pl, r.lo);
    if (ORDER == 2) {
      r = two_sum(r.hi, ph[ORDER]);
      pl = __fadd_rn(pl, r.lo);
    }
    acc = ff_add(acc, ff_mul_f(fast_two_sum(r.hi, pl), ay.w[b]));
  }
  return acc;
}

// floor(V s_a s_b / 2^r + 1/2) (the nearest integer, ties up) for r >= 32,
// given m = V s_b (|V| < 2^31, s <= 2^23, so |V s_a s_b| < 2^77): with m =
// mh 2^32 + ml (mh signed, ml unsigned), m s_a + 2^(r-1) = (mh s_a + ((ml s_a +
// 2^(r-1)) >> 32)) 2^32 + the low word, and the floor of its quotient by 2^r is
// the arithmetic shift of the first factor by r - 32.
__device__ __forceinline__ long long deposit_term(long long m, uint32_t sa,
                                                  const Em2dMixConst &c) {
  const uint64_t lo = (uint64_t)(uint32_t)m * sa + (uint64_t)c.rnd;
  const long long hi = (long long)(int)(m >> 32) * (long long)sa + (long long)(lo >> 32);
  return hi >> (c.rshift - 32);
}

template <int ORDER>
__device__ __forceinline__ void deposit_c(long long *J, int nx, const AxisMix<ORDER> &ax,
                                          const AxisMix<ORDER> &ay, int V,
                                          const Em2dMixConst &c) {
  if (V == 0) return;
#pragma unroll
  for (int b = 0; b <= ORDER; b++) {
    const long long m = (long long)V * ay.s[b];
    long long *row = J + ay.k[b] * nx;
#pragma unroll
    for (int a = 0; a <= ORDER; a++)
      atomicAdd((unsigned long long *)(row + ax.k[a]),
                (unsigned long long)deposit_term(m, ax.s[a], c));
  }
}

// j of velocity V at the shape's point: Jx on (H, I), Jy on (I, H), Jz on (I, I)
template <int ORDER>
__device__ __forceinline__ void deposit_j(const Em2dMixConst &c, long long *J,
                                          const Shape2Mix<ORDER> &S, const int V[3]) {
  const int nx = c.nx, nc = c.nx * c.ny;
  deposit_c<ORDER>(J, nx, S.xH, S.yI, V[0], c);
  deposit_c<ORDER>(J + nc, nx, S.xI, S.yH, V[1], c);
  deposit_c<ORDER>(J + 2 * nc, nx, S.xI, S.yI, V[2], c);
}

// Segments of a warp's lanes: neighbouring lanes with equal keys (the quarter
// cell of their deposit runs) form a segment.  With the markers sorted by
// quarter cell, the lanes of a warp hold a few segments, and each segment's
// deposits can be summed over its lanes before one atomic per node: exact
// integer sums, so the result is the per-marker atomics' bit for bit, whatever
// the order (an unsorted warp only gets shorter segments).
struct WarpSegments {
  int start;  // first lane of this lane's segment
  bool tail;  // this lane ends its segment
  __device__ __forceinline__ explicit WarpSegments(int key) {
    const unsigned lane = threadIdx.x & 31u;
    const int prev = __shfl_up_sync(0xffffffffu, key, 1);
    const unsigned heads = __ballot_sync(0xffffffffu, lane == 0u || key != prev);
    start = 31 - __clz(heads & (0xffffffffu >> (31u - lane)));
    tail = lane == 31u || ((heads >> (lane + 1u)) & 1u);
  }
  // inclusive sum of v over the lanes of the segment up to this one
  __device__ __forceinline__ long long scan(long long v) const {
    const int lane = (int)(threadIdx.x & 31u);
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const long long t = __shfl_up_sync(0xffffffffu, v, d);
      if (lane - d >= start) v += t;
    }
    return v;
  }
};

// The quarter cell floor(2x / hx) + 2 nx floor(2y / hy) of a point: within a
// quarter cell every current component's stencil starts at the same node
// (order 1 and 2, integer and half nodes).
__device__ __forceinline__ int quarter_key(uint32_t X, uint32_t Y, int nx, int ny) {
  const int qx = (int)(((uint64_t)X * (uint32_t)(2 * nx)) >> 32);
  const int qy = (int)(((uint64_t)Y * (uint32_t)(2 * ny)) >> 32);
  return PIC_INDEX(qx + 2 * nx * qy, 4 * nx * ny);
}

// The deposits of a thread's consecutive markers (sorted by quarter cell),
// summed in registers while they fall in one quarter cell: a marker in
// another quarter cell first sends the run's sums to the grid, and the last
// run of each thread goes through the warp's segmented sums (flush_warp), one
// atomic per segment and node.  The sums are exact integers, so the grid gets
// the per-marker atomics' result bit for bit, in any order.
template <int ORDER>
struct DepositRun {
  static constexpr int K = (ORDER + 1) * (ORDER + 1);
  long long s[3][K];  // Jx, Jy, Jz terms, node (a, b) at b (ORDER + 1) + a
  int key;            // quarter cell of the run, or -1 - lane while empty
  uint32_t X, Y;      // a deposit point of the run

  __device__ __forceinline__ explicit DepositRun(unsigned lane)
      : key(-1 - (int)lane), X(0u), Y(0u) {
#pragma unroll
    for (int d = 0; d < 3; d++)
#pragma unroll
      for (int t = 0; t < K; t++) s[d][t] = 0;
  }

  __device__ __forceinline__ static void add_terms(const AxisMix<ORDER> &ax,
                                                   const AxisMix<ORDER> &ay, int V,
                                                   const Em2dMixConst &c, long long *t) {
#pragma unroll
    for (int b = 0; b <= ORDER; b++) {
      const long long m = (long long)V * ay.s[b];
#pragma unroll
      for (int a = 0; a <= ORDER; a++) t[b * (ORDER + 1) + a] += deposit_term(m, ax.s[a], c);
    }
  }

  // adds sum(d, i) to node i of component d's stencil at the run's point (zero
  // sums skipped)
  template <typename F>
  __device__ __forceinline__ void to_grid(const Em2dMixConst &c, long long *J, F &&sum) const {
    const int nx = c.nx, nc = c.nx * c.ny;
    const Shape2Mix<ORDER> S(X, Y, c.nx, c.ny);
    const AxisMix<ORDER> *ax[3] = {&S.xH, &S.xI, &S.xI}, *ay[3] = {&S.yI, &S.yH, &S.yI};
#pragma unroll
    for (int d = 0; d < 3; d++)
#pragma unroll
      for (int b = 0; b <= ORDER; b++)
#pragma unroll
        for (int a = 0; a <= ORDER; a++) {
          const long long v = sum(d, b * (ORDER + 1) + a);
          if (v != 0)
            atomicAdd((unsigned long long *)(J + d * nc + ay[d]->k[b] * nx + ax[d]->k[a]),
                      (unsigned long long)v);
        }
  }

  // one marker with deposit point (Xd, Yd), shape S there and velocity V
  __device__ __forceinline__ void add(const Em2dMixConst &c, long long *J, uint32_t Xd,
                                      uint32_t Yd, const Shape2Mix<ORDER> &S, const int V[3]) {
    const int k = quarter_key(Xd, Yd, c.nx, c.ny);
    if (k != key) {
      if (key >= 0) to_grid(c, J, [&](int d, int i) { return s[d][i]; });
      key = k;
      X = Xd;
      Y = Yd;
#pragma unroll
      for (int d = 0; d < 3; d++)
#pragma unroll
        for (int i = 0; i < K; i++) s[d][i] = 0;
    }
    add_terms(S.xH, S.yI, V[0], c, s[0]);
    add_terms(S.xI, S.yH, V[1], c, s[1]);
    add_terms(S.xI, S.yI, V[2], c, s[2]);
  }

  // called by every lane of the warp: the last lane of each segment of equal
  // keys adds the segment's sums
  __device__ __forceinline__ void flush_warp(const Em2dMixConst &c, long long *J) {
    const WarpSegments seg(key);
#pragma unroll
    for (int d = 0; d < 3; d++)
#pragma unroll
      for (int i = 0; i < K; i++) s[d][i] = seg.scan(s[d][i]);
    if (seg.tail && key >= 0) to_grid(c, J, [&](int d, int i) { return s[d][i]; });
  }
};

__device__ __forceinline__ void report_bad(unsigned bad, unsigned *err) {
  bad = __reduce_or_sync(0xffffffffu, bad);
  if ((threadIdx.x & 31u) == 0u && bad) atomicOr(err, bad);
}

// An exact integer as a float pair (|V| < 2^31).
__device__ __forceinline__ ff ff_from_int(int V) {
  const float hi = __int2float_rn(V);
  return {hi, __int2float_rn(V - __float2int_rn(hi))};
}

// The non-series path of correct_velocity3: the R < 0 test and Gamma - 1 in
// FP64 (mixed_common.cuh); returns false for the fallback.
__device__ __forceinline__ bool gamma3_fp64(float vh0, float vh1, float vh2, float vl0, float vl1,
                                         float vl2, int V0, int V1, int V2, ff D0, ff D1, ff D2,
                                         ff u0, ff u1, ff u2, double &g) {
  const double a = ff_to_double(D0) * bracket_fp64(vh0, vl0, V0, D0) +
                   ff_to_double(D1) * bracket_fp64(vh1, vl1, V1, D1) +
                   ff_to_double(D2) * bracket_fp64(vh2, vl2, V2, D2);
  const double x = ff_to_double(u0), y = ff_to_double(u1), z = ff_to_double(u2);
  return gamma_minus_one_fp64(a, x * x + y * y + z * z, g);
}

// v^dag = v^n + Delta and v^{n+1} = Gamma v^dag (Eq. opt_solution) in float
// pairs, three components.  R - |v^dag|^2 = 2a with a = Delta . b and
// b = V* - v^n - Delta/2: each b_i is formed from the exact difference
// V*_i - rint(vh_i) and the exact remainders, the small product in FP32.
// Gamma - 1 = sqrt(1 + t) - 1, t = 2a / |v^dag|^2; for |t| < 2^-8 the
// series t/2 - t^2/8 + t^3/16 - 5t^4/128 (relative error < 2^-33); every
// other marker, among them every candidate for the fallback, takes
// gamma3_fp64: R < 0 (t < -1) and v^dag = 0 (t not finite) fall back to
// Gamma = 1, counted.
__device__ __forceinline__ void correct_velocity3(const float vh[3], const float vl[3],
                                                  const int Vs[3], const ff D[3], bool on,
                                                  unsigned &nfb, ff vn[3]) {
  ff vd[3];
#pragma unroll
  for (int d = 0; d < 3; d++) vd[d] = ff_add(ff{vh[d], vl[d]}, D[d]);
  float gm = 0.0f;
  if (on) {
    float a2 = 0.0f, vd2 = 0.0f;
#pragma unroll
    for (int d = 0; d < 3; d++) {
      const int ih = __float2int_rn(vh[d]);
      const float fr = __fsub_rn(vh[d], __int2float_rn(ih));
      const ff q = two_sum(__int2float_rn(Vs[d] - ih), __fmul_rn(-0.5f, D[d].hi));
      const float small =
          __fsub_rn(__fsub_rn(__fsub_rn(q.lo, fr), vl[d]), __fmul_rn(0.5f, D[d].lo));
      const float bq = __fadd_rn(q.hi, small);
      a2 = __fmaf_rn(__fadd_rn(D[d].hi, D[d].hi), bq, a2);
      vd2 = __fmaf_rn(vd[d].hi, vd[d].hi, vd2);
    }
    const float t = div_rcp_residual(a2, vd2);
    if (fabsf(t) < 0.00390625f) {
      gm = __fmul_rn(
          t, __fmaf_rn(t, __fmaf_rn(t, __fmaf_rn(t, -0.0390625f, 0.0625f), -0.125f), 0.5f));
    } else {
      double g;
      if (!gamma3_fp64(vh[0], vh[1], vh[2], vl[0], vl[1], vl[2], Vs[0], Vs[1], Vs[2], D[0], D[1],
                       D[2], vd[0], vd[1], vd[2], g)) {
        nfb++;
      } else {
#pragma unroll
        for (int d = 0; d < 3; d++) vn[d] = scale_by_gamma_fp64(vd[d], g);
        return;
      }
    }
  }
#pragma unroll
  for (int d = 0; d < 3; d++) {
    ff p = two_prod(vd[d].hi, gm);
    p.lo = __fmaf_rn(vd[d].lo, gm, p.lo);
    vn[d] = ff_add(vd[d], p);
  }
}

// K1: e_half E* (ESEC2: E^n + dt/2 (c^2 curl B^{n+1/2} - j^{n,*}); ESEC1: E^n)
// and t_half B^{n+1/2} as FP32 tables; clear J2.  One more block may reduce
// the previous step's total energy (its partials are complete).
__global__ void mix2_k1_kernel(Em2dConst c, Em2dMixConst m, Em2dMixBufs mb, Em2dBufs b,
                               int fin_slot, int nkb, int nfb) {
  griddep_wait();
  griddep_launch_dependents();
  // with fin_slot >= 0 the last block reduces the previous step's TE instead
  const int nb = fin_slot >= 0 ? (int)gridDim.x - 1 : (int)gridDim.x;
  if ((int)blockIdx.x == nb) {
    __shared__ double red[33];
    finalize_block(c, b, fin_slot, nkb, nfb, red);
    return;
  }
  const int nc = c.nx * c.ny;
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < 3 * nc; a += nb * blockDim.x) {
    const int d = a / nc, ij = a % nc, i = ij % c.nx, j = ij / c.nx;
    double es = b.E[a];
    if (m.scheme == 2)
      es = es + 0.5 * c.dt * (c.c2 * curl_b(c, b.Bp, i, j, d) - m.jscale * (double)mb.J1[a]);
    mb.T1[a] = (float)(m.e_half * es);
    mb.T1[3 * nc + a] = (float)(m.t_half * b.Bp[a]);
    mb.J2[a] = 0;
  }
}

// K3: E^{n+1} (FP64), kick E^{n+1/2} as float pairs, m_full B^{n+1/2}; clear J1
__global__ void mix2_k3_kernel(Em2dConst c, Em2dMixConst m, Em2dMixBufs mb, Em2dBufs b) {
  griddep_wait();
  griddep_launch_dependents();
  const int nc = c.nx * c.ny;
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < 3 * nc; a += gridDim.x * blockDim.x) {
    const int d = a / nc, ij = a % nc, i = ij % c.nx, j = ij / c.nx;
    const double en =
        b.E[a] + c.dt * (c.c2 * curl_b(c, b.Bp, i, j, d) - m.jscale * (double)mb.J2[a]);
    const ff k = ff_from_double(m.kick * (0.5 * (b.E[a] + en)));
    b.En[a] = en;
    mb.T2[a] = make_float2(k.hi, k.lo);
    mb.B2[a] = (float)(m.m_full * b.Bp[a]);
    mb.J1[a] = 0;
  }
}

// Pass C for marker p up to v*: x*, E* and B at x*, the integer V* (stored)
// and the deposit point x^{n+1/2} = (Xd, Yd)
template <int ORDER>
__device__ __forceinline__ void pass_c_marker(const Em2dMixConst &c, const Em2dMixBufs &b,
                                              int64_t p, unsigned &bad, int Vs[3],
                                              uint32_t &Xd, uint32_t &Yd) {
  const int nx = c.nx, nc = c.nx * c.ny;
  const uint32_t X = b.X[p], Y = b.Y[p];
  float vh[3], vl[3];
#pragma unroll
  for (int d = 0; d < 3; d++) {
    vh[d] = b.vh[d][p];
    vl[d] = b.vl[d][p];
  }
  const Shape2Mix<ORDER> S1(X + half_shift(to_fixed(vh[0], bad), c),
                            Y + half_shift(to_fixed(vh[1], bad), c), c.nx, c.ny);
  const float *T = b.T1;
  float e[3], t[3];
  e[0] = gather_f<ORDER>(T, nx, S1.xH, S1.yI);
  e[1] = gather_f<ORDER>(T + nc, nx, S1.xI, S1.yH);
  e[2] = gather_f<ORDER>(T + 2 * nc, nx, S1.xI, S1.yI);
  t[0] = gather_f<ORDER>(T + 3 * nc, nx, S1.xI, S1.yH);
  t[1] = gather_f<ORDER>(T + 4 * nc, nx, S1.xH, S1.yI);
  t[2] = gather_f<ORDER>(T + 5 * nc, nx, S1.xH, S1.yH);
  // v* - v* x t = u = v^n + e: v* = u + (u x t + (u.t) t - |t|^2 u) / (1 + |t|^2)
  float u[3];
#pragma unroll
  for (int d = 0; d < 3; d++) u[d] = __fadd_rn(vh[d], e[d]);
  const float ut = __fmaf_rn(u[2], t[2], __fmaf_rn(u[1], t[1], __fmul_rn(u[0], t[0])));
  const float tt = __fmaf_rn(t[2], t[2], __fmaf_rn(t[1], t[1], __fmul_rn(t[0], t[0])));
  const float inv = __frcp_rn(__fadd_rn(1.0f, tt));
  const float r[3] = {__fsub_rn(__fmul_rn(u[1], t[2]), __fmul_rn(u[2], t[1])),
                      __fsub_rn(__fmul_rn(u[2], t[0]), __fmul_rn(u[0], t[2])),
                      __fsub_rn(__fmul_rn(u[0], t[1]), __fmul_rn(u[1], t[0]))};
#pragma unroll
  for (int d = 0; d < 3; d++) {
    const float corr = __fmul_rn(__fmaf_rn(ut, t[d], __fmaf_rn(-tt, u[d], r[d])), inv);
    Vs[d] = vstar_fixed(vh[d], vl[d], __fadd_rn(e[d], corr), bad);
  }
  Xd = X + half_shift(Vs[0], c);
  Yd = Y + half_shift(Vs[1], c);
}

// The lanes of a warp with equal keys (a match over the warp) take their
// slots in cnt[key] with one atomic: each lane gets the old count plus its
// rank among them.  Called by all 32 lanes; a lane with key < 0 has no
// marker (its key is -1 - lane, so it matches no other lane).
__device__ __forceinline__ unsigned warp_slot(unsigned *cnt, int key) {
  const unsigned lane = threadIdx.x & 31u;
  const unsigned grp = __match_any_sync(0xffffffffu, key);
  const int leader = __ffs(grp) - 1;
  unsigned base = 0u;
  if (key >= 0 && lane == (unsigned)leader) base = atomicAdd(&cnt[key], (unsigned)__popc(grp));
  base = __shfl_sync(0xffffffffu, base, leader);
  return base + (unsigned)__popc(grp & ((1u << lane) - 1u));
}

// Markers a thread takes in a row on sorted markers, their deposits summed in
// a DepositRun: each warp takes 32 kRunMarkers consecutive markers, lane l
// those from kRunMarkers l on (every lane the same trips).  Unsorted markers:
// one per thread and trip, per-marker atomics.
constexpr int kRunMarkers = 4;

// Pass C: x*, E* and B at x*, v* (integer V*), x^{n+1/2}, deposit of j^{*,n+1/2};
// on sorted markers, with cnt set (the step that ends a sort period), the
// count of each quarter cell of x^{n+1} = X + 2 [V*]
template <int ORDER, bool SORTED>
__global__ void __launch_bounds__(256, SORTED ? (ORDER == 1 ? 3 : 2) : 0)
    mix2_pass_c_kernel(Em2dMixConst c, Em2dMixBufs b, unsigned *cnt) {
  griddep_wait();
  griddep_launch_dependents();
  const unsigned lane = threadIdx.x & 31u;
  unsigned bad = 0;
  if constexpr (SORTED) {
    constexpr int M = kRunMarkers;
    for (int64_t pw = (blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31u)) * M; pw < c.n;
         pw += (int64_t)gridDim.x * blockDim.x * M) {
      DepositRun<ORDER> run(lane);
#pragma unroll 1
      for (int j = 0; j < M; j++) {
        const int64_t p = pw + (int64_t)lane * M + j;
        int key = -1 - (int)lane;
        if (p < c.n) {
          int Vs[3];
          uint32_t Xd, Yd;
          pass_c_marker<ORDER>(c, b, p, bad, Vs, Xd, Yd);
          run.add(c, b.J2, Xd, Yd, Shape2Mix<ORDER>(Xd, Yd, c.nx, c.ny), Vs);
#pragma unroll
          for (int d = 0; d < 3; d++) b.Vs[d][p] = Vs[d];
          key = quarter_key(Xd + half_shift(Vs[0], c), Yd + half_shift(Vs[1], c), c.nx, c.ny);
        }
        if (cnt) warp_slot(cnt, key);
      }
      run.flush_warp(c, b.J2);
    }
  } else {
    for (int64_t pw = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31u); pw < c.n;
         pw += (int64_t)gridDim.x * blockDim.x) {
      const int64_t p = pw + lane;
      if (p >= c.n) break;
      int Vs[3];
      uint32_t Xd, Yd;
      pass_c_marker<ORDER>(c, b, p, bad, Vs, Xd, Yd);
      deposit_j<ORDER>(c, b.J2, Shape2Mix<ORDER>(Xd, Yd, c.nx, c.ny), Vs);
#pragma unroll
      for (int d = 0; d < 3; d++) b.Vs[d][p] = Vs[d];
    }
  }
  report_bad(bad, b.err);
}

// Pass E for marker p: the gather at x^{n+1/2} = X + [V*], v^dag, Gamma,
// the kinetic energy; returns x^{n+1} = (Xn, Yn), v^{n+1} = vn and (ESEC2)
// the next step's deposit point (Xd, Yd) and V* estimate Vn1
template <int ORDER>
__device__ __forceinline__ void pass_e_marker(const Em2dMixConst &c, const Em2dMixBufs &b,
                                              int64_t p, unsigned &bad, unsigned &nfb,
                                              float &ke_hi, float &ke_lo, int Vn1[3],
                                              uint32_t &Xd, uint32_t &Yd, uint32_t &Xn,
                                              uint32_t &Yn, ff vn[3]) {
  const int nx = c.nx, nc = c.nx * c.ny;
  const uint32_t X = b.X[p], Y = b.Y[p];
  float vh[3], vl[3];
  int Vs[3];
#pragma unroll
  for (int d = 0; d < 3; d++) {
    vh[d] = b.vh[d][p];
    vl[d] = b.vl[d][p];
    Vs[d] = b.Vs[d][p];
  }
  const uint32_t hx = half_shift(Vs[0], c), hy = half_shift(Vs[1], c);
  const Shape2Mix<ORDER> S(X + hx, Y + hy, c.nx, c.ny);
  ff D[3];
  D[0] = gather_ff<ORDER>(b.T2, nx, S.xH, S.yI);
  D[1] = gather_ff<ORDER>(b.T2 + nc, nx, S.xI, S.yH);
  D[2] = gather_ff<ORDER>(b.T2 + 2 * nc, nx, S.xI, S.yI);
  const float bb[3] = {gather_f<ORDER>(b.B2, nx, S.xI, S.yH),
                       gather_f<ORDER>(b.B2 + nc, nx, S.xH, S.yI),
                       gather_f<ORDER>(b.B2 + 2 * nc, nx, S.xH, S.yH)};
  // Delta = d + dt (q/m) V* x B, the cross product in float pairs of the exact V*
  const ff vs[3] = {ff_from_int(Vs[0]), ff_from_int(Vs[1]), ff_from_int(Vs[2])};
  D[0] = ff_add(D[0], ff_sub(ff_mul_f(vs[1], bb[2]), ff_mul_f(vs[2], bb[1])));
  D[1] = ff_add(D[1], ff_sub(ff_mul_f(vs[2], bb[0]), ff_mul_f(vs[0], bb[2])));
  D[2] = ff_add(D[2], ff_sub(ff_mul_f(vs[0], bb[1]), ff_mul_f(vs[1], bb[0])));
  correct_velocity3(vh, vl, Vs, D, c.gamma_on != 0, nfb, vn);
#pragma unroll
  for (int d = 0; d < 3; d++) {
    ff s2 = two_prod(vn[d].hi, vn[d].hi);
    s2.lo = __fmaf_rn(__fadd_rn(vn[d].hi, vn[d].hi), vn[d].lo, s2.lo);
    const ff acc = two_sum(ke_hi, s2.hi);
    ke_hi = acc.hi;
    ke_lo = __fadd_rn(ke_lo, __fadd_rn(acc.lo, s2.lo));
  }
  Xn = X + 2u * hx;
  Yn = Y + 2u * hy;
  if (c.scheme == 2) {
#pragma unroll
    for (int d = 0; d < 3; d++) Vn1[d] = to_fixed(vn[d].hi, bad);
    Xd = Xn + half_shift(Vn1[0], c);
    Yd = Yn + half_shift(Vn1[1], c);
  }
#pragma unroll
  for (int d = 0; d < 3; d++)
    if (!isfinite(vn[d].hi)) bad |= kErrNonfinite;
}

__device__ __forceinline__ void store_marker(const Em2dMixBufs &b, int64_t q, uint32_t Xn,
                                             uint32_t Yn, const ff vn[3]) {
  b.X[q] = Xn;
  b.Y[q] = Yn;
#pragma unroll
  for (int d = 0; d < 3; d++) {
    b.vh[d][q] = vn[d].hi;
    b.vl[d][q] = vn[d].lo;
  }
}

// Pass E: gather at x^{n+1/2} = X + [V*], v^dag, Gamma, x^{n+1}, v^{n+1}, the
// kinetic energy and (ESEC2) the next step's j^{n+1,*}.  On sorted markers
// with so.off set (the step that ends a sort period) each marker goes to the
// next free slot of its quarter cell in so.dst (its id with it), else back to
// its own slot.
//
// The last nk5 blocks run K5 on the FP64 fields (fc, fb) instead: it reads
// E^{n+1} and B^{n+1/2} and writes B^{n+3/2} and the field energies, nothing
// the markers touch.
template <int ORDER, bool SORTED>
__global__ void __launch_bounds__(256, SORTED ? 2 : 0)
    mix2_pass_e_kernel(Em2dMixConst c, Em2dMixBufs b, int slot, Em2dSortIO so, Em2dConst fc,
                       Em2dBufs fb, int nk5) {
  __shared__ double red[33];
  griddep_wait();
  griddep_launch_dependents();
  const int npass = (int)gridDim.x - nk5;
  if ((int)blockIdx.x >= npass) {
    k5_block(fc, fb, (int)blockIdx.x - npass, nk5, red);
    return;
  }
  const unsigned lane = threadIdx.x & 31u;
  float ke_hi = 0.0f, ke_lo = 0.0f;
  unsigned nfb = 0, bad = 0;
  if constexpr (SORTED) {
    constexpr int M = kRunMarkers;
    for (int64_t pw = (blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31u)) * M; pw < c.n;
         pw += (int64_t)npass * blockDim.x * M) {
      DepositRun<ORDER> run(lane);
#pragma unroll 1
      for (int j = 0; j < M; j++) {
        const int64_t p = pw + (int64_t)lane * M + j;
        const bool valid = p < c.n;
        int key = -1 - (int)lane;
        uint32_t Xn = 0u, Yn = 0u;
        ff vn[3];
        int Vn1[3];
        uint32_t Xd = 0u, Yd = 0u;
        if (valid) {
          pass_e_marker<ORDER>(c, b, p, bad, nfb, ke_hi, ke_lo, Vn1, Xd, Yd, Xn, Yn, vn);
          if (so.off)
            key = quarter_key(Xn, Yn, c.nx, c.ny);
          else
            store_marker(b, p, Xn, Yn, vn);
        }
        if (so.off) {
          const unsigned q = PIC_INDEX(warp_slot(so.off, key), c.n);
          if (valid) {
            store_marker(so.dst, q, Xn, Yn, vn);
            if (so.ids_in) so.ids_out[q] = so.ids_in[p];
          }
        }
        if (valid && c.scheme == 2)
          run.add(c, b.J1, Xd, Yd, Shape2Mix<ORDER>(Xd, Yd, c.nx, c.ny), Vn1);
      }
      if (c.scheme == 2) run.flush_warp(c, b.J1);
    }
  } else {
    for (int64_t pw = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31u); pw < c.n;
         pw += (int64_t)npass * blockDim.x) {
      const int64_t p = pw + lane;
      if (p >= c.n) break;
      int Vn1[3];
      uint32_t Xd, Yd, Xn, Yn;
      ff vn[3];
      pass_e_marker<ORDER>(c, b, p, bad, nfb, ke_hi, ke_lo, Vn1, Xd, Yd, Xn, Yn, vn);
      store_marker(b, p, Xn, Yn, vn);
      if (c.scheme == 2) deposit_j<ORDER>(c, b.J1, Shape2Mix<ORDER>(Xd, Yd, c.nx, c.ny), Vn1);
    }
  }
  for (int o = 16; o > 0; o >>= 1) nfb += __shfl_xor_sync(0xffffffffu, nfb, o);
  if ((threadIdx.x & 31) == 0 && nfb) atomicAdd(&b.fallback[slot], (unsigned long long)nfb);
  report_bad(bad, b.err);
  const double t = block_sum2((double)ke_hi + (double)ke_lo, red);
  if (threadIdx.x == 0) b.ke_part[blockIdx.x] = c.ke_scale * t;
}

// j^{n,*} of the current state (start-up and after a state change), the same
// deposit pass E makes for the next step
template <int ORDER>
__global__ void __launch_bounds__(256) mix2_deposit_initial_kernel(Em2dMixConst c,
                                                                   Em2dMixBufs b) {
  unsigned bad = 0;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < c.n;
       p += (int64_t)gridDim.x * blockDim.x) {
    int V[3];
#pragma unroll
    for (int d = 0; d < 3; d++) V[d] = to_fixed(b.vh[d][p], bad);
    const Shape2Mix<ORDER> S(b.X[p] + half_shift(V[0], c), b.Y[p] + half_shift(V[1], c), c.nx,
                             c.ny);
    deposit_j<ORDER>(c, b.J1, S, V);
  }
  report_bad(bad, b.err);
}

__global__ void mix2_from_fp64_kernel(Em2dMixConst c, Em2dMixBufs mb, Em2dBufs b) {
  const double *v[3] = {b.vx, b.vy, b.vz};
  const double scale = 4294967296.0 / c.L;   // one multiply per coordinate, no divide
  unsigned bad = 0;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < c.n;
       p += (int64_t)gridDim.x * blockDim.x) {
    mb.X[p] = (uint32_t)((unsigned long long)llrint(b.x[p] * scale) & 0xFFFFFFFFull);
    mb.Y[p] = (uint32_t)((unsigned long long)llrint(b.y[p] * scale) & 0xFFFFFFFFull);
#pragma unroll
    for (int d = 0; d < 3; d++) {
      const double vv = v[d][p] * c.cxk;
      if (!isfinite(vv)) bad |= kErrNonfinite;
      if (!(fabs(vv) < 2147483520.0)) bad |= kErrVelocityRange;
      const float h = (float)vv;
      mb.vh[d][p] = h;
      mb.vl[d][p] = (float)(vv - (double)h);
    }
  }
  report_bad(bad, b.err);
}

__global__ void mix2_to_fp64_kernel(Em2dMixConst c, Em2dMixBufs mb, Em2dBufs b) {
  double *v[3] = {b.vx, b.vy, b.vz};
  const double inv = 1.0 / c.cxk;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < c.n;
       p += (int64_t)gridDim.x * blockDim.x) {
    b.x[p] = (double)mb.X[p] * (c.L / 4294967296.0);
    b.y[p] = (double)mb.Y[p] * (c.L / 4294967296.0);
#pragma unroll
    for (int d = 0; d < 3; d++) v[d][p] = ((double)mb.vh[d][p] + (double)mb.vl[d][p]) * inv;
  }
}

__global__ void __launch_bounds__(256) mix2_kinetic_kernel(Em2dMixConst c, Em2dMixBufs mb,
                                                           double *out) {
  __shared__ double red[33];
  double acc = 0.0;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < c.n;
       p += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int d = 0; d < 3; d++) {
      const double v = (double)mb.vh[d][p] + (double)mb.vl[d][p];
      acc += v * v;
    }
  }
  const double t = block_sum2(acc, red);
  if (threadIdx.x == 0) out[blockIdx.x] = c.ke_scale * t;
}

// max |v| over the three staging components (non-negative doubles order like
// their bit patterns)
__global__ void mix2_absmax_kernel(Em2dBufs b, int64_t n, unsigned long long *out) {
  double m = 0.0;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x)
    m = fmax(m, fmax(fabs(b.vx[p]), fmax(fabs(b.vy[p]), fabs(b.vz[p]))));
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

// ------------------------------------------------------------ quarter-cell sort
// The markers in the order of their quarter cell (quarter_key), written so by
// pass E of the step that ends a sort period: pass C counts the quarter cells
// of x^{n+1} (known once V* is), the scan below turns the counts into
// offsets, and pass E puts each marker (and its id) at the next free slot of
// its quarter cell.  The order within a quarter cell is not fixed, which
// changes no result (the currents are exact integer sums).
//
// Exclusive scan of cnt[0 .. nk) into off[] (nk a multiple of 4) in tiles of
// 4096 keys, a block of 1024 threads per tile, 4 keys a thread: the tiles'
// totals first, then each tile's scan from the sum of the totals before it.
// The second kernel leaves the counts zero for the next sort.
constexpr int kScanThreads = 1024, kScanTile = 4 * kScanThreads;

__device__ __forceinline__ unsigned block_sum_u(unsigned v, unsigned *red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31u) == 0u) red[threadIdx.x >> 5] = v;
  __syncthreads();
  unsigned t = 0;
  for (int w = 0; w < kScanThreads / 32; w++) t += red[w];
  return t;
}

__global__ void __launch_bounds__(kScanThreads) mix2_sort_tilesum_kernel(const unsigned *cnt,
                                                                        int nk, unsigned *tsum) {
  __shared__ unsigned red[kScanThreads / 32];
  griddep_wait();
  griddep_launch_dependents();
  const int i = blockIdx.x * kScanTile + 4 * (int)threadIdx.x;
  unsigned v = 0;
  if (i < nk) {
    const uint4 q = *(const uint4 *)(cnt + i);
    v = q.x + q.y + q.z + q.w;
  }
  v = block_sum_u(v, red);
  if (threadIdx.x == 0) tsum[blockIdx.x] = v;
}

__global__ void __launch_bounds__(kScanThreads) mix2_sort_offsets_kernel(unsigned *cnt, int nk,
                                                                        const unsigned *tsum,
                                                                        unsigned *off) {
  __shared__ unsigned red[kScanThreads / 32];
  __shared__ unsigned wsum[kScanThreads / 32];
  griddep_wait();
  griddep_launch_dependents();
  unsigned before = 0;
  for (int t = threadIdx.x; t < (int)blockIdx.x; t += kScanThreads) before += tsum[t];
  before = block_sum_u(before, red);
  const int i = blockIdx.x * kScanTile + 4 * (int)threadIdx.x;
  uint4 q = make_uint4(0u, 0u, 0u, 0u);
  if (i < nk) {
    q = *(const uint4 *)(cnt + i);
    *(uint4 *)(cnt + i) = make_uint4(0u, 0u, 0u, 0u);
  }
  const unsigned mine = q.x + q.y + q.z + q.w;
  // inclusive scan of the threads' totals: over the warp, then over the warps
  const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  unsigned inc = mine;
  for (int d = 1; d < 32; d <<= 1) {
    const unsigned t = __shfl_up_sync(0xffffffffu, inc, d);
    if ((int)lane >= d) inc += t;
  }
  if (lane == 31u) wsum[warp] = inc;
  __syncthreads();
  unsigned wbefore = 0;
  for (unsigned w = 0; w < warp; w++) wbefore += wsum[w];
  if (i < nk) {
    const unsigned o = before + wbefore + inc - mine;
    *(uint4 *)(off + i) = make_uint4(o, o + q.x, o + q.x + q.y, o + q.x + q.y + q.z);
  }
}

}  // namespace

PIC_BOUNDS_READER(bounds_site_em2d_mixed)

LaunchShape em2dm_pass_shape(int64_t n, bool sorted, LaunchShape lp) {
  if (!sorted) return lp;
  const int64_t per_block = 256 * (int64_t)kRunMarkers;
  return {(int)std::max<int64_t>(1, (n + per_block - 1) / per_block), 256};
}

size_t em2dm_sort_count_words(int nx, int ny) {
  const size_t nk = 4 * (size_t)nx * ny;
  return nk + (nk + kScanTile - 1) / kScanTile;
}

void em2dm_sort_scan(const Em2dMixConst &m, unsigned *cnt, unsigned *off, cudaStream_t st) {
  const int nk = 4 * m.nx * m.ny, tiles = (nk + kScanTile - 1) / kScanTile;
  unsigned *tsum = cnt + nk;  // [tiles] after the counts
  launch_dependent(mix2_sort_tilesum_kernel, LaunchShape{tiles, kScanThreads}, 0, st, true, cnt,
                   nk, tsum);
  launch_dependent(mix2_sort_offsets_kernel, LaunchShape{tiles, kScanThreads}, 0, st, true, cnt,
                   nk, (const unsigned *)tsum, off);
}

void em2dm_k1(const Em2dConst &c, const Em2dMixConst &m, const Em2dMixBufs &mb,
              const Em2dBufs &b, int fin_slot, LaunchShape lp, LaunchShape lg, cudaStream_t st) {
  const LaunchShape ls{lg.grid + (fin_slot >= 0 ? 1 : 0), lg.block};
  launch_dependent(mix2_k1_kernel, ls, 0, st, true, c, m, mb, b, fin_slot, lp.grid, lg.grid);
}

void em2dm_k3(const Em2dConst &c, const Em2dMixConst &m, const Em2dMixBufs &mb,
              const Em2dBufs &b, LaunchShape lg, cudaStream_t st) {
  launch_dependent(mix2_k3_kernel, lg, 0, st, true, c, m, mb, b);
}

void em2dm_pass_c(const Em2dMixConst &m, const Em2dMixBufs &mb, unsigned *cnt, LaunchShape lp,
                  cudaStream_t st) {
  auto k = m.order == 1 ? (m.sorted ? mix2_pass_c_kernel<1, true> : mix2_pass_c_kernel<1, false>)
                        : (m.sorted ? mix2_pass_c_kernel<2, true> : mix2_pass_c_kernel<2, false>);
  launch_dependent(k, LaunchShape{lp.grid, 256}, 0, st, true, m, mb, cnt);
}

void em2dm_pass_e(const Em2dMixConst &m, const Em2dMixBufs &mb, int slot, const Em2dSortIO &so,
                  const Em2dConst &c, const Em2dBufs &b, LaunchShape lp, LaunchShape lg,
                  cudaStream_t st) {
  auto k = m.order == 1 ? (m.sorted ? mix2_pass_e_kernel<1, true> : mix2_pass_e_kernel<1, false>)
                        : (m.sorted ? mix2_pass_e_kernel<2, true> : mix2_pass_e_kernel<2, false>);
  launch_dependent(k, LaunchShape{lp.grid + lg.grid, 256}, 0, st, true, m, mb, slot, so, c, b,
                   lg.grid);
}

void em2dm_from_fp64(const Em2dMixConst &m, const Em2dMixBufs &mb, const Em2dBufs &b,
                     LaunchShape lp, cudaStream_t st) {
  mix2_from_fp64_kernel<<<lp.grid, 256, 0, st>>>(m, mb, b);
}

void em2dm_to_fp64(const Em2dMixConst &m, const Em2dMixBufs &mb, const Em2dBufs &b,
                   LaunchShape lp, cudaStream_t st) {
  mix2_to_fp64_kernel<<<lp.grid, 256, 0, st>>>(m, mb, b);
}

void em2dm_deposit_initial(const Em2dMixConst &m, const Em2dMixBufs &mb, LaunchShape lp,
                           cudaStream_t st) {
  if (m.order == 1)
    mix2_deposit_initial_kernel<1><<<lp.grid, 256, 0, st>>>(m, mb);
  else
    mix2_deposit_initial_kernel<2><<<lp.grid, 256, 0, st>>>(m, mb);
}

void em2dm_kinetic(const Em2dMixConst &m, const Em2dMixBufs &mb, double *out, LaunchShape lp,
                   cudaStream_t st) {
  mix2_kinetic_kernel<<<lp.grid, 256, 0, st>>>(m, mb, out);
}

void em2dm_absmax(const Em2dBufs &b, int64_t n, unsigned long long *out, LaunchShape lp,
                  cudaStream_t st) {
  mix2_absmax_kernel<<<lp.grid, 256, 0, st>>>(b, n, out);
}

}  // namespace pic
