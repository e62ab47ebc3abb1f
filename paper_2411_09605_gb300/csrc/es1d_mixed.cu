// 1D1V electrostatic ESEC1 / ESEC2 step, mixed-precision form.
//
// On GB300 the FP64 pipe issues 1/64 of the FP32 rate (and converts between
// float and double at that rate too), so this form keeps FP64 out of the
// per-marker work and still conserves energy to the FP64 bound:
//   * position: one uint32 word X, x = X L / 2^32.  Cell index and in-cell
//     fraction come from the 64-bit product X nc; the periodic wrap is the
//     integer overflow of X.
//   * velocity: an unevaluated float pair (vh, vl) stored in "V units", v times
//     cxk = (dt 2^31 / L) 2^kv: one V unit moves a marker 2^-kv position units
//     in half a step.  kv >= 1 is fixed at set-up from the initial velocity range.
//   * v* (Eq. good_translation) is the integer V* = rint(v*), so x* , x^{n+1/2}
//     = X + [V*]_kv and x^{n+1} = X + 2 [V*]_kv are exact integer additions and
//     x^{n+1/2} is exactly the midpoint.
//   * shape weights are exact integers in units of 2^-23 computed from the
//     fraction (partition of unity is exact); gather and deposit at x^{n+1/2}
//     use the same integers, as Eq. exp_econs_simple requires.
//   * current: each marker adds round(V* s_k / 2^r) to node k as an exact
//     integer (order independent, r chosen so no sum overflows; the rounding
//     is independent per marker and far below the FP64 energy bound), through
//     a shared-memory tile of split 32-bit counters; one global 64-bit atomic
//     per node per block at the end.  Unsorted markers on grids of up to 512
//     nodes use one tile copy per lane (no bank conflicts); cell-sorted markers
//     are first summed over the warp in a window of nodes.
//   * the shared field tables and tiles carry ghost nodes, so the nodes of a
//     shape never wrap.
//   * gather #2 reads dt (q/m) cxk E^{n+1/2} as a float pair with error-free
//     weight products, and v^dag = v^n + d in float pairs.
//   * Gamma (Eq. opt_solution) from the exact difference
//     |v^{n+1}|^2 - |v^dag|^2 = 2a, a = d (v* - v^n - d/2) (float pairs for
//     the cancelling subtraction, FP32 for the small product):
//     g = Gamma - 1, t = 2a/|v^dag|^2: for |t| < 2^-8 an FP32 series of
//     sqrt(1 + t) - 1 and v^{n+1} = v^dag + g v^dag in float pairs; every
//     other marker takes FP64, R = |v^dag|^2 + 2a and v^{n+1} = sqrt(R) with
//     the sign of v^dag.  R < 0 is 1 + t < 0.
//   * energies: per-thread float-pair sums of v^2, block sums in FP64.
// Gather #1 and deposit #1 only shape v* (not the conservation), so they use
// plain FP32 weights and the same integer deposit.
// Optionally the markers are kept cell-sorted: by a counting sort every
// sort_period steps, or written in (cell, sign of v) order by every pass E.
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "ff.cuh"
#include "mixed_common.cuh"
#include "pdl.cuh"
#include "pic_internal.cuh"

namespace pic {
namespace {

// b.A[i] for a two-entry pointer array in a kernel parameter, selected
// without indexing (indexing would copy the parameter block to local memory)
#define PSEL(A, i) ((i) ? (A)[1] : (A)[0])

__device__ __forceinline__ int cell_of(uint32_t X, int nc) {
  return (int)(((uint64_t)X * (uint32_t)nc) >> 32);
}




__device__ __forceinline__ SplitTerm deposit_split(int V, int s, const Es1dMixConst &c) {
  return split_term(V, s, c.rshift, c.rnd, c.lomask, c.hishift);
}

__device__ __forceinline__ long long deposit_term(int V, int s, const Es1dMixConst &c) {
  return ((long long)V * (long long)s + c.rnd) >> c.rshift;
}


// V units -> position units for half a step (kv >= 1)
__device__ __forceinline__ uint32_t half_shift(int V, const Es1dMixConst &c) {
  return (uint32_t)((V + c.hround) >> c.kv);
}

// Shared-memory current tile.  Every padded node holds two 32-bit counters per
// copy: the low b = c.split bits of each added amount (unsigned) and the
// signed rest; an amount A is added exactly as (A mod 2^b, A >> b) and the
// node's value is rest 2^b + low.  Two 32-bit shared atomics run faster than
// one 64-bit one.  With at most 2^(32-b) amounts per copy in a launch the low
// counter cannot overflow, and the rounding shift r is chosen so that the
// signed rest cannot either.  The tile is laid out [node][half][copy] with RT
// copies; lane l of every warp adds into copy l mod RT (Jl = tile + l mod RT).
// With RT = 32 the lanes of a warp always address 32 different banks, so the
// random-address atomics of unsorted markers never conflict.
template <int RT>
__device__ __forceinline__ void tile_add(unsigned *Jl, int q, long long a, int b) {
  atomicAdd(&Jl[q * 2 * RT], (unsigned)a & ((1u << b) - 1u));
  atomicAdd(&Jl[q * 2 * RT + RT], (unsigned)(int)(a >> b));
}

template <int ORDER, int RT>
__device__ __forceinline__ void deposit_direct(unsigned *Jl, const ShapeMix<ORDER> &S, int V,
                                               const Es1dMixConst &c) {
#pragma unroll
  for (int k = 0; k <= ORDER; k++) {
    const SplitTerm t = deposit_split(V, S.s[k], c);
    atomicAdd(&Jl[(S.p + k) * 2 * RT], t.lo);
    atomicAdd(&Jl[(S.p + k) * 2 * RT + RT], (unsigned)t.hi);
  }
}

// Deposit window for cell-sorted markers (single-copy tile): a thread adds the
// terms of its four markers into kWin consecutive padded nodes starting one
// below the warp's smallest first node, then the warp sums each node over its
// 32 lanes (two 32-bit halves: 4 terms of |t| < 2^37 per lane, so the low 20
// bits and the signed rest sum without overflow) and one lane adds the 128
// markers' total with one split atomic per node.  Markers whose nodes fall
// outside the window use direct atomics.
constexpr int kWin = 6;

template <int ORDER>
struct DepositWindow {
  long long acc[kWin];
  int base;
  __device__ __forceinline__ void start(int p, bool valid, int npad) {
#pragma unroll
    for (int w = 0; w < kWin; w++) acc[w] = 0;
    const int m = __reduce_min_sync(0xffffffffu, valid ? p : 0x7fffffff);
    base = m == 0x7fffffff ? 0 : m - 1;
    base = base < 0 ? 0 : (base > npad - kWin ? npad - kWin : base);
  }
  __device__ __forceinline__ void add(unsigned *Jt, const ShapeMix<ORDER> &S, int V,
                                      const Es1dMixConst &c, bool valid) {
    if (!valid) return;
    const int off = S.p - base;
    const bool inwin = off >= 0 && off <= kWin - 1 - ORDER;
    long long t[ORDER + 1];
#pragma unroll
    for (int k = 0; k <= ORDER; k++) t[k] = deposit_term(V, S.s[k], c);
    if (inwin) {
#pragma unroll
      for (int w = 0; w < kWin; w++) {
        long long a = 0;
#pragma unroll
        for (int k = 0; k <= ORDER; k++) a = (w - k == off) ? t[k] : a;
        acc[w] += a;
      }
    } else {
#pragma unroll
      for (int k = 0; k <= ORDER; k++) tile_add<1>(Jt, S.p + k, t[k], c.split);
    }
  }
  __device__ __forceinline__ void flush(unsigned *Jt, int b) {
    const bool lead = (threadIdx.x & 31u) == 0u;
#pragma unroll
    for (int w = 0; w < kWin; w++) {
      if (__any_sync(0xffffffffu, acc[w] != 0)) {
        const int hs = __reduce_add_sync(0xffffffffu, (int)(acc[w] >> 20));
        const int ls = __reduce_add_sync(0xffffffffu, (int)(acc[w] & 0xFFFFF));
        if (lead) tile_add<1>(Jt, base + w, ((long long)hs << 20) + (long long)ls, b);
      }
    }
  }
};

__device__ void block_exclusive_scan(const uint32_t *T, uint32_t *base, int nc, uint32_t *tmp);

// Sort key of a marker after the step: its cell and the sign of its velocity
// (counter-streaming markers of one cell then sit in separate runs).
__device__ __forceinline__ int sort_key(uint32_t X, int V, int nc) {
  return PIC_INDEX(2 * cell_of(X, nc) + (V > 0 ? 1 : 0), 2 * nc);
}

// Warp-aggregated increment of a shared counter array: returns this lane's
// slot (the counter's old value plus the lane's rank among the warp's lanes
// with the same key).  Cell-sorted markers give one or a few distinct keys
// per warp; each distinct key costs one ballot, two shuffles and one atomic.
__device__ __forceinline__ uint32_t warp_rank(uint32_t *cnt, int key, bool valid) {
  const unsigned lane = threadIdx.x & 31u;
  const unsigned lt = (1u << lane) - 1u;
  unsigned todo = __ballot_sync(0xffffffffu, valid);
  uint32_t mine = 0;
  while (todo) {
    const int leader = __ffs(todo) - 1;
    const int kk = __shfl_sync(0xffffffffu, key, leader);
    const unsigned grp = __ballot_sync(0xffffffffu, ((todo >> lane) & 1u) && key == kk);
    uint32_t first = 0;
    if ((int)lane == leader) first = atomicAdd(&cnt[kk], (uint32_t)__popc(grp));
    first = __shfl_sync(0xffffffffu, first, leader);
    if ((grp >> lane) & 1u) mine = first + (uint32_t)__popc(grp & lt);
    todo &= ~grp;
  }
  return mine;
}

__device__ __forceinline__ double block_sum_d(double s, double *red) {
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[warp] = s;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int k = 0; k < (int)(blockDim.x >> 5); k++) t += red[k];
  return t;  // thread 0
}

// An int64 as a float pair (about 48 bits): the rounded value and the exact
// integer remainder.
__device__ __forceinline__ ff ff_from_i64(long long J) {
  const float hi = __ll2float_rn(J);
  const long long rem = J - __float2ll_rz(hi);  // hi holds an integer value
  return {hi, __ll2float_rn(rem)};
}

// Grid mean <J> of integer node sums from their exact total (read by every
// thread; no block reduction): in J units as a float pair.
__device__ __forceinline__ ff mean_of_total(long long total, const Es1dMixConst &c) {
  return ff_mul(ff_from_i64(total), c.inv_nc);
}

// Stores one table value into RE consecutive copies (RE = 16: 16-byte stores).
template <int RE, typename T>
__device__ __forceinline__ void store_copies(T *row, T v) {
  if (RE == 1) {
    row[0] = v;
  } else {
    static_assert(16 % sizeof(T) == 0, "copies are written 16 bytes at a time");
    constexpr int kPer = 16 / sizeof(T);
    union {
      T t[kPer];
      uint4 u;
    } pk;
#pragma unroll
    for (int k = 0; k < kPer; k++) pk.t[k] = v;
    uint4 *r4 = reinterpret_cast<uint4 *>(row);
#pragma unroll
    for (int k = 0; k < RE / kPer; k++) r4[k] = pk.u;
  }
}

// The RE copies of the 32 nodes q of a warp's lanes (lane l holds the value v
// of node q = q0 + l; called by all 32 lanes, node q written when q < npad),
// the warp together: its CPN = 16 RE / sizeof(T) stores of 16 bytes per lane
// cover consecutive 512-byte spans of the table, so no two lanes of a quarter
// warp address the same banks.  (Each lane writing its own node's copies puts
// the lanes 16 RE bytes apart, all on the same four banks.)
template <int RE, typename T>
__device__ __forceinline__ void store_copies_warp(T *table, int q, T v, int npad) {
  constexpr int kPer = 16 / sizeof(T);
  if constexpr (RE < kPer || RE % kPer != 0) {
    if (q < npad) store_copies<RE>(table + q * RE, v);
  } else {
    constexpr int CPN = RE / kPer;  // 16-byte chunks per node
    const int lane = (int)(threadIdx.x & 31u), q0 = q - lane;
    uint4 *base = reinterpret_cast<uint4 *>(table + q0 * RE);
#pragma unroll
    for (int s = 0; s < CPN; s++) {
      const int src = (32 * s + lane) / CPN;  // the lane whose node this chunk is
      union {
        T t[kPer];
        uint4 u;
      } pk;
      T w;
      static_assert(sizeof(T) == 4 || sizeof(T) == 8, "4- or 8-byte table entries");
      if constexpr (sizeof(T) == 4) {
        w = __int_as_float(__shfl_sync(0xffffffffu, __float_as_int(v), src));
      } else {
        w = make_float2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
      }
#pragma unroll
      for (int k = 0; k < kPer; k++) pk.t[k] = w;
      if (q0 + src < npad) base[32 * s + lane] = pk.u;
    }
  }
}

// The binomial filter F (the periodic 1-2-1 stencil, p passes) inside the
// scheme, put in energy-consistently: both Ampere updates use F j and both
// gathers read F E* and F E^{n+1/2}; F is symmetric and keeps the mean, so
// sum E (F j) = sum (F E) j.  A table entry is a stencil over the unfiltered
// grid: F E* = F E^n - dt/2 (F^2 j1 - <j1>), with F^p's weights C(2p, p + k) /
// 4^p and F^2p's (b.filt).  Node i + k of the periodic grid, any k:
__device__ __forceinline__ int node_at(int i, int k, int nc) {
  const int j = (i + k) % nc;
  return j < 0 ? j + nc : j;
}

// The filtered tables are built out of line (noinline), so that the kernels
// without the filter keep their code.  e_scale F E* on the padded nodes in
// FP32 (gather #1 only shapes v*), RE copies each:
template <int SCHEME, int RE, int PAD>
__device__ __noinline__ void estar_table_filtered(int nc, int p, float c_jstar, const float2 *filt,
                                                  const float2 *Ek, const long long *J1,
                                                  float mean, float *Es, int npad) {
  const float2 *f2 = filt + 2 * p + 1;
  // whole warps in every trip (the copies are written by the warp together)
  for (int q = threadIdx.x; q - (int)(threadIdx.x & 31u) < npad; q += blockDim.x) {
    float e = 0.0f;
    if (q < npad) {
      const int i = wrap_node(q - PAD, nc);
      for (int k = -p; k <= p; k++) {
        const float2 ek = Ek[node_at(i, k, nc)];
        e = __fmaf_rn(filt[k + p].x, __fmul_rn(0.5f, __fadd_rn(ek.x, ek.y)), e);
      }
      if (SCHEME == 2) {
        float j = 0.0f;
        for (int k = -2 * p; k <= 2 * p; k++)
          j = __fmaf_rn(f2[k + 2 * p].x, __ll2float_rn(J1[node_at(i, k, nc) * kJStride]), j);
        e = __fmaf_rn(-c_jstar, __fsub_rn(j, mean), e);
      }
    }
    store_copies_warp<RE>(Es, q, e, npad);
  }
}

// kick F E^{n+1/2} = kick F E^n - kick dt/2 jscale (F^2 j2 - <j2>) on the
// padded nodes in float pairs, RE copies each
template <int RE, int PAD>
__device__ __noinline__ void ehalf_table_filtered(int nc, int p, ff kick_jhalf, const float2 *filt,
                                                  const float2 *Ek, const long long *J2, ff mean,
                                                  float2 *Eh2, int npad) {
  const float2 *f2 = filt + 2 * p + 1;
  // whole warps in every trip (the copies are written by the warp together)
  for (int q = threadIdx.x; q - (int)(threadIdx.x & 31u) < npad; q += blockDim.x) {
    float2 v = make_float2(0.0f, 0.0f);
    if (q < npad) {
      const int i = wrap_node(q - PAD, nc);
      ff e{0.0f, 0.0f}, j{0.0f, 0.0f};
      for (int k = -p; k <= p; k++) {
        const float2 ek = Ek[node_at(i, k, nc)], f = filt[k + p];
        e = ff_add(e, ff_mul(ff{f.x, f.y}, ff{ek.x, ek.y}));
      }
      for (int k = -2 * p; k <= 2 * p; k++) {
        const float2 f = f2[k + 2 * p];
        j = ff_add(j, ff_mul(ff{f.x, f.y}, ff_from_i64(J2[node_at(i, k, nc) * kJStride])));
      }
      const ff eh = ff_sub(e, ff_mul(kick_jhalf, ff_sub(j, mean)));
      v = make_float2(eh.hi, eh.lo);
    }
    store_copies_warp<RE>(Eh2, q, v, npad);
  }
}

// (F^p j2)_i in FP64, as the state's Ampere update uses it
__device__ __noinline__ double filtered_j(int nc, int p, const float2 *filt, const long long *J2,
                                          int i) {
  double j = 0.0;
  for (int k = -p; k <= p; k++) {
    const float2 f = filt[k + p];
    j = fma((double)f.x + (double)f.y, (double)J2[node_at(i, k, nc) * kJStride], j);
  }
  return j;
}

// Zeroes 2 RT npad counters (RT > 1: the count is a multiple of 4, 16-byte aligned).
template <int RT>
__device__ __forceinline__ void clear_tile(unsigned *Jt, int npad) {
  if (RT > 1) {
    uint4 *t4 = reinterpret_cast<uint4 *>(Jt);
    for (int i = threadIdx.x; i < npad * RT / 2; i += blockDim.x) t4[i] = make_uint4(0, 0, 0, 0);
  } else {
    for (int i = threadIdx.x; i < 2 * npad; i += blockDim.x) Jt[i] = 0;
  }
}

// Sums the tile's copies node by node (one thread per padded node), adds each
// node's total to J[node kJStride] with one 64-bit global atomic (ghost nodes
// add to the node they stand for) and the block's total to *total (exact
// integers, so the grid total does not depend on the order of the blocks).
template <int ORDER, int RT>
__device__ __forceinline__ void flush_tile(const unsigned *Jt, long long *J, long long *total,
                                           int nc, int b) {
  __shared__ long long tred[32];
  const int npad = npad_of(nc);
  long long mine = 0;
  for (int q = threadIdx.x; q < npad; q += blockDim.x) {
    long long lo = 0, hi = 0;
    // copies read in an order skewed by the node: the 32 lanes of a warp
    // (consecutive nodes) then read 32 different banks
#pragma unroll
    for (int k = 0; k < RT; k++) {
      const int kk = (k + q) & (RT - 1);
      lo += Jt[q * 2 * RT + kk];
      hi += (int)Jt[q * 2 * RT + RT + kk];
    }
    const long long a = hi * (1ll << b) + lo;
    mine += a;
    if (a != 0)
      atomicAdd((unsigned long long *)&J[PIC_INDEX(wrap_node(q - Pad<ORDER>::kPad, nc), nc) *
                                         kJStride],
                (unsigned long long)a);
  }
  for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
  if ((threadIdx.x & 31u) == 0u) tred[threadIdx.x >> 5] = mine;
  __syncthreads();
  if (threadIdx.x < 32) {
    long long t = threadIdx.x < (blockDim.x >> 5) ? tred[threadIdx.x] : 0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0 && t != 0) atomicAdd((unsigned long long *)total, (unsigned long long)t);
  }
}

// TE of a finished step from the blocks' partials of the kinetic energy and
// of sum E^2 (pass E), by one warp: lane l sums the partials l, l + 32, ...,
// then the lanes are summed by a butterfly.  Lane 0 stores TE.  The passes run
// it in one warp before that warp's markers, off the path between launches.
__device__ __forceinline__ void finalize_stats_warp(const Es1dMixBufs &b, double h, int slot,
                                                    int nblocks) {
  const int lane = threadIdx.x & 31;
  double s = 0.0;
#pragma unroll 4
  for (int i = lane; i < nblocks; i += 32) s += b.ke_part[i] + 0.5 * h * b.we_part[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) {
    b.te[slot] = s;
    if (!isfinite(s)) atomicOr(b.err, kErrNonfinite);
  }
}

__device__ __forceinline__ bool last_warp() {
  return (threadIdx.x >> 5) == (blockDim.x >> 5) - 1;
}

// The passes are launched as programmatic dependent launches (pdl.cuh): each
// one sets up its shared memory before griddep_wait().

// Ors the flags of a warp's lanes into the error word (one atomic per warp).
__device__ __forceinline__ void report_flags(unsigned bad, unsigned *err) {
  bad = __reduce_or_sync(0xffffffffu, bad);
  if ((threadIdx.x & 31u) == 0u && bad) atomicOr(err, bad);
}



// The correction of Eq. opt_solution in FP64 from the float-pair state: R =
// |v^dag|^2 + 2a (a from bracket_fp64), the R < 0 test, and in 1D v^{n+1} =
// Gamma v^dag = sqrt(R) with the sign of v^dag (one root, no quotient; v^dag
// is exact in FP64, so R carries FP64's precision), rounded to a float pair;
// a fallback (R < 0 or v^dag = 0) keeps v^dag and is counted (Sec. 3.2,
// Sec. 5.1).
__device__ __forceinline__ ff correct_velocity_fp64(float vh, float vl, int Vs, ff d, ff vd,
                                                 unsigned &nfb) {
  const double vdd = ff_to_double(vd);
  const double R = fma(vdd, vdd, 2.0 * (ff_to_double(d) * bracket_fp64(vh, vl, Vs, d)));
  if (!(R >= 0.0) || vdd == 0.0) {
    nfb++;
    return vd;
  }
  return ff_from_double(copysign(sqrt(R), vdd));
}

// v^dag = v^n + d and v^{n+1} = Gamma v^dag (Eq. opt_solution) in float pairs.
// t = 2a / |v^dag|^2 (see correct_velocity_fp64) is first formed in FP32 from
// the same exact pieces: V* - v^n = (V* - ih) - fr - vl with V* - ih a small
// exact integer, its sum with -d/2 split exactly by a two-sum and only the
// small terms rounded.  For |t| < 2^-8 (|Gamma - 1| < 2^-9: every marker whose
// speed is not small against its kick) Gamma - 1 is the series t/2 - t^2/8 +
// t^3/16 - 5t^4/128 in FP32 (relative error below 2^-22, so Gamma is within
// 2^-31 of its value); every other marker, among them every candidate for
// the fallback, takes correct_velocity_fp64, which decides R < 0 and forms
// Gamma in FP64.  With G64 every marker takes correct_velocity_fp64.
template <bool G64>
__device__ __forceinline__ ff correct_velocity(float vh, float vl, int Vs, ff d, bool on,
                                               unsigned &nfb) {
  const ff vd = ff_add(ff{vh, vl}, d);
  if (!on) return vd;
  if (G64) return correct_velocity_fp64(vh, vl, Vs, d, vd, nfb);
  const int ih = __float2int_rn(vh);
  const float fr = __fsub_rn(vh, __int2float_rn(ih));
  const ff q = two_sum(__int2float_rn(Vs - ih), __fmul_rn(-0.5f, d.hi));
  const float small = __fsub_rn(__fsub_rn(__fsub_rn(q.lo, fr), vl), __fmul_rn(0.5f, d.lo));
  const float bq = __fadd_rn(q.hi, small);
  const float t = div_rcp_residual(__fmul_rn(__fadd_rn(d.hi, d.hi), bq), __fmul_rn(vd.hi, vd.hi));
  if (fabsf(t) < 0.00390625f) {
    const float gm = __fmul_rn(
        t, __fmaf_rn(t, __fmaf_rn(t, __fmaf_rn(t, -0.0390625f, 0.0625f), -0.125f), 0.5f));
    // |gm| < 2^-8, so gm v^dag is far below v^dag
    ff p = two_prod(vd.hi, gm);
    p.lo = __fmaf_rn(vd.lo, gm, p.lo);
    const ff s = fast_two_sum(vd.hi, p.hi);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(vd.lo, p.lo)));
  }
  return correct_velocity_fp64(vh, vl, Vs, d, vd, nfb);
}

// dt (q/m) cxk E^{n+1/2}_p of two markers (lane x: S0, lane y: S1) as float
// pairs: error-free products of the pair table with the quantised weights,
// the high parts summed with two-sums, in packed FP32
template <int ORDER, int RE>
__device__ __forceinline__ ff2 gather_kick2(const float2 *El, const ShapeMix<ORDER> &S0,
                                            const ShapeMix<ORDER> &S1) {
  float2 ph[ORDER + 1], pl = make_float2(0.0f, 0.0f);
#pragma unroll
  for (int k = 0; k <= ORDER; k++) {
    const float2 e0 = El[(S0.p + k) * RE], e1 = El[(S1.p + k) * RE];
    const float2 w = make_float2(S0.w[k], S1.w[k]);
    const ff2 p = two_prod2(make_float2(e0.x, e1.x), w);
    ph[k] = p.hi;
    pl = add2(pl, fma2(make_float2(e0.y, e1.y), w, p.lo));
  }
  ff2 Ep = two_sum2(ph[0], ph[1]);
  pl = add2(pl, Ep.lo);
  if (ORDER == 2) {
    Ep = two_sum2(Ep.hi, ph[ORDER]);
    pl = add2(pl, Ep.lo);
  }
  return fast_two_sum2(Ep.hi, pl);
}

// correct_velocity for two markers at once.  The packed path covers the
// common case, both markers corrected with |t| < 2^-8; any other pair runs
// correct_velocity per marker, so each lane gets exactly the scalar result.
template <bool G64>
__device__ __forceinline__ ff2 correct_velocity2(float2 vh, float2 vl, int Vs0, int Vs1, ff2 d,
                                                 bool on0, bool on1, unsigned &nfb) {
  if (G64) {
    const ff v0 = correct_velocity<true>(vh.x, vl.x, Vs0, ff{d.hi.x, d.lo.x}, on0, nfb);
    const ff v1 = correct_velocity<true>(vh.y, vl.y, Vs1, ff{d.hi.y, d.lo.y}, on1, nfb);
    return ff2{make_float2(v0.hi, v1.hi), make_float2(v0.lo, v1.lo)};
  }
  const ff2 vd = ff_add2(ff2{vh, vl}, d);
  bool packed = on0 && on1;
  float2 gm = make_float2(0.0f, 0.0f);
  if (packed) {
    const int ih0 = __float2int_rn(vh.x), ih1 = __float2int_rn(vh.y);
    const float2 fr = sub2(vh, make_float2(__int2float_rn(ih0), __int2float_rn(ih1)));
    const ff2 q = two_sum2(make_float2(__int2float_rn(Vs0 - ih0), __int2float_rn(Vs1 - ih1)),
                           mul2(splat2(-0.5f), d.hi));
    const float2 small = sub2(sub2(sub2(q.lo, fr), vl), mul2(splat2(0.5f), d.lo));
    const float2 bq = add2(q.hi, small);
    // t = a / b by div_rcp_residual, lane by lane
    const float2 a = mul2(add2(d.hi, d.hi), bq), b = mul2(vd.hi, vd.hi);
    float2 r;
    asm("rcp.approx.f32 %0, %1;" : "=f"(r.x) : "f"(b.x));
    asm("rcp.approx.f32 %0, %1;" : "=f"(r.y) : "f"(b.y));
    const float2 q0 = mul2(a, r);
    const float2 t = fma2(fma2(neg2(q0), b, a), r, q0);
    packed = fabsf(t.x) < 0.00390625f && fabsf(t.y) < 0.00390625f;
    if (packed)
      gm = mul2(t, fma2(t, fma2(t, fma2(t, splat2(-0.0390625f), splat2(0.0625f)), splat2(-0.125f)),
                        splat2(0.5f)));
  }
  if (!packed) {
    const ff v0 = correct_velocity<false>(vh.x, vl.x, Vs0, ff{d.hi.x, d.lo.x}, on0, nfb);
    const ff v1 = correct_velocity<false>(vh.y, vl.y, Vs1, ff{d.hi.y, d.lo.y}, on1, nfb);
    return ff2{make_float2(v0.hi, v1.hi), make_float2(v0.lo, v1.lo)};
  }
  ff2 p = two_prod2(vd.hi, gm);
  p.lo = fma2(vd.lo, gm, p.lo);
  const ff2 s = fast_two_sum2(vd.hi, p.hi);
  return fast_two_sum2(s.hi, add2(s.lo, add2(vd.lo, p.lo)));
}

// Adds a 64-bit padded tile to J[node stride] with one global atomic per node
// and, when total is not null, the tile's sum to *total.
template <int ORDER>
__device__ __forceinline__ void flush_tile_i64(const long long *Jt, long long *J, int nc,
                                               int stride, long long *total) {
  long long mine = 0;
  for (int q = threadIdx.x; q < npad_of(nc); q += blockDim.x) {
    const long long a = Jt[q];
    mine += a;
    if (a != 0)
      atomicAdd((unsigned long long *)&J[PIC_INDEX(wrap_node(q - Pad<ORDER>::kPad, nc), nc) *
                                         stride],
                (unsigned long long)a);
  }
  if (total) {
    for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
    if ((threadIdx.x & 31u) == 0u && mine != 0)
      atomicAdd((unsigned long long *)total, (unsigned long long)mine);
  }
}

// A block's place among the blocks that share one run's markers: rb of nb.  A
// single-run launch uses (blockIdx.x, gridDim.x); a batched launch over several
// runs takes it from its work list.
struct BlockPlace {
  int rb, nb;
};
__device__ __forceinline__ BlockPlace grid_place() { return {(int)blockIdx.x, (int)gridDim.x}; }

// State of G consecutive markers of one thread (vector loads of 4 G bytes).
template <int G>
struct MarkerGroup {
  uint32_t X[G];
  float vh[G], vl[G];
  int V[G];
};

template <int G, typename T>
__device__ __forceinline__ void load_vec(const T *base, int64_t g, bool ok, T (&out)[G]) {
  static_assert(sizeof(T) == 4 && (G == 2 || G == 4), "groups of 2 or 4 words");
  if (G == 4) {
    uint4 u = make_uint4(0, 0, 0, 0);
    if (ok) u = reinterpret_cast<const uint4 *>(base)[g];
    memcpy(&out, &u, sizeof u);
  } else {
    uint2 u = make_uint2(0, 0);
    if (ok) u = reinterpret_cast<const uint2 *>(base)[g];
    memcpy(&out, &u, sizeof u);
  }
}

template <int G, typename T>
__device__ __forceinline__ void store_vec(T *base, int64_t g, const T (&in)[G]) {
  if (G == 4) {
    uint4 u;
    memcpy(&u, &in, sizeof u);
    reinterpret_cast<uint4 *>(base)[g] = u;
  } else {
    uint2 u;
    memcpy(&u, &in, sizeof u);
    reinterpret_cast<uint2 *>(base)[g] = u;
  }
}

template <int G, bool WITH_V>
__device__ __forceinline__ void load_group(const Es1dMixBufs &b, int64_t g, bool ok,
                                           MarkerGroup<G> &m) {
  load_vec<G>(b.X, g, ok, m.X);
  load_vec<G>(b.vh, g, ok, m.vh);
  load_vec<G>(b.vl, g, ok, m.vl);
  if (WITH_V) load_vec<G>(b.Vs, g, ok, m.V);
}

// Runs body(check, g, m) over the groups g of G consecutive markers of this
// thread.  With PREFETCH the state of the next group is loaded while the
// current one is processed (the unsorted passes; the windowed deposits of the
// sorted modes need those registers).  All lanes of a warp run the same trips
// (warp-level deposits and ranks need them): trips in which the warp's 32
// groups are all full run without validity tests (check = false_type), the
// last one or two with them.
template <int G, bool WITH_V, bool PREFETCH, typename F>
__device__ __forceinline__ void for_groups(const Es1dMixBufs &b, int64_t n, BlockPlace P, F body) {
  // block rb of nb takes the groups [ngroups rb / nb, ngroups (rb + 1) / nb)
  const int64_t nfull = n / G, ngroups = (n + G - 1) / G;
  const int64_t beg = ngroups * P.rb / P.nb;
  const int64_t end = ngroups * (P.rb + 1) / P.nb;
  const int64_t full_end = end < nfull ? end : nfull;
  int64_t gw = beg + (threadIdx.x & ~31u);
  int64_t g = gw + (threadIdx.x & 31u);
  MarkerGroup<G> cur;
  if (PREFETCH) load_group<G, WITH_V>(b, g, g < end, cur);
  for (; gw < end; gw += blockDim.x, g += blockDim.x) {
    MarkerGroup<G> nxt;
    if (PREFETCH)
      load_group<G, WITH_V>(b, g + blockDim.x, g + blockDim.x < end, nxt);
    else
      load_group<G, WITH_V>(b, g, g < end, cur);
    if (gw + 31 < full_end)
      body(std::false_type(), g, cur, end);
    else
      body(std::true_type(), g, cur, end);
    if (PREFETCH) cur = nxt;
  }
}

// Markers per group of a thread in passes C and E, and whether the next
// group's state is loaded while the current one is processed (unsorted modes).
constexpr int kGroupC = 4;
constexpr int kGroupE = 4;
constexpr bool kPrefetchC = true;
constexpr bool kPrefetchE = false;

// FILT: the unsorted kernels are built with and without the filter's table
// code (the sorted ones test c.passes at run time)
template <int ORDER, int SCHEME, int MODE, int RT, int RE, bool FILT = false>
__device__ __forceinline__ void pass_c_body(const Es1dMixConst &c, const Es1dMixBufs &b, int par,
                                            int prev_slot, int prev_nblocks, BlockPlace P) {
  constexpr bool AGG = MODE > 0;
  constexpr bool kFilterCode = FILT || MODE > 0;
  constexpr int PAD = Pad<ORDER>::kPad;
  static_assert(!AGG || RT == 1, "sorted modes use a single tile copy");
  extern __shared__ __align__(16) unsigned char smraw[];
  const int npad = npad_of(c.nc);
  unsigned *Jt = (unsigned *)smraw;           // [npad][2][RT]
  float *Es = (float *)(Jt + 2 * RT * npad);  // [npad][RE]: dt/2 (q/m) cxk E*
  uint32_t *hist = (uint32_t *)(Es + RE * npad);  // MODE 2: keys of the markers after the step
  // shared-memory set-up needs nothing from the previous kernel
  clear_tile<RT>(Jt, npad);
  if (MODE == 2)
    for (int i = threadIdx.x; i < 2 * c.nc; i += blockDim.x) hist[i] = 0;
  griddep_wait();
  {
    // e_scale E* = e_scale E - e_scale dt/2 jscale (J1 - <J1>) at every padded
    // node in FP32, from the float-pair table kick E (e_scale = kick / 2); the
    // first node's loads are issued before the grid mean
    const float2 *Ek = PSEL(b.Ek, par);
    const long long *J1 = PSEL(b.J1, par);
    const int i0 = wrap_node((int)threadIdx.x - PAD, c.nc);
    const bool has0 = (int)threadIdx.x < npad;
    const float2 E0 = has0 ? Ek[i0] : make_float2(0.0f, 0.0f);
    const long long J0 = (SCHEME == 2 && has0) ? J1[i0 * kJStride] : 0;
    const float mean = (SCHEME == 2 && c.remove_mean) ? mean_of_total(b.Jtot[par], c).hi : 0.0f;
    if (kFilterCode && c.passes > 0) {
      estar_table_filtered<SCHEME, RE, PAD>(c.nc, c.passes, c.c_jstar, b.filt, Ek, J1, mean, Es,
                                            npad);
    } else {
      // whole warps in every trip (the copies are written by the warp together)
      for (int q = threadIdx.x; q - (int)(threadIdx.x & 31u) < npad; q += blockDim.x) {
        float e = 0.0f;
        if (q < npad) {
          const int i = wrap_node(q - PAD, c.nc);
          const bool first = q == (int)threadIdx.x;
          const float2 ek = first ? E0 : Ek[i];
          e = __fmul_rn(0.5f, __fadd_rn(ek.x, ek.y));
          if (SCHEME == 2) {
            const float dj = __fsub_rn(__ll2float_rn(first ? J0 : J1[i * kJStride]), mean);
            e = __fmaf_rn(-c.c_jstar, dj, e);
          }
        }
        store_copies_warp<RE>(Es, q, e, npad);
      }
    }
  }
  if (P.rb == 0 && SCHEME == 2) {
    for (int i = threadIdx.x; i < c.nc; i += blockDim.x) PSEL(b.J1, par ^ 1)[i * kJStride] = 0;
    if (threadIdx.x == 0) b.Jtot[par ^ 1] = 0;
  }
  __syncthreads();
  const unsigned lane = threadIdx.x & 31u;
  unsigned *Jl = Jt + (lane & (RT - 1));
  const float *El = Es + (lane & (RE - 1));
  unsigned bad = 0;
  // TE of the previous step (its pass E partials are complete after the wait)
  if (P.rb == 0 && prev_slot >= 0 && last_warp())
    finalize_stats_warp(b, c.h, prev_slot, prev_nblocks);
  constexpr int G = kGroupC;
  for_groups<G, false, !AGG && kPrefetchC>(b, c.n, P, [&](auto check, int64_t g, const MarkerGroup<G> &m, int64_t end) {
    constexpr bool CHECK = decltype(check)::value;
    const bool gv = !CHECK || g < end;
    int Vout[G];
    DepositWindow<ORDER> win;
    static_assert(G % 2 == 0, "markers are processed in pairs");
#pragma unroll
    for (int j = 0; j < G; j += 2) {
      // gather #1 at x* and v* of two markers, the float work in packed FP32
      ShapeMix<ORDER> Sx0, Sx1;
      shape_mix_pair<ORDER>(m.X[j] + half_shift(to_fixed(m.vh[j], bad), c),
                            m.X[j + 1] + half_shift(to_fixed(m.vh[j + 1], bad), c), c.nc, Sx0, Sx1);
      float2 e = make_float2(0.0f, 0.0f);
#pragma unroll
      for (int k = 0; k <= ORDER; k++)
        e = fma2(make_float2(Sx0.w[k], Sx1.w[k]),
                 make_float2(El[(Sx0.p + k) * RE], El[(Sx1.p + k) * RE]), e);
      int Vs2[2];
      vstar_fixed2(make_float2(m.vh[j], m.vh[j + 1]), make_float2(m.vl[j], m.vl[j + 1]), e, bad,
                   Vs2);
      const uint32_t hs0 = half_shift(Vs2[0], c), hs1 = half_shift(Vs2[1], c);
      ShapeMix<ORDER> Sh0, Sh1;
      shape_mix_pair<ORDER>(m.X[j] + hs0, m.X[j + 1] + hs1, c.nc, Sh0, Sh1);
#pragma unroll
      for (int u = 0; u < 2; u++) {
        const int jj = j + u;
        const bool valid = !CHECK || (gv && G * g + jj < c.n);
        const int Vs = Vs2[u];
        const ShapeMix<ORDER> &Sh = u ? Sh1 : Sh0;
        if (AGG) {
          if (jj == 0) win.start(Sh.p, valid, npad);
          win.add(Jt, Sh, Vs, c, valid);
        } else if (valid) {
          deposit_direct<ORDER, RT>(Jl, Sh, Vs, c);
        }
        if (MODE == 2) warp_rank(hist, sort_key(m.X[jj] + 2u * (u ? hs1 : hs0), Vs, c.nc), valid);
        Vout[jj] = Vs;
      }
    }
    if (AGG) win.flush(Jt, c.split);
    if (gv) store_vec<G>(b.Vs, g, Vout);
  });
  griddep_launch_dependents();
  report_flags(bad, b.err);
  __syncthreads();
  flush_tile<ORDER, RT>(Jt, PSEL(b.J2, par), b.Jtot + 2 + par, c.nc, c.split);
  if (MODE == 2)
    for (int i = threadIdx.x; i < 2 * c.nc; i += blockDim.x)
      b.H[(int64_t)i * P.nb + P.rb] = hist[i];
}

template <int ORDER, int SCHEME, int MODE, int RT, int RE, bool FILT>
__global__ void __launch_bounds__(RT > 1 ? 1024 : 512, RT > 1 ? 1 : 2)
    mix_pass_c_kernel(Es1dMixConst c, Es1dMixBufs b, int par, int prev_slot, int prev_nblocks) {
  pass_c_body<ORDER, SCHEME, MODE, RT, RE, FILT>(c, b, par, prev_slot, prev_nblocks, grid_place());
}

// pass E: E^{n+1} and dt (q/m) cxk E^{n+1/2} (float pairs) in the prologue; per
// marker the gather at x^{n+1/2} = X + [V*], v^dag, Gamma, x^{n+1}, v^{n+1},
// the kinetic energy and (ESEC2) the next step's x* and j^{n+1,*} deposit.
template <int ORDER, int SCHEME, int MODE, int RT, int RE, bool G64 = false, bool FILT = false>
__device__ __forceinline__ void pass_e_body(const Es1dMixConst &c, const Es1dMixBufs &b, int par,
                                            int slot, BlockPlace P) {
  constexpr bool AGG = MODE > 0;
  constexpr bool kFilterCode = FILT || MODE > 0;
  constexpr int PAD = Pad<ORDER>::kPad;
  static_assert(!AGG || RT == 1, "sorted modes use a single tile copy");
  extern __shared__ __align__(16) unsigned char smraw[];
  const int npad = npad_of(c.nc);
  unsigned *Jt = (unsigned *)smraw;              // [npad][2][RT]
  float2 *Eh2 = (float2 *)(Jt + 2 * RT * npad);  // [npad][RE]: dt (q/m) cxk E^{n+1/2}
  uint32_t *off = (uint32_t *)(Eh2 + RE * npad); // MODE 2: next free slot of each key
  clear_tile<RT>(Jt, npad);  // needs nothing from the previous kernel
  griddep_wait();
  const long long *J2 = PSEL(b.J2, par);
  struct {
    ff j;
  } mean2{{0.0f, 0.0f}};
  if (MODE == 2) {
    __shared__ uint32_t tmp[512];
    block_exclusive_scan(b.T, off, 2 * c.nc, tmp);
    for (int i = threadIdx.x; i < 2 * c.nc; i += blockDim.x)
      off[i] += b.H[(int64_t)i * P.nb + P.rb];
  }
  {
    // kick E^{n+1/2} = kick E^n - kick dt/2 jscale (J2 - <J2>) at every padded
    // node in float pairs (no FP64 per node); the first node's loads are issued
    // before the grid mean
    const float2 *Ek = PSEL(b.Ek, par);
    const int i0 = wrap_node((int)threadIdx.x - PAD, c.nc);
    const bool has0 = (int)threadIdx.x < npad;
    const float2 E0 = has0 ? Ek[i0] : make_float2(0.0f, 0.0f);
    const long long J0 = has0 ? J2[i0 * kJStride] : 0;
    if (c.remove_mean) mean2.j = mean_of_total(b.Jtot[2 + par], c);
    if (kFilterCode && c.passes > 0) {
      ehalf_table_filtered<RE, PAD>(c.nc, c.passes, c.kick_jhalf, b.filt, Ek, J2, mean2.j, Eh2,
                                    npad);
    } else {
      // whole warps in every trip (the copies are written by the warp together)
      for (int q = threadIdx.x; q - (int)(threadIdx.x & 31u) < npad; q += blockDim.x) {
        float2 v = make_float2(0.0f, 0.0f);
        if (q < npad) {
          const int i = wrap_node(q - PAD, c.nc);
          const bool first = q == (int)threadIdx.x;
          const float2 ek = first ? E0 : Ek[i];
          const ff dj = ff_sub(ff_from_i64(first ? J0 : J2[i * kJStride]), mean2.j);
          const ff eh = ff_sub(ff{ek.x, ek.y}, ff_mul(c.kick_jhalf, dj));
          v = make_float2(eh.hi, eh.lo);
        }
        store_copies_warp<RE>(Eh2, q, v, npad);
      }
    }
  }
  __syncthreads();

  // E^{n+1} = E^n - dt (jscale J2 - jscale <J2>) (F^p J2 with the filter) in
  // FP64 on the nodes [b nc / grid, (b + 1) nc / grid) by the last warp of
  // block b, before its markers (with a block's groups not a multiple of its
  // threads, the last warp has one trip fewer): the field, its float-pair
  // table for the next step, the cleared J2 of the next step and this
  // block's part of sum (E^{n+1})^2.  Nothing in this pass reads what it
  // writes.
  if (last_warp()) {
    const unsigned lane = threadIdx.x & 31u;
    const double *E = PSEL(b.E, par);
    const double mean_e = c.remove_mean ? (double)b.Jtot[2 + par] * c.jscale / c.nc : 0.0;
    if (P.rb == 0 && lane == 0) b.Jtot[2 + (par ^ 1)] = 0;
    const int n0 = (int)((int64_t)c.nc * P.rb / P.nb);
    const int n1 = (int)((int64_t)c.nc * (P.rb + 1) / P.nb);
    double w = 0.0;
    for (int i = n0 + (int)lane; i < n1; i += 32) {
      const double j = kFilterCode && c.passes > 0 ? filtered_j(c.nc, c.passes, b.filt, J2, i)
                                                   : (double)J2[i * kJStride];
      const double en = E[i] - c.dt * (j * c.jscale - mean_e);
      PSEL(b.E, par ^ 1)[i] = en;
      const ff k = ff_from_double(c.kick * en);
      PSEL(b.Ek, par ^ 1)[i] = make_float2(k.hi, k.lo);
      PSEL(b.J2, par ^ 1)[i * kJStride] = 0;
      w = fma(en, en, w);
    }
    if (n1 > n0)
      for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
    if (lane == 0) b.we_part[P.rb] = w;
  }
  const unsigned lane = threadIdx.x & 31u;
  unsigned *Jl = Jt + (lane & (RT - 1));
  const float2 *El = Eh2 + (lane & (RE - 1));
  // kinetic sums of the even (x) and odd (y) markers of each group
  float2 ke2h = make_float2(0.0f, 0.0f), ke2l = make_float2(0.0f, 0.0f);
  unsigned nfb = 0, bad = 0;
  constexpr int G = kGroupE;
  static_assert(G % 2 == 0, "markers are processed in pairs");
  for_groups<G, true, !AGG && kPrefetchE>(b, c.n, P, [&](auto check, int64_t g, const MarkerGroup<G> &m, int64_t end) {
    constexpr bool CHECK = decltype(check)::value;
    const bool gv = !CHECK || g < end;
    MarkerGroup<G> o;
    DepositWindow<ORDER> win;
#pragma unroll
    for (int j = 0; j < G; j += 2) {
      const bool valid0 = !CHECK || (gv && G * g + j < c.n);
      const bool valid1 = !CHECK || (gv && G * g + j + 1 < c.n);
      const uint32_t hs0 = half_shift(m.V[j], c), hs1 = half_shift(m.V[j + 1], c);
      // gather #2 at x^{n+1/2}: d = dt (q/m) E^{n+1/2}_p in V units, two markers at once
      ShapeMix<ORDER> Sh0, Sh1;
      shape_mix_pair<ORDER>(m.X[j] + hs0, m.X[j + 1] + hs1, c.nc, Sh0, Sh1);
      const ff2 d = gather_kick2<ORDER, RE>(El, Sh0, Sh1);
      const ff2 vn2 = correct_velocity2<G64>(make_float2(m.vh[j], m.vh[j + 1]),
                                        make_float2(m.vl[j], m.vl[j + 1]), m.V[j], m.V[j + 1], d,
                                        c.gamma_on && valid0, c.gamma_on && valid1, nfb);
      {
        // |v^{n+1}|^2 in float pairs into the two lanes' sums (0 for a marker past the end)
        const float2 h = make_float2(valid0 ? vn2.hi.x : 0.0f, valid1 ? vn2.hi.y : 0.0f);
        const float2 l = make_float2(valid0 ? vn2.lo.x : 0.0f, valid1 ? vn2.lo.y : 0.0f);
        ff2 s2 = two_prod2(h, h);
        s2.lo = fma2(add2(h, h), l, s2.lo);
        const ff2 acc = two_sum2(ke2h, s2.hi);
        ke2h = acc.hi;
        ke2l = add2(ke2l, add2(acc.lo, s2.lo));
      }
      const uint32_t Xn0 = m.X[j] + 2u * hs0, Xn1 = m.X[j + 1] + 2u * hs1;
      // x* of the next step and its shapes (ESEC2's j^{n+1,*} deposit)
      int Vn1s[2] = {0, 0};
      ShapeMix<ORDER> S10, S11;
      if (SCHEME == 2) {
        Vn1s[0] = to_fixed(vn2.hi.x, bad);
        Vn1s[1] = to_fixed(vn2.hi.y, bad);
        shape_mix_pair<ORDER>(Xn0 + half_shift(Vn1s[0], c), Xn1 + half_shift(Vn1s[1], c), c.nc,
                              S10, S11);
      }
#pragma unroll
      for (int u = 0; u < 2; u++) {
        const int jj = j + u;
        const uint32_t X = m.X[jj];
        const int Vs = m.V[jj];
        const bool valid = u ? valid1 : valid0;
        const ff vn = u ? ff{vn2.hi.y, vn2.lo.y} : ff{vn2.hi.x, vn2.lo.x};
        const uint32_t Xn = u ? Xn1 : Xn0;
        if (SCHEME == 2) {
          const int Vn1 = Vn1s[u];
          const ShapeMix<ORDER> &S1 = u ? S11 : S10;
          if (AGG) {
            if (jj == 0) win.start(S1.p, valid, npad);
            win.add(Jt, S1, Vn1, c, valid);
          } else if (valid) {
            deposit_direct<ORDER, RT>(Jl, S1, Vn1, c);
          }
        }
        if (MODE == 2) {
          // sort on write: the marker's slot in key order, from pass C's counts
          const uint32_t dst = PIC_INDEX(warp_rank(off, sort_key(Xn, Vs, c.nc), valid), c.n);
          if (valid) {
            b.Xo[dst] = Xn;
            b.vho[dst] = vn.hi;
            b.vlo[dst] = vn.lo;
            if (b.ids) b.ido[dst] = b.ids[G * g + jj];
          }
        }
        o.X[jj] = valid ? Xn : X;
        o.vh[jj] = valid ? vn.hi : m.vh[jj];
        o.vl[jj] = valid ? vn.lo : m.vl[jj];
      }
    }
    if (AGG && SCHEME == 2) win.flush(Jt, c.split);
    if (MODE != 2 && gv) {
      store_vec<G>(b.X, g, o.X);
      store_vec<G>(b.vh, g, o.vh);
      store_vec<G>(b.vl, g, o.vl);
    }
  });
  griddep_launch_dependents();
  // the two lanes' kinetic sums; a non-finite v^{n+1} leaves them non-finite
  const ff ke_t = ff_add(ff{ke2h.x, ke2l.x}, ff{ke2h.y, ke2l.y});
  const float ke_hi = ke_t.hi, ke_lo = ke_t.lo;
  if (!isfinite(ke_hi) || !isfinite(ke_lo)) bad |= kErrNonfinite;
  report_flags(bad, b.err);
  nfb = __reduce_add_sync(0xffffffffu, nfb);
  if (lane == 0 && nfb) atomicAdd(&b.fallback[slot], (unsigned long long)nfb);
  // kinetic energy: float-pair sums over each warp, then over the warps by
  // warp 0, FP64 for the block total only
  {
    __shared__ float2 kred[32];
    ff k = {ke_hi, ke_lo};
    for (int o = 16; o > 0; o >>= 1)
      k = ff_add(k, ff{__shfl_xor_sync(0xffffffffu, k.hi, o), __shfl_xor_sync(0xffffffffu, k.lo, o)});
    if (lane == 0) kred[threadIdx.x >> 5] = make_float2(k.hi, k.lo);
    __syncthreads();
    if (threadIdx.x < 32) {
      k = threadIdx.x < (blockDim.x >> 5) ? ff{kred[lane].x, kred[lane].y} : ff{0.0f, 0.0f};
      for (int o = 16; o > 0; o >>= 1)
        k = ff_add(k, ff{__shfl_xor_sync(0xffffffffu, k.hi, o), __shfl_xor_sync(0xffffffffu, k.lo, o)});
      if (lane == 0) b.ke_part[P.rb] = c.ke_scale * ((double)k.hi + (double)k.lo);
    }
  }
  if (SCHEME == 2) flush_tile<ORDER, RT>(Jt, PSEL(b.J1, par ^ 1), b.Jtot + (par ^ 1), c.nc, c.split);
}

template <int ORDER, int SCHEME, int MODE, int RT, int RE, bool G64, bool FILT>
__global__ void __launch_bounds__(RT > 1 ? 1024 : 512, RT > 1 ? 1 : 2)
    mix_pass_e_kernel(Es1dMixConst c, Es1dMixBufs b, int par, int slot) {
  pass_e_body<ORDER, SCHEME, MODE, RT, RE, G64, FILT>(c, b, par, slot, grid_place());
}

// ESEC1 in one pass per step (Eq. naivetranslation with the correction of Eq.
// PICmodification).  ESEC1 has no j^{n,*}: the only grid quantity a step
// needs before its first gather is E^n, so the update of step n (pass E: the
// gather at x^{n+1/2}, Gamma, x^{n+1}, v^{n+1}) and the push of step n+1
// (pass C: the gather of E^{n+1} at x*, v*, the deposit of j^{*,n+3/2}) run
// on each marker in one visit: 16 bytes read and 16 written per
// particle-step.  The block prologue builds both tables from the same inputs
// the two separate passes use (kick E^{n+1/2} in float pairs; e_scale E^{n+1}
// in FP32 from the FP64 E^{n+1} that the last warp also writes back), so the
// results are those of the two-launch form bit for bit.  Currents rotate
// through three buffers (RingIO): this launch reads j^{*,n+1/2}, deposits
// j^{*,n+3/2} and clears the one the previous launch read.
template <int ORDER, int RT, int RE, int RE1>
__global__ void __launch_bounds__(RT > 1 ? kFusedThreads : 512, RT > 1 ? 1 : 2)
    mix_pass_ec_kernel(Es1dMixConst c, Es1dMixBufs b, RingIO io, int par, int slot,
                       int prev_slot, int prev_nblocks) {
  constexpr int PAD = Pad<ORDER>::kPad;
  const BlockPlace P = grid_place();
  extern __shared__ __align__(16) unsigned char smraw[];
  const int npad = npad_of(c.nc);
  unsigned *Jt = (unsigned *)smraw;              // [npad][2][RT]
  float2 *Eh2 = (float2 *)(Jt + 2 * RT * npad);  // [npad][RE]: kick E^{n+1/2}
  float *Es = (float *)(Eh2 + RE * npad);         // [npad][RE1]: e_scale E^{n+1}
  clear_tile<RT>(Jt, npad);  // needs nothing from the previous kernel
  griddep_wait();
  const double mean_e = c.remove_mean ? (double)(*io.Tr) * c.jscale / c.nc : 0.0;
  {
    const float2 *Ek = PSEL(b.Ek, par);
    const double *E = PSEL(b.E, par);
    const ff meanj = c.remove_mean ? mean_of_total(*io.Tr, c) : ff{0.0f, 0.0f};
    // whole warps in every trip (the copies are written by the warp together)
    for (int q = threadIdx.x; q - (int)(threadIdx.x & 31u) < npad; q += blockDim.x) {
      float2 vh = make_float2(0.0f, 0.0f);
      float vs = 0.0f;
      if (q < npad) {
        const int i = wrap_node(q - PAD, c.nc);
        const float2 ek = Ek[i];
        const long long j2 = io.Jr[i * kJStride];
        const ff dj = ff_sub(ff_from_i64(j2), meanj);
        const ff eh = ff_sub(ff{ek.x, ek.y}, ff_mul(c.kick_jhalf, dj));
        vh = make_float2(eh.hi, eh.lo);
        const double en = E[i] - c.dt * ((double)j2 * c.jscale - mean_e);
        const ff k = ff_from_double(c.kick * en);
        vs = __fmul_rn(0.5f, __fadd_rn(k.hi, k.lo));
      }
      store_copies_warp<RE>(Eh2, q, vh, npad);
      store_copies_warp<RE1>(Es, q, vs, npad);
    }
  }
  __syncthreads();
  const unsigned lane = threadIdx.x & 31u;
  if (last_warp()) {
    // TE of the previous step from its partials (io.ke_prev, io.we_prev)
    if (P.rb == 0 && prev_slot >= 0) {
      Es1dMixBufs bp = b;
      bp.ke_part = const_cast<double *>(io.ke_prev);
      bp.we_part = const_cast<double *>(io.we_prev);
      finalize_stats_warp(bp, c.h, prev_slot, prev_nblocks);
    }
    // E^{n+1} on this block's slice of nodes, its float-pair table, the
    // cleared current buffer of step n+2 and this block's part of sum E^2
    const double *E = PSEL(b.E, par);
    if (P.rb == 0 && lane == 0) *io.Tc = 0;
    const int n0 = (int)((int64_t)c.nc * P.rb / P.nb);
    const int n1 = (int)((int64_t)c.nc * (P.rb + 1) / P.nb);
    double w = 0.0;
    for (int i = n0 + (int)lane; i < n1; i += 32) {
      const double en = E[i] - c.dt * ((double)io.Jr[i * kJStride] * c.jscale - mean_e);
      PSEL(b.E, par ^ 1)[i] = en;
      const ff k = ff_from_double(c.kick * en);
      PSEL(b.Ek, par ^ 1)[i] = make_float2(k.hi, k.lo);
      io.Jc[i * kJStride] = 0;
      w = fma(en, en, w);
    }
    if (n1 > n0)
      for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
    if (lane == 0) io.we_out[P.rb] = w;
  }
  unsigned *Jl = Jt + (lane & (RT - 1));
  const float2 *El = Eh2 + (lane & (RE - 1));
  const float *Ex = Es + (lane & (RE1 - 1));
  float2 ke2h = make_float2(0.0f, 0.0f), ke2l = make_float2(0.0f, 0.0f);
  unsigned nfb = 0, bad = 0;
  constexpr int G = kGroupE;
  for_groups<G, true, false>(b, c.n, P, [&](auto check, int64_t g, const MarkerGroup<G> &m, int64_t end) {
    constexpr bool CHECK = decltype(check)::value;
    const bool gv = !CHECK || g < end;
    MarkerGroup<G> o;
#pragma unroll
    for (int j = 0; j < G; j += 2) {
      const bool valid0 = !CHECK || (gv && G * g + j < c.n);
      const bool valid1 = !CHECK || (gv && G * g + j + 1 < c.n);
      // step n: gather #2 at x^{n+1/2} = X + [V*], Gamma, x^{n+1}, v^{n+1}
      const uint32_t hs0 = half_shift(m.V[j], c), hs1 = half_shift(m.V[j + 1], c);
      ShapeMix<ORDER> Sh0, Sh1;
      shape_mix_pair<ORDER>(m.X[j] + hs0, m.X[j + 1] + hs1, c.nc, Sh0, Sh1);
      const ff2 d = gather_kick2<ORDER, RE>(El, Sh0, Sh1);
      const ff2 vn2 = correct_velocity2<false>(make_float2(m.vh[j], m.vh[j + 1]),
                                               make_float2(m.vl[j], m.vl[j + 1]), m.V[j],
                                               m.V[j + 1], d, c.gamma_on && valid0,
                                               c.gamma_on && valid1, nfb);
      {
        const float2 h = make_float2(valid0 ? vn2.hi.x : 0.0f, valid1 ? vn2.hi.y : 0.0f);
        const float2 l = make_float2(valid0 ? vn2.lo.x : 0.0f, valid1 ? vn2.lo.y : 0.0f);
        ff2 s2 = two_prod2(h, h);
        s2.lo = fma2(add2(h, h), l, s2.lo);
        const ff2 acc = two_sum2(ke2h, s2.hi);
        ke2h = acc.hi;
        ke2l = add2(ke2l, add2(acc.lo, s2.lo));
      }
      const uint32_t Xn0 = m.X[j] + 2u * hs0, Xn1 = m.X[j + 1] + 2u * hs1;
      // step n+1: gather #1 of E^{n+1} at x* = x^{n+1} + dt/2 v^{n+1}, V*,
      // x^{n+3/2} and the deposit of j^{*,n+3/2}
      ShapeMix<ORDER> Sx0, Sx1;
      shape_mix_pair<ORDER>(Xn0 + half_shift(to_fixed(vn2.hi.x, bad), c),
                            Xn1 + half_shift(to_fixed(vn2.hi.y, bad), c), c.nc, Sx0, Sx1);
      float2 e = make_float2(0.0f, 0.0f);
#pragma unroll
      for (int k = 0; k <= ORDER; k++)
        e = fma2(make_float2(Sx0.w[k], Sx1.w[k]),
                 make_float2(Ex[(Sx0.p + k) * RE1], Ex[(Sx1.p + k) * RE1]), e);
      int Vs2[2];
      vstar_fixed2(vn2.hi, vn2.lo, e, bad, Vs2);
      const uint32_t h20 = half_shift(Vs2[0], c), h21 = half_shift(Vs2[1], c);
      ShapeMix<ORDER> S20, S21;
      shape_mix_pair<ORDER>(Xn0 + h20, Xn1 + h21, c.nc, S20, S21);
#pragma unroll
      for (int u = 0; u < 2; u++) {
        const int jj = j + u;
        const bool valid = u ? valid1 : valid0;
        if (valid) deposit_direct<ORDER, RT>(Jl, u ? S21 : S20, Vs2[u], c);
        o.X[jj] = valid ? (u ? Xn1 : Xn0) : m.X[jj];
        o.vh[jj] = valid ? (u ? vn2.hi.y : vn2.hi.x) : m.vh[jj];
        o.vl[jj] = valid ? (u ? vn2.lo.y : vn2.lo.x) : m.vl[jj];
        o.V[jj] = valid ? Vs2[u] : m.V[jj];
      }
    }
    if (gv) {
      store_vec<G>(b.X, g, o.X);
      store_vec<G>(b.vh, g, o.vh);
      store_vec<G>(b.vl, g, o.vl);
      store_vec<G>(b.Vs, g, o.V);
    }
  });
  griddep_launch_dependents();
  const ff ke_t = ff_add(ff{ke2h.x, ke2l.x}, ff{ke2h.y, ke2l.y});
  if (!isfinite(ke_t.hi) || !isfinite(ke_t.lo)) bad |= kErrNonfinite;
  report_flags(bad, b.err);
  nfb = __reduce_add_sync(0xffffffffu, nfb);
  if (lane == 0 && nfb) atomicAdd(&b.fallback[slot], (unsigned long long)nfb);
  {
    __shared__ float2 kred[32];
    ff k = ke_t;
    for (int o = 16; o > 0; o >>= 1)
      k = ff_add(k, ff{__shfl_xor_sync(0xffffffffu, k.hi, o), __shfl_xor_sync(0xffffffffu, k.lo, o)});
    if (lane == 0) kred[threadIdx.x >> 5] = make_float2(k.hi, k.lo);
    __syncthreads();
    if (threadIdx.x < 32) {
      k = threadIdx.x < (blockDim.x >> 5) ? ff{kred[lane].x, kred[lane].y} : ff{0.0f, 0.0f};
      for (int o = 16; o > 0; o >>= 1)
        k = ff_add(k, ff{__shfl_xor_sync(0xffffffffu, k.hi, o), __shfl_xor_sync(0xffffffffu, k.lo, o)});
      if (lane == 0) io.ke_out[P.rb] = c.ke_scale * ((double)k.hi + (double)k.lo);
    }
  }
  flush_tile<ORDER, RT>(Jt, io.Jw, io.Tw, c.nc, c.split);
}

template <int ORDER>
__global__ void __launch_bounds__(512) mix_deposit_initial_kernel(Es1dMixConst c, Es1dMixBufs b,
                                                                  int par) {
  extern __shared__ __align__(16) unsigned char smraw[];
  long long *Jt = (long long *)smraw;
  const int npad = npad_of(c.nc);
  for (int i = threadIdx.x; i < npad; i += blockDim.x) Jt[i] = 0;
  __syncthreads();
  unsigned bad = 0;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < c.n;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int Vn = to_fixed(b.vh[p], bad);
    const ShapeMix<ORDER> S(b.X[p] + half_shift(Vn, c), c.nc);
#pragma unroll
    for (int k = 0; k <= ORDER; k++)
      atomicAdd((unsigned long long *)&Jt[S.p + k], (unsigned long long)deposit_term(Vn, S.s[k], c));
  }
  if (bad) atomicOr(b.err, bad);
  __syncthreads();
  flush_tile_i64<ORDER>(Jt, PSEL(b.J1, par), c.nc, kJStride, b.Jtot + par);
}

// The same j^{n,*} for the wide layout (nc <= kWideMaxNodes, unsorted): 1024-thread
// blocks of the passes' launch, each lane adding into its own copy of the split
// tile; the per-copy marker count stays within the bound the rounding shift is
// chosen for (a thread takes at most 4 markers per trip of the passes), and the
// integer totals equal the single-tile kernel's.
template <int ORDER>
__global__ void __launch_bounds__(1024, 1)
    mix_deposit_initial_wide_kernel(Es1dMixConst c, Es1dMixBufs b, int par) {
  constexpr int RT = 32;
  extern __shared__ __align__(16) unsigned char smraw[];
  unsigned *Jt = (unsigned *)smraw;  // [npad][2][RT]
  const int npad = npad_of(c.nc);
  clear_tile<RT>(Jt, npad);
  __syncthreads();
  unsigned *Jl = Jt + (threadIdx.x & (RT - 1));
  unsigned bad = 0;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < c.n;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int Vn = to_fixed(b.vh[p], bad);
    const ShapeMix<ORDER> S(b.X[p] + half_shift(Vn, c), c.nc);
    deposit_direct<ORDER, RT>(Jl, S, Vn, c);
  }
  if (bad) atomicOr(b.err, bad);
  __syncthreads();
  flush_tile<ORDER, RT>(Jt, PSEL(b.J1, par), b.Jtot + par, c.nc, c.split);
}

// Charge of the markers for the initial Poisson solve: the integer weights
// summed exactly per node (order independent), in units of 2^-23.
template <int ORDER>
__global__ void __launch_bounds__(512) mix_charge_kernel(Es1dMixConst c, Es1dMixBufs b,
                                                         long long *count) {
  extern __shared__ __align__(16) unsigned char smraw[];
  long long *Jt = (long long *)smraw;
  const int npad = npad_of(c.nc);
  for (int i = threadIdx.x; i < npad; i += blockDim.x) Jt[i] = 0;
  __syncthreads();
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < c.n;
       p += (int64_t)gridDim.x * blockDim.x) {
    const ShapeMix<ORDER> S(b.X[p], c.nc);
#pragma unroll
    for (int k = 0; k <= ORDER; k++)
      atomicAdd((unsigned long long *)&Jt[S.p + k], (unsigned long long)S.s[k]);
  }
  __syncthreads();
  flush_tile_i64<ORDER>(Jt, count, c.nc, 1, nullptr);
}

// ------------------------------------------------------------- batched runs
// One launch per pass over a work list: block i steps block items[i].rb of the
// items[i].nb blocks of run items[i].run, with that run's constants and
// buffers (read-only arrays, read before the dependency wait) and the same
// pass bodies as a single-run launch; the kernel boundaries remain the only
// barriers between the passes.
// Batch blocks of NT threads: 1024 (32 tile copies, 16 table copies, one
// block per SM) for runs of many markers, 256 (8 and 8, up to eight blocks per
// SM) for batches of small runs, where a 1024-thread block would sit mostly
// idle.  A copy takes at most 2048 markers a launch in both (16 trips).
template <int NT>
struct BatchLayout {
  static constexpr int RT = NT == 1024 ? 32 : 8;
  static constexpr int RE = NT == 1024 ? 16 : 8;
  static constexpr int kMinBlocks = NT == 1024 ? 1 : 3;
};

template <int SCHEME, int NT>
__global__ void __launch_bounds__(NT, BatchLayout<NT>::kMinBlocks)
    mix_batch_pass_c_kernel(const Es1dMixConst *__restrict__ cs, const Es1dMixBufs *__restrict__ bs,
                            const BatchItem *__restrict__ items, int par, int prev_slot) {
  constexpr int RT = BatchLayout<NT>::RT, RE = BatchLayout<NT>::RE;
  const BatchItem it = items[blockIdx.x];
  const Es1dMixConst &c = cs[it.run];
  const Es1dMixBufs &b = bs[it.run];
  const BlockPlace P{it.rb, it.nb};
  if (c.order == 1)
    pass_c_body<1, SCHEME, 0, RT, RE>(c, b, par, prev_slot, it.nb, P);
  else
    pass_c_body<2, SCHEME, 0, RT, RE>(c, b, par, prev_slot, it.nb, P);
}

template <int SCHEME, int NT>
__global__ void __launch_bounds__(NT, BatchLayout<NT>::kMinBlocks)
    mix_batch_pass_e_kernel(const Es1dMixConst *__restrict__ cs, const Es1dMixBufs *__restrict__ bs,
                            const BatchItem *__restrict__ items, int par, int slot) {
  constexpr int RT = BatchLayout<NT>::RT, RE = BatchLayout<NT>::RE;
  const BatchItem it = items[blockIdx.x];
  const Es1dMixConst &c = cs[it.run];
  const Es1dMixBufs &b = bs[it.run];
  const BlockPlace P{it.rb, it.nb};
  if (c.order == 1)
    pass_e_body<1, SCHEME, 0, RT, RE>(c, b, par, slot, P);
  else
    pass_e_body<2, SCHEME, 0, RT, RE>(c, b, par, slot, P);
}

// TE of step `slot` of every run (one warp per run).
__global__ void mix_batch_finalize_kernel(const Es1dMixConst *cs, const Es1dMixBufs *bs,
                                          const int *nblocks, int slot) {
  const Es1dMixBufs &b = bs[blockIdx.x];
  const double h = cs[blockIdx.x].h;
  finalize_stats_warp(b, h, slot, nblocks[blockIdx.x]);
}

// Copies the first n per-step counts and energies of every run into one
// buffer ([run][step]) and clears the counts for the next steps.
__global__ void mix_batch_gather_kernel(const Es1dMixBufs *bs, int n, unsigned long long *fb,
                                        double *te) {
  const Es1dMixBufs &b = bs[blockIdx.x];
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    fb[(int64_t)blockIdx.x * n + k] = b.fallback[k];
    te[(int64_t)blockIdx.x * n + k] = b.te[k];
    b.fallback[k] = 0;
  }
}

__global__ void mix_set_ek_kernel(const double *E, float2 *Ek, int nc, double kick) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += gridDim.x * blockDim.x) {
    const ff k = ff_from_double(kick * E[i]);
    Ek[i] = make_float2(k.hi, k.lo);
  }
}

__global__ void mix_finalize_kernel(Es1dMixBufs b, double h, int slot, int nblocks) {
  finalize_stats_warp(b, h, slot, nblocks);
}

// FP64 (x, v) <-> (X, vh, vl) with v stored in V units (v * cxk)
__global__ void to_mix_kernel(const double *x, const double *v, int64_t n, double L, double cxk,
                              uint32_t *X, float *vh, float *vl, unsigned *err) {
  // x 2^32 / L with one multiply per marker (the FP64 divide is many FP64
  // instructions); X is the rounded product, within a rounding of x / L 2^32
  const double scale = 4294967296.0 / L;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    double xx = x[p], vv = v[p] * cxk;
    if (!(xx >= 0.0 && xx < L)) atomicOr(err, kErrBounds);
    if (!isfinite(vv)) atomicOr(err, kErrNonfinite);
    if (!(fabs(vv) < 2147483520.0)) atomicOr(err, kErrVelocityRange);
    double u = xx * scale;
    unsigned long long q = (unsigned long long)llrint(u);
    X[p] = (uint32_t)(q & 0xFFFFFFFFull);
    float h = (float)vv;
    vh[p] = h;
    vl[p] = (float)(vv - (double)h);
  }
}

__global__ void from_mix_kernel(const uint32_t *X, const float *vh, const float *vl, int64_t n,
                                double L, double inv_cxk, double *x, double *v) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    x[p] = (double)X[p] * (L / 4294967296.0);
    v[p] = ((double)vh[p] + (double)vl[p]) * inv_cxk;
  }
}

__global__ void __launch_bounds__(512) mix_kinetic_kernel(const float *vh, const float *vl,
                                                          int64_t n, double ke_scale,
                                                          double *part) {
  __shared__ double red[33];
  double acc = 0.0;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    double v = (double)vh[p] + (double)vl[p];
    acc += v * v;
  }
  double t = block_sum_d(acc, red);
  if (threadIdx.x == 0) part[blockIdx.x] = ke_scale * t;
}

// max |v| over the markers (non-negative doubles order like their bit patterns)
__global__ void absmax_kernel(const double *v, int64_t n, unsigned long long *out) {
  double m = 0.0;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    double a = fabs(v[p]);
    if (a > m) m = a;
  }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

// ---------------------------------------------------------------- counting sort
// Markers are split into G contiguous chunks, one per block.  (1) each block
// counts its markers per cell; (2) one block scans the counts in cell-major,
// block-minor order; (3) each block moves its markers to their cell's range.
// Within a warp, markers of a cell keep their order; the order across warps of
// a block is not fixed (the mixed form's results do not depend on marker order:
// the current is an exact integer sum).

__global__ void __launch_bounds__(512) sort_count_kernel(const uint32_t *X, int64_t n, int nc,
                                                         int64_t chunk, uint32_t *H) {
  extern __shared__ __align__(16) unsigned char smraw[];
  uint32_t *cnt = (uint32_t *)smraw;
  for (int i = threadIdx.x; i < nc; i += blockDim.x) cnt[i] = 0;
  __syncthreads();
  int64_t beg = blockIdx.x * chunk, end = beg + chunk < n ? beg + chunk : n;
  for (int64_t base = beg; base < end; base += blockDim.x) {
    int64_t p = base + threadIdx.x;
    bool valid = p < end;
    int key = valid ? cell_of(X[p], nc) : -1;
    warp_rank(cnt, key, valid);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nc; i += blockDim.x) H[(int64_t)i * gridDim.x + blockIdx.x] = cnt[i];
}

// Per cell (one warp each): exclusive prefix of the per-block counts H[c][b]
// over b (written back in place) and the cell's total T[c].
__global__ void sort_cellscan_kernel(uint32_t *H, uint32_t *T, int nc, int G) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const unsigned lane = threadIdx.x & 31u;
  if (warp >= nc) return;
  uint32_t *row = H + (int64_t)warp * G;
  uint32_t carry = 0;
  for (int b0 = 0; b0 < G; b0 += 32) {
    int b = b0 + (int)lane;
    uint32_t v = b < G ? row[b] : 0u;
    uint32_t inc = v;
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t u = __shfl_up_sync(0xffffffffu, inc, o);
      if ((int)lane >= o) inc += u;
    }
    if (b < G) row[b] = carry + inc - v;
    carry += __shfl_sync(0xffffffffu, inc, 31);
  }
  if (lane == 0) T[warp] = carry;
}

// Exclusive scan of T[0..nc) into base[] by one block (nc <= 8192).
__device__ void block_exclusive_scan(const uint32_t *T, uint32_t *base, int nc, uint32_t *tmp) {
  const int per = (nc + blockDim.x - 1) / blockDim.x;
  const int beg = threadIdx.x * per, end = beg + per < nc ? beg + per : nc;
  uint32_t s = 0;
  for (int i = beg; i < end; i++) s += T[i];
  tmp[threadIdx.x] = s;
  __syncthreads();
  for (int o = 1; o < (int)blockDim.x; o <<= 1) {
    uint32_t v = threadIdx.x >= (unsigned)o ? tmp[threadIdx.x - o] : 0u;
    __syncthreads();
    tmp[threadIdx.x] += v;
    __syncthreads();
  }
  uint32_t run = tmp[threadIdx.x] - s;
  for (int i = beg; i < end; i++) {
    base[i] = run;
    run += T[i];
  }
  __syncthreads();
}

// Moves each block's markers (and ids) to their cell's range: the cell base
// (scan of the totals, computed redundantly per block) plus this block's
// prefix within the cell; lanes of a warp with the same cell keep their order.
__global__ void __launch_bounds__(512) sort_move_kernel(Es1dMixBufs src, Es1dMixBufs dst,
                                                        const int64_t *ids_in, int64_t *ids_out,
                                                        int64_t n, int nc, int64_t chunk,
                                                        const uint32_t *H, const uint32_t *T) {
  extern __shared__ __align__(16) unsigned char smraw[];
  uint32_t *off = (uint32_t *)smraw;
  __shared__ uint32_t tmp[512];
  block_exclusive_scan(T, off, nc, tmp);
  for (int i = threadIdx.x; i < nc; i += blockDim.x) off[i] += H[(int64_t)i * gridDim.x + blockIdx.x];
  __syncthreads();
  int64_t beg = blockIdx.x * chunk, end = beg + chunk < n ? beg + chunk : n;
  for (int64_t base = beg; base < end; base += blockDim.x) {
    int64_t p = base + threadIdx.x;
    bool valid = p < end;
    uint32_t X = valid ? src.X[p] : 0u;
    int key = valid ? cell_of(X, nc) : -1;
    const uint32_t dest = PIC_INDEX(warp_rank(off, key, valid), n);
    if (valid) {
      dst.X[dest] = X;
      dst.vh[dest] = src.vh[p];
      dst.vl[dest] = src.vl[p];
      ids_out[dest] = ids_in[p];
    }
  }
}

template <typename F>
void dispatch_mix(const Es1dMixConst &c, F f) {
  using I1 = std::integral_constant<int, 1>;
  using I2 = std::integral_constant<int, 2>;
  using M0 = std::integral_constant<int, 0>;
  using M1 = std::integral_constant<int, 1>;
  using M2 = std::integral_constant<int, 2>;
  using R1 = std::integral_constant<int, 1>;
  using R16 = std::integral_constant<int, 16>;
  using R32 = std::integral_constant<int, 32>;
  using G0 = std::false_type;
  using G1 = std::true_type;
  using F0 = std::false_type;
  using F1 = std::true_type;
  // the FP64 correction for every marker (gamma64) is built for the unsorted
  // mode without the filter; the unsorted kernels with the filter (F1) are
  // separate instantiations, the sorted ones test c.passes at run time
  const bool filt = c.passes > 0;
  auto go = [&](auto O, auto S) {
    if (c.mode == 0 && c.wide && !c.gamma64 && !filt) f(O, S, M0(), R32(), R16(), G0(), F0());
    if (c.mode == 0 && c.wide && !c.gamma64 && filt) f(O, S, M0(), R32(), R16(), G0(), F1());
    if (c.mode == 0 && c.wide && c.gamma64) f(O, S, M0(), R32(), R16(), G1(), F0());
    if (c.mode == 0 && !c.wide && !c.gamma64 && !filt) f(O, S, M0(), R1(), R1(), G0(), F0());
    if (c.mode == 0 && !c.wide && !c.gamma64 && filt) f(O, S, M0(), R1(), R1(), G0(), F1());
    if (c.mode == 0 && !c.wide && c.gamma64) f(O, S, M0(), R1(), R1(), G1(), F0());
    if (c.mode == 1) f(O, S, M1(), R1(), R1(), G0(), F0());
    if (c.mode == 2) f(O, S, M2(), R1(), R1(), G0(), F0());
  };
  if (c.order == 1 && c.scheme == 1) go(I1(), I1());
  if (c.order == 1 && c.scheme == 2) go(I1(), I2());
  if (c.order == 2 && c.scheme == 1) go(I2(), I1());
  if (c.order == 2 && c.scheme == 2) go(I2(), I2());
}

int tile_copies(const Es1dMixConst &c) { return c.mode == 0 && c.wide ? 32 : 1; }
int table_copies(const Es1dMixConst &c) { return c.mode == 0 && c.wide ? 16 : 1; }
size_t npad_host(const Es1dMixConst &c) { return (size_t)c.nc + 3; }
size_t smem_c(const Es1dMixConst &c) {
  return npad_host(c) * (8 * tile_copies(c) + 4 * table_copies(c)) + (c.mode == 2 ? 8 * c.nc : 0);
}
size_t smem_e(const Es1dMixConst &c) {
  return npad_host(c) * (8 * tile_copies(c) + 8 * table_copies(c)) + (c.mode == 2 ? 8 * c.nc : 0);
}
// the fused ESEC1 pass: the tile, the float-pair table and an FP32 table with
// half the copies (the three fit 227 KB at 512 nodes)
int fused_table_copies(const Es1dMixConst &c) { return c.wide ? 8 : 1; }
size_t smem_ec(const Es1dMixConst &c) {
  return npad_host(c) * (8 * tile_copies(c) + 8 * table_copies(c) + 4 * fused_table_copies(c));
}

template <typename F>
void dispatch_fused(const Es1dMixConst &c, F f) {
  using I1 = std::integral_constant<int, 1>;
  using I2 = std::integral_constant<int, 2>;
  using R1 = std::integral_constant<int, 1>;
  using R8 = std::integral_constant<int, 8>;
  using R16 = std::integral_constant<int, 16>;
  using R32 = std::integral_constant<int, 32>;
  auto go = [&](auto O) {
    if (c.wide)
      f(O, R32(), R16(), R8());
    else
      f(O, R1(), R1(), R1());
  };
  if (c.order == 1) go(I1());
  if (c.order == 2) go(I2());
}

}  // namespace

PIC_BOUNDS_READER(bounds_site_es1d_mixed)

cudaError_t es1d_mix_prepare(const Es1dMixConst &c) {
  cudaError_t e = cudaSuccess;
  dispatch_mix(c, [&](auto O, auto S, auto M, auto RT, auto RE, auto G, auto F) {
    constexpr int ORDER = decltype(O)::value, SCHEME = decltype(S)::value;
    constexpr int MODE = decltype(M)::value, NT = decltype(RT)::value, NE = decltype(RE)::value;
    constexpr bool G64 = decltype(G)::value, FILT = decltype(F)::value;
    e = cudaFuncSetAttribute(mix_pass_c_kernel<ORDER, SCHEME, MODE, NT, NE, FILT>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_c(c));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(mix_pass_e_kernel<ORDER, SCHEME, MODE, NT, NE, G64, FILT>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_e(c));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(mix_deposit_initial_kernel<ORDER>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(8 * npad_host(c)));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(mix_charge_kernel<ORDER>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(8 * npad_host(c)));
    if (e == cudaSuccess && c.wide)
      e = cudaFuncSetAttribute(mix_deposit_initial_wide_kernel<ORDER>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)(2 * 32 * 4 * npad_host(c)));
  });
  if (e == cudaSuccess && c.scheme == 1 && c.mode == 0)
    dispatch_fused(c, [&](auto O, auto RT, auto RE, auto RE1) {
      e = cudaFuncSetAttribute(mix_pass_ec_kernel<decltype(O)::value, decltype(RT)::value,
                                                  decltype(RE)::value, decltype(RE1)::value>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_ec(c));
    });
  return e;
}

void es1d_mix_pass_c(const Es1dMixConst &c, const Es1dMixBufs &b, int64_t step_index, int slot,
                     LaunchShape ls, cudaStream_t st) {
  int par = (int)(step_index & 1);
  dispatch_mix(c, [&](auto O, auto S, auto M, auto RT, auto RE, auto, auto F) {
    constexpr int ORDER = decltype(O)::value, SCHEME = decltype(S)::value;
    constexpr int MODE = decltype(M)::value, NT = decltype(RT)::value, NE = decltype(RE)::value;
    launch_dependent(mix_pass_c_kernel<ORDER, SCHEME, MODE, NT, NE, decltype(F)::value>, ls,
                     smem_c(c), st, true, c, b, par, slot - 1, ls.grid);
  });
}

void es1d_mix_pass_e(const Es1dMixConst &c, const Es1dMixBufs &b, int64_t step_index, int slot,
                     LaunchShape ls, cudaStream_t st) {
  int par = (int)(step_index & 1);
  dispatch_mix(c, [&](auto O, auto S, auto M, auto RT, auto RE, auto G, auto F) {
    constexpr int ORDER = decltype(O)::value, SCHEME = decltype(S)::value;
    constexpr int MODE = decltype(M)::value, NT = decltype(RT)::value, NE = decltype(RE)::value;
    launch_dependent(
        mix_pass_e_kernel<ORDER, SCHEME, MODE, NT, NE, decltype(G)::value, decltype(F)::value>,
        ls, smem_e(c), st, true, c, b, par, slot);
  });
}

void es1d_mix_pass_ec(const Es1dMixConst &c, const Es1dMixBufs &b, const RingIO &io,
                      int64_t step_index, int slot, LaunchShape ls, cudaStream_t st) {
  const int par = (int)(step_index & 1);
  dispatch_fused(c, [&](auto O, auto RT, auto RE, auto RE1) {
    launch_dependent(mix_pass_ec_kernel<decltype(O)::value, decltype(RT)::value,
                                        decltype(RE)::value, decltype(RE1)::value>,
                     ls, smem_ec(c), st, true, c, b, io, par, slot, slot - 1, ls.grid);
  });
}

void es1d_mix_deposit_initial(const Es1dMixConst &c, const Es1dMixBufs &b, int parity,
                              LaunchShape ls, cudaStream_t st) {
  if (c.wide && ls.block == 1024) {
    const size_t smw = 2 * 32 * 4 * npad_host(c);
    if (c.order == 1)
      mix_deposit_initial_wide_kernel<1><<<ls.grid, 1024, smw, st>>>(c, b, parity);
    else
      mix_deposit_initial_wide_kernel<2><<<ls.grid, 1024, smw, st>>>(c, b, parity);
    return;
  }
  const size_t sm = 8 * npad_host(c);
  if (c.order == 1)
    mix_deposit_initial_kernel<1><<<ls.grid, 512, sm, st>>>(c, b, parity);
  else
    mix_deposit_initial_kernel<2><<<ls.grid, 512, sm, st>>>(c, b, parity);
}

void es1d_mix_charge(const Es1dMixConst &c, const Es1dMixBufs &b, long long *count,
                     LaunchShape ls, cudaStream_t st) {
  const size_t sm = 8 * npad_host(c);
  if (c.order == 1)
    mix_charge_kernel<1><<<ls.grid, 512, sm, st>>>(c, b, count);
  else
    mix_charge_kernel<2><<<ls.grid, 512, sm, st>>>(c, b, count);
}

void es1d_mix_finalize(const Es1dMixConst &c, const Es1dMixBufs &b, int slot, int nblocks,
                       cudaStream_t st) {
  mix_finalize_kernel<<<1, 32, 0, st>>>(b, c.h, slot, nblocks);
}

void es1d_mix_set_ek(const Es1dMixConst &c, const Es1dMixBufs &b, int parity, cudaStream_t st) {
  mix_set_ek_kernel<<<(c.nc + 255) / 256, 256, 0, st>>>(PSEL(b.E, parity), PSEL(b.Ek, parity), c.nc,
                                                         c.kick);
}

cudaError_t es1d_batch_prepare(size_t smem, int threads) {
  cudaError_t e = cudaSuccess;
  const void *ks[4] = {(const void *)mix_batch_pass_c_kernel<1, 1024>,
                       (const void *)mix_batch_pass_c_kernel<2, 1024>,
                       (const void *)mix_batch_pass_e_kernel<1, 1024>,
                       (const void *)mix_batch_pass_e_kernel<2, 1024>};
  const void *ks_small[4] = {(const void *)mix_batch_pass_c_kernel<1, 256>,
                             (const void *)mix_batch_pass_c_kernel<2, 256>,
                             (const void *)mix_batch_pass_e_kernel<1, 256>,
                             (const void *)mix_batch_pass_e_kernel<2, 256>};
  for (const void *k : threads == 1024 ? ks : ks_small)
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  return e;
}

size_t es1d_mix_smem_max(const Es1dMixConst &c) {
  const size_t a = smem_c(c), b = smem_e(c);
  return a > b ? a : b;
}

size_t es1d_batch_smem(const Es1dMixConst &c, int threads) {
  if (threads == 1024) return es1d_mix_smem_max(c);
  constexpr int RT = BatchLayout<256>::RT, RE = BatchLayout<256>::RE;
  return npad_host(c) * (8 * RT + 8 * RE);  // pass E's (pass C's table is FP32)
}

void es1d_batch_pass_c(const Es1dMixConst *cs, const Es1dMixBufs *bs, const BatchItem *items,
                       int nitems, int scheme, int threads, size_t smem, int64_t step_index,
                       int prev_slot, cudaStream_t st) {
  const int par = (int)(step_index & 1);
  const LaunchShape ls{nitems, threads};
  auto k = threads == 1024 ? (scheme == 1 ? mix_batch_pass_c_kernel<1, 1024>
                                          : mix_batch_pass_c_kernel<2, 1024>)
                           : (scheme == 1 ? mix_batch_pass_c_kernel<1, 256>
                                          : mix_batch_pass_c_kernel<2, 256>);
  launch_dependent(k, ls, smem, st, true, cs, bs, items, par, prev_slot);
}

void es1d_batch_pass_e(const Es1dMixConst *cs, const Es1dMixBufs *bs, const BatchItem *items,
                       int nitems, int scheme, int threads, size_t smem, int64_t step_index,
                       int slot, cudaStream_t st) {
  const int par = (int)(step_index & 1);
  const LaunchShape ls{nitems, threads};
  auto k = threads == 1024 ? (scheme == 1 ? mix_batch_pass_e_kernel<1, 1024>
                                          : mix_batch_pass_e_kernel<2, 1024>)
                           : (scheme == 1 ? mix_batch_pass_e_kernel<1, 256>
                                          : mix_batch_pass_e_kernel<2, 256>);
  launch_dependent(k, ls, smem, st, true, cs, bs, items, par, slot);
}

void es1d_batch_finalize(const Es1dMixConst *cs, const Es1dMixBufs *bs, const int *nblocks,
                         int nruns, int slot, cudaStream_t st) {
  mix_batch_finalize_kernel<<<nruns, 32, 0, st>>>(cs, bs, nblocks, slot);
}

void es1d_batch_gather_stats(const Es1dMixBufs *bs, int nruns, int n, unsigned long long *fb,
                             double *te, cudaStream_t st) {
  mix_batch_gather_kernel<<<nruns, 256, 0, st>>>(bs, n, fb, te);
}

void es1d_mix_from_fp64(const Es1dMixConst &c, const double *x, const double *v, Es1dMixBufs &b,
                        LaunchShape ls, cudaStream_t st) {
  es1d_mix_from_fp64_part(c, x, v, b, 0, c.n, ls, st);
}

void es1d_mix_to_fp64(const Es1dMixConst &c, const Es1dMixBufs &b, double *x, double *v,
                      LaunchShape ls, cudaStream_t st) {
  es1d_mix_to_fp64_part(c, b, x, v, 0, c.n, ls, st);
}

void es1d_mix_from_fp64_part(const Es1dMixConst &c, const double *x, const double *v,
                             Es1dMixBufs &b, int64_t begin, int64_t count, LaunchShape ls,
                             cudaStream_t st) {
  to_mix_kernel<<<ls.grid, 256, 0, st>>>(x + begin, v + begin, count, c.L, c.cxk, b.X + begin,
                                         b.vh + begin, b.vl + begin, b.err);
}

void es1d_mix_to_fp64_part(const Es1dMixConst &c, const Es1dMixBufs &b, double *x, double *v,
                           int64_t begin, int64_t count, LaunchShape ls, cudaStream_t st) {
  from_mix_kernel<<<ls.grid, 256, 0, st>>>(b.X + begin, b.vh + begin, b.vl + begin, count, c.L,
                                           1.0 / c.cxk, x + begin, v + begin);
}

void es1d_mix_kinetic(const Es1dMixConst &c, const Es1dMixBufs &b, double *part, int nblocks,
                      cudaStream_t st) {
  mix_kinetic_kernel<<<nblocks, 512, 0, st>>>(b.vh, b.vl, c.n, c.ke_scale, part);
}

void es1d_absmax(const double *v, int64_t n, unsigned long long *out, LaunchShape ls,
                 cudaStream_t st) {
  absmax_kernel<<<ls.grid, 256, 0, st>>>(v, n, out);
}

void es1d_mix_fused_scan(const Es1dMixConst &c, const Es1dMixBufs &b, int G, cudaStream_t st) {
  const int nkeys = 2 * c.nc;
  sort_cellscan_kernel<<<(nkeys * 32 + 255) / 256, 256, 0, st>>>(b.H, b.T, nkeys, G);
}

int es1d_mix_sort_blocks(const Es1dMixConst &c, int nsm) {
  int64_t want = (c.n + 4095) / 4096;
  int64_t cap = (int64_t)nsm * 2;
  return (int)(want < 1 ? 1 : (want < cap ? want : cap));
}

cudaError_t es1d_mix_sort(const Es1dMixConst &c, const Es1dMixBufs &src, const Es1dMixBufs &dst,
                          const int64_t *ids_in, int64_t *ids_out, uint32_t *H, int G,
                          cudaStream_t st) {
  // H holds nc * G per-block counts followed by nc cell totals
  int64_t chunk = (c.n + G - 1) / G;
  size_t sm = sizeof(uint32_t) * c.nc;
  uint32_t *T = H + (int64_t)c.nc * G;
  sort_count_kernel<<<G, 512, sm, st>>>(src.X, c.n, c.nc, chunk, H);
  sort_cellscan_kernel<<<(c.nc * 32 + 255) / 256, 256, 0, st>>>(H, T, c.nc, G);
  sort_move_kernel<<<G, 512, sm, st>>>(src, dst, ids_in, ids_out, c.n, c.nc, chunk, H, T);
  return cudaGetLastError();
}

}  // namespace pic
