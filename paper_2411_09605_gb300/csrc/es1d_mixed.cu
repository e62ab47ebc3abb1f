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
//     in half a step.  kv is fixed at set-up from the initial velocity range.
//   * v* (Eq. good_translation) is the integer V* = rint(v*), so x* , x^{n+1/2}
//     = X + [V*]_kv and x^{n+1} = X + 2 [V*]_kv are exact integer additions and
//     x^{n+1/2} is exactly the midpoint.
//   * shape weights are exact integers in units of 2^-23 computed from the
//     fraction (partition of unity is exact); gather and deposit at x^{n+1/2}
//     use the same integers, as Eq. exp_econs_simple requires.
//   * current: each marker adds round(V* s_k / 2^r) to node k in 64-bit
//     integers (exact and order independent, r chosen so no sum overflows; the
//     rounding is independent per marker and far below the FP64 energy bound).
//     Lanes of a warp that deposit into the same cell are summed first with
//     warp reductions (cell-sorted markers make most warps single-cell), then
//     one shared-memory atomic per cell group; one global atomic per node per
//     block at the end.
//   * gather #2 reads E^{n+1/2} as a float pair with error-free weight
//     products; d = dt (q/m) E_p and v^dag = v^n + d in float pairs.
//   * Gamma (Eq. opt_solution) from the exact difference
//     |v^{n+1}|^2 - |v^dag|^2 = 2a, a = d (v* - v^n - d/2) (float pairs for
//     the cancelling subtraction, FP32 for the small product):
//     g = Gamma - 1 = t / (1 + sqrt(1 + t)), t = 2a/|v^dag|^2, and
//     v^{n+1} = v^dag + g v^dag in float pairs.  R < 0 is 1 + t < 0.
//   * energies: per-thread float-pair sums of v^2, block sums in FP64.
// Gather #1 and deposit #1 only shape v* (not the conservation), so they use
// plain FP32 weights and the same integer deposit.
// The markers are kept cell-sorted by a counting sort every sort_period steps.
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "ff.cuh"
#include "pic_internal.cuh"

namespace pic {
namespace {

// b.A[i] for a two-entry pointer array in a kernel parameter, selected
// without indexing (indexing would copy the parameter block to local memory)
#define PSEL(A, i) ((i) ? (A)[1] : (A)[0])

__device__ __forceinline__ int cell_of(uint32_t X, int nc) {
  return (int)(((uint64_t)X * (uint32_t)nc) >> 32);
}

// Shape of a marker at X: nodes and weights.  The weights are quantised
// B-spline values, multiples of 2^-23, available both as floats (w, for the
// gathers) and as integers (s = w 2^23, for the deposits); gather and deposit
// at the same X therefore use exactly the same numbers and sum to 1 exactly.
// Order 1: w = (1 - f, f).  Order 2: with f = xi - i0 + 1/2 in [0, 1),
// w = (1/2 (1 - f)^2, 1 - w0 - w2, 1/2 f^2) at nodes i0 - 1, i0, i0 + 1.
template <int ORDER>
struct ShapeMix {
  int key;  // base cell
  int idx[ORDER + 1];
  float w[ORDER + 1];
  int s[ORDER + 1];
  __device__ __forceinline__ ShapeMix(uint32_t X, int nc) {
    uint32_t lo = X * (uint32_t)nc;
    int hi = (int)__umulhi(X, (uint32_t)nc);
    if (ORDER == 2) {
      uint32_t lo2 = lo + 0x80000000u;
      hi += lo2 < lo ? 1 : 0;
      lo = lo2;
      if (hi >= nc) hi -= nc;
    }
    const uint32_t f23 = lo >> 9;
    const float f = __fsub_rn(__uint_as_float(0x3F800000u | f23), 1.0f);  // exact
    key = hi;
    if (ORDER == 1) {
      idx[0] = hi;
      idx[1] = (hi + 1 == nc) ? 0 : hi + 1;
      w[0] = __fsub_rn(1.0f, f);
      w[1] = f;
      s[0] = (1 << 23) - (int)f23;
      s[1] = (int)f23;
    } else {
      const float a = __fsub_rn(1.0f, f);
      const float q0 = __fadd_rn(__fmul_rn(0.5f, __fmul_rn(a, a)), 1.0f);  // 1 + w0 on the 2^-23 grid
      const float q2 = __fadd_rn(__fmul_rn(0.5f, __fmul_rn(f, f)), 1.0f);
      w[0] = __fsub_rn(q0, 1.0f);
      w[ORDER] = __fsub_rn(q2, 1.0f);
      w[1] = __fsub_rn(__fsub_rn(1.0f, w[0]), w[ORDER]);
      s[0] = __float_as_int(q0) & 0x7FFFFF;
      s[ORDER] = __float_as_int(q2) & 0x7FFFFF;
      s[1] = (1 << 23) - s[0] - s[ORDER];
      idx[0] = (hi == 0) ? nc - 1 : hi - 1;
      idx[1] = hi;
      idx[ORDER] = (hi + 1 == nc) ? 0 : hi + 1;
    }
  }
};

__device__ __forceinline__ long long deposit_term(int V, int s, int r) {
  long long t = (long long)V * (long long)s;
  return (t + (1ll << (r - 1))) >> r;
}

// V units -> position units for half a step
__device__ __forceinline__ uint32_t half_shift(int V, int kv) {
  return kv == 0 ? (uint32_t)V : (uint32_t)((V + (1 << (kv - 1))) >> kv);
}

__device__ __forceinline__ int to_fixed(float y, unsigned *err) {
  if (!(fabsf(y) < 2147483520.0f)) atomicOr(err, kErrVelocityRange);
  return __float2int_rn(y);
}

// Adds round(V s_k / 2^r) at the nodes of S to the block tile.  AGG = false:
// one shared atomic per lane and node (markers in arbitrary order spread over
// the tile's banks).  AGG = true (cell-sorted markers): lanes of the warp with
// the same base cell, found by one match instruction, are summed first with
// warp reductions of the two 32-bit halves of each term (|term| < 2^37: the low
// 20 bits and the signed rest sum over 32 lanes without overflow), then one
// lane adds the sum; warps spread over more than 8 cells fall back to per-lane
// atomics.
// The block tile holds each node's integer current as two 32-bit counters:
// the low 16 bits of every added amount (unsigned) and the rest (signed).  An
// amount A is added exactly as (A & 0xFFFF, A >> 16); the tile value is
// hi 2^16 + lo.  Two 32-bit shared atomics run about 2.7 times faster than one
// 64-bit atomic on random addresses, and the rounding shift r is chosen so that
// neither counter can overflow for the markers a block processes.
__device__ __forceinline__ void tile_add(unsigned *Jt, int node, long long a) {
  atomicAdd(&Jt[2 * node], (unsigned)(a & 0xFFFF));
  atomicAdd(&Jt[2 * node + 1], (unsigned)(int)(a >> 16));
}

// Direct deposit: one split atomic per node (markers in arbitrary order spread
// over the tile's banks).
template <int ORDER>
__device__ __forceinline__ void deposit_direct(unsigned *Jt, const ShapeMix<ORDER> &S, int V,
                                               int r) {
#pragma unroll
  for (int k = 0; k <= ORDER; k++) tile_add(Jt, S.idx[k], deposit_term(V, S.s[k], r));
}

// Deposit window for cell-sorted markers: a thread adds the terms of its four
// markers into kWin consecutive nodes starting at the first node of base cell
// `base` (one below the warp's smallest first key), then the warp sums each
// node over its 32
// lanes (two 32-bit halves: 4 terms of |t| < 2^37 per lane, so the low 20
// bits and the signed rest sum without overflow) and one lane adds the 128
// markers' total with a single shared atomic per node.  Markers whose base
// cell falls outside the window use direct atomics.
constexpr int kWin = 6;

template <int ORDER>
struct DepositWindow {
  long long acc[kWin];
  int base;
  // The window starts one cell below the smallest base cell among the warp's
  // first markers (the other three per lane usually fall within two cells).
  __device__ __forceinline__ void start(int key, bool valid) {
#pragma unroll
    for (int w = 0; w < kWin; w++) acc[w] = 0;
    const int m = __reduce_min_sync(0xffffffffu, valid ? key : 0x7fffffff);
    base = m == 0x7fffffff ? 0 : m - 1;
  }
  __device__ __forceinline__ void add(unsigned *Jt, const ShapeMix<ORDER> &S, int V, int r,
                                      bool valid) {
    if (!valid) return;
    const int off = S.key - base;
    const bool inwin = off >= 0 && off <= kWin - 1 - ORDER;
    long long t[ORDER + 1];
#pragma unroll
    for (int k = 0; k <= ORDER; k++) t[k] = deposit_term(V, S.s[k], r);
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
      for (int k = 0; k <= ORDER; k++) tile_add(Jt, S.idx[k], t[k]);
    }
  }
  __device__ __forceinline__ void flush(unsigned *Jt, int nc) {
    int first = (ORDER == 2 ? base - 1 : base) % nc;
    if (first < 0) first += nc;
    const bool lead = (threadIdx.x & 31u) == 0u;
#pragma unroll
    for (int w = 0; w < kWin; w++) {
      if (__any_sync(0xffffffffu, acc[w] != 0)) {
        const int hs = __reduce_add_sync(0xffffffffu, (int)(acc[w] >> 20));
        const int ls = __reduce_add_sync(0xffffffffu, (int)(acc[w] & 0xFFFFF));
        if (lead) {
          int node = first + w;
          if (node >= nc) node -= nc;
          tile_add(Jt, node, ((long long)hs << 20) + (long long)ls);
        }
      }
    }
  }
};

__device__ void block_exclusive_scan(const uint32_t *T, uint32_t *base, int nc, uint32_t *tmp);

// Sort key of a marker after the step: its cell and the sign of its velocity
// (counter-streaming markers of one cell then sit in separate runs).
__device__ __forceinline__ int sort_key(uint32_t X, int V, int nc) {
  return 2 * cell_of(X, nc) + (V > 0 ? 1 : 0);
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

// mean of jscale * J over the grid, identical in every block
__device__ __forceinline__ double block_mean_j(const long long *J, int n, double jscale, double *red) {
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += (double)J[i] * jscale;
  double t = block_sum_d(s, red);
  if (threadIdx.x == 0) red[32] = t / (double)n;
  __syncthreads();
  double m = red[32];
  __syncthreads();
  return m;
}

template <int SCHEME>
__device__ __forceinline__ void build_estar_mix(const Es1dMixConst &c, const double *E, const long long *J1,
                                float *Es, double *red) {
  if (SCHEME == 2) {
    double mean = c.remove_mean ? block_mean_j(J1, c.nc, c.jscale, red) : 0.0;
    double hdt = 0.5 * c.dt;
    for (int i = threadIdx.x; i < c.nc; i += blockDim.x)
      Es[i] = (float)(E[i] - hdt * ((double)J1[i] * c.jscale - mean));
  } else {
    for (int i = threadIdx.x; i < c.nc; i += blockDim.x) Es[i] = (float)E[i];
  }
}

__device__ __forceinline__ void flush_tile_split(const unsigned *Jt, long long *J, int nc) {
  for (int i = threadIdx.x; i < nc; i += blockDim.x) {
    const long long a = (long long)(int)Jt[2 * i + 1] * 65536ll + (long long)Jt[2 * i];
    if (a != 0) atomicAdd((unsigned long long *)&J[i], (unsigned long long)a);
  }
}

__device__ __forceinline__ void flush_tile_i64(const long long *Jt, long long *J, int nc) {
  for (int i = threadIdx.x; i < nc; i += blockDim.x) {
    long long a = Jt[i];
    if (a != 0) atomicAdd((unsigned long long *)&J[i], (unsigned long long)a);
  }
}

__device__ __forceinline__ void finalize_stats_mix(const Es1dMixBufs &b, int slot, int nblocks, double *red) {
  double s = 0.0;
  for (int i = threadIdx.x; i < nblocks; i += blockDim.x) s += b.ke_part[i];
  double t = block_sum_d(s, red);
  if (threadIdx.x == 0) {
    double te = t + b.we[0];
    b.te[slot] = te;
    if (!isfinite(te)) atomicOr(b.err, kErrNonfinite);
  }
}

// Every thread walks groups of 4 consecutive markers (16-byte loads).  All 32
// lanes of a warp stay in the loop together (the warp-level deposit needs
// them), so the trip count is rounded up to whole warps.
__device__ __forceinline__ int64_t warp_trips(int64_t ngroups) {
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t first = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31u);
  return first < ngroups ? (ngroups - first + stride - 1) / stride : 0;
}

// V* = rint(v^n + e) to one V unit: v^n is the pair (vh, vl), and above 2^24
// a float cannot hold every integer, so the sum is split into an integer part
// and an exact remainder.
__device__ __forceinline__ int vstar_fixed(float vh, float vl, float e, unsigned *err) {
  const ff s = two_sum(vh, e);
  const int vi = to_fixed(s.hi, err);
  const float rem = __fadd_rn(__fadd_rn(__fsub_rn(s.hi, (float)vi), s.lo), vl);
  return vi + __float2int_rn(rem);
}

// pass C: x*, E**_p (FP32), v* as the integer V* (stored for pass E),
// x^{n+1/2} and the exact deposit of j^{*,n+1/2}.
template <int ORDER, int SCHEME, int MODE>
__global__ void __launch_bounds__(512) mix_pass_c_kernel(Es1dMixConst c, Es1dMixBufs b, int par,
                                                         int prev_slot, int prev_nblocks) {
  constexpr bool AGG = MODE > 0;
  extern __shared__ __align__(16) unsigned char smraw[];
  unsigned *Jt = (unsigned *)smraw;           // split tile: 2 counters per node
  float *Es = (float *)(Jt + 2 * c.nc);
  uint32_t *hist = (uint32_t *)(Es + c.nc);   // MODE 2: keys of the markers after the step
  __shared__ double red[33];
  build_estar_mix<SCHEME>(c, PSEL(b.E, par), PSEL(b.J1, par), Es, red);
  for (int i = threadIdx.x; i < 2 * c.nc; i += blockDim.x) Jt[i] = 0;
  if (MODE == 2)
    for (int i = threadIdx.x; i < 2 * c.nc; i += blockDim.x) hist[i] = 0;
  if (blockIdx.x == 0) {
    if (SCHEME == 2)
      for (int i = threadIdx.x; i < c.nc; i += blockDim.x) PSEL(b.J1, par ^ 1)[i] = 0;
    if (prev_slot >= 0) finalize_stats_mix(b, prev_slot, prev_nblocks, red);
  }
  __syncthreads();
  const int64_t ngroups = (c.n + 3) >> 2;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t trips = warp_trips(ngroups);
  int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  for (int64_t it = 0; it < trips; it++, g += stride) {
    const bool gv = g < ngroups;
    uint4 X4 = make_uint4(0, 0, 0, 0);
    float4 h4 = make_float4(0.f, 0.f, 0.f, 0.f), l4 = h4;
    if (gv) {
      X4 = reinterpret_cast<const uint4 *>(b.X)[g];
      h4 = reinterpret_cast<const float4 *>(b.vh)[g];
      l4 = reinterpret_cast<const float4 *>(b.vl)[g];
    }
    int Vout[4];
    DepositWindow<ORDER> win;
#pragma unroll
    for (int j = 0; j < 4; j++) {
      const uint32_t X = j == 0 ? X4.x : j == 1 ? X4.y : j == 2 ? X4.z : X4.w;
      const float vh = j == 0 ? h4.x : j == 1 ? h4.y : j == 2 ? h4.z : h4.w;
      const float vl = j == 0 ? l4.x : j == 1 ? l4.y : j == 2 ? l4.z : l4.w;
      const bool valid = gv && (4 * g + j < c.n);
      const int Vn = to_fixed(vh, b.err);
      const ShapeMix<ORDER> Sx(X + half_shift(Vn, c.kv), c.nc);
      float e = 0.0f;
#pragma unroll
      for (int k = 0; k <= ORDER; k++) e = __fmaf_rn(Sx.w[k], Es[Sx.idx[k]], e);
      const int Vs = vstar_fixed(vh, vl, __fmul_rn(c.e_scale, e), b.err);
      const uint32_t hs = half_shift(Vs, c.kv);
      const ShapeMix<ORDER> Sh(X + hs, c.nc);
      if (AGG) {
        if (j == 0) win.start(Sh.key, valid);
        win.add(Jt, Sh, Vs, c.rshift, valid);
      } else if (valid) {
        deposit_direct<ORDER>(Jt, Sh, Vs, c.rshift);
      }
      if (MODE == 2) warp_rank(hist, sort_key(X + 2u * hs, Vs, c.nc), valid);
      Vout[j] = Vs;
    }
    if (AGG) win.flush(Jt, c.nc);
    if (gv) reinterpret_cast<int4 *>(b.Vs)[g] = make_int4(Vout[0], Vout[1], Vout[2], Vout[3]);
  }
  __syncthreads();
  flush_tile_split(Jt, PSEL(b.J2, par), c.nc);
  if (MODE == 2)
    for (int i = threadIdx.x; i < 2 * c.nc; i += blockDim.x)
      b.H[(int64_t)i * gridDim.x + blockIdx.x] = hist[i];
}

// pass E: E^{n+1}, E^{n+1/2} (float pairs) in the prologue; per marker the
// gather at x^{n+1/2} = X + [V*], v^dag, Gamma, x^{n+1}, v^{n+1}, the kinetic
// energy and (ESEC2) the next step's x* and j^{n+1,*} deposit.
template <int ORDER, int SCHEME, int MODE>
__global__ void __launch_bounds__(512) mix_pass_e_kernel(Es1dMixConst c, Es1dMixBufs b, int par,
                                                         int slot) {
  constexpr bool AGG = MODE > 0;
  extern __shared__ __align__(16) unsigned char smraw[];
  unsigned *Jt = (unsigned *)smraw;           // split tile: 2 counters per node
  float2 *Eh2 = (float2 *)(Jt + 2 * c.nc);
  uint32_t *off = (uint32_t *)(Eh2 + c.nc);   // MODE 2: next free slot of each key
  __shared__ double red[33];
  if (MODE == 2) {
    __shared__ uint32_t tmp[512];
    block_exclusive_scan(b.T, off, 2 * c.nc, tmp);
    for (int i = threadIdx.x; i < 2 * c.nc; i += blockDim.x)
      off[i] += b.H[(int64_t)i * gridDim.x + blockIdx.x];
  }
  const double *E = PSEL(b.E, par);
  const long long *J2 = PSEL(b.J2, par);
  double mean2 = c.remove_mean ? block_mean_j(J2, c.nc, c.jscale, red) : 0.0;
  double we_loc = 0.0;
  for (int i = threadIdx.x; i < c.nc; i += blockDim.x) {
    double en = E[i] - c.dt * ((double)J2[i] * c.jscale - mean2);
    ff s = ff_from_double(0.5 * (E[i] + en));
    Eh2[i] = make_float2(s.hi, s.lo);
    Jt[2 * i] = 0;
    Jt[2 * i + 1] = 0;
    if (blockIdx.x == 0) {
      PSEL(b.E, par ^ 1)[i] = en;
      PSEL(b.J2, par ^ 1)[i] = 0;
      we_loc += en * en;
    }
  }
  if (blockIdx.x == 0) {
    double t = block_sum_d(we_loc, red);
    if (threadIdx.x == 0) b.we[0] = 0.5 * c.h * t;
  }
  __syncthreads();

  float ke_hi = 0.0f, ke_lo = 0.0f;
  unsigned nfb = 0;
  const int64_t ngroups = (c.n + 3) >> 2;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t trips = warp_trips(ngroups);
  int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  for (int64_t it = 0; it < trips; it++, g += stride) {
    const bool gv = g < ngroups;
    uint4 X4 = make_uint4(0, 0, 0, 0);
    float4 h4 = make_float4(0.f, 0.f, 0.f, 0.f), l4 = h4;
    int4 V4 = make_int4(0, 0, 0, 0);
    if (gv) {
      X4 = reinterpret_cast<const uint4 *>(b.X)[g];
      h4 = reinterpret_cast<const float4 *>(b.vh)[g];
      l4 = reinterpret_cast<const float4 *>(b.vl)[g];
      V4 = reinterpret_cast<const int4 *>(b.Vs)[g];
    }
    uint32_t Xo[4];
    float ho[4], lo[4];
    DepositWindow<ORDER> win;
#pragma unroll
    for (int j = 0; j < 4; j++) {
      const uint32_t X = j == 0 ? X4.x : j == 1 ? X4.y : j == 2 ? X4.z : X4.w;
      const float vh = j == 0 ? h4.x : j == 1 ? h4.y : j == 2 ? h4.z : h4.w;
      const float vl = j == 0 ? l4.x : j == 1 ? l4.y : j == 2 ? l4.z : l4.w;
      const int Vs = j == 0 ? V4.x : j == 1 ? V4.y : j == 2 ? V4.z : V4.w;
      const bool valid = gv && (4 * g + j < c.n);
      const uint32_t hs = half_shift(Vs, c.kv);
      // gather #2: E^{n+1/2}_p as a float pair from exact weight products
      const ShapeMix<ORDER> Sh(X + hs, c.nc);
      float ph[ORDER + 1], pl = 0.0f;
#pragma unroll
      for (int k = 0; k <= ORDER; k++) {
        const float2 eh = Eh2[Sh.idx[k]];
        const ff p = two_prod(eh.x, Sh.w[k]);
        ph[k] = p.hi;
        pl = __fadd_rn(pl, __fmaf_rn(eh.y, Sh.w[k], p.lo));
      }
      ff Ep = two_sum(ph[0], ph[1]);
      pl = __fadd_rn(pl, Ep.lo);
      if (ORDER == 2) {
        Ep = two_sum(Ep.hi, ph[ORDER]);
        pl = __fadd_rn(pl, Ep.lo);
      }
      Ep = fast_two_sum(Ep.hi, pl);
      const ff d = ff_mul(Ep, c.cd);        // dt (q/m) E^{n+1/2}_p, V units
      const ff v = {vh, vl};
      const ff vd = ff_add(v, d);           // v^dag
      // b = v* - v^n - d/2 with v* = V* exactly (two exact float parts)
      const int vlo8 = Vs & 0xFF;
      const float vst_hi = (float)(Vs - vlo8);
      const float vst_lo = __fsub_rn(__uint_as_float(0x4B000000u | (unsigned)vlo8), 8388608.0f);
      const ff q1 = two_sum(vst_hi, -vh);
      const float q1l = __fadd_rn(q1.lo, __fsub_rn(vst_lo, vl));
      const ff q2 = two_sum(q1.hi, __fmul_rn(-0.5f, d.hi));
      const float bq = __fadd_rn(q2.hi, __fadd_rn(q2.lo, __fadd_rn(q1l, __fmul_rn(-0.5f, d.lo))));
      const float a = __fmul_rn(d.hi, bq);  // |v^{n+1}|^2 - |v^dag|^2 = 2a
      const float vd2 = __fmul_rn(vd.hi, vd.hi);
      ff vn = vd;
      if (c.gamma_on && valid) {
        const float t = __fdiv_rn(__fmul_rn(2.0f, a), vd2);
        const float op = __fadd_rn(1.0f, t);
        if (vd2 > 0.0f && op >= 0.0f && fabsf(t) < 1e30f) {
          // Gamma - 1 = sqrt(1 + t) - 1 = t / (1 + sqrt(1 + t)): for |t| < 2^-8 the
          // series t/2 - t^2/8 + t^3/16 - 5t^4/128 (relative error < 2^-33),
          // otherwise correctly rounded sqrt and divide
          float gm;
          if (fabsf(t) < 0.00390625f) {
            gm = __fmul_rn(t, __fmaf_rn(t, __fmaf_rn(t, __fmaf_rn(t, -0.0390625f, 0.0625f),
                                                     -0.125f), 0.5f));
          } else {
            gm = __fdiv_rn(t, __fadd_rn(1.0f, __fsqrt_rn(op)));
          }
          ff p = two_prod(vd.hi, gm);
          p.lo = __fmaf_rn(vd.lo, gm, p.lo);
          vn = ff_add(vd, p);
        } else {
          nfb++;
        }
      }
      if (valid) {
        ff s2 = two_prod(vn.hi, vn.hi);
        s2.lo = __fmaf_rn(__fmul_rn(2.0f, vn.hi), vn.lo, s2.lo);
        const ff acc = two_sum(ke_hi, s2.hi);
        ke_hi = acc.hi;
        ke_lo = __fadd_rn(ke_lo, __fadd_rn(acc.lo, s2.lo));
        if (!isfinite(vn.hi)) atomicOr(b.err, kErrNonfinite);
      }
      const uint32_t Xn = X + 2u * hs;
      if (SCHEME == 2) {
        const int Vn1 = to_fixed(vn.hi, b.err);
        const ShapeMix<ORDER> S1(Xn + half_shift(Vn1, c.kv), c.nc);
        if (AGG) {
          if (j == 0) win.start(S1.key, valid);
          win.add(Jt, S1, Vn1, c.rshift, valid);
        } else if (valid) {
          deposit_direct<ORDER>(Jt, S1, Vn1, c.rshift);
        }
      }
      if (MODE == 2) {
        // sort on write: the marker's slot in key order, from pass C's counts
        const uint32_t dst = warp_rank(off, sort_key(Xn, Vs, c.nc), valid);
        if (valid) {
          b.Xo[dst] = Xn;
          b.vho[dst] = vn.hi;
          b.vlo[dst] = vn.lo;
          if (b.ids) b.ido[dst] = b.ids[4 * g + j];
        }
      }
      Xo[j] = valid ? Xn : X;
      ho[j] = valid ? vn.hi : vh;
      lo[j] = valid ? vn.lo : vl;
    }
    if (AGG && SCHEME == 2) win.flush(Jt, c.nc);
    if (MODE != 2 && gv) {
      reinterpret_cast<uint4 *>(b.X)[g] = make_uint4(Xo[0], Xo[1], Xo[2], Xo[3]);
      reinterpret_cast<float4 *>(b.vh)[g] = make_float4(ho[0], ho[1], ho[2], ho[3]);
      reinterpret_cast<float4 *>(b.vl)[g] = make_float4(lo[0], lo[1], lo[2], lo[3]);
    }
  }
  for (int o = 16; o > 0; o >>= 1) nfb += __shfl_xor_sync(0xffffffffu, nfb, o);
  if ((threadIdx.x & 31) == 0 && nfb) atomicAdd(&b.fallback[slot], (unsigned long long)nfb);
  double t = block_sum_d((double)ke_hi + (double)ke_lo, red);
  if (threadIdx.x == 0) b.ke_part[blockIdx.x] = c.ke_scale * t;
  if (SCHEME == 2) {
    __syncthreads();
    flush_tile_split(Jt, PSEL(b.J1, par ^ 1), c.nc);
  }
}

template <int ORDER>
__global__ void __launch_bounds__(512) mix_deposit_initial_kernel(Es1dMixConst c, Es1dMixBufs b,
                                                                  int par) {
  extern __shared__ __align__(16) unsigned char smraw[];
  long long *Jt = (long long *)smraw;
  for (int i = threadIdx.x; i < c.nc; i += blockDim.x) Jt[i] = 0;
  __syncthreads();
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < c.n;
       p += (int64_t)gridDim.x * blockDim.x) {
    int Vn = to_fixed(b.vh[p], b.err);
    ShapeMix<ORDER> S(b.X[p] + half_shift(Vn, c.kv), c.nc);
#pragma unroll
    for (int k = 0; k <= ORDER; k++)
      atomicAdd((unsigned long long *)&Jt[S.idx[k]],
                (unsigned long long)deposit_term(Vn, S.s[k], c.rshift));
  }
  __syncthreads();
  flush_tile_i64(Jt, PSEL(b.J1, par), c.nc);
}

// Charge of the markers for the initial Poisson solve: the integer weights
// summed exactly per node (order independent), in units of 2^-23.
template <int ORDER>
__global__ void __launch_bounds__(512) mix_charge_kernel(Es1dMixConst c, Es1dMixBufs b,
                                                         long long *count) {
  extern __shared__ __align__(16) unsigned char smraw[];
  long long *Jt = (long long *)smraw;
  for (int i = threadIdx.x; i < c.nc; i += blockDim.x) Jt[i] = 0;
  __syncthreads();
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < c.n;
       p += (int64_t)gridDim.x * blockDim.x) {
    ShapeMix<ORDER> S(b.X[p], c.nc);
#pragma unroll
    for (int k = 0; k <= ORDER; k++)
      atomicAdd((unsigned long long *)&Jt[S.idx[k]], (unsigned long long)S.s[k]);
  }
  __syncthreads();
  flush_tile_i64(Jt, count, c.nc);
}

__global__ void mix_finalize_kernel(Es1dMixBufs b, int slot, int nblocks) {
  __shared__ double red[33];
  finalize_stats_mix(b, slot, nblocks, red);
}

// FP64 (x, v) <-> (X, vh, vl) with v stored in V units (v * cxk)
__global__ void to_mix_kernel(const double *x, const double *v, int64_t n, double L, double cxk,
                              uint32_t *X, float *vh, float *vl, unsigned *err) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    double xx = x[p], vv = v[p] * cxk;
    if (!(xx >= 0.0 && xx < L)) atomicOr(err, kErrBounds);
    if (!isfinite(vv)) atomicOr(err, kErrNonfinite);
    if (!(fabs(vv) < 2147483520.0)) atomicOr(err, kErrVelocityRange);
    double u = xx / L * 4294967296.0;
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
  const unsigned lane = threadIdx.x & 31u;
  int64_t beg = blockIdx.x * chunk, end = beg + chunk < n ? beg + chunk : n;
  for (int64_t base = beg; base < end; base += blockDim.x) {
    int64_t p = base + threadIdx.x;
    bool valid = p < end;
    uint32_t X = valid ? src.X[p] : 0u;
    int key = valid ? cell_of(X, nc) : -1;
    const uint32_t dest = warp_rank(off, key, valid);
    if (valid) {
      dst.X[dest] = X;
      dst.vh[dest] = src.vh[p];
      dst.vl[dest] = src.vl[p];
      ids_out[dest] = ids_in[p];
    }
  }
}

template <typename F>
void dispatch_mix(int order, int scheme, int mode, F f) {
  using I1 = std::integral_constant<int, 1>;
  using I2 = std::integral_constant<int, 2>;
  using M0 = std::integral_constant<int, 0>;
  using M1 = std::integral_constant<int, 1>;
  using M2 = std::integral_constant<int, 2>;
  auto go = [&](auto O, auto S) {
    if (mode == 0) f(O, S, M0());
    if (mode == 1) f(O, S, M1());
    if (mode == 2) f(O, S, M2());
  };
  if (order == 1 && scheme == 1) go(I1(), I1());
  if (order == 1 && scheme == 2) go(I1(), I2());
  if (order == 2 && scheme == 1) go(I2(), I1());
  if (order == 2 && scheme == 2) go(I2(), I2());
}

size_t smem_c(const Es1dMixConst &c) { return (size_t)c.nc * (8 + 4 + (c.mode == 2 ? 8 : 0)); }
size_t smem_e(const Es1dMixConst &c) { return (size_t)c.nc * (8 + 8 + (c.mode == 2 ? 8 : 0)); }

}  // namespace

cudaError_t es1d_mix_prepare(const Es1dMixConst &c) {
  cudaError_t e = cudaSuccess;
  dispatch_mix(c.order, c.scheme, c.mode, [&](auto O, auto S, auto M) {
    constexpr int ORDER = decltype(O)::value, SCHEME = decltype(S)::value;
    constexpr int MODE = decltype(M)::value;
    e = cudaFuncSetAttribute(mix_pass_c_kernel<ORDER, SCHEME, MODE>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_c(c));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(mix_pass_e_kernel<ORDER, SCHEME, MODE>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_e(c));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(mix_deposit_initial_kernel<ORDER>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(8 * c.nc));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(mix_charge_kernel<ORDER>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(8 * c.nc));
  });
  return e;
}

void es1d_mix_pass_c(const Es1dMixConst &c, const Es1dMixBufs &b, int64_t step_index, int slot,
                     LaunchShape ls, cudaStream_t st) {
  int par = (int)(step_index & 1);
  dispatch_mix(c.order, c.scheme, c.mode, [&](auto O, auto S, auto M) {
    constexpr int ORDER = decltype(O)::value, SCHEME = decltype(S)::value;
    constexpr int MODE = decltype(M)::value;
    mix_pass_c_kernel<ORDER, SCHEME, MODE><<<ls.grid, ls.block, smem_c(c), st>>>(c, b, par,
                                                                                 slot - 1, ls.grid);
  });
}

void es1d_mix_pass_e(const Es1dMixConst &c, const Es1dMixBufs &b, int64_t step_index, int slot,
                     LaunchShape ls, cudaStream_t st) {
  int par = (int)(step_index & 1);
  dispatch_mix(c.order, c.scheme, c.mode, [&](auto O, auto S, auto M) {
    constexpr int ORDER = decltype(O)::value, SCHEME = decltype(S)::value;
    constexpr int MODE = decltype(M)::value;
    mix_pass_e_kernel<ORDER, SCHEME, MODE><<<ls.grid, ls.block, smem_e(c), st>>>(c, b, par, slot);
  });
}

void es1d_mix_deposit_initial(const Es1dMixConst &c, const Es1dMixBufs &b, int parity,
                              LaunchShape ls, cudaStream_t st) {
  if (c.order == 1)
    mix_deposit_initial_kernel<1><<<ls.grid, ls.block, 8 * c.nc, st>>>(c, b, parity);
  else
    mix_deposit_initial_kernel<2><<<ls.grid, ls.block, 8 * c.nc, st>>>(c, b, parity);
}

void es1d_mix_charge(const Es1dMixConst &c, const Es1dMixBufs &b, long long *count,
                     LaunchShape ls, cudaStream_t st) {
  if (c.order == 1)
    mix_charge_kernel<1><<<ls.grid, ls.block, 8 * c.nc, st>>>(c, b, count);
  else
    mix_charge_kernel<2><<<ls.grid, ls.block, 8 * c.nc, st>>>(c, b, count);
}

void es1d_mix_finalize(const Es1dMixBufs &b, int slot, int nblocks, cudaStream_t st) {
  mix_finalize_kernel<<<1, 256, 0, st>>>(b, slot, nblocks);
}

void es1d_mix_from_fp64(const Es1dMixConst &c, const double *x, const double *v, Es1dMixBufs &b,
                        LaunchShape ls, cudaStream_t st) {
  to_mix_kernel<<<ls.grid, 256, 0, st>>>(x, v, c.n, c.L, c.cxk, b.X, b.vh, b.vl, b.err);
}

void es1d_mix_to_fp64(const Es1dMixConst &c, const Es1dMixBufs &b, double *x, double *v,
                      LaunchShape ls, cudaStream_t st) {
  from_mix_kernel<<<ls.grid, 256, 0, st>>>(b.X, b.vh, b.vl, c.n, c.L, 1.0 / c.cxk, x, v);
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
