// 1D2V electromagnetic step with a pseudospectral field solve, FP64 form:
// EMEC(LI), the Crank-Nicolson scheme of Sec. 4.1 (Eq. EMbasic), and
// EMEC(PSATD) of Sec. 4.3 (Eq. EM_PSATD), in the geometry of the paper's
// Weibel test: one periodic coordinate y, velocities (vx, vy), E = (Ex, Ey),
// B = Bz, all on n collocated nodes.  With only d/dy non-zero,
//   dEx/dt = c^2 dBz/dy - jx,   dEy/dt = -jy,   dBz/dt = dEx/dy,
// so Ey's update is pointwise and only the pair (Ex, Bz) needs a transform.
// d/dy multiplies Fourier mode m by i kk, kk = 2 pi m / L (m signed); the
// Nyquist mode gets kk = 0, which keeps the discrete curl antisymmetric
// (Eq. curlIdentity), so both energy proofs hold exactly.
//
// Two launches per step, like the other particle paths:
//   pass C  every block: E*, B* tables in shared memory; per marker y*,
//           E**, B**, the closed-form v* of v* = v^n + dt/2 (q/m)(E** + v* x B**),
//           y^{n+1/2}, deposit of j^{*,n+1/2}.  The block that finishes last
//           does the full field step: (E^{n+1}, B^{n+1}) by Crank-Nicolson or
//           PSATD over dt with j^{*,n+1/2}, the E that v^dag uses (E^{n+1/2},
//           or PSATD's time average <E>) and B^{n+1/2} = (B^n + B^{n+1})/2.
//   pass E  every block: v* as pass C stored it and y^{n+1/2} formed with the
//           same rounding (cheaper than recomputing on the FP64 pipe), the
//           gather of that E and B^{n+1/2}, v^dag, Gamma (Eq. opt_solution;
//           fallback counted), y^{n+1}, v^{n+1}, the kinetic-energy partial and
//           (ESEC2 form) the deposit of j^{n+1,*} at y^{n+1} + dt/2 vy^{n+1}.
//           The block that finishes last writes TE of the new state and the
//           next step's half step: (E*, B*) from E^{n+1}, B^{n+1}, j^{n+1,*}
//           by the explicit half step (Crank-Nicolson scheme) or PSATD over
//           dt/2.
// "Last block" is a counter taken with one atomic per block after a memory
// fence; nothing waits.  The field solve is an in-block radix-2 FFT over n
// (a power of two, 4 <= n <= 1024) in shared memory, with its twiddles and
// the PSATD per-mode coefficients tabulated once at set-up.
//
// Mixed form (Em1dMixConst / Em1dMixBufs): the same two passes and the same
// FP64 field solve, with the per-marker work of the 1D1V mixed form: y as a
// 32-bit fixed-point word, (vx, vy) as float pairs in V units, v* as the
// integers (V*x, V*y), quantised shape weights, and the currents as exact
// integer sums (split 32-bit counters in per-lane tile copies, one int64
// global atomic per node and block); the last block hands the field solve
// jscale times those sums.  Gather #1 (E*, B* at y*) runs in FP32; gather #2
// reads the E of v^dag as float pairs with error-free weight products, and the
// magnetic part dt (q/m) (V*y Bz, -V*x Bz) is formed in float pairs of the
// exact V*, so it does no work; Gamma from the exact bracket
// Delta . (V* - v^n - Delta/2), as in the 1D1V mixed form.
//
// Deposits: each lane of a block adds into its own copy of the block's
// current tile (rt copies, laid out [node][component][copy], rt up to 32 as
// shared memory allows), so FP64 shared atomics rarely meet; the flush sums
// the copies and adds the block's tile into one of kJSlices slices of the
// global current, which spreads the blocks' global atomics over kJSlices
// addresses per node; the field solve sums the slices.
#include <cuda_runtime.h>

#include "es1d_fp64_common.cuh"
#include "ff.cuh"
#include "mixed_common.cuh"
#include "pic_internal.cuh"
#include "spectral_common.cuh"

namespace pic {
namespace {

constexpr int kEm1Threads = 256;

__device__ __forceinline__ int species_of1(const Em1dConst &c, int64_t p) {
  int s = 0;
  while (s < c.nsp - 1 && p >= c.sp_end[s]) s++;
  return s;
}

// y*, E**, B**, v*, y^{n+1/2} with explicitly rounded operations: pass C
// deposits at exactly the y^{n+1/2} and v* that pass E gathers at.
// The shape at y* = y + dt/2 vy, with the rounding every kernel of this form
// uses for it.
template <int ORDER>
__device__ __forceinline__ Shape64<ORDER> em1d_shape_at_ystar(const Em1dConst &c, double y,
                                                              double vy, unsigned *err) {
  const double ys = wrap_periodic(__fma_rn(0.5 * c.dt, vy, y), c.L, err);
  return Shape64<ORDER>(__dmul_rn(ys, c.inv_h), c.n);
}

// E**, B**, v*, y^{n+1/2} from the shape S at y*
template <int ORDER>
__device__ __forceinline__ void em1d_half_push(const Em1dConst &c, const double *Esx,
                                               const double *Esy, const double *Bs,
                                               const Shape64<ORDER> &S, double y, double vx,
                                               double vy, double qm, unsigned *err, double &vsx,
                                               double &vsy, double &yh) {
  const double hdt = 0.5 * c.dt;
  const double ex = S.gather(Esx), ey = S.gather(Esy), bz = S.gather(Bs);
  const double a = __dmul_rn(hdt, qm);
  const double ux = __fma_rn(a, ex, vx), uy = __fma_rn(a, ey, vy);
  const double t = __dmul_rn(a, bz);
  const double inv = __ddiv_rn(1.0, __fma_rn(t, t, 1.0));
  vsx = __dmul_rn(__fma_rn(uy, t, ux), inv);
  vsy = __dmul_rn(__fma_rn(-ux, t, uy), inv);
  yh = wrap_periodic(__fma_rn(hdt, vsy, y), c.L, err);
}

// ---------------------------------------------------------------- field solve

// Signed wavenumber of mode k (0 for the Nyquist mode).
__device__ __forceinline__ double mode_kk(const Em1dConst &c, int k) {
  if (2 * k == c.n) return 0.0;
  const int m = (k <= c.n / 2) ? k : k - c.n;
  return 2.0 * 3.141592653589793 * (double)m / c.L;
}

// Sum of the kJSlices slices of a sliced current at entry i of [2][n].
__device__ __forceinline__ double jsum(const double *J, int n, int i) {
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kJSlices; k++) s += __ldcg(J + (size_t)k * 2 * n + i);
  return s;
}

// Per-mode coefficients of the three field advances over tau with j fixed.
// Each maps the transverse spectra (Ex, Bz, jx) of mode k to
//   Ex' = a1 Ex + i a2 Bz - a3 jx,   Bz' = a1 Bz + i a4 Ex - i a5 jx,
// and PSATD's time average <Ex> = b1 Ex + i b2 Bz - b3 jx:
//   explicit Euler (the half step of Eq. EMbasic): a = (1, c^2 kk tau, tau, kk tau, 0);
//   Crank-Nicolson (its full step), al = kk tau / 2, d = 1 + c^2 al^2:
//     a = ((1 - c^2 al^2)/d, 2 c^2 al / d, tau / d, 2 al / d, al tau / d);
//   PSATD (Eq. PSATDformula with Delta t -> tau), x = |kk| c tau, s = sign kk:
//     a = (cos x, s c sin x, sin x / (|kk| c), s sin x / c, s (1 - cos x)/(|kk| c^2)),
//     b = (sin x / x, s (1 - cos x)/(|kk| tau), (1 - cos x)/(kk^2 c^2 tau)),
//   and for kk = 0 the limits a = (1, 0, tau, 0, 0), b = (1, 0, tau / 2).
// 1 - cos x is formed as 2 sin^2 (x/2).
__device__ void mode_coefficients(const Em1dConst &c, int kind, double tau, int k, double *q) {
  const double kk = mode_kk(c, k), c2 = c.c2;
  for (int i = 0; i < kEm1Coef; i++) q[i] = 0.0;
  if (kind == 0) {
    q[0] = 1.0;
    q[1] = c2 * kk * tau;
    q[2] = tau;
    q[3] = kk * tau;
  } else if (kind == 1) {
    const double al = 0.5 * kk * tau, d = 1.0 + c2 * al * al;
    q[0] = (1.0 - c2 * al * al) / d;
    q[1] = 2.0 * c2 * al / d;
    q[2] = tau / d;
    q[3] = 2.0 * al / d;
    q[4] = al * tau / d;
  } else if (kk == 0.0) {
    q[0] = 1.0;
    q[2] = tau;
    q[5] = 1.0;
    q[7] = 0.5 * tau;
  } else {
    const double ka = fabs(kk), sg = kk > 0.0 ? 1.0 : -1.0, cc = c.c, x = ka * cc * tau;
    double S, C, sh, ch;
    sincos(x, &S, &C);
    sincos(0.5 * x, &sh, &ch);
    const double omc = 2.0 * sh * sh;
    q[0] = C;
    q[1] = sg * S * cc;
    q[2] = S / (ka * cc);
    q[3] = sg * S / cc;
    q[4] = sg * omc / (ka * c2);
    q[5] = S / x;
    q[6] = sg * omc / (ka * tau);
    q[7] = omc / (ka * ka * c2 * tau);
  }
}

// Field advance over tau with j held fixed, from the per-mode coefficients cf
// [n/2 + 1][kEm1Coef] of mode_coefficients; psatd selects <E> (else the
// average (E + Eo)/2) for Ea.  Reads E [2][n], B [n] and the sliced J
// [kJSlices][2][n] from global memory (written by other blocks of this
// kernel: read through L2), writes Eo, Bo and, when non-null, Ea (the E of
// v^dag) and Bh = (B + Bo)/2.  Z1: shared scratch of at least 9n + 8 doubles
// (the two transforms, the twiddles and the coefficients, loaded together).
__device__ void field_advance(const Em1dConst &c, bool psatd, double tau, const double *cf_g,
                              const double2 *tw_g, const double *E, const double *B,
                              const double *J, double *Eo, double *Bo, double *Ea, double *Bh,
                              double2 *Z1) {
  const int n = c.n;
  double2 *Z2 = Z1 + n, *tw = Z1 + 2 * n;
  double *cf = (double *)(tw + n / 2);
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    Z1[i] = make_double2(__ldcg(E + i), __ldcg(B + i));
    Z2[i] = make_double2(jsum(J, n, i), 0.0);
  }
  for (int i = threadIdx.x; i < n / 2; i += blockDim.x) tw[i] = __ldg(tw_g + i);
  for (int i = threadIdx.x; i < kEm1Coef * (n / 2 + 1); i += blockDim.x) cf[i] = __ldg(cf_g + i);
  __syncthreads();
  block_fft(Z1, n, c.log2n, -1, tw);
  block_fft(Z2, n, c.log2n, -1, tw);
  // modes k and n - k by one thread: Z1 holds Ex + i Bz, so
  // Ex_k = (Z_k + conj Z_{n-k}) / 2 and Bz_k = (Z_k - conj Z_{n-k}) / (2i)
  for (int k = threadIdx.x; k <= n / 2; k += blockDim.x) {
    const int k2 = (n - k) & (n - 1);
    const double2 zk = Z1[k], zm = Z1[k2];
    const double2 A = cscale(0.5, cadd(zk, cconj(zm)));
    const double2 Bm = cscale(0.5, {zk.y + zm.y, zm.x - zk.x});   // (zk - conj zm) / (2i)
    const double2 Jk = Z2[k];
    const double *q = cf + kEm1Coef * k;
    const double2 Ox = csub(cadd(cscale(q[0], A), cscale(q[1], ctimes_i(Bm))), cscale(q[2], Jk));
    const double2 Ob = csub(cadd(cscale(q[0], Bm), cscale(q[3], ctimes_i(A))),
                            cscale(q[4], ctimes_i(Jk)));
    const double2 Ax =
        csub(cadd(cscale(q[5], A), cscale(q[6], ctimes_i(Bm))), cscale(q[7], Jk));
    // repack Ex' + i Bz' (and <Ex>) for the inverse transform; mode n - k holds
    // the conjugates
    Z1[k] = cadd(Ox, ctimes_i(Ob));
    Z2[k] = Ax;
    if (k2 != k) {
      Z1[k2] = cadd(cconj(Ox), ctimes_i(cconj(Ob)));
      Z2[k2] = cconj(Ax);
    }
  }
  __syncthreads();
  block_fft(Z1, n, c.log2n, 1, tw);
  if (psatd && Ea) block_fft(Z2, n, c.log2n, 1, tw);
  const double inv_n = 1.0 / (double)n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double ex = __ldcg(E + i), ey = __ldcg(E + n + i), bz = __ldcg(B + i);
    const double jy = jsum(J, n, n + i);
    const double exn = Z1[i].x * inv_n, bzn = Z1[i].y * inv_n;
    Eo[i] = exn;
    Eo[n + i] = ey - tau * jy;
    Bo[i] = bzn;
    if (Ea) {
      Ea[i] = psatd ? Z2[i].x * inv_n : 0.5 * (ex + exn);
      Ea[n + i] = ey - 0.5 * tau * jy;
    }
    if (Bh) Bh[i] = 0.5 * (bz + bzn);
  }
  __syncthreads();
}

__device__ __forceinline__ double marker_qw(const Em1dConst &c, const Em1dBufs &b, int s,
                                            int64_t p) {
  return b.w ? c.q_h[s] * b.w[p] : c.qw_h[s];
}

// ------------------------------------------------------------ current tiles

__device__ __forceinline__ void clear_tile(double *Jt, int len) {
  for (int i = threadIdx.x; i < len; i += blockDim.x) Jt[i] = 0.0;
}

// (ax, ay) S(y_h - y) into this lane's copy of the tile [n][2][rt].
template <int ORDER>
__device__ __forceinline__ void tile_deposit(double *Jt, int rt, const Shape64<ORDER> &S,
                                             double ax, double ay) {
  const int l = threadIdx.x & (rt - 1);
#pragma unroll
  for (int k = 0; k <= ORDER; k++) {
    double *q = Jt + (size_t)S.idx[k] * 2 * rt + l;
    atomicAdd(q, ax * S.w[k]);
    atomicAdd(q + rt, ay * S.w[k]);
  }
}

// Sums each (node, component)'s copies (starting at a rotating copy, so the
// threads of a warp read different banks) and adds the non-zero totals into
// this block's slice of the global current J [kJSlices][2][n].
__device__ void flush_tile(const double *Jt, int rt, double *J, int n) {
  double *Js = J + (size_t)(blockIdx.x & (kJSlices - 1)) * 2 * n;
  for (int i = threadIdx.x; i < 2 * n; i += blockDim.x) {
    const int node = i >> 1, comp = i & 1;
    const double *q = Jt + (size_t)i * rt;
    double a = 0.0;
    for (int r = 0; r < rt; r++) a += q[(r + i) & (rt - 1)];
    if (a != 0.0) atomicAdd(&Js[comp * n + node], a);
  }
}

// ---------------------------------------------------------------- passes

template <int ORDER>
__global__ void __launch_bounds__(kEm1Threads) em1d_pass_c_kernel(Em1dConst c, Em1dBufs b) {
  extern __shared__ double sm[];
  const int n = c.n;
  double *Esx = sm, *Esy = sm + n, *Bs = sm + 2 * n, *Jt = sm + 3 * n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    Esx[i] = b.Es[i];
    Esy[i] = b.Es[n + i];
    Bs[i] = b.Bs[i];
  }
  clear_tile(Jt, 2 * n * c.rt);
  __syncthreads();
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < c.n_total;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int s = species_of1(c, p);
    double vsx, vsy, yh;
    // ESEC2: the shape at y* that the previous pass E (or the initial deposit)
    // deposited j^{n,*} with, the same bits as forming it here
    Shape64<ORDER> Sy;
    if (b.sws)
      Sy.load(b.sws, b.sis, p, c.n_total, n);
    else
      Sy = em1d_shape_at_ystar<ORDER>(c, b.y[p], b.vy[p], b.err);
    em1d_half_push<ORDER>(c, Esx, Esy, Bs, Sy, b.y[p], b.vx[p], b.vy[p], c.qm[s], b.err, vsx, vsy,
                          yh);
    b.vsx[p] = vsx;   // pass E forms y^{n+1/2} from v* with the same rounding
    b.vsy[p] = vsy;
    const Shape64<ORDER> S(__dmul_rn(yh, c.inv_h), n);
    const double qw = marker_qw(c, b, s, p);
    tile_deposit<ORDER>(Jt, c.rt, S, qw * vsx, qw * vsy);
    if (b.sw) S.store(b.sw, b.si, p, c.n_total);  // pass E gathers with it
  }
  __syncthreads();
  flush_tile(Jt, c.rt, b.J2, n);
  if (arrive_last(b.done)) {
    double2 *Z = (double2 *)sm;
    field_advance(c, c.solver == 2, c.dt, b.coef, b.tw, b.E, b.B, b.J2, b.En, b.Bn, b.Ea, b.Bh, Z);
    for (int i = threadIdx.x; i < kJSlices * 2 * n; i += blockDim.x) b.J1[i] = 0.0;
  }
}

template <int ORDER>
__global__ void __launch_bounds__(kEm1Threads) em1d_pass_e_kernel(Em1dConst c, Em1dBufs b,
                                                                   int slot) {
  extern __shared__ double sm[];
  __shared__ double red[33];
  const int n = c.n;
  double *Esx = sm, *Esy = sm + n, *Bs = sm + 2 * n;
  double *Eax = sm + 3 * n, *Eay = sm + 4 * n, *Bh = sm + 5 * n, *Jt = sm + 6 * n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    Esx[i] = b.Es[i];
    Esy[i] = b.Es[n + i];
    Bs[i] = b.Bs[i];
    Eax[i] = b.Ea[i];
    Eay[i] = b.Ea[n + i];
    Bh[i] = b.Bh[i];
  }
  clear_tile(Jt, 2 * n * c.rt);
  __syncthreads();
  const double dt = c.dt, hdt = 0.5 * c.dt;
  double ke = 0.0;
  unsigned nfb = 0;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < c.n_total;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int s = species_of1(c, p);
    const double qm = c.qm[s];
    const double y = b.y[p], vx = b.vx[p], vy = b.vy[p];
    const double vsx = b.vsx[p], vsy = b.vsy[p];
    // the shape at y^{n+1/2} that pass C deposited with (loaded: on this
    // FP64-bound pass bytes are cheaper than its arithmetic), else formed
    // again with pass C's rounding
    Shape64<ORDER> S;
    if (b.sw) {
      S.load(b.sw, b.si, p, c.n_total, n);
    } else {
      const double yh = wrap_periodic(__fma_rn(hdt, vsy, y), c.L, b.err);
      S = Shape64<ORDER>(__dmul_rn(yh, c.inv_h), n);
    }
    const double ex = S.gather(Eax), ey = S.gather(Eay), bz = S.gather(Bh);
    const double a = dt * qm;
    const double dx = fma(a, fma(vsy, bz, ex), vx);
    const double dy = fma(a, fma(-vsx, bz, ey), vy);
    // R = |v^n|^2 + 2 v* . (v^dag - v^n), Gamma = sqrt(R) / |v^dag| (Eq. opt_solution)
    const double R = fma(vx, vx, vy * vy) + 2.0 * fma(vsx, dx - vx, vsy * (dy - vy));
    const double vd2 = fma(dx, dx, dy * dy);
    double g = 1.0;
    if (c.gamma_on) {
      if (R < 0.0 || vd2 == 0.0)
        nfb++;
      else
        g = sqrt(R / vd2);
    }
    const double v1x = g * dx, v1y = g * dy;
    const double y1 = wrap_periodic(fma(dt, vsy, y), c.L, b.err);
    b.y[p] = y1;
    b.vx[p] = v1x;
    b.vy[p] = v1y;
    ke = fma(c.half_m[s] * (b.w ? b.w[p] : c.w0[s]), fma(v1x, v1x, v1y * v1y), ke);
    if (c.scheme == 2) {
      const Shape64<ORDER> S2 = em1d_shape_at_ystar<ORDER>(c, y1, v1y, b.err);
      const double qw = marker_qw(c, b, s, p);
      tile_deposit<ORDER>(Jt, c.rt, S2, qw * v1x, qw * v1y);
      if (b.sws) S2.store(b.sws, b.sis, p, c.n_total);  // the next pass C gathers with it
    }
  }
  if (!isfinite(ke)) atomicOr(b.err, kErrNonfinite);
  const unsigned fbw = __reduce_add_sync(0xffffffffu, nfb);
  if ((threadIdx.x & 31) == 0 && fbw) atomicAdd(&b.fallback[slot], (unsigned long long)fbw);
  const double kb = block_sum_d(ke, red);
  if (threadIdx.x == 0) b.ke_part[blockIdx.x] = kb;
  __syncthreads();
  if (c.scheme == 2) flush_tile(Jt, c.rt, b.J1, n);
  if (arrive_last(b.done + 1)) {
    // TE of the new state: KE from the block partials in block order, W_E + W_B
    double wf = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const double ex = __ldcg(b.En + i), ey = __ldcg(b.En + n + i), bz = __ldcg(b.Bn + i);
      wf += 0.5 * c.h * (ex * ex + ey * ey) + 0.5 * c.c2 * c.h * bz * bz;
    }
    // the block partials, each thread a fixed stride of them, then a fixed-order
    // block reduction: the same sum every step for the same partials
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) wf += __ldcg(b.ke_part + i);
    const double tsum = block_sum_d(wf, red);
    if (threadIdx.x == 0) b.te[slot] = tsum;
    double2 *Z = (double2 *)sm;
    if (c.scheme == 2) {
      field_advance(c, c.solver == 2, hdt, b.coef + kEm1Coef * (n / 2 + 1), b.tw, b.En, b.Bn,
                    b.J1, b.Es, b.Bs, nullptr, nullptr, Z);
    } else {
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        b.Es[i] = __ldcg(b.En + i);
        b.Es[n + i] = __ldcg(b.En + n + i);
        b.Bs[i] = __ldcg(b.Bn + i);
      }
    }
    for (int i = threadIdx.x; i < kJSlices * 2 * n; i += blockDim.x) b.J2[i] = 0.0;
  }
}

// j^{0,*} of the initial state (ESEC2 form): deposit of v^n at y^n + dt/2 vy^n.
template <int ORDER>
__global__ void __launch_bounds__(kEm1Threads) em1d_deposit_initial_kernel(Em1dConst c,
                                                                            Em1dBufs b) {
  extern __shared__ double sm[];
  double *Jt = sm;
  clear_tile(Jt, 2 * c.n * c.rt);
  __syncthreads();
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < c.n_total;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int s = species_of1(c, p);
    const Shape64<ORDER> S = em1d_shape_at_ystar<ORDER>(c, b.y[p], b.vy[p], b.err);
    const double qw = marker_qw(c, b, s, p);
    tile_deposit<ORDER>(Jt, c.rt, S, qw * b.vx[p], qw * b.vy[p]);
    if (b.sws) S.store(b.sws, b.sis, p, c.n_total);  // pass C gathers with it
  }
  __syncthreads();
  flush_tile(Jt, c.rt, b.J1, c.n);
}

// Twiddles tw[j] = exp(-2 pi i j / n), j < n/2, and the per-mode coefficients
// of the full step over dt (coef[0 .. n/2]: Crank-Nicolson or PSATD) and of
// the half step over dt/2 (coef[n/2 + 1 ..]: explicit Euler or PSATD); one
// block, once per set-up.
__global__ void em1d_tables_kernel(Em1dConst c, Em1dBufs b) {
  const int n = c.n;
  for (int j = threadIdx.x; j < n / 2; j += blockDim.x) {
    double s, co;
    sincospi(-2.0 * (double)j / (double)n, &s, &co);
    b.tw[j] = make_double2(co, s);
  }
  for (int k = threadIdx.x; k <= n / 2; k += blockDim.x) {
    mode_coefficients(c, c.solver == 1 ? 1 : 2, c.dt, k, b.coef + kEm1Coef * k);
    mode_coefficients(c, c.solver == 1 ? 0 : 2, 0.5 * c.dt, k,
                      b.coef + kEm1Coef * (n / 2 + 1 + k));
  }
}

// The first half step (E*, B*) from (E^n, B^n, j^{n,*}); one block.
__global__ void __launch_bounds__(kEm1Threads) em1d_half_kernel(Em1dConst c, Em1dBufs b) {
  extern __shared__ double sm[];
  double2 *Z = (double2 *)sm;
  if (c.scheme == 2) {
    field_advance(c, c.solver == 2, 0.5 * c.dt, b.coef + kEm1Coef * (c.n / 2 + 1), b.tw, b.E,
                  b.B, b.J1, b.Es, b.Bs, nullptr, nullptr, Z);
  } else {
    for (int i = threadIdx.x; i < c.n; i += blockDim.x) {
      b.Es[i] = b.E[i];
      b.Es[c.n + i] = b.E[c.n + i];
      b.Bs[i] = b.B[i];
    }
  }
}

// Kinetic energy per species (block partials [nsp][grid]) and, from block 0,
// W_E and W_B of the current fields (wf[0], wf[1]).
__global__ void __launch_bounds__(kEm1Threads) em1d_energy_kernel(Em1dConst c, Em1dBufs b,
                                                                   double *ke_out, double *wf) {
  __shared__ double red[33];
  for (int s = 0; s < c.nsp; s++) {
    const int64_t lo = s == 0 ? 0 : c.sp_end[s - 1], hi = c.sp_end[s];
    double acc = 0.0;
    for (int64_t p = lo + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < hi;
         p += (int64_t)gridDim.x * blockDim.x)
      acc = fma(b.w ? b.w[p] : c.w0[s], fma(b.vx[p], b.vx[p], b.vy[p] * b.vy[p]), acc);
    const double t = block_sum_d(acc, red);
    if (threadIdx.x == 0) ke_out[(size_t)s * gridDim.x + blockIdx.x] = c.half_m[s] * t;
    __syncthreads();
  }
  if (blockIdx.x == 0) {
    double we = 0.0, wb = 0.0;
    for (int i = threadIdx.x; i < c.n; i += blockDim.x) {
      we = fma(b.E[i], b.E[i], fma(b.E[c.n + i], b.E[c.n + i], we));
      wb = fma(b.B[i], b.B[i], wb);
    }
    const double a = block_sum_d(we, red);
    const double d = block_sum_d(wb, red);
    if (threadIdx.x == 0) {
      wf[0] = 0.5 * c.h * a;
      wf[1] = 0.5 * c.c2 * c.h * d;
    }
  }
}

// ------------------------------------------------------------ mixed form

// V units -> position units for half a step (kv >= 1)
__device__ __forceinline__ uint32_t half_shift1(int V, const Em1dMixConst &m) {
  return (uint32_t)((V + m.hround) >> m.kv);
}

// Split tile of the mixed passes: [padded node][component][half][copy], the
// low 16 bits of each term (unsigned) and the signed rest, so a node's value
// is rest 2^16 + low; lane l adds into copy l mod rt.
template <int ORDER>
__device__ __forceinline__ void mix_tile_deposit(unsigned *Jl, int rt, const ShapeMix<ORDER> &S,
                                                 int Vx, int Vy, const Em1dMixConst &m) {
#pragma unroll
  for (int k = 0; k <= ORDER; k++) {
    unsigned *q = Jl + (S.p + k) * 4 * rt;
    const SplitTerm tx = split_term(Vx, S.s[k], m.rshift, m.rnd, 0xFFFFu, m.rshift - 16);
    const SplitTerm ty = split_term(Vy, S.s[k], m.rshift, m.rnd, 0xFFFFu, m.rshift - 16);
    atomicAdd(q, tx.lo);
    atomicAdd(q + rt, (unsigned)tx.hi);
    atomicAdd(q + 2 * rt, ty.lo);
    atomicAdd(q + 3 * rt, (unsigned)ty.hi);
  }
}

// Sums each (padded node, component)'s copies and adds the non-zero totals to
// J [2][n] with one int64 atomic (ghost nodes add to the node they stand for).
template <int ORDER>
__device__ void mix_flush_tile(const unsigned *Jt, int rt, long long *J, int n) {
  for (int i = threadIdx.x; i < 2 * npad_of(n); i += blockDim.x) {
    const int q = i >> 1, comp = i & 1;
    const unsigned *lo = Jt + (size_t)(q * 2 + comp) * 2 * rt, *hi = lo + rt;
    unsigned long long sl = 0;
    long long sh = 0;
    for (int r = 0; r < rt; r++) {
      const int k = (r + i) & (rt - 1);
      sl += lo[k];
      sh += (int)hi[k];
    }
    const long long a = sh * 65536 + (long long)sl;
    if (a != 0)
      atomicAdd((unsigned long long *)&J[comp * n + wrap_node(q - Pad<ORDER>::kPad, n)],
                (unsigned long long)a);
  }
}

// jscale times an integer current into slice 0 of an FP64 sliced current
// (the field solve's input; the other slices stay zero); the block's threads.
__device__ __forceinline__ void mix_current_to_fp64(const long long *Ji, double *J, int n,
                                                    double jscale) {
  for (int i = threadIdx.x; i < 2 * n; i += blockDim.x) J[i] = jscale * (double)__ldcg(Ji + i);
}

__device__ __forceinline__ void clear_words(unsigned *a, int len) {
  for (int i = threadIdx.x; i < len; i += blockDim.x) a[i] = 0u;
}

// The non-series path of correct_velocity_xy: the R < 0 test and Gamma - 1 in
// FP64 (mixed_common.cuh).
__device__ __noinline__ ff2 correct_velocity_xy_fp64(float2 vh, float2 vl, int Vx, int Vy, ff2 D,
                                                     ff2 vd, unsigned &nfb) {
  const ff Dx{D.hi.x, D.lo.x}, Dy{D.hi.y, D.lo.y};
  const ff vx{vd.hi.x, vd.lo.x}, vy{vd.hi.y, vd.lo.y};
  const double a = ff_to_double(Dx) * bracket_fp64(vh.x, vl.x, Vx, Dx) +
                   ff_to_double(Dy) * bracket_fp64(vh.y, vl.y, Vy, Dy);
  const double ux = ff_to_double(vx), uy = ff_to_double(vy);
  double g;
  if (!gamma_minus_one_fp64(a, ux * ux + uy * uy, g)) {
    nfb++;
    return vd;
  }
  const ff nx = scale_by_gamma_fp64(vx, g), ny = scale_by_gamma_fp64(vy, g);
  return ff2{make_float2(nx.hi, ny.hi), make_float2(nx.lo, ny.lo)};
}

// v^dag = v^n + Delta and v^{n+1} = Gamma v^dag for the pair (vx, vy) of one
// marker, the components in the two lanes (x, y) of packed float pairs:
// b = V* - v^n - Delta/2 from the exact differences, a = Delta . b, and
// Gamma - 1 from t = 2a / |v^dag|^2 as in the 1D1V mixed form: the FP32
// series for |t| < 2^-8, else the R < 0 test and Gamma in FP64.
__device__ __forceinline__ ff2 correct_velocity_xy(float2 vh, float2 vl, int Vx, int Vy, ff2 D,
                                                   bool on, unsigned &nfb) {
  const ff2 vd = ff_add2(ff2{vh, vl}, D);
  if (!on) return vd;
  const int ihx = __float2int_rn(vh.x), ihy = __float2int_rn(vh.y);
  const float2 fr = sub2(vh, make_float2(__int2float_rn(ihx), __int2float_rn(ihy)));
  const ff2 q = two_sum2(make_float2(__int2float_rn(Vx - ihx), __int2float_rn(Vy - ihy)),
                         mul2(splat2(-0.5f), D.hi));
  const float2 bq = add2(q.hi, sub2(sub2(sub2(q.lo, fr), vl), mul2(splat2(0.5f), D.lo)));
  const float2 db = mul2(add2(D.hi, D.hi), bq);
  const float2 v2 = mul2(vd.hi, vd.hi);
  const float t = div_rcp_residual(__fadd_rn(db.x, db.y), __fadd_rn(v2.x, v2.y));
  if (!(fabsf(t) < 0.00390625f)) return correct_velocity_xy_fp64(vh, vl, Vx, Vy, D, vd, nfb);
  const float gm = __fmul_rn(
      t, __fmaf_rn(t, __fmaf_rn(t, __fmaf_rn(t, -0.0390625f, 0.0625f), -0.125f), 0.5f));
  ff2 p = two_prod2(vd.hi, splat2(gm));
  p.lo = fma2(vd.lo, splat2(gm), p.lo);
  return ff_add2(vd, p);
}

template <int ORDER>
__global__ void __launch_bounds__(kEm1Threads, 4) em1m_pass_c_kernel(Em1dConst c, Em1dBufs b,
                                                                   Em1dMixConst m,
                                                                   Em1dMixBufs mb) {
  extern __shared__ __align__(16) unsigned char smraw[];
  constexpr int PAD = Pad<ORDER>::kPad;
  const int n = c.n, npad = npad_of(n), rt = m.rt;
  unsigned *Jt = (unsigned *)smraw;                      // [npad][2][2][rt]
  float4 *T = (float4 *)(Jt + 4 * rt * npad);            // e_half E*x, e_half E*y, t_half B*z
  uint4 *stage = (uint4 *)(T + npad);                    // [5][blockDim]: next group's words
  clear_words(Jt, 4 * rt * npad);
  for (int q = threadIdx.x; q < npad; q += blockDim.x) {
    const int i = wrap_node(q - PAD, n);
    T[q] = make_float4((float)(m.e_half * b.Es[i]), (float)(m.e_half * b.Es[n + i]),
                       (float)(m.t_half * b.Bs[i]), 0.0f);
  }
  unsigned *Jl = Jt + (threadIdx.x & (rt - 1));
  unsigned bad = 0;
  // four consecutive markers per thread and trip, 16 bytes per array (the
  // arrays are padded to a multiple of four).  Each thread copies its next
  // group into its own five stage slots with asynchronous copies while it
  // works on the current one; it reads only its own slots, so the wait is on
  // its own copies and needs no block barrier.
  const int64_t ngroups = (m.N + 3) / 4;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const unsigned slot0 = (unsigned)__cvta_generic_to_shared(stage + threadIdx.x);
  const unsigned sstep = 16u * blockDim.x;
  const auto fetch = [&](int64_t gg) {
    cp_async16(slot0, reinterpret_cast<const uint4 *>(mb.Y) + gg);
    cp_async16(slot0 + sstep, reinterpret_cast<const uint4 *>(mb.vh[0]) + gg);
    cp_async16(slot0 + 2 * sstep, reinterpret_cast<const uint4 *>(mb.vl[0]) + gg);
    cp_async16(slot0 + 3 * sstep, reinterpret_cast<const uint4 *>(mb.vh[1]) + gg);
    cp_async16(slot0 + 4 * sstep, reinterpret_cast<const uint4 *>(mb.vl[1]) + gg);
    cp_async_commit();
  };
  int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g < ngroups) fetch(g);
  __syncthreads();
  for (; g < ngroups; g += stride) {
    cp_async_wait_all();
    const uint4 Yq = stage[threadIdx.x];
    const float4 xh4 = uint_as_float4(stage[blockDim.x + threadIdx.x]);
    const float4 xl4 = uint_as_float4(stage[2 * blockDim.x + threadIdx.x]);
    const float4 yh4 = uint_as_float4(stage[3 * blockDim.x + threadIdx.x]);
    const float4 yl4 = uint_as_float4(stage[4 * blockDim.x + threadIdx.x]);
    if (g + stride < ngroups) fetch(g + stride);
    const uint32_t Ya[4] = {Yq.x, Yq.y, Yq.z, Yq.w};
    const float xha[4] = {xh4.x, xh4.y, xh4.z, xh4.w}, xla[4] = {xl4.x, xl4.y, xl4.z, xl4.w};
    const float yha[4] = {yh4.x, yh4.y, yh4.z, yh4.w}, yla[4] = {yl4.x, yl4.y, yl4.z, yl4.w};
    int Vxa[4], Vya[4];
#pragma unroll
    for (int j = 0; j < 4; j++) {
      const bool valid = 4 * g + j < m.N;
      const uint32_t Y = Ya[j];
      const float vxh = xha[j], vxl = xla[j], vyh = yha[j], vyl = yla[j];
      unsigned flags = 0;
      // gather #1 at y* = y^n + dt/2 vy^n: e_half E*, t = t_half B*z
      const ShapeMix<ORDER> S1(Y + half_shift1(to_fixed(vyh, flags), m), n);
      float ex = 0.0f, ey = 0.0f, t = 0.0f;
#pragma unroll
      for (int k = 0; k <= ORDER; k++) {
        const float4 f = T[S1.p + k];
        ex = __fmaf_rn(S1.w[k], f.x, ex);
        ey = __fmaf_rn(S1.w[k], f.y, ey);
        t = __fmaf_rn(S1.w[k], f.z, t);
      }
      // v* = (ux + t uy, uy - t ux) / (1 + t^2), u = v^n + e: v* = u + correction
      const float ux = __fadd_rn(vxh, ex), uy = __fadd_rn(vyh, ey);
      const float tt = __fmul_rn(t, t), inv = __frcp_rn(__fadd_rn(1.0f, tt));
      const float cx = __fmul_rn(__fmaf_rn(t, uy, -__fmul_rn(tt, ux)), inv);
      const float cy = __fmul_rn(__fmaf_rn(-t, ux, -__fmul_rn(tt, uy)), inv);
      Vxa[j] = vstar_fixed(vxh, vxl, __fadd_rn(ex, cx), flags);
      Vya[j] = vstar_fixed(vyh, vyl, __fadd_rn(ey, cy), flags);
      if (valid) {
        bad |= flags;
        const ShapeMix<ORDER> Sh(Y + half_shift1(Vya[j], m), n);
        mix_tile_deposit<ORDER>(Jl, rt, Sh, Vxa[j], Vya[j], m);
      }
    }
    reinterpret_cast<int4 *>(mb.Vs[0])[g] = make_int4(Vxa[0], Vxa[1], Vxa[2], Vxa[3]);
    reinterpret_cast<int4 *>(mb.Vs[1])[g] = make_int4(Vya[0], Vya[1], Vya[2], Vya[3]);
  }
  if (bad) atomicOr(b.err, bad);
  __syncthreads();
  mix_flush_tile<ORDER>(Jt, rt, mb.J2, n);
  if (arrive_last(b.done)) {
    mix_current_to_fp64(mb.J2, b.J2, n, m.jscale);
    for (int i = threadIdx.x; i < 2 * n; i += blockDim.x) mb.J1[i] = 0;
    __syncthreads();
    double2 *Z = (double2 *)smraw;
    field_advance(c, c.solver == 2, c.dt, b.coef, b.tw, b.E, b.B, b.J2, b.En, b.Bn, b.Ea, b.Bh, Z);
  }
}

template <int ORDER>
__global__ void __launch_bounds__(kEm1Threads, 4) em1m_pass_e_kernel(Em1dConst c, Em1dBufs b,
                                                                   Em1dMixConst m,
                                                                   Em1dMixBufs mb, int slot) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ double red[33];
  constexpr int PAD = Pad<ORDER>::kPad;
  const int n = c.n, npad = npad_of(n), rt = m.rt;
  unsigned *Jt = (unsigned *)smraw;                      // [npad][2][2][rt]
  float4 *Ta = (float4 *)(Jt + 4 * rt * npad);           // kick Ea as pairs (x hi, x lo, y hi, y lo)
  float *Tb = (float *)(Ta + npad);                      // m_full B^{n+1/2}
  clear_words(Jt, 4 * rt * npad);
  for (int q = threadIdx.x; q < npad; q += blockDim.x) {
    const int i = wrap_node(q - PAD, n);
    const ff ax = ff_from_double(m.kick * b.Ea[i]), ay = ff_from_double(m.kick * b.Ea[n + i]);
    Ta[q] = make_float4(ax.hi, ax.lo, ay.hi, ay.lo);
    Tb[q] = (float)(m.m_full * b.Bh[i]);
  }
  __syncthreads();
  unsigned *Jl = Jt + (threadIdx.x & (rt - 1));
  float2 keh = make_float2(0.0f, 0.0f), kel = make_float2(0.0f, 0.0f);
  unsigned nfb = 0, bad = 0;
  // four consecutive markers per thread and trip, loaded and stored 16 bytes
  // at a time (the arrays are padded to a multiple of four)
  const int64_t ngroups = (m.N + 3) / 4;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < ngroups;
       g += (int64_t)gridDim.x * blockDim.x) {
    const uint4 Yq = reinterpret_cast<const uint4 *>(mb.Y)[g];
    const float4 xh4 = reinterpret_cast<const float4 *>(mb.vh[0])[g];
    const float4 xl4 = reinterpret_cast<const float4 *>(mb.vl[0])[g];
    const float4 yh4 = reinterpret_cast<const float4 *>(mb.vh[1])[g];
    const float4 yl4 = reinterpret_cast<const float4 *>(mb.vl[1])[g];
    const int4 vx4 = reinterpret_cast<const int4 *>(mb.Vs[0])[g];
    const int4 vy4 = reinterpret_cast<const int4 *>(mb.Vs[1])[g];
    uint32_t Ya[4] = {Yq.x, Yq.y, Yq.z, Yq.w};
    float xha[4] = {xh4.x, xh4.y, xh4.z, xh4.w}, xla[4] = {xl4.x, xl4.y, xl4.z, xl4.w};
    float yha[4] = {yh4.x, yh4.y, yh4.z, yh4.w}, yla[4] = {yl4.x, yl4.y, yl4.z, yl4.w};
    const int Vxa[4] = {vx4.x, vx4.y, vx4.z, vx4.w}, Vya[4] = {vy4.x, vy4.y, vy4.z, vy4.w};
#pragma unroll
    for (int j = 0; j < 4; j++) {
      const bool valid = 4 * g + j < m.N;
      const uint32_t Y = Ya[j];
      const float2 vh = make_float2(xha[j], yha[j]), vl = make_float2(xla[j], yla[j]);
      const int Vx = Vxa[j], Vy = Vya[j];
      const uint32_t hs = half_shift1(Vy, m);
      const ShapeMix<ORDER> S(Y + hs, n);
      // gather #2 at y^{n+1/2}: kick E as float pairs (lane x: Ex, lane y: Ey)
      float2 ph[ORDER + 1], pl = make_float2(0.0f, 0.0f);
      float bz = 0.0f;
#pragma unroll
      for (int k = 0; k <= ORDER; k++) {
        const float4 e = Ta[S.p + k];
        const float2 w = splat2(S.w[k]);
        const ff2 pr = two_prod2(make_float2(e.x, e.z), w);
        ph[k] = pr.hi;
        pl = add2(pl, fma2(make_float2(e.y, e.w), w, pr.lo));
        bz = __fmaf_rn(S.w[k], Tb[S.p + k], bz);
      }
      ff2 Ep = two_sum2(ph[0], ph[1]);
      pl = add2(pl, Ep.lo);
      if (ORDER == 2) {
        Ep = two_sum2(Ep.hi, ph[ORDER]);
        pl = add2(pl, Ep.lo);
      }
      // Delta = d + dt (q/m) (V*y Bz, -V*x Bz), the products in float pairs of the exact V*
      const float fx = __int2float_rn(Vx), fy = __int2float_rn(Vy);
      const ff2 vs{make_float2(fy, fx), make_float2(__int2float_rn(Vy - __float2int_rn(fy)),
                                                    __int2float_rn(Vx - __float2int_rn(fx)))};
      ff2 mu = two_prod2(vs.hi, splat2(bz));
      mu.lo = fma2(vs.lo, splat2(bz), mu.lo);
      mu = fast_two_sum2(mu.hi, mu.lo);
      mu.hi.y = -mu.hi.y;
      mu.lo.y = -mu.lo.y;
      const ff2 D = ff_add2(fast_two_sum2(Ep.hi, pl), mu);
      const ff2 vn = correct_velocity_xy(vh, vl, Vx, Vy, D, c.gamma_on != 0 && valid, nfb);
      if (!valid) continue;
      {
        ff2 s2 = two_prod2(vn.hi, vn.hi);
        s2.lo = fma2(add2(vn.hi, vn.hi), vn.lo, s2.lo);
        const ff2 acc = two_sum2(keh, s2.hi);
        keh = acc.hi;
        kel = add2(kel, add2(acc.lo, s2.lo));
      }
      const uint32_t Y1 = Y + 2u * hs;
      if (c.scheme == 2) {
        const int V1x = to_fixed(vn.hi.x, bad), V1y = to_fixed(vn.hi.y, bad);
        const ShapeMix<ORDER> S1(Y1 + half_shift1(V1y, m), n);
        mix_tile_deposit<ORDER>(Jl, rt, S1, V1x, V1y, m);
      }
      Ya[j] = Y1;
      xha[j] = vn.hi.x;
      xla[j] = vn.lo.x;
      yha[j] = vn.hi.y;
      yla[j] = vn.lo.y;
    }
    reinterpret_cast<uint4 *>(mb.Y)[g] = make_uint4(Ya[0], Ya[1], Ya[2], Ya[3]);
    reinterpret_cast<float4 *>(mb.vh[0])[g] = make_float4(xha[0], xha[1], xha[2], xha[3]);
    reinterpret_cast<float4 *>(mb.vl[0])[g] = make_float4(xla[0], xla[1], xla[2], xla[3]);
    reinterpret_cast<float4 *>(mb.vh[1])[g] = make_float4(yha[0], yha[1], yha[2], yha[3]);
    reinterpret_cast<float4 *>(mb.vl[1])[g] = make_float4(yla[0], yla[1], yla[2], yla[3]);
  }
  const ff kt = ff_add(ff{keh.x, kel.x}, ff{keh.y, kel.y});
  if (!isfinite(kt.hi) || !isfinite(kt.lo)) bad |= kErrNonfinite;
  if (bad) atomicOr(b.err, bad);
  const unsigned fbw = __reduce_add_sync(0xffffffffu, nfb);
  if ((threadIdx.x & 31) == 0 && fbw) atomicAdd(&b.fallback[slot], (unsigned long long)fbw);
  const double kb = block_sum_d((double)kt.hi + (double)kt.lo, red);
  if (threadIdx.x == 0) b.ke_part[blockIdx.x] = m.ke_scale * kb;
  __syncthreads();
  if (c.scheme == 2) mix_flush_tile<ORDER>(Jt, rt, mb.J1, n);
  if (arrive_last(b.done + 1)) {
    // TE of the new state: KE from the block partials in block order, W_E + W_B
    double wf = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const double ex = __ldcg(b.En + i), ey = __ldcg(b.En + n + i), bz = __ldcg(b.Bn + i);
      wf += 0.5 * c.h * (ex * ex + ey * ey) + 0.5 * c.c2 * c.h * bz * bz;
    }
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) wf += __ldcg(b.ke_part + i);
    const double tsum = block_sum_d(wf, red);
    if (threadIdx.x == 0) b.te[slot] = tsum;
    double2 *Z = (double2 *)smraw;
    if (c.scheme == 2) {
      mix_current_to_fp64(mb.J1, b.J1, n, m.jscale);
      __syncthreads();
      field_advance(c, c.solver == 2, 0.5 * c.dt, b.coef + kEm1Coef * (n / 2 + 1), b.tw, b.En,
                    b.Bn, b.J1, b.Es, b.Bs, nullptr, nullptr, Z);
    } else {
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        b.Es[i] = __ldcg(b.En + i);
        b.Es[n + i] = __ldcg(b.En + n + i);
        b.Bs[i] = __ldcg(b.Bn + i);
      }
    }
    for (int i = threadIdx.x; i < 2 * n; i += blockDim.x) mb.J2[i] = 0;
  }
}

// j^{0,*} of the current state (ESEC2): V^n at y^n + dt/2 vy^n into mb.J1.
template <int ORDER>
__global__ void __launch_bounds__(kEm1Threads) em1m_deposit_initial_kernel(Em1dConst c,
                                                                            Em1dMixConst m,
                                                                            Em1dMixBufs mb,
                                                                            unsigned *err) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int n = c.n, rt = m.rt;
  unsigned *Jt = (unsigned *)smraw;
  clear_words(Jt, 4 * rt * npad_of(n));
  __syncthreads();
  unsigned *Jl = Jt + (threadIdx.x & (rt - 1));
  unsigned bad = 0;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < m.N;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int Vx = to_fixed(mb.vh[0][p], bad), Vy = to_fixed(mb.vh[1][p], bad);
    const ShapeMix<ORDER> S(mb.Y[p] + half_shift1(Vy, m), n);
    mix_tile_deposit<ORDER>(Jl, rt, S, Vx, Vy, m);
  }
  if (bad) atomicOr(err, bad);
  __syncthreads();
  mix_flush_tile<ORDER>(Jt, rt, mb.J1, n);
}

__global__ void em1m_j1_to_fp64_kernel(Em1dConst c, Em1dBufs b, Em1dMixConst m,
                                       Em1dMixBufs mb) {
  mix_current_to_fp64(mb.J1, b.J1, c.n, m.jscale);
}

__global__ void em1m_from_fp64_kernel(Em1dBufs b, Em1dMixConst m, Em1dMixBufs mb) {
  const double scale = 4294967296.0 / m.L;   // one multiply per marker, no divide
  const double *v[2] = {b.vx, b.vy};
  unsigned bad = 0;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < m.N;
       p += (int64_t)gridDim.x * blockDim.x) {
    mb.Y[p] = (uint32_t)((unsigned long long)llrint(b.y[p] * scale) & 0xFFFFFFFFull);
#pragma unroll
    for (int d = 0; d < 2; d++) {
      const double vv = v[d][p] * m.cxk;
      if (!isfinite(vv)) bad |= kErrNonfinite;
      if (!(fabs(vv) < 2147483520.0)) bad |= kErrVelocityRange;
      const float hi = (float)vv;
      mb.vh[d][p] = hi;
      mb.vl[d][p] = (float)(vv - (double)hi);
    }
  }
  if (bad) atomicOr(b.err, bad);
}

__global__ void em1m_to_fp64_kernel(Em1dBufs b, Em1dMixConst m, Em1dMixBufs mb) {
  double *v[2] = {b.vx, b.vy};
  const double inv = 1.0 / m.cxk;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < m.N;
       p += (int64_t)gridDim.x * blockDim.x) {
    b.y[p] = (double)mb.Y[p] * (m.L / 4294967296.0);
#pragma unroll
    for (int d = 0; d < 2; d++) v[d][p] = ((double)mb.vh[d][p] + (double)mb.vl[d][p]) * inv;
  }
}

__global__ void __launch_bounds__(kEm1Threads) em1m_energy_kernel(Em1dConst c, Em1dBufs b,
                                                                   Em1dMixConst m,
                                                                   Em1dMixBufs mb, double *ke_out,
                                                                   double *wf) {
  __shared__ double red[33];
  double acc = 0.0;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < m.N;
       p += (int64_t)gridDim.x * blockDim.x) {
    const double vx = (double)mb.vh[0][p] + (double)mb.vl[0][p];
    const double vy = (double)mb.vh[1][p] + (double)mb.vl[1][p];
    acc = fma(vx, vx, fma(vy, vy, acc));
  }
  const double t = block_sum_d(acc, red);
  if (threadIdx.x == 0) ke_out[blockIdx.x] = m.ke_scale * t;
  __syncthreads();
  if (blockIdx.x == 0) {
    double we = 0.0, wb = 0.0;
    for (int i = threadIdx.x; i < c.n; i += blockDim.x) {
      we = fma(b.E[i], b.E[i], fma(b.E[c.n + i], b.E[c.n + i], we));
      wb = fma(b.B[i], b.B[i], wb);
    }
    const double a = block_sum_d(we, red);
    const double d = block_sum_d(wb, red);
    if (threadIdx.x == 0) {
      wf[0] = 0.5 * c.h * a;
      wf[1] = 0.5 * c.c2 * c.h * d;
    }
  }
}

__global__ void em1m_absmax_kernel(Em1dBufs b, int64_t n, unsigned long long *out) {
  double mx = 0.0;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x)
    mx = fmax(mx, fmax(fabs(b.vx[p]), fabs(b.vy[p])));
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(mx));
}

// the mixed passes' tile and tables, or the field solve's 9n + 8 doubles
size_t mix_smem(const Em1dConst &c, const Em1dMixConst &m) {
  const size_t npad = (size_t)c.n + 3;
  const size_t a = 4 * sizeof(unsigned) * m.rt * npad + (sizeof(float4) + sizeof(float)) * npad;
  const size_t f = sizeof(double) * (9 * (size_t)c.n + 8);
  return a > f ? a : f;
}

// pass C: tile copies, its table and the stage of the next groups (five
// 16-byte words a thread), or the field solve
size_t mix_smem_c(const Em1dConst &c, const Em1dMixConst &m) {
  const size_t npad = (size_t)c.n + 3;
  const size_t a = 4 * sizeof(unsigned) * m.rt * npad + sizeof(float4) * npad +
                   5 * sizeof(uint4) * kEm1Threads;
  const size_t f = sizeof(double) * (9 * (size_t)c.n + 8);
  return a > f ? a : f;
}

// the passes' tables and tile copies, or the field solve's 9n + 8 doubles
size_t pass_smem(const Em1dConst &c) {
  const size_t a = (6 + 2 * (size_t)c.rt) * c.n, f = 9 * (size_t)c.n + 8;
  return sizeof(double) * (a > f ? a : f);
}

template <typename K>
cudaError_t allow_smem(K kernel, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

PIC_BOUNDS_READER(bounds_site_em1d_spectral)

int em1d_tile_copies(int n) {
  int rt = 32;
  while (rt > 1 && sizeof(double) * (6 + 2 * (size_t)rt) * n > kEm1TileBudget) rt >>= 1;
  return rt;
}

__global__ void em1d_validate_kernel(const double *y, const double *vx, const double *vy,
                                     int64_t n, double L, unsigned *err) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    if (!(y[p] >= 0.0 && y[p] < L)) atomicOr(err, kErrBounds);
    if (!isfinite(vx[p]) || !isfinite(vy[p])) atomicOr(err, kErrNonfinite);
  }
}

cudaError_t em1d_prepare(const Em1dConst &c, const Em1dBufs &b, cudaStream_t st) {
  const size_t sm = pass_smem(c);
  cudaError_t e = cudaSuccess;
  if (c.order == 1) {
    if ((e = allow_smem(em1d_pass_c_kernel<1>, sm))) return e;
    if ((e = allow_smem(em1d_pass_e_kernel<1>, sm))) return e;
    if ((e = allow_smem(em1d_deposit_initial_kernel<1>, sm))) return e;
  } else {
    if ((e = allow_smem(em1d_pass_c_kernel<2>, sm))) return e;
    if ((e = allow_smem(em1d_pass_e_kernel<2>, sm))) return e;
    if ((e = allow_smem(em1d_deposit_initial_kernel<2>, sm))) return e;
  }
  if ((e = allow_smem(em1d_half_kernel, sm))) return e;
  em1d_tables_kernel<<<1, kEm1Threads, 0, st>>>(c, b);
  return cudaGetLastError();
}

void em1d_pass_c(const Em1dConst &c, const Em1dBufs &b, LaunchShape lp, cudaStream_t st) {
  const size_t sm = pass_smem(c);
  if (c.order == 1)
    em1d_pass_c_kernel<1><<<lp.grid, kEm1Threads, sm, st>>>(c, b);
  else
    em1d_pass_c_kernel<2><<<lp.grid, kEm1Threads, sm, st>>>(c, b);
}

void em1d_pass_e(const Em1dConst &c, const Em1dBufs &b, int slot, LaunchShape lp,
                 cudaStream_t st) {
  const size_t sm = pass_smem(c);
  if (c.order == 1)
    em1d_pass_e_kernel<1><<<lp.grid, kEm1Threads, sm, st>>>(c, b, slot);
  else
    em1d_pass_e_kernel<2><<<lp.grid, kEm1Threads, sm, st>>>(c, b, slot);
}

void em1d_start(const Em1dConst &c, const Em1dBufs &b, LaunchShape lp, cudaStream_t st) {
  const size_t sm = pass_smem(c);
  if (c.scheme == 2) {
    if (c.order == 1)
      em1d_deposit_initial_kernel<1><<<lp.grid, kEm1Threads, sm, st>>>(c, b);
    else
      em1d_deposit_initial_kernel<2><<<lp.grid, kEm1Threads, sm, st>>>(c, b);
  }
  em1d_half_kernel<<<1, kEm1Threads, sm, st>>>(c, b);
}

void em1d_energy(const Em1dConst &c, const Em1dBufs &b, double *ke_out, double *wf,
                 LaunchShape lp, cudaStream_t st) {
  em1d_energy_kernel<<<lp.grid, kEm1Threads, 0, st>>>(c, b, ke_out, wf);
}

int em1m_tile_copies(int n) {
  const size_t npad = (size_t)n + 3;
  int rt = 32;
  while (rt > 1 && 4 * sizeof(unsigned) * rt * npad + (sizeof(float4) + sizeof(float)) * npad >
                       kEm1TileBudget)
    rt >>= 1;
  return rt;
}

cudaError_t em1m_prepare(const Em1dConst &c, const Em1dMixConst &m) {
  const size_t sm = mix_smem(c, m);
  cudaError_t e = cudaSuccess;
  const size_t smc = mix_smem_c(c, m);
  if (c.order == 1) {
    if ((e = allow_smem(em1m_pass_c_kernel<1>, smc))) return e;
    if ((e = allow_smem(em1m_pass_e_kernel<1>, sm))) return e;
    if ((e = allow_smem(em1m_deposit_initial_kernel<1>, sm))) return e;
  } else {
    if ((e = allow_smem(em1m_pass_c_kernel<2>, smc))) return e;
    if ((e = allow_smem(em1m_pass_e_kernel<2>, sm))) return e;
    if ((e = allow_smem(em1m_deposit_initial_kernel<2>, sm))) return e;
  }
  return allow_smem(em1d_half_kernel, pass_smem(c) > sm ? pass_smem(c) : sm);
}

void em1m_pass_c(const Em1dConst &c, const Em1dBufs &b, const Em1dMixConst &m,
                 const Em1dMixBufs &mb, LaunchShape lp, cudaStream_t st) {
  const size_t sm = mix_smem_c(c, m);
  if (c.order == 1)
    em1m_pass_c_kernel<1><<<lp.grid, kEm1Threads, sm, st>>>(c, b, m, mb);
  else
    em1m_pass_c_kernel<2><<<lp.grid, kEm1Threads, sm, st>>>(c, b, m, mb);
}

void em1m_pass_e(const Em1dConst &c, const Em1dBufs &b, const Em1dMixConst &m,
                 const Em1dMixBufs &mb, int slot, LaunchShape lp, cudaStream_t st) {
  const size_t sm = mix_smem(c, m);
  if (c.order == 1)
    em1m_pass_e_kernel<1><<<lp.grid, kEm1Threads, sm, st>>>(c, b, m, mb, slot);
  else
    em1m_pass_e_kernel<2><<<lp.grid, kEm1Threads, sm, st>>>(c, b, m, mb, slot);
}

void em1m_start(const Em1dConst &c, const Em1dBufs &b, const Em1dMixConst &m,
                const Em1dMixBufs &mb, LaunchShape lp, cudaStream_t st) {
  const size_t sm = mix_smem(c, m);
  if (c.scheme == 2) {
    if (c.order == 1)
      em1m_deposit_initial_kernel<1><<<lp.grid, kEm1Threads, sm, st>>>(c, m, mb, b.err);
    else
      em1m_deposit_initial_kernel<2><<<lp.grid, kEm1Threads, sm, st>>>(c, m, mb, b.err);
    em1m_j1_to_fp64_kernel<<<1, kEm1Threads, 0, st>>>(c, b, m, mb);
  }
  const size_t hs = pass_smem(c) > sm ? pass_smem(c) : sm;
  em1d_half_kernel<<<1, kEm1Threads, hs, st>>>(c, b);
}

void em1m_from_fp64(const Em1dConst &c, const Em1dBufs &b, const Em1dMixConst &m,
                    const Em1dMixBufs &mb, LaunchShape lp, cudaStream_t st) {
  (void)c;
  em1m_from_fp64_kernel<<<lp.grid, kEm1Threads, 0, st>>>(b, m, mb);
}

void em1m_to_fp64(const Em1dConst &c, const Em1dBufs &b, const Em1dMixConst &m,
                  const Em1dMixBufs &mb, LaunchShape lp, cudaStream_t st) {
  (void)c;
  em1m_to_fp64_kernel<<<lp.grid, kEm1Threads, 0, st>>>(b, m, mb);
}

void em1m_energy(const Em1dConst &c, const Em1dBufs &b, const Em1dMixConst &m,
                 const Em1dMixBufs &mb, double *ke_out, double *wf, LaunchShape lp,
                 cudaStream_t st) {
  em1m_energy_kernel<<<lp.grid, kEm1Threads, 0, st>>>(c, b, m, mb, ke_out, wf);
}

void em1m_absmax(const Em1dBufs &b, int64_t n, unsigned long long *out, LaunchShape lp,
                 cudaStream_t st) {
  em1m_absmax_kernel<<<lp.grid, kEm1Threads, 0, st>>>(b, n, out);
}

}  // namespace pic
