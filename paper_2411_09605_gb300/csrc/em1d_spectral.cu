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
// Deposits: each lane of a block adds into its own copy of the block's
// current tile (rt copies, laid out [node][component][copy], rt up to 32 as
// shared memory allows), so FP64 shared atomics rarely meet; the flush sums
// the copies and adds the block's tile into one of kJSlices slices of the
// global current, which spreads the blocks' global atomics over kJSlices
// addresses per node; the field solve sums the slices.
#include <cuda_runtime.h>

#include "es1d_fp64_common.cuh"
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
template <int ORDER>
__device__ __forceinline__ void em1d_half_push(const Em1dConst &c, const double *Esx,
                                               const double *Esy, const double *Bs, double y,
                                               double vx, double vy, double qm, unsigned *err,
                                               double &vsx, double &vsy, double &yh) {
  const double hdt = 0.5 * c.dt;
  const double ys = wrap_periodic(__fma_rn(hdt, vy, y), c.L, err);
  const Shape64<ORDER> S(__dmul_rn(ys, c.inv_h), c.n);
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
    em1d_half_push<ORDER>(c, Esx, Esy, Bs, b.y[p], b.vx[p], b.vy[p], c.qm[s], b.err, vsx, vsy, yh);
    b.vsx[p] = vsx;   // pass E forms y^{n+1/2} from v* with the same rounding
    b.vsy[p] = vsy;
    const Shape64<ORDER> S(__dmul_rn(yh, c.inv_h), n);
    const double qw = marker_qw(c, b, s, p);
    tile_deposit<ORDER>(Jt, c.rt, S, qw * vsx, qw * vsy);
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
    const double yh = wrap_periodic(__fma_rn(hdt, vsy, y), c.L, b.err);
    const Shape64<ORDER> S(__dmul_rn(yh, c.inv_h), n);
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
      const double ys = wrap_periodic(fma(hdt, v1y, y1), c.L, b.err);
      const Shape64<ORDER> S2(ys * c.inv_h, n);
      const double qw = marker_qw(c, b, s, p);
      tile_deposit<ORDER>(Jt, c.rt, S2, qw * v1x, qw * v1y);
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
    const double ys = wrap_periodic(fma(0.5 * c.dt, b.vy[p], b.y[p]), c.L, b.err);
    const Shape64<ORDER> S(ys * c.inv_h, c.n);
    const double qw = marker_qw(c, b, s, p);
    tile_deposit<ORDER>(Jt, c.rt, S, qw * b.vx[p], qw * b.vy[p]);
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

}  // namespace pic
