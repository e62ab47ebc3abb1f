// 1D1V electrostatic ESEC1 / ESEC2 step, plain FP64 form.
//
// Two particle passes per ESEC2 step, separated by the only global dependencies
// of the scheme (Sec. 3.3, Eq. good_translation): the deposited currents.
//   pass C: E* = E^n - dt/2 (j^{n,*} - <j^{n,*}>) in the prologue (every block,
//           redundantly, from the tiny grid), then per particle
//           x* -> E**_p -> v* -> x^{n+1/2} -> deposit j^{*,n+1/2}; v* is stored.
//   pass E: E^{n+1} = E^n - dt (j^{*,n+1/2} - <.>) and E^{n+1/2} in the prologue,
//           then per particle v* loaded and x^{n+1/2} formed with pass C's
//           rounding (the FP64 pipe, not HBM, bounds this form: a load is
//           cheaper than recomputing x*, E**_p and v*),
//           E^{n+1/2}_p, v^dag, Gamma (Eq. opt_solution) with the imaginary-root
//           fallback of Sec. 3.2, x^{n+1}, v^{n+1}; for ESEC2 the next step's
//           x* and j^{n+1,*} deposit are fused in (Eq. doublestardef).
// The whole 1D grid lives in shared memory; each block accumulates its current
// in a shared tile and flushes it with one global atomic per touched node.
// ESEC1 (Eq. naivetranslation + Eq. PICmodification) gathers E^n at x* and
// skips the j^{n,*} deposit.
#include <cuda_runtime.h>

#include <type_traits>

#include "es1d_fp64_common.cuh"
#include "pic_internal.cuh"

namespace pic {
namespace {

// Block-wide mean of a grid array (fixed summation order: every block gets the
// identical value).
__device__ double block_mean(const double *a, int n, double *red) {
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += a[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) red[warp] = s;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0) {
    for (int k = 0; k < (int)(blockDim.x >> 5); k++) t += red[k];
    red[32] = t / (double)n;
  }
  __syncthreads();
  double m = red[32];
  __syncthreads();
  return m;
}

__device__ double block_sum(double s, double *red) {
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[warp] = s;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int k = 0; k < (int)(blockDim.x >> 5); k++) t += red[k];
  return t;  // valid in thread 0
}

// E* = E^n - dt/2 (J1 - <J1>) (ESEC2) or E^n (ESEC1), into shared memory.
template <int SCHEME>
__device__ void build_estar(const Es1dConst &c, const double *E, const double *J1, double *Es,
                            double *red) {
  if (SCHEME == 2) {
    double mean = c.remove_mean ? block_mean(J1, c.nc, red) : 0.0;
    double hdt = 0.5 * c.dt;
    for (int i = threadIdx.x; i < c.nc; i += blockDim.x) Es[i] = E[i] - hdt * (J1[i] - mean);
  } else {
    for (int i = threadIdx.x; i < c.nc; i += blockDim.x) Es[i] = E[i];
  }
}

// a <- F^passes a in shared memory (the 1-2-1 filter, periodic), ping-ponging
// with tmp; returns the buffer that holds the result.
__device__ double *smem_filter(double *a, double *tmp, int nc, int passes) {
  for (int k = 0; k < passes; k++) {
    __syncthreads();
    for (int i = threadIdx.x; i < nc; i += blockDim.x) {
      const int im = i == 0 ? nc - 1 : i - 1, ip = i + 1 == nc ? 0 : i + 1;
      tmp[i] = 0.25 * (a[im] + 2.0 * a[i] + a[ip]);
    }
    double *t = a;
    a = tmp;
    tmp = t;
  }
  __syncthreads();
  return a;
}

// With filtering: Es = F E*, E* = E^n - dt/2 (F J1 - <J1>) (ESEC2) or E^n;
// T is nc doubles of scratch (the filter keeps the mean, <F J1> = <J1>).
template <int SCHEME>
__device__ void build_estar_filtered(const Es1dConst &c, const double *E, const double *J1,
                                     double *Es, double *T, double *red) {
  double *o = T;
  if (SCHEME == 2) {
    const double mean = c.remove_mean ? block_mean(J1, c.nc, red) : 0.0;
    for (int i = threadIdx.x; i < c.nc; i += blockDim.x) T[i] = J1[i];
    double *fj = smem_filter(T, Es, c.nc, c.passes);
    o = fj == T ? Es : T;
    const double hdt = 0.5 * c.dt;
    for (int i = threadIdx.x; i < c.nc; i += blockDim.x) o[i] = E[i] - hdt * (fj[i] - mean);
    double *r = smem_filter(o, fj, c.nc, c.passes);
    if (r != Es)
      for (int i = threadIdx.x; i < c.nc; i += blockDim.x) Es[i] = r[i];
  } else {
    for (int i = threadIdx.x; i < c.nc; i += blockDim.x) T[i] = E[i];
    double *r = smem_filter(T, Es, c.nc, c.passes);
    if (r != Es)
      for (int i = threadIdx.x; i < c.nc; i += blockDim.x) Es[i] = r[i];
  }
  __syncthreads();
}

__device__ void flush_tile(const double *Jt, double *J, int nc) {
  for (int i = threadIdx.x; i < nc; i += blockDim.x) {
    double a = Jt[i];
    if (a != 0.0) atomicAdd(&J[i], a);
  }
}

// Reduces the previous step's block partials into te[slot] (block 0 only).
__device__ void finalize_stats(const Es1dFp64Bufs &b, int slot, int nblocks, double *red) {
  double s = 0.0;
  for (int i = threadIdx.x; i < nblocks; i += blockDim.x) s += b.ke_part[i];
  double t = block_sum(s, red);
  if (threadIdx.x == 0) {
    double te = t + b.we[0];
    b.te[slot] = te;
    if (!isfinite(te)) atomicOr(b.err, kErrNonfinite);
  }
}

template <int ORDER, int SCHEME>
__global__ void __launch_bounds__(512) pass_c_kernel(Es1dConst c, Es1dFp64Bufs b, int par,
                                                     int prev_slot, int prev_nblocks) {
  extern __shared__ double sm[];
  double *Es = sm;
  double *Jt = sm + c.nc;
  __shared__ double red[33];
  if (c.passes > 0)
    build_estar_filtered<SCHEME>(c, b.E[par], b.J1[par], Es, Jt, red);
  else
    build_estar<SCHEME>(c, b.E[par], b.J1[par], Es, red);
  for (int i = threadIdx.x; i < c.nc; i += blockDim.x) Jt[i] = 0.0;
  if (blockIdx.x == 0) {
    if (SCHEME == 2)
      for (int i = threadIdx.x; i < c.nc; i += blockDim.x) b.J1[par ^ 1][i] = 0.0;
    if (prev_slot >= 0) finalize_stats(b, prev_slot, prev_nblocks, red);
  }
  __syncthreads();
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < c.n_total;
       p += (int64_t)gridDim.x * blockDim.x) {
    int s = species_of(c, p);
    double x = b.x[p], v = b.v[p];
    double vs, xh;
    if (SCHEME == 2 && b.sws) {
      // the shape at x* that the previous pass E (or the initial deposit)
      // deposited j^{n,*} with, the same bits as forming it here
      Shape64<ORDER> Sx;
      Sx.load(b.sws, b.sis, p, c.n_total, c.nc);
      half_push_at<ORDER>(c, Es, Sx, x, v, c.qm[s], b.err, vs, xh);
    } else {
      half_push<ORDER>(c, Es, x, v, c.qm[s], b.err, vs, xh);
    }
    if (b.vs) b.vs[p] = vs;   // pass E forms x^{n+1/2} from it with the same rounding
    double coef = (b.w ? c.q_h[s] * b.w[p] : c.qw_h[s]) * vs;
    Shape64<ORDER> S(__dmul_rn(xh, c.inv_h), c.nc);
    S.deposit(Jt, coef);
    if (b.sw) S.store(b.sw, b.si, p, c.n_total);  // pass E gathers with it
  }
  __syncthreads();
  flush_tile(Jt, b.J2[par], c.nc);
}

template <int ORDER, int SCHEME>
__global__ void __launch_bounds__(512) pass_e_kernel(Es1dConst c, Es1dFp64Bufs b, int par,
                                                     int slot) {
  extern __shared__ double sm[];
  double *Es = sm;
  double *Eh = sm + c.nc;
  double *Jt = sm + 2 * c.nc;
  __shared__ double red[33];
  const double *E = b.E[par];
  const double *J2 = b.J2[par];
  double mean2 = c.remove_mean ? block_mean(J2, c.nc, red) : 0.0;
  double we_loc = 0.0;
  if (c.passes > 0) {
    // E^{n+1} = E^n - dt (F J2 - <J2>) (the state, unfiltered), gather table
    // F E^{n+1/2}; Jt and Eh serve as scratch before the tile is cleared
    for (int i = threadIdx.x; i < c.nc; i += blockDim.x) Jt[i] = J2[i];
    double *fj = smem_filter(Jt, Eh, c.nc, c.passes);
    double *o = fj == Jt ? Eh : Jt;
    for (int i = threadIdx.x; i < c.nc; i += blockDim.x) {
      double en = E[i] - c.dt * (fj[i] - mean2);
      o[i] = 0.5 * (E[i] + en);
      if (blockIdx.x == 0) {
        b.E[par ^ 1][i] = en;
        b.J2[par ^ 1][i] = 0.0;
        we_loc += en * en;
      }
    }
    double *r = smem_filter(o, fj, c.nc, c.passes);
    if (r != Eh)
      for (int i = threadIdx.x; i < c.nc; i += blockDim.x) Eh[i] = r[i];
    __syncthreads();
    build_estar_filtered<SCHEME>(c, E, b.J1[par], Es, Jt, red);
    for (int i = threadIdx.x; i < c.nc; i += blockDim.x) Jt[i] = 0.0;
  } else {
    for (int i = threadIdx.x; i < c.nc; i += blockDim.x) {
      double en = E[i] - c.dt * (J2[i] - mean2);
      Eh[i] = 0.5 * (E[i] + en);
      Jt[i] = 0.0;
      if (blockIdx.x == 0) {
        b.E[par ^ 1][i] = en;
        b.J2[par ^ 1][i] = 0.0;
        we_loc += en * en;
      }
    }
    build_estar<SCHEME>(c, E, b.J1[par], Es, red);
  }
  if (blockIdx.x == 0) {
    double t = block_sum(we_loc, red);
    if (threadIdx.x == 0) b.we[0] = 0.5 * c.h * t;
  }
  __syncthreads();
  double ke = 0.0;
  unsigned nfb = 0;
  const double hdt = 0.5 * c.dt;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < c.n_total;
       p += (int64_t)gridDim.x * blockDim.x) {
    int s = species_of(c, p);
    double x = b.x[p], v = b.v[p];
    double qm = c.qm[s];
    // v* and the shape at x^{n+1/2} that pass C deposited with (loaded: on
    // this FP64-bound pass bytes are cheaper than the shape's arithmetic);
    // without those arrays (the entry point without allocation), half_push
    // again on the same E* table, which gives the same bits
    double vs;
    Shape64<ORDER> Sh;
    if (b.vs && b.sw) {
      vs = b.vs[p];
      Sh.load(b.sw, b.si, p, c.n_total, c.nc);
    } else {
      double xh;
      if (b.vs) {
        vs = b.vs[p];
        xh = wrap_periodic(__fma_rn(hdt, vs, x), c.L, b.err);
      } else {
        half_push<ORDER>(c, Es, x, v, qm, b.err, vs, xh);
      }
      Sh = Shape64<ORDER>(__dmul_rn(xh, c.inv_h), c.nc);
    }
    double Ep = Sh.gather(Eh);
    double vd = v + c.dt * qm * Ep;
    double R = v * v + 2.0 * vs * (vd - v);
    double vd2 = vd * vd;
    double vn = vd;
    if (c.gamma_on) {
      // v^{n+1} = Gamma v^dag with Gamma = sqrt(R) / |v^dag| (Eq. opt_solution):
      // in 1D that is sqrt(R) with the sign of v^dag (one square root, no
      // division)
      if (R < 0.0 || vd2 == 0.0)
        nfb++;
      else
        vn = copysign(sqrt(R), vd);
    }
    double xn = wrap_periodic(x + c.dt * vs, c.L, b.err);
    double wp = b.w ? b.w[p] : 1.0;
    ke += (b.w ? c.half_m[s] * wp : c.half_mw[s]) * vn * vn;
    if (SCHEME == 2) {
      Shape64<ORDER> S2(__dmul_rn(xstar(c, xn, vn, b.err), c.inv_h), c.nc);
      S2.deposit(Jt, (b.w ? c.q_h[s] * wp : c.qw_h[s]) * vn);
      if (b.sws) S2.store(b.sws, b.sis, p, c.n_total);  // the next pass C gathers with it
    }
    b.x[p] = xn;
    b.v[p] = vn;
  }
  // per-warp fallback count -> one atomic per warp
  for (int o = 16; o > 0; o >>= 1) nfb += __shfl_xor_sync(0xffffffffu, nfb, o);
  if ((threadIdx.x & 31) == 0 && nfb) atomicAdd(&b.fallback[slot], (unsigned long long)nfb);
  double t = block_sum(ke, red);
  if (threadIdx.x == 0) b.ke_part[blockIdx.x] = t;
  if (SCHEME == 2) {
    __syncthreads();
    flush_tile(Jt, b.J1[par ^ 1], c.nc);
  }
}

// j^{n,*} of the current state (ESEC2 start-up and after a state change).
template <int ORDER>
__global__ void __launch_bounds__(512) deposit_initial_kernel(Es1dConst c, Es1dFp64Bufs b,
                                                              int par) {
  extern __shared__ double sm[];
  double *Jt = sm;
  for (int i = threadIdx.x; i < c.nc; i += blockDim.x) Jt[i] = 0.0;
  __syncthreads();
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < c.n_total;
       p += (int64_t)gridDim.x * blockDim.x) {
    int s = species_of(c, p);
    double x = b.x[p], v = b.v[p];
    Shape64<ORDER> S(__dmul_rn(xstar(c, x, v, b.err), c.inv_h), c.nc);
    S.deposit(Jt, (b.w ? c.q_h[s] * b.w[p] : c.qw_h[s]) * v);
    if (b.sws) S.store(b.sws, b.sis, p, c.n_total);  // pass C gathers with it
  }
  __syncthreads();
  flush_tile(Jt, b.J1[par], c.nc);
}

__global__ void finalize_kernel(Es1dFp64Bufs b, int slot, int nblocks) {
  __shared__ double red[33];
  finalize_stats(b, slot, nblocks, red);
}

// rho = (1/h) sum q w S(x_h - x_p) (for the initial Poisson solve).
template <int ORDER>
__global__ void __launch_bounds__(512) charge_kernel(Es1dConst c, const double *x,
                                                     const double *w, double *rho) {
  extern __shared__ double sm[];
  double *Jt = sm;
  for (int i = threadIdx.x; i < c.nc; i += blockDim.x) Jt[i] = 0.0;
  __syncthreads();
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < c.n_total;
       p += (int64_t)gridDim.x * blockDim.x) {
    int s = species_of(c, p);
    Shape64<ORDER> S(x[p] * c.inv_h, c.nc);
    S.deposit(Jt, w ? c.q_h[s] * w[p] : c.qw_h[s]);
  }
  __syncthreads();
  flush_tile(Jt, rho, c.nc);
}

// KE per species: (1/2) m sum w v^2, one block per species slice, fixed order.
__global__ void __launch_bounds__(512) kinetic_kernel(Es1dConst c, const double *v,
                                                      const double *w, double *ke_sp) {
  __shared__ double red[33];
  int s = blockIdx.x;
  int64_t beg = s == 0 ? 0 : c.sp_end[s - 1], end = c.sp_end[s];
  double acc = 0.0;
  for (int64_t p = beg + threadIdx.x; p < end; p += blockDim.x) {
    double vv = v[p] * v[p];
    acc += w ? c.half_m[s] * w[p] * vv : c.half_mw[s] * vv;
  }
  double t = block_sum(acc, red);
  if (threadIdx.x == 0) ke_sp[s] = t;
}

template <typename F>
void dispatch(int order, int scheme, F f) {
  if (order == 1 && scheme == 1) f(std::integral_constant<int, 1>(), std::integral_constant<int, 1>());
  if (order == 1 && scheme == 2) f(std::integral_constant<int, 1>(), std::integral_constant<int, 2>());
  if (order == 2 && scheme == 1) f(std::integral_constant<int, 2>(), std::integral_constant<int, 1>());
  if (order == 2 && scheme == 2) f(std::integral_constant<int, 2>(), std::integral_constant<int, 2>());
}

}  // namespace

void es1d_fp64_deposit_initial(const Es1dConst &c, const Es1dFp64Bufs &b, int parity,
                               LaunchShape ls, cudaStream_t st) {
  size_t smem = sizeof(double) * c.nc;
  if (c.order == 1)
    deposit_initial_kernel<1><<<ls.grid, ls.block, smem, st>>>(c, b, parity);
  else
    deposit_initial_kernel<2><<<ls.grid, ls.block, smem, st>>>(c, b, parity);
}

void es1d_fp64_pass_c(const Es1dConst &c, const Es1dFp64Bufs &b, int64_t step_index, int slot,
                      LaunchShape ls, cudaStream_t st) {
  int par = (int)(step_index & 1);
  int prev_slot = slot - 1;  // the stats of the previous step in this window
  dispatch(c.order, c.scheme, [&](auto O, auto S) {
    constexpr int ORDER = decltype(O)::value, SCHEME = decltype(S)::value;
    size_t smc = sizeof(double) * 2 * c.nc;
    pass_c_kernel<ORDER, SCHEME><<<ls.grid, ls.block, smc, st>>>(c, b, par, prev_slot, ls.grid);
  });
}

void es1d_fp64_pass_e(const Es1dConst &c, const Es1dFp64Bufs &b, int64_t step_index, int slot,
                      LaunchShape ls, cudaStream_t st) {
  int par = (int)(step_index & 1);
  dispatch(c.order, c.scheme, [&](auto O, auto S) {
    constexpr int ORDER = decltype(O)::value, SCHEME = decltype(S)::value;
    size_t sme = sizeof(double) * 3 * c.nc;
    pass_e_kernel<ORDER, SCHEME><<<ls.grid, ls.block, sme, st>>>(c, b, par, slot);
  });
}

cudaError_t es1d_fp64_prepare(const Es1dConst &c) {
  cudaError_t e = cudaSuccess;
  dispatch(c.order, c.scheme, [&](auto O, auto S) {
    constexpr int ORDER = decltype(O)::value, SCHEME = decltype(S)::value;
    int smc = (int)(sizeof(double) * 2 * c.nc), sme = (int)(sizeof(double) * 3 * c.nc);
    e = cudaFuncSetAttribute(pass_c_kernel<ORDER, SCHEME>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, smc);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(pass_e_kernel<ORDER, SCHEME>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, sme);
    int sm1 = (int)(sizeof(double) * c.nc);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(deposit_initial_kernel<ORDER>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, sm1);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(charge_kernel<ORDER>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               sm1);
  });
  return e;
}

void es1d_fp64_finalize(const Es1dConst &c, const Es1dFp64Bufs &b, int slot, int nblocks,
                        cudaStream_t st) {
  (void)c;
  finalize_kernel<<<1, 256, 0, st>>>(b, slot, nblocks);
}

void es1d_fp64_charge(const Es1dConst &c, const double *x, const double *w, double *rho,
                      LaunchShape ls, cudaStream_t st) {
  size_t smem = sizeof(double) * c.nc;
  if (c.order == 1)
    charge_kernel<1><<<ls.grid, ls.block, smem, st>>>(c, x, w, rho);
  else
    charge_kernel<2><<<ls.grid, ls.block, smem, st>>>(c, x, w, rho);
}

void es1d_fp64_kinetic(const Es1dConst &c, const double *v, const double *w, double *ke_sp,
                       cudaStream_t st) {
  kinetic_kernel<<<c.nsp, 512, 0, st>>>(c, v, w, ke_sp);
}

}  // namespace pic
