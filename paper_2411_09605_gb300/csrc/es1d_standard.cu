// Standard explicit PIC, the comparison scheme of Sec. 5: Vlasov-Poisson with
// the classical leapfrog push (in 1D1V the Boris push without B) and a
// binomially filtered charge density, FP64, 1D1V.  It does not conserve
// energy; it is here to measure the energy-conserving schemes against.
//
// State: x^n, v^{n-1/2} and E^n, the field of the filtered charge of x^n.
// One launch per step:
//   every block: E^n table in shared memory; per marker E^n_p,
//     v^{n+1/2} = v^{n-1/2} + dt (q/m) E^n_p, x^{n+1} = x^n + dt v^{n+1/2},
//     the kinetic partial (1/2) m w (v^{n-1/2}^2 + v^{n+1/2}^2) / 2, and the
//     charge q w S(x_h - x^{n+1}) / h into this lane's copy of the block tile;
//   the block that finishes last (a counter after a fence; nothing waits):
//     TE^n = KE^n + (h/2) sum (E^n)^2, then E^{n+1} from the charge: forward
//     FFT, E_k = rho_k F_k / (i kk_k) with the filter gain
//     F_k = cos^{2p}(pi k / n) of p passes of the 1-2-1 filter (its exact
//     effect on mode k) and 0 for k = 0 (the ion background) and the Nyquist
//     mode, inverse FFT.
#include <cuda_runtime.h>

#include "es1d_fp64_common.cuh"
#include "pic_internal.cuh"
#include "spectral_common.cuh"

namespace pic {
namespace {

constexpr int kStdThreads = 256;

__device__ __forceinline__ int species_of_std(const StdConst &c, int64_t p) {
  int s = 0;
  while (s < c.nsp - 1 && p >= c.sp_end[s]) s++;
  return s;
}

__device__ __forceinline__ double std_qw(const StdConst &c, const StdBufs &b, int s, int64_t p) {
  return b.w ? c.q_h[s] * b.w[p] : c.qw_h[s];
}

// The marker's charge into this lane's copy of the tile [n][rt].
template <int ORDER>
__device__ __forceinline__ void charge_deposit(double *Jt, int rt, const Shape64<ORDER> &S,
                                               double a) {
  const int l = threadIdx.x & (rt - 1);
#pragma unroll
  for (int k = 0; k <= ORDER; k++) atomicAdd(&Jt[(size_t)S.idx[k] * rt + l], a * S.w[k]);
}

// Sums each node's copies (rotated start: different banks per thread) and adds
// the non-zero totals into this block's slice of rho [kJSlices][n].
__device__ void flush_charge(const double *Jt, int rt, double *rho, int n) {
  double *r = rho + (size_t)(blockIdx.x & (kJSlices - 1)) * n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double *q = Jt + (size_t)i * rt;
    double a = 0.0;
    for (int k = 0; k < rt; k++) a += q[(k + i) & (rt - 1)];
    if (a != 0.0) atomicAdd(&r[i], a);
  }
}

// E from the sliced charge (one block; shared scratch of 4n + 2 doubles):
// E_k = -i sign(kk_k) g_{|k|} rho_k with g = F / |kk| tabulated; the slices
// are cleared for the next deposit.
__device__ void poisson_from_charge(const StdConst &c, const StdBufs &b, double2 *Z) {
  const int n = c.n;
  double2 *tw = Z + n;
  double *g = (double *)(tw + n / 2);
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kJSlices; k++) s += __ldcg(b.rho + (size_t)k * n + i);
    Z[i] = make_double2(s, 0.0);
  }
  for (int i = threadIdx.x; i < n / 2; i += blockDim.x) tw[i] = __ldg(b.tw + i);
  for (int i = threadIdx.x; i <= n / 2; i += blockDim.x) g[i] = __ldg(b.g + i);
  __syncthreads();
  block_fft(Z, n, c.log2n, -1, tw);
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const bool neg = k > n / 2;
    const double gk = neg ? -g[n - k] : g[k];
    const double2 r = Z[k];
    Z[k] = make_double2(gk * r.y, -gk * r.x);   // -i gk rho_k
  }
  __syncthreads();
  block_fft(Z, n, c.log2n, 1, tw);
  const double inv_n = 1.0 / (double)n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) b.E[i] = Z[i].x * inv_n;
  for (int i = threadIdx.x; i < kJSlices * n; i += blockDim.x) b.rho[i] = 0.0;
  __syncthreads();
}

template <int ORDER>
__global__ void __launch_bounds__(kStdThreads) std_step_kernel(StdConst c, StdBufs b, int slot) {
  extern __shared__ double sm[];
  __shared__ double red[33];
  const int n = c.n;
  double *Es = sm, *Jt = sm + n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) Es[i] = b.E[i];
  for (int i = threadIdx.x; i < n * c.rt; i += blockDim.x) Jt[i] = 0.0;
  __syncthreads();
  double ke = 0.0;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < c.n_total;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int s = species_of_std(c, p);
    const double x = b.x[p], v = b.v[p];
    const Shape64<ORDER> S(x * c.inv_h, n);
    const double vn = fma(c.dt * c.qm[s], S.gather(Es), v);
    ke = fma(c.half_m[s] * (b.w ? b.w[p] : c.w0[s]), 0.5 * fma(v, v, vn * vn), ke);
    const double x1 = wrap_periodic(fma(c.dt, vn, x), c.L, b.err);
    b.x[p] = x1;
    b.v[p] = vn;
    const Shape64<ORDER> S1(x1 * c.inv_h, n);
    charge_deposit<ORDER>(Jt, c.rt, S1, std_qw(c, b, s, p));
  }
  if (!isfinite(ke)) atomicOr(b.err, kErrNonfinite);
  const double kb = block_sum_d(ke, red);
  if (threadIdx.x == 0) b.ke_part[blockIdx.x] = kb;
  __syncthreads();
  flush_charge(Jt, c.rt, b.rho, n);
  if (arrive_last(b.done)) {
    // TE^n: the kinetic partials in a fixed order and W_E of the E^n used
    double t = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) t = fma(0.5 * c.h * Es[i], Es[i], t);
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) t += __ldcg(b.ke_part + i);
    const double te = block_sum_d(t, red);
    if (threadIdx.x == 0) b.te[slot] = te;
    __syncthreads();
    poisson_from_charge(c, b, (double2 *)sm);
  }
}

// rho^0 of x^0 and, from the last block, E^0.
template <int ORDER>
__global__ void __launch_bounds__(kStdThreads) std_charge_kernel(StdConst c, StdBufs b) {
  extern __shared__ double sm[];
  double *Jt = sm;
  for (int i = threadIdx.x; i < c.n * c.rt; i += blockDim.x) Jt[i] = 0.0;
  __syncthreads();
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < c.n_total;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int s = species_of_std(c, p);
    const Shape64<ORDER> S(b.x[p] * c.inv_h, c.n);
    charge_deposit<ORDER>(Jt, c.rt, S, std_qw(c, b, s, p));
  }
  __syncthreads();
  flush_charge(Jt, c.rt, b.rho, c.n);
  if (arrive_last(b.done)) poisson_from_charge(c, b, (double2 *)sm);
}

// v^{-1/2} = v^0 - dt/2 (q/m) E^0_p (the start of the leapfrog).
template <int ORDER>
__global__ void __launch_bounds__(kStdThreads) std_kick_back_kernel(StdConst c, StdBufs b) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < c.n_total;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int s = species_of_std(c, p);
    const Shape64<ORDER> S(b.x[p] * c.inv_h, c.n);
    b.v[p] = fma(-0.5 * c.dt * c.qm[s], S.gather(b.E), b.v[p]);
  }
}

// KE^n per species with v^{n+1/2} formed but not stored (block partials
// [nsp][grid]), and from block 0 W_E^n.
template <int ORDER>
__global__ void __launch_bounds__(kStdThreads) std_energy_kernel(StdConst c, StdBufs b,
                                                                  double *ke_out, double *we) {
  __shared__ double red[33];
  for (int s = 0; s < c.nsp; s++) {
    const int64_t lo = s == 0 ? 0 : c.sp_end[s - 1], hi = c.sp_end[s];
    double acc = 0.0;
    for (int64_t p = lo + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < hi;
         p += (int64_t)gridDim.x * blockDim.x) {
      const Shape64<ORDER> S(b.x[p] * c.inv_h, c.n);
      const double v = b.v[p], vn = fma(c.dt * c.qm[s], S.gather(b.E), v);
      acc = fma(b.w ? b.w[p] : c.w0[s], 0.5 * fma(v, v, vn * vn), acc);
    }
    const double t = block_sum_d(acc, red);
    if (threadIdx.x == 0) ke_out[(size_t)s * gridDim.x + blockIdx.x] = c.half_m[s] * t;
    __syncthreads();
  }
  if (blockIdx.x == 0) {
    double a = 0.0;
    for (int i = threadIdx.x; i < c.n; i += blockDim.x) a = fma(b.E[i], b.E[i], a);
    const double t = block_sum_d(a, red);
    if (threadIdx.x == 0) *we = 0.5 * c.h * t;
  }
}

// Twiddles and g_k = cos^{2p}(pi k / n) / |kk_k| for k = 0 .. n/2 (0 for k = 0
// and the Nyquist mode); one block, once per set-up.
__global__ void std_tables_kernel(StdConst c, StdBufs b) {
  const int n = c.n;
  for (int j = threadIdx.x; j < n / 2; j += blockDim.x) {
    double s, co;
    sincospi(-2.0 * (double)j / (double)n, &s, &co);
    b.tw[j] = make_double2(co, s);
  }
  for (int k = threadIdx.x; k <= n / 2; k += blockDim.x) {
    if (k == 0 || 2 * k == n) {
      b.g[k] = 0.0;
      continue;
    }
    const double cs = cospi((double)k / (double)n);
    double f = 1.0;
    for (int q = 0; q < c.passes; q++) f *= cs * cs;
    b.g[k] = f / (2.0 * 3.141592653589793 * (double)k / c.L);
  }
}

size_t std_smem(const StdConst &c) {
  const size_t a = (1 + (size_t)c.rt) * c.n, f = 4 * (size_t)c.n + 2;
  return sizeof(double) * (a > f ? a : f);
}

template <typename K>
cudaError_t allow(K kernel, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

int std_tile_copies(int n) {
  int rt = 32;
  while (rt > 1 && sizeof(double) * (1 + (size_t)rt) * n > kEm1TileBudget) rt >>= 1;
  return rt;
}

cudaError_t std_prepare(const StdConst &c, const StdBufs &b, cudaStream_t st) {
  const size_t sm = std_smem(c);
  cudaError_t e = cudaSuccess;
  if (c.order == 1) {
    if ((e = allow(std_step_kernel<1>, sm)) || (e = allow(std_charge_kernel<1>, sm))) return e;
  } else {
    if ((e = allow(std_step_kernel<2>, sm)) || (e = allow(std_charge_kernel<2>, sm))) return e;
  }
  std_tables_kernel<<<1, kStdThreads, 0, st>>>(c, b);
  return cudaGetLastError();
}

void std_step(const StdConst &c, const StdBufs &b, int slot, LaunchShape lp, cudaStream_t st) {
  const size_t sm = std_smem(c);
  if (c.order == 1)
    std_step_kernel<1><<<lp.grid, kStdThreads, sm, st>>>(c, b, slot);
  else
    std_step_kernel<2><<<lp.grid, kStdThreads, sm, st>>>(c, b, slot);
}

void std_start(const StdConst &c, const StdBufs &b, LaunchShape lp, cudaStream_t st) {
  const size_t sm = std_smem(c);
  if (c.order == 1) {
    std_charge_kernel<1><<<lp.grid, kStdThreads, sm, st>>>(c, b);
    std_kick_back_kernel<1><<<lp.grid, kStdThreads, 0, st>>>(c, b);
  } else {
    std_charge_kernel<2><<<lp.grid, kStdThreads, sm, st>>>(c, b);
    std_kick_back_kernel<2><<<lp.grid, kStdThreads, 0, st>>>(c, b);
  }
}

void std_energy(const StdConst &c, const StdBufs &b, double *ke_out, double *we, LaunchShape lp,
                cudaStream_t st) {
  if (c.order == 1)
    std_energy_kernel<1><<<lp.grid, kStdThreads, 0, st>>>(c, b, ke_out, we);
  else
    std_energy_kernel<2><<<lp.grid, kStdThreads, 0, st>>>(c, b, ke_out, we);
}

}  // namespace pic
