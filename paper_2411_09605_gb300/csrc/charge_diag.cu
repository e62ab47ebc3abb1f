// Charge diagnostics of a state (Sec. 2.1): the deposited charge density, its
// total, and the residual of Gauss's law, which continuity (d rho/dt + div j =
// 0) keeps constant in time when the deposit conserves charge discretely
// (Sec. 3.5).
//
// 1D grids (Ampere solver): rho_j = (1/h) sum_p q w_p S(x_j - x_p) with the
// deposit's own shape; the residual r = D E - (rho - <rho>) with the spectral
// derivative D of the initial Poisson solve, on the Fourier modes m = 1 ..
// (nc - 1) / 2 (the k = 0 mode is the neutralising background; D does not
// represent the Nyquist mode).  gauss1d_modes_kernel forms r_m = i kappa_m E_m
// - rho_m mode by mode with direct sums over the nodes; gauss1d_nodes_kernel
// transforms r and the same modes of rho back to the nodes and sums their
// squares per block.  Both read a table of exp(2 pi i t / nc), t = m j mod nc,
// built once on the host.
//
// 2D Yee grids: rho on the nodes (i, j) with the bilinear shape of the
// charge-conserving option, and r = div_h E - (rho - <rho>) with the Yee
// divergence (Ex(i+1/2,j) - Ex(i-1/2,j)) / hx + (Ey(i,j+1/2) - Ey(i,j-1/2)) / hy.
#include <cuda_runtime.h>

#include "pic_internal.cuh"

namespace pic {
namespace {

constexpr int kDiagThreads = 256;

// Sums K doubles over a block in a fixed order (deterministic); thread 0 holds
// the result.
template <int K>
__device__ __forceinline__ void block_sum_k(double (&v)[K], double (*red)[32]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < K; k++)
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < K; k++) red[k][warp] = v[k];
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; k++) {
      double s = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += red[k][w];
      v[k] = s;
    }
  }
}

__global__ void rho_from_counts_kernel(const long long *cnt, int nc, double scale, double *rho) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += gridDim.x * blockDim.x)
    rho[i] = scale * (double)cnt[i];
}

// One block per mode m = 1 + blockIdx.x: E_m, rho_m = sum_j F_j exp(-2 pi i m j /
// nc), then r_m = i kappa_m E_m - rho_m.
__global__ void __launch_bounds__(kDiagThreads)
    gauss1d_modes_kernel(const double *E, const double *rho, int nc, double two_pi_over_L,
                         const double2 *tw, double2 *rm, double2 *pm) {
  __shared__ double red[4][32];
  const int m = blockIdx.x + 1;
  double v[4] = {0.0, 0.0, 0.0, 0.0};  // Re E_m, Im E_m, Re rho_m, Im rho_m
  for (int j = threadIdx.x; j < nc; j += blockDim.x) {
    const double2 e = tw[(int)(((long long)m * j) % nc)];
    v[0] += E[j] * e.x;
    v[1] -= E[j] * e.y;
    v[2] += rho[j] * e.x;
    v[3] -= rho[j] * e.y;
  }
  block_sum_k<4>(v, red);
  if (threadIdx.x == 0) {
    const double kappa = two_pi_over_L * (double)m;
    rm[m - 1] = make_double2(-kappa * v[1] - v[2], kappa * v[0] - v[3]);
    pm[m - 1] = make_double2(v[2], v[3]);
  }
}

// r_j = (2 / nc) sum_m Re(r_m exp(2 pi i m j / nc)) and the same for rho; per
// block: sum r_j^2, sum rhot_j^2 and sum rho_j (the raw charge, for Q).
__global__ void __launch_bounds__(kDiagThreads)
    gauss1d_nodes_kernel(const double2 *rm, const double2 *pm, const double *rho, int nc, int M,
                         const double2 *tw, double *r, double *part) {
  __shared__ double red[3][32];
  double v[3] = {0.0, 0.0, 0.0};
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < nc) {
    double rr = 0.0, rt = 0.0;
    for (int m = 1; m <= M; m++) {
      const double2 e = tw[(int)(((long long)m * j) % nc)];
      const double2 a = rm[m - 1], b = pm[m - 1];
      rr += a.x * e.x - a.y * e.y;
      rt += b.x * e.x - b.y * e.y;
    }
    rr *= 2.0 / nc;
    rt *= 2.0 / nc;
    r[j] = rr;
    v[0] = rr * rr;
    v[1] = rt * rt;
    v[2] = rho[j];
  }
  block_sum_k<3>(v, red);
  if (threadIdx.x == 0)
    for (int k = 0; k < 3; k++) part[3 * blockIdx.x + k] = v[k];
}

// Per block: sum of a[beg, end) (weights of one species).
__global__ void __launch_bounds__(kDiagThreads)
    sum_range_kernel(const double *a, int64_t n, double *part) {
  __shared__ double red[1][32];
  double v[1] = {0.0};
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x)
    v[0] += a[p];
  block_sum_k<1>(v, red);
  if (threadIdx.x == 0) part[blockIdx.x] = v[0];
}

__device__ __forceinline__ int em2d_species_of(const Em2dConst &c, int64_t p) {
  int s = 0;
  while (s < c.nsp - 1 && p >= c.sp_end[s]) s++;
  return s;
}

__device__ __forceinline__ int wrap_index(int i, int n) {
  i %= n;
  return i < 0 ? i + n : i;
}

// rho = sum_p q w_p B1(x/hx - i) B1(y/hy - j) / |h| on the nodes (i, j) (FP64
// global atomics; rho cleared by the caller).
__global__ void em2d_charge_kernel(Em2dConst c, const double *x, const double *y, const double *w,
                                   double *rho) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < c.n_total;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int s = em2d_species_of(c, p);
    const double qa = w ? c.q_a[s] * w[p] : c.qw_a[s];
    const double xi = x[p] * c.inv_hx, yj = y[p] * c.inv_hy;
    const double fx = floor(xi), fy = floor(yj);
    const double ax = xi - fx, ay = yj - fy;
    const int i0 = wrap_index((int)fx, c.nx), j0 = wrap_index((int)fy, c.ny);
    const int i1 = i0 + 1 == c.nx ? 0 : i0 + 1, j1 = j0 + 1 == c.ny ? 0 : j0 + 1;
    const double wx[2] = {1.0 - ax, ax}, wy[2] = {1.0 - ay, ay};
    const int ix[2] = {i0, i1}, iy[2] = {j0, j1};
    for (int b = 0; b < 2; b++)
      for (int a = 0; a < 2; a++) atomicAdd(&rho[iy[b] * c.nx + ix[a]], qa * wx[a] * wy[b]);
  }
}

// r = div_h E - (rho - mean) on the nodes; per block: sum r^2, sum (rho -
// mean)^2 and sum rho.
__global__ void __launch_bounds__(kDiagThreads)
    em2d_gauss_kernel(Em2dConst c, const double *E, const double *rho, double mean, double *r,
                      double *part) {
  __shared__ double red[3][32];
  double v[3] = {0.0, 0.0, 0.0};
  const int ncell = c.nx * c.ny;
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a < ncell) {
    const int i = a % c.nx, j = a / c.nx;
    const int im = i == 0 ? c.nx - 1 : i - 1, jm = j == 0 ? c.ny - 1 : j - 1;
    const double *Ex = E, *Ey = E + ncell;
    const double div = (Ex[a] - Ex[j * c.nx + im]) * c.inv_hx + (Ey[a] - Ey[jm * c.nx + i]) * c.inv_hy;
    const double rt = rho[a] - mean;
    const double rr = div - rt;
    r[a] = rr;
    v[0] = rr * rr;
    v[1] = rt * rt;
    v[2] = rho[a];
  }
  block_sum_k<3>(v, red);
  if (threadIdx.x == 0)
    for (int k = 0; k < 3; k++) part[3 * blockIdx.x + k] = v[k];
}

}  // namespace

int diag_blocks(int nodes) { return (nodes + kDiagThreads - 1) / kDiagThreads; }

void diag_rho_from_counts(const long long *cnt, int nc, double scale, double *rho,
                          cudaStream_t st) {
  rho_from_counts_kernel<<<diag_blocks(nc), kDiagThreads, 0, st>>>(cnt, nc, scale, rho);
}

void diag_gauss1d(const double *E, const double *rho, int nc, double L, const double2 *tw,
                  double2 *rm, double2 *pm, double *r, double *part, cudaStream_t st) {
  const int M = (nc - 1) / 2;
  if (M > 0)
    gauss1d_modes_kernel<<<M, kDiagThreads, 0, st>>>(E, rho, nc, 6.283185307179586476925286766559 / L,
                                                     tw, rm, pm);
  gauss1d_nodes_kernel<<<diag_blocks(nc), kDiagThreads, 0, st>>>(rm, pm, rho, nc, M, tw, r, part);
}

void diag_sum_range(const double *a, int64_t n, double *part, int blocks, cudaStream_t st) {
  sum_range_kernel<<<blocks, kDiagThreads, 0, st>>>(a, n, part);
}

void diag_em2d_charge(const Em2dConst &c, const double *x, const double *y, const double *w,
                      double *rho, LaunchShape lp, cudaStream_t st) {
  em2d_charge_kernel<<<lp.grid, 256, 0, st>>>(c, x, y, w, rho);
}

void diag_em2d_gauss(const Em2dConst &c, const double *E, const double *rho, double mean,
                     double *r, double *part, cudaStream_t st) {
  em2d_gauss_kernel<<<diag_blocks(c.nx * c.ny), kDiagThreads, 0, st>>>(c, E, rho, mean, r, part);
}

}  // namespace pic
