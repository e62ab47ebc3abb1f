// Grid helpers shared by the FP64 and mixed forms of the 2D3V Yee step
// (Sec. 4.1, Eq. EMleapfrog): periodic index wrap, the discrete curls on the
// staggered lattice, a block sum, the B update with the field energies (K5)
// and the step's total energy.  Both forms advance the fields with the
// same FP64 curls, so their field energies are computed the same way.
#pragma once

#include <cuda_runtime.h>

#include "pic_internal.cuh"

namespace pic {
namespace {

__device__ __forceinline__ int wrapi(int i, int n) {
  if ((unsigned)i < (unsigned)n) return i;
  int r = i % n;
  return r < 0 ? r + n : r;
}

// Sum over the block of one double per thread (valid in thread 0).
__device__ double block_sum2(double s, double *red) {
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[warp] = s;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int k = 0; k < (int)(blockDim.x >> 5); k++) t += red[k];
  return t;
}

// curl of B on the E locations at (i, j), component d
__device__ __forceinline__ double curl_b(const Em2dConst &c, const double *B, int i, int j, int d) {
  const int nx = c.nx, ny = c.ny, nc = nx * ny;
  const double *Bx = B, *By = B + nc, *Bz = B + 2 * nc;
  const int im = i == 0 ? nx - 1 : i - 1, jm = j == 0 ? ny - 1 : j - 1;
  if (d == 0) return (Bz[j * nx + i] - Bz[jm * nx + i]) * c.inv_hy;
  if (d == 1) return -(Bz[j * nx + i] - Bz[j * nx + im]) * c.inv_hx;
  return (By[j * nx + i] - By[j * nx + im]) * c.inv_hx - (Bx[j * nx + i] - Bx[jm * nx + i]) * c.inv_hy;
}

// curl of E on the B locations at (i, j), component d
__device__ __forceinline__ double curl_e(const Em2dConst &c, const double *E, int i, int j, int d) {
  const int nx = c.nx, ny = c.ny, nc = nx * ny;
  const double *Ex = E, *Ey = E + nc, *Ez = E + 2 * nc;
  const int ip = i + 1 == nx ? 0 : i + 1, jp = j + 1 == ny ? 0 : j + 1;
  if (d == 0) return (Ez[jp * nx + i] - Ez[j * nx + i]) * c.inv_hy;
  if (d == 1) return -(Ez[j * nx + ip] - Ez[j * nx + i]) * c.inv_hx;
  return (Ey[j * nx + ip] - Ey[j * nx + i]) * c.inv_hx - (Ex[jp * nx + i] - Ex[j * nx + i]) * c.inv_hy;
}

// K5 as block blk of nblk: B^{n+3/2} = B^{n+1/2} - dt curl E^{n+1} and the
// block's partials of W_E and W_B (wf_part[2 blk], wf_part[2 blk + 1])
__device__ __forceinline__ void k5_block(const Em2dConst &c, const Em2dBufs &b, int blk, int nblk,
                                         double *red) {
  const int nc = c.nx * c.ny;
  double we = 0.0, wb = 0.0;
  for (int a = blk * blockDim.x + threadIdx.x; a < 3 * nc; a += nblk * blockDim.x) {
    const int d = a / nc, ij = a % nc, i = ij % c.nx, j = ij / c.nx;
    const double bpp = b.Bp[a] - c.dt * curl_e(c, b.En, i, j, d);
    b.Bpp[a] = bpp;
    we += b.En[a] * b.En[a];
    wb += b.Bp[a] * bpp;
  }
  double t = block_sum2(we, red);
  if (threadIdx.x == 0) b.wf_part[2 * blk] = t;
  t = block_sum2(wb, red);
  if (threadIdx.x == 0) b.wf_part[2 * blk + 1] = t;
}

// TE of the step in slot from its nkb kinetic and nfb field partials (one block)
__device__ __forceinline__ void finalize_block(const Em2dConst &c, const Em2dBufs &b, int slot,
                                               int nkb, int nfb, double *red) {
  double ke = 0.0, we = 0.0, wb = 0.0;
  for (int i = threadIdx.x; i < nkb; i += blockDim.x) ke += b.ke_part[i];
  for (int i = threadIdx.x; i < nfb; i += blockDim.x) {
    we += b.wf_part[2 * i];
    wb += b.wf_part[2 * i + 1];
  }
  const double k = block_sum2(ke, red);
  const double e = block_sum2(we, red);
  const double m = block_sum2(wb, red);
  if (threadIdx.x == 0) {
    const double te = k + 0.5 * c.area * e + 0.5 * c.c2 * c.area * m;
    b.te[slot] = te;
    if (!isfinite(te)) atomicOr(b.err, kErrNonfinite);
  }
}

}  // namespace
}  // namespace pic
