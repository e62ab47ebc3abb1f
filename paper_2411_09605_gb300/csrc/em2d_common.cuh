// Grid helpers shared by the FP64 and mixed forms of the 2D3V Yee step
// (Sec. 4.1, Eq. EMleapfrog): periodic index wrap, the discrete curls on the
// staggered lattice, and a block sum.  Both forms advance the fields with the
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

}  // namespace
}  // namespace pic
