// Block-level helpers of the spectral field solves (the 1D2V electromagnetic
// path and the standard-PIC Poisson solve): complex arithmetic on double2, an
// in-block radix-2 FFT over shared memory, the "last block to finish"
// detection and a fixed-order block sum.
#pragma once

#include <cuda_runtime.h>

namespace pic {
namespace {

__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return {a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return {a.x - b.x, a.y - b.y}; }
__device__ __forceinline__ double2 cscale(double s, double2 a) { return {s * a.x, s * a.y}; }
__device__ __forceinline__ double2 ctimes_i(double2 a) { return {-a.y, a.x}; }   // i a
__device__ __forceinline__ double2 cconj(double2 a) { return {a.x, -a.y}; }

// In-place radix-2 transform of n = 2^log2n values in shared memory:
// a_k <- sum_j a_j exp(sign 2 pi i j k / n) (unnormalised), sign = -1 or +1.
// tw[j] = exp(-2 pi i j / n), j < n/2.  Every thread of the block takes part.
__device__ void block_fft(double2 *a, int n, int log2n, int sign, const double2 *tw) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int r = (int)(__brev((unsigned)i) >> (32 - log2n));
    if (r > i) {
      const double2 t = a[i];
      a[i] = a[r];
      a[r] = t;
    }
  }
  __syncthreads();
  for (int len = 2, step = n >> 1; len <= n; len <<= 1, step >>= 1) {
    const int half = len >> 1;
    for (int b = threadIdx.x; b < (n >> 1); b += blockDim.x) {
      const int grp = b / half, j = b - grp * half;
      const int i0 = grp * len + j, i1 = i0 + half;
      double2 w = tw[j * step];
      if (sign > 0) w.y = -w.y;
      const double2 u = a[i0], v = a[i1];
      const double2 t = {v.x * w.x - v.y * w.y, v.x * w.y + v.y * w.x};
      a[i0] = cadd(u, t);
      a[i1] = csub(u, t);
    }
    __syncthreads();
  }
}

// True in the one block that arrives last at this counter; every thread first
// fences its own global writes, so the last block sees all blocks' results.
// That block resets the counter for the next launch.
__device__ bool arrive_last(unsigned *counter) {
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned prev = atomicAdd(counter, 1u);
    last = prev == gridDim.x - 1;
    if (last) *counter = 0u;
  }
  __syncthreads();
  if (last) __threadfence();
  return last;
}

__device__ double block_sum_d(double s, double *red) {
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[warp] = s;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int k = 0; k < (int)(blockDim.x >> 5); k++) t += red[k];
  return t;  // valid in thread 0
}

}  // namespace
}  // namespace pic
