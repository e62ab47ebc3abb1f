// Reverse mode of the FP64 1D1V step: adjoints of a final objective with
// respect to the markers, their weights and the field one step earlier.
//
// Forward step (Sec. 3.3, Eq. good_translation; per marker p, node i):
//   x* = x + dt/2 v,  J1_i = (q/h) sum w v S_i(x*),  E* = E - dt/2 (J1 - <J1>)
//   a = sum E*_i S_i(x*),  u = v + dt/2 (q/m) a,  y = x + dt/2 u
//   J2_i = (q/h) sum w u S_i(y),  F = E - dt (J2 - <J2>),  H = (E + F)/2
//   b = sum H_i S_i(y),  d = v + dt (q/m) b,  R = v^2 + 2 u (d - v)
//   v' = sign(d) sqrt(R) (Sec. 3.2; d itself on a fallback),  x' = x + dt u
// Reverse, three marker kernels and two grid kernels separated by the global
// sums of the adjoint "currents":
//   rev1: v', x' -> d, R -> adjoint of H deposited at y (gather <-> deposit)
//   grid1: adjoint of F and of E, J2_bar = -dt (F_bar - <F_bar>)
//   rev2: J2_bar gathered at y -> u, y, w; u -> v, a; adjoint of E* deposited at x*
//   grid2: J1_bar = -dt/2 (E*_bar - <E*_bar>) (ESEC2), adjoint of E
//   rev3: J1_bar gathered at x* -> v, w, x*; x* -> x, v
// Shape derivatives dS/dx = (dS/dxi)/h enter wherever a position is
// differentiated; the quadratic B-spline is continuously differentiable.  The
// periodic wrap has derivative 1.
#include <cuda_runtime.h>

#include "es1d_fp64_common.cuh"
#include "pic_internal.cuh"

namespace pic {
namespace {

// dS/dxi of the shape at xi (same nodes as Shape64).
template <int ORDER>
__device__ __forceinline__ void shape_deriv(double xi, double (&dw)[ORDER + 1]) {
  if (ORDER == 1) {
    dw[0] = -1.0;
    dw[1] = 1.0;
  } else {
    const double d = xi - floor(xi + 0.5);
    dw[0] = -(0.5 - d);
    dw[1] = -2.0 * d;
    dw[ORDER] = 0.5 + d;
  }
}

// q/h of marker p's species and the marker's weight.
__device__ __forceinline__ double marker_qh(const Es1dConst &c, const Es1dGradBufs &g, int s,
                                            int64_t p, double &w) {
  w = g.w ? g.w[p] : g.w0[s];
  return c.q_h[s];
}

// x*, u = v*, y = x^{n+1/2} of a marker, exactly as the forward kernels
// evaluate them.
template <int ORDER>
__device__ __forceinline__ void recompute(const Es1dConst &c, const Es1dGradBufs &g, double x,
                                          double v, double qm, double &xs, double &u,
                                          double &y) {
  xs = wrap_periodic(__fma_rn(0.5 * c.dt, v, x), c.L, g.err);
  half_push<ORDER>(c, g.Estar, x, v, qm, g.err, u, y);
}

__device__ __forceinline__ void block_flush(const double *t, double *J, int nc) {
  for (int i = threadIdx.x; i < nc; i += blockDim.x)
    if (t[i] != 0.0) atomicAdd(&J[i], t[i]);
}

// Block mean of a grid array (single-block kernels), 0 without mean removal.
__device__ __forceinline__ double grid_mean(const Es1dConst &c, const double *a, double *red) {
  double s = 0.0;
  for (int i = threadIdx.x; i < c.nc; i += blockDim.x) s += a[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); k++) t += red[k];
    red[32] = c.remove_mean ? t / c.nc : 0.0;
  }
  __syncthreads();
  return red[32];
}

// rev1: from the adjoints of x', v' to those of d, R and the deposit of H_bar.
template <int ORDER>
__global__ void __launch_bounds__(256) rev1_kernel(Es1dConst c, Es1dGradBufs g) {
  extern __shared__ double tile[];
  for (int i = threadIdx.x; i < c.nc; i += blockDim.x) tile[i] = 0.0;
  __syncthreads();
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < c.n_total;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int s = species_of(c, p);
    const double qm = c.qm[s], x = g.x[p], v = g.v[p];
    double xs, u, y;
    recompute<ORDER>(c, g, x, v, qm, xs, u, y);
    const double yi = __dmul_rn(y, c.inv_h);
    Shape64<ORDER> S(yi, c.nc);
    double dw[ORDER + 1];
    shape_deriv<ORDER>(yi, dw);
    double b = 0.0, bp = 0.0;
#pragma unroll
    for (int k = 0; k <= ORDER; k++) {
      b += g.H[S.idx[k]] * S.w[k];
      bp += g.H[S.idx[k]] * dw[k];
    }
    const double d = v + c.dt * qm * b;
    const double R = v * v + 2.0 * u * (d - v);
    const double xb1 = g.xbar[p], vb1 = g.vbar[p];
    double ubar = c.dt * xb1, vb = 0.0, db = 0.0;
    if (c.gamma_on && !(R < 0.0 || d * d == 0.0)) {
      const double Rb = vb1 * (d > 0.0 ? 1.0 : -1.0) / (2.0 * sqrt(R));
      vb += Rb * (2.0 * v - 2.0 * u);
      ubar += Rb * 2.0 * (d - v);
      db += Rb * 2.0 * u;
    } else {
      db += vb1;
    }
    vb += db;
    const double bb = db * c.dt * qm;
#pragma unroll
    for (int k = 0; k <= ORDER; k++) atomicAdd(&tile[S.idx[k]], bb * S.w[k]);
    g.vbar[p] = vb;  // xbar keeps the adjoint of x'
    g.ub[p] = ubar;
    g.yb[p] = bb * bp * c.inv_h;
  }
  __syncthreads();
  block_flush(tile, g.Hbar, c.nc);
}

// Single block: the adjoint of F = E^{n+1} (incoming E_bar plus half of H_bar),
// E_bar of E^n so far, and J2_bar = -dt (F_bar - <F_bar>).
__global__ void grid1_kernel(Es1dConst c, Es1dGradBufs g) {
  __shared__ double red[33];
  for (int i = threadIdx.x; i < c.nc; i += blockDim.x) g.Esbar[i] = g.Ebar[i] + 0.5 * g.Hbar[i];
  __syncthreads();
  const double mean = grid_mean(c, g.Esbar, red);
  for (int i = threadIdx.x; i < c.nc; i += blockDim.x) {
    const double fb = g.Esbar[i];
    g.Ebar[i] = 0.5 * g.Hbar[i] + fb;
    g.Jbar[i] = -c.dt * (fb - mean);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < c.nc; i += blockDim.x) g.Esbar[i] = 0.0;
}

// rev2: J2_bar gathered at y -> adjoints of u, y and w; then through y, u, a.
template <int ORDER>
__global__ void __launch_bounds__(256) rev2_kernel(Es1dConst c, Es1dGradBufs g) {
  extern __shared__ double tile[];
  for (int i = threadIdx.x; i < c.nc; i += blockDim.x) tile[i] = 0.0;
  __syncthreads();
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < c.n_total;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int s = species_of(c, p);
    const double qm = c.qm[s], x = g.x[p], v = g.v[p];
    double w;
    const double qh = marker_qh(c, g, s, p, w);
    double xs, u, y;
    recompute<ORDER>(c, g, x, v, qm, xs, u, y);
    const double xsi = __dmul_rn(xs, c.inv_h), yi = __dmul_rn(y, c.inv_h);
    Shape64<ORDER> Sx(xsi, c.nc), Sy(yi, c.nc);
    double dwx[ORDER + 1], dwy[ORDER + 1];
    shape_deriv<ORDER>(xsi, dwx);
    shape_deriv<ORDER>(yi, dwy);
    double gj = 0.0, gjp = 0.0, ap = 0.0;
#pragma unroll
    for (int k = 0; k <= ORDER; k++) {
      gj += g.Jbar[Sy.idx[k]] * Sy.w[k];
      gjp += g.Jbar[Sy.idx[k]] * dwy[k];
      ap += g.Estar[Sx.idx[k]] * dwx[k];
    }
    double ubar = g.ub[p] + qh * w * gj;
    const double ybar = g.yb[p] + qh * w * u * gjp * c.inv_h;
    g.wbar[p] += qh * u * gj;
    g.xbar[p] += ybar;
    ubar += 0.5 * c.dt * ybar;
    g.vbar[p] += ubar;
    const double abar = 0.5 * c.dt * qm * ubar;
#pragma unroll
    for (int k = 0; k <= ORDER; k++) atomicAdd(&tile[Sx.idx[k]], abar * Sx.w[k]);
    g.ub[p] = abar * ap * c.inv_h;  // adjoint of x* so far
  }
  __syncthreads();
  block_flush(tile, g.Esbar, c.nc);
}

// Single block: E* = E - dt/2 (J1 - <J1>) (ESEC2) or E (ESEC1).
__global__ void grid2_kernel(Es1dConst c, Es1dGradBufs g) {
  __shared__ double red[33];
  const double mean = grid_mean(c, g.Esbar, red);
  for (int i = threadIdx.x; i < c.nc; i += blockDim.x) {
    g.Ebar[i] += g.Esbar[i];
    g.Jbar[i] = c.scheme == 2 ? -0.5 * c.dt * (g.Esbar[i] - mean) : 0.0;
  }
}

// rev3: J1_bar gathered at x* (ESEC2) -> v, w, x*; then x* = x + dt/2 v.
template <int ORDER>
__global__ void __launch_bounds__(256) rev3_kernel(Es1dConst c, Es1dGradBufs g) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < c.n_total;
       p += (int64_t)gridDim.x * blockDim.x) {
    const double x = g.x[p], v = g.v[p];
    double xsb = g.ub[p];
    if (c.scheme == 2) {
      const int s = species_of(c, p);
      double w;
      const double qh = marker_qh(c, g, s, p, w);
      const double xs = wrap_periodic(__fma_rn(0.5 * c.dt, v, x), c.L, g.err);
      const double xsi = __dmul_rn(xs, c.inv_h);
      Shape64<ORDER> S(xsi, c.nc);
      double dw[ORDER + 1];
      shape_deriv<ORDER>(xsi, dw);
      double gj = 0.0, gjp = 0.0;
#pragma unroll
      for (int k = 0; k <= ORDER; k++) {
        gj += g.Jbar[S.idx[k]] * S.w[k];
        gjp += g.Jbar[S.idx[k]] * dw[k];
      }
      g.wbar[p] += qh * v * gj;
      g.vbar[p] += qh * w * gj;
      xsb += qh * w * v * gjp * c.inv_h;
    }
    g.xbar[p] += xsb;
    g.vbar[p] += 0.5 * c.dt * xsb;
  }
}

// Grid quantities of the forward step: E* (from J1 of the step, deposited by
// dep_j1_kernel into g.J1) and H = (E^n + E^{n+1})/2; clears H_bar.
__global__ void prep_kernel(Es1dConst c, Es1dGradBufs g, const double *E, const double *Enew) {
  __shared__ double red[33];
  const double mean = c.scheme == 2 ? grid_mean(c, g.J1, red) : 0.0;
  for (int i = threadIdx.x; i < c.nc; i += blockDim.x) {
    g.Estar[i] = c.scheme == 2 ? E[i] - 0.5 * c.dt * (g.J1[i] - mean) : E[i];
    g.H[i] = 0.5 * (E[i] + Enew[i]);
    g.Hbar[i] = 0.0;
  }
}

// J1 = (q/h) sum w v S(x*) of the step's markers (ESEC2).
template <int ORDER>
__global__ void __launch_bounds__(256) dep_j1_kernel(Es1dConst c, Es1dGradBufs g) {
  extern __shared__ double tile[];
  for (int i = threadIdx.x; i < c.nc; i += blockDim.x) tile[i] = 0.0;
  __syncthreads();
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < c.n_total;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int s = species_of(c, p);
    double w;
    const double qh = marker_qh(c, g, s, p, w);
    const double xs = wrap_periodic(__fma_rn(0.5 * c.dt, g.v[p], g.x[p]), c.L, g.err);
    Shape64<ORDER> S(__dmul_rn(xs, c.inv_h), c.nc);
#pragma unroll
    for (int k = 0; k <= ORDER; k++) atomicAdd(&tile[S.idx[k]], qh * w * g.v[p] * S.w[k]);
  }
  __syncthreads();
  block_flush(tile, g.J1, c.nc);
}

template <int ORDER>
void grad_step(const Es1dConst &c, const Es1dGradBufs &g, const double *E, const double *Enew,
               LaunchShape ls, cudaStream_t st) {
  const size_t sm = sizeof(double) * c.nc;
  const int gb = ls.grid;
  if (c.scheme == 2) {
    cudaMemsetAsync(g.J1, 0, sm, st);
    dep_j1_kernel<ORDER><<<gb, 256, sm, st>>>(c, g);
  }
  prep_kernel<<<1, 1024, 0, st>>>(c, g, E, Enew);
  rev1_kernel<ORDER><<<gb, 256, sm, st>>>(c, g);
  grid1_kernel<<<1, 1024, 0, st>>>(c, g);
  rev2_kernel<ORDER><<<gb, 256, sm, st>>>(c, g);
  grid2_kernel<<<1, 1024, 0, st>>>(c, g);
  rev3_kernel<ORDER><<<gb, 256, 0, st>>>(c, g);
}

}  // namespace

void es1d_grad_step(const Es1dConst &c, const Es1dGradBufs &g, const double *E,
                    const double *Enew, LaunchShape ls, cudaStream_t st) {
  if (c.order == 1)
    grad_step<1>(c, g, E, Enew, ls, st);
  else
    grad_step<2>(c, g, E, Enew, ls, st);
}

cudaError_t es1d_grad_prepare(const Es1dConst &c) {
  const int sm = (int)(sizeof(double) * c.nc);
  cudaError_t e = cudaSuccess;
  for (auto k : {(const void *)dep_j1_kernel<1>, (const void *)dep_j1_kernel<2>,
                 (const void *)rev1_kernel<1>, (const void *)rev1_kernel<2>,
                 (const void *)rev2_kernel<1>, (const void *)rev2_kernel<2>})
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  return e;
}

}  // namespace pic
