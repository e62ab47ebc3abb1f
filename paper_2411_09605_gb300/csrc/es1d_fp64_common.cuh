// Marker-side helpers of the FP64 1D form, shared by the stepping kernels and
// their reverse mode: periodic wrap, shape weights, species lookup and the
// half push x* -> E**_p -> v* -> x^{n+1/2}, all with explicitly rounded
// operations so that every kernel that evaluates them gets the same values.
#pragma once

#include <cuda_runtime.h>

#include "pic_internal.cuh"

namespace pic {
namespace {

__device__ __forceinline__ double wrap_periodic(double y, double L, unsigned *err) {
  if (y < 0.0) y += L;
  if (y >= L) y -= L;
  if (!(y >= 0.0 && y < L)) atomicOr(err, kErrBounds);
  return y;
}

// Node index reduced into [0, nc) whatever the input (a position that left the
// domain is flagged by wrap_periodic; this keeps every access in bounds).
__device__ __forceinline__ int safe_mod(int i, int nc) {
  if ((unsigned)i < (unsigned)nc) return i;
  int r = i % nc;
  return r < 0 ? r + nc : r;
}

template <int ORDER>
struct Shape64 {
  int idx[ORDER + 1];
  double w[ORDER + 1];
  Shape64() = default;
  // the shape a pass stored (store()), node i0 = idx[ORDER - 1]
  __device__ __forceinline__ void load(const double *sw, const int *si, int64_t p, int64_t n,
                                       int nc) {
    const int i0 = si[p];
    if (ORDER == 1) {
      idx[0] = i0;
      idx[1] = i0 + 1 == nc ? 0 : i0 + 1;
    } else {
      idx[0] = i0 - 1 < 0 ? i0 - 1 + nc : i0 - 1;
      idx[1] = i0;
      idx[ORDER] = i0 + 1 >= nc ? i0 + 1 - nc : i0 + 1;
    }
#pragma unroll
    for (int k = 0; k <= ORDER; k++) w[k] = sw[k * n + p];
  }
  __device__ __forceinline__ void store(double *sw, int *si, int64_t p, int64_t n) const {
    si[p] = idx[ORDER - 1];
#pragma unroll
    for (int k = 0; k <= ORDER; k++) sw[k * n + p] = w[k];
  }
  __device__ __forceinline__ Shape64(double xi, int nc) {
    if (ORDER == 1) {
      double fl = floor(xi);
      double f = xi - fl;
      int i = safe_mod((int)fl, nc);
      idx[0] = i;
      idx[1] = (i + 1 == nc) ? 0 : i + 1;
      w[0] = __dadd_rn(1.0, -f);
      w[1] = f;
    } else {
      double fl = floor(xi + 0.5);
      double d = xi - fl;
      int i0 = safe_mod((int)fl, nc);
      int im = i0 - 1 < 0 ? i0 - 1 + nc : i0 - 1;
      int ip = i0 + 1 >= nc ? i0 + 1 - nc : i0 + 1;
      idx[0] = im;
      idx[1] = i0;
      idx[ORDER] = ip;
      // explicit roundings: both passes must produce identical weights
      double a = __dadd_rn(0.5, -d), b = __dadd_rn(0.5, d);
      w[0] = __dmul_rn(0.5, __dmul_rn(a, a));
      w[1] = __fma_rn(-d, d, 0.75);
      w[ORDER] = __dmul_rn(0.5, __dmul_rn(b, b));
    }
  }
  __device__ __forceinline__ double gather(const double *F) const {
    double s = F[idx[0]] * w[0];
#pragma unroll
    for (int k = 1; k <= ORDER; k++) s = fma(F[idx[k]], w[k], s);
    return s;
  }
  __device__ __forceinline__ void deposit(double *J, double coef) const {
#pragma unroll
    for (int k = 0; k <= ORDER; k++) atomicAdd(&J[idx[k]], coef * w[k]);
  }
};

__device__ __forceinline__ int species_of(const Es1dConst &c, int64_t p) {
  int s = 0;
  while (s < c.nsp - 1 && p >= c.sp_end[s]) s++;
  return s;
}

// x*, E**_p, v*, x^{n+1/2}: evaluated by both passes with explicitly rounded
// operations so that the two passes agree bit for bit (the deposit of pass C
// and the gather of pass E must use the same x^{n+1/2} and v*, Eq.
// exp_econs_simple).
// x* = x + dt/2 v with the rounding every kernel of this form uses for it
__device__ __forceinline__ double xstar(const Es1dConst &c, double x, double v, unsigned *err) {
  return wrap_periodic(__fma_rn(0.5 * c.dt, v, x), c.L, err);
}

// E**_p, v*, x^{n+1/2} from the shape S at x*
template <int ORDER>
__device__ __forceinline__ void half_push_at(const Es1dConst &c, const double *Es,
                                             const Shape64<ORDER> &S, double x, double v,
                                             double qm, unsigned *err, double &vs, double &xh) {
  double hdt = 0.5 * c.dt;
  double Ess = __fma_rn(Es[S.idx[0]], S.w[0], 0.0);
#pragma unroll
  for (int k = 1; k <= ORDER; k++) Ess = __fma_rn(Es[S.idx[k]], S.w[k], Ess);
  vs = __fma_rn(__dmul_rn(hdt, qm), Ess, v);
  xh = wrap_periodic(__fma_rn(hdt, vs, x), c.L, err);
}

template <int ORDER>
__device__ __forceinline__ void half_push(const Es1dConst &c, const double *Es, double x,
                                          double v, double qm, unsigned *err, double &vs,
                                          double &xh) {
  double hdt = 0.5 * c.dt;
  double xs = wrap_periodic(__fma_rn(hdt, v, x), c.L, err);
  Shape64<ORDER> S(__dmul_rn(xs, c.inv_h), c.nc);
  double Ess = __fma_rn(Es[S.idx[0]], S.w[0], 0.0);
#pragma unroll
  for (int k = 1; k <= ORDER; k++) Ess = __fma_rn(Es[S.idx[k]], S.w[k], Ess);
  vs = __fma_rn(__dmul_rn(hdt, qm), Ess, v);
  xh = wrap_periodic(__fma_rn(hdt, vs, x), c.L, err);
}

}  // namespace
}  // namespace pic
