// 2D3V electromagnetic step with the leapfrog / Yee field update (Sec. 4.1,
// Eq. EMleapfrog), FP64 form.
//
// Yee lattice on a periodic nx x ny grid, component-major [3][ny][nx] arrays:
//   Ex (i+1/2, j)  Ey (i, j+1/2)  Ez (i, j)      (J the same)
//   Bx (i, j+1/2)  By (i+1/2, j)  Bz (i+1/2, j+1/2)
// Gather of E_c and deposit of J_c use the same tensor-product B-spline
// centred on component c's nodes, so Eq. exp_econs_simple holds per component.
//
// Per step (the state is E^n, B^{n-1/2}, Bp = B^{n+1/2} and, for ESEC2,
// j^{n,*} deposited at the end of the previous step):
//   K1 grid     E* = E^n + dt/2 (c^2 curl Bp - j^{n,*}); clear j^{*,n+1/2}
//   K2 markers  x*, E**, B at x*, v* (closed form of the implicit relation,
//               stored), x^{n+1/2}, deposit of j^{*,n+1/2}
//   K3 grid     E^{n+1} = E^n + dt (c^2 curl Bp - j^{*,n+1/2}), E^{n+1/2}
//   K4 markers  v* loaded, x^{n+1/2} with K2's rounding; gather E^{n+1/2}, B at x^{n+1/2};
//               v^dag, Gamma (fallback counted), x^{n+1}, v^{n+1}, KE, next j^{n+1,*}
//   K5 grid     B^{n+3/2} = Bp - dt curl E^{n+1}; W_E^{n+1}, W_B^{n+1} =
//               (c^2/2)|h| sum Bp . B^{n+3/2} (the energy of the new state)
// Fields stay in global memory (0.8 MB at 128 x 128, L2-resident); the
// current is accumulated with FP64 global atomics.
//
// Charge-conserving option (Sec. 3.5, Eq. detbal; order 1): with the bilinear
// charge shape, each component takes the tent on the axes where it sits on
// integer nodes and the degree-0 box on the axes where it sits on half nodes
// (Jx, Ex: box x tent; Jy, Ey: tent x box; Jz, Ez: tent x tent), and the
// deposit of j^{*,n+1/2} and the gather of E^{n+1/2} sum, over the pieces of
// the path x^n -> x^{n+1} between grid lines, the piece's fraction times the
// shape at its midpoint.  The continuity equation then holds exactly with the
// Yee divergence, and the energy pairing is unchanged.
#include <cuda_runtime.h>

#include <type_traits>

#include "em2d_common.cuh"
#include "pdl.cuh"
#include "pic_internal.cuh"

namespace pic {
namespace {


__device__ __forceinline__ double wrapd(double y, double L, unsigned *err) {
  if (y < 0.0) y += L;
  if (y >= L) y -= L;
  if (!(y >= 0.0 && y < L)) atomicOr(err, kErrBounds);
  return y;
}

// 1D B-spline weights of coordinate xi (cell units) on nodes i0 .. i0+ORDER
// (ORDER 0: the box, weight 1 at the nearest node)
template <int ORDER>
struct W1 {
  int i0;
  double w[ORDER + 1];
  __device__ __forceinline__ void set(double xi) {
    if (ORDER == 0) {
      i0 = (int)floor(__dadd_rn(xi, 0.5));
      w[0] = 1.0;
    } else if (ORDER == 1) {
      double fl = floor(xi);
      double f = __dadd_rn(xi, -fl);
      i0 = (int)fl;
      w[0] = __dadd_rn(1.0, -f);
      w[1] = f;
    } else {
      double fl = floor(__dadd_rn(xi, 0.5));
      double d = __dadd_rn(xi, -fl);
      i0 = (int)fl - 1;
      double a = __dadd_rn(0.5, -d), b = __dadd_rn(0.5, d);
      w[0] = __dmul_rn(0.5, __dmul_rn(a, a));
      w[1] = __fma_rn(-d, d, 0.75);
      w[ORDER] = __dmul_rn(0.5, __dmul_rn(b, b));
    }
  }
};

// Weights of a point for integer-node (I) and half-node (H) components in x,
// y: order OI on integer-node axes, OH on half-node axes.
template <int OI, int OH>
struct Shape2 {
  W1<OI> xI, yI;
  W1<OH> xH, yH;
  static constexpr int kWeights = 2 * (OI + 1) + 2 * (OH + 1);
  Shape2() = default;
  // the four axes' first nodes and weights, as store() wrote them for marker p
  __device__ __forceinline__ void load(const double *sw, const int *si, int64_t p, int64_t n) {
    xI.i0 = si[p];
    xH.i0 = si[n + p];
    yI.i0 = si[2 * n + p];
    yH.i0 = si[3 * n + p];
    int k = 0;
#pragma unroll
    for (int a = 0; a <= OI; a++) xI.w[a] = sw[(k++) * n + p];
#pragma unroll
    for (int a = 0; a <= OH; a++) xH.w[a] = sw[(k++) * n + p];
#pragma unroll
    for (int a = 0; a <= OI; a++) yI.w[a] = sw[(k++) * n + p];
#pragma unroll
    for (int a = 0; a <= OH; a++) yH.w[a] = sw[(k++) * n + p];
  }
  __device__ __forceinline__ void store(double *sw, int *si, int64_t p, int64_t n) const {
    si[p] = xI.i0;
    si[n + p] = xH.i0;
    si[2 * n + p] = yI.i0;
    si[3 * n + p] = yH.i0;
    int k = 0;
#pragma unroll
    for (int a = 0; a <= OI; a++) sw[(k++) * n + p] = xI.w[a];
#pragma unroll
    for (int a = 0; a <= OH; a++) sw[(k++) * n + p] = xH.w[a];
#pragma unroll
    for (int a = 0; a <= OI; a++) sw[(k++) * n + p] = yI.w[a];
#pragma unroll
    for (int a = 0; a <= OH; a++) sw[(k++) * n + p] = yH.w[a];
  }
  __device__ __forceinline__ Shape2(const Em2dConst &c, double x, double y) {
    const double xi = __dmul_rn(x, c.inv_hx), yi = __dmul_rn(y, c.inv_hy);
    xI.set(xi);
    xH.set(__dadd_rn(xi, -0.5));
    yI.set(yi);
    yH.set(__dadd_rn(yi, -0.5));
  }
};

template <int OX, int OY>
__device__ __forceinline__ double gather_c(const double *F, int nx, int ny, const W1<OX> &wx,
                                           const W1<OY> &wy) {
  double s = 0.0;
#pragma unroll
  for (int b = 0; b <= OY; b++) {
    const int row = wrapi(wy.i0 + b, ny) * nx;
    double r = 0.0;
#pragma unroll
    for (int a = 0; a <= OX; a++) r = fma(__ldg(&F[row + wrapi(wx.i0 + a, nx)]), wx.w[a], r);
    s = fma(r, wy.w[b], s);
  }
  return s;
}

template <int OX, int OY>
__device__ __forceinline__ void deposit_c(double *J, int nx, int ny, const W1<OX> &wx,
                                          const W1<OY> &wy, double coef) {
#pragma unroll
  for (int b = 0; b <= OY; b++) {
    const int row = wrapi(wy.i0 + b, ny) * nx;
    const double cb = coef * wy.w[b];
#pragma unroll
    for (int a = 0; a <= OX; a++) atomicAdd(&J[row + wrapi(wx.i0 + a, nx)], cb * wx.w[a]);
  }
}

// E (Ex: H,I; Ey: I,H; Ez: I,I) and B (Bx: I,H; By: H,I; Bz: H,H) at a point
template <int OI, int OH>
__device__ __forceinline__ void gather_eb(const Em2dConst &c, const double *E, const double *B,
                                          const Shape2<OI, OH> &S, double e[3], double bb[3]) {
  const int nx = c.nx, ny = c.ny, nc = c.nx * c.ny;
  if (E) {
    e[0] = gather_c<OH, OI>(E, nx, ny, S.xH, S.yI);
    e[1] = gather_c<OI, OH>(E + nc, nx, ny, S.xI, S.yH);
    e[2] = gather_c<OI, OI>(E + 2 * nc, nx, ny, S.xI, S.yI);
  }
  if (B) {
    bb[0] = gather_c<OI, OH>(B, nx, ny, S.xI, S.yH);
    bb[1] = gather_c<OH, OI>(B + nc, nx, ny, S.xH, S.yI);
    bb[2] = gather_c<OH, OH>(B + 2 * nc, nx, ny, S.xH, S.yH);
  }
}

template <int OI, int OH>
__device__ __forceinline__ void deposit_j(const Em2dConst &c, double *J, const Shape2<OI, OH> &S,
                                          double coef, const double u[3]) {
  const int nx = c.nx, ny = c.ny, nc = c.nx * c.ny;
  deposit_c<OH, OI>(J, nx, ny, S.xH, S.yI, coef * u[0]);
  deposit_c<OI, OH>(J + nc, nx, ny, S.xI, S.yH, coef * u[1]);
  deposit_c<OI, OI>(J + 2 * nc, nx, ny, S.xI, S.yI, coef * u[2]);
}

// Shape orders of a form: the order on both axis kinds, or for the
// charge-conserving form the tent on integer-node and the box on half-node axes
template <int ORDER, bool CC>
struct Orders {
  static constexpr int I = CC ? 1 : ORDER;
  static constexpr int H = CC ? 0 : ORDER;
};

// The pieces of the straight path from (x0, y0) by (dx, dy) between the grid
// lines x = i hx and y = j hy, in path order: f(tau, xm, ym) with the piece's
// fraction of the path and its (wrapped) midpoint.  The lines of each axis are
// met in order, so the two sequences of crossing parameters are merged; there
// are 1 + (lines crossed) pieces.
template <class F>
__device__ __forceinline__ void for_pieces(const Em2dConst &c, double x0, double y0, double dx,
                                           double dy, unsigned *err, F f) {
  const double ax = x0 * c.inv_hx, bx = (x0 + dx) * c.inv_hx;   // in cells
  const double ay = y0 * c.inv_hy, by = (y0 + dy) * c.inv_hy;
  const double fx0 = floor(ax), fx1 = floor(bx), fy0 = floor(ay), fy1 = floor(by);
  const int nxc = (int)fabs(fx1 - fx0), nyc = (int)fabs(fy1 - fy0);
  const double stx = fx1 > fx0 ? 1.0 : -1.0, sty = fy1 > fy0 ? 1.0 : -1.0;
  double lx = fx1 > fx0 ? fx0 + 1.0 : fx0;   // next line to cross on each axis
  double ly = fy1 > fy0 ? fy0 + 1.0 : fy0;
  int kx = 0, ky = 0;
  double s0 = 0.0;
  for (int it = 0; it <= nxc + nyc; it++) {
    const double tx = kx < nxc ? (lx - ax) / (bx - ax) : 2.0;
    const double ty = ky < nyc ? (ly - ay) / (by - ay) : 2.0;
    double s1;
    if (it == nxc + nyc) {
      s1 = 1.0;
    } else if (tx <= ty) {
      s1 = fmin(tx, 1.0);
      kx++;
      lx += stx;
    } else {
      s1 = fmin(ty, 1.0);
      ky++;
      ly += sty;
    }
    s1 = fmax(s1, s0);
    const double mid = 0.5 * (s0 + s1);
    f(s1 - s0, wrapd(x0 + mid * dx, c.Lx, err), wrapd(y0 + mid * dy, c.Ly, err));
    s0 = s1;
  }
}

__device__ __forceinline__ int species_of2(const Em2dConst &c, int64_t p) {
  int s = 0;
  while (s < c.nsp - 1 && p >= c.sp_end[s]) s++;
  return s;
}

// The shape at x* = x + dt/2 v, with the rounding every kernel of this form
// uses for it.
template <int OI, int OH>
__device__ __forceinline__ Shape2<OI, OH> shape_at_xstar(const Em2dConst &c, const Em2dBufs &b,
                                                         double x, double y, const double v[3]) {
  const double hdt = 0.5 * c.dt;
  const double xs = wrapd(__fma_rn(hdt, v[0], x), c.Lx, b.err);
  const double ys = wrapd(__fma_rn(hdt, v[1], y), c.Ly, b.err);
  return Shape2<OI, OH>(c, xs, ys);
}

// E**, B at x* (shape S), v* and x^{n+1/2}.
template <int OI, int OH>
__device__ __forceinline__ void half_push_em(const Em2dConst &c, const Em2dBufs &b, int s,
                                             const Shape2<OI, OH> &S, double x, double y,
                                             const double v[3], double vs[3], double &xh,
                                             double &yh) {
  const double hdt = 0.5 * c.dt;
  double e[3], bb[3];
  gather_eb<OI, OH>(c, b.Es, b.Bp, S, e, bb);
  const double k = __dmul_rn(hdt, c.qm[s]);
  double u[3], t[3];
#pragma unroll
  for (int d = 0; d < 3; d++) {
    u[d] = __fma_rn(k, e[d], v[d]);
    t[d] = __dmul_rn(k, bb[d]);
  }
  // v* - v* x t = u  ->  v* = (u + u x t + (u.t) t) / (1 + |t|^2)
  const double uxt0 = __dadd_rn(__dmul_rn(u[1], t[2]), -__dmul_rn(u[2], t[1]));
  const double uxt1 = __dadd_rn(__dmul_rn(u[2], t[0]), -__dmul_rn(u[0], t[2]));
  const double uxt2 = __dadd_rn(__dmul_rn(u[0], t[1]), -__dmul_rn(u[1], t[0]));
  const double ut = __fma_rn(u[2], t[2], __fma_rn(u[1], t[1], __dmul_rn(u[0], t[0])));
  const double tt = __fma_rn(t[2], t[2], __fma_rn(t[1], t[1], __dmul_rn(t[0], t[0])));
  const double inv = __drcp_rn(__dadd_rn(1.0, tt));
  vs[0] = __dmul_rn(__fma_rn(ut, t[0], __dadd_rn(u[0], uxt0)), inv);
  vs[1] = __dmul_rn(__fma_rn(ut, t[1], __dadd_rn(u[1], uxt1)), inv);
  vs[2] = __dmul_rn(__fma_rn(ut, t[2], __dadd_rn(u[2], uxt2)), inv);
  xh = wrapd(__fma_rn(hdt, vs[0], x), c.Lx, b.err);
  yh = wrapd(__fma_rn(hdt, vs[1], y), c.Ly, b.err);
}




// K1: E* (ESEC2: with j^{n,*}; ESEC1: E^n), clear J2
__global__ void em_k1_kernel(Em2dConst c, Em2dBufs b) {
  const int nc = c.nx * c.ny;
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < 3 * nc; a += gridDim.x * blockDim.x) {
    const int d = a / nc, ij = a % nc, i = ij % c.nx, j = ij / c.nx;
    double es = b.E[a];
    if (c.scheme == 2) es = es + 0.5 * c.dt * (c.c2 * curl_b(c, b.Bp, i, j, d) - b.J1[a]);
    b.Es[a] = es;
    b.J2[a] = 0.0;
  }
}

// K3: E^{n+1}, E^{n+1/2}; clear J1 (it receives j^{n+1,*})
__global__ void em_k3_kernel(Em2dConst c, Em2dBufs b) {
  const int nc = c.nx * c.ny;
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < 3 * nc; a += gridDim.x * blockDim.x) {
    const int d = a / nc, ij = a % nc, i = ij % c.nx, j = ij / c.nx;
    const double en = b.E[a] + c.dt * (c.c2 * curl_b(c, b.Bp, i, j, d) - b.J2[a]);
    b.Eh[a] = 0.5 * (b.E[a] + en);
    b.En[a] = en;
    b.J1[a] = 0.0;
  }
}

// K5: B^{n+3/2} = Bp - dt curl E^{n+1}, block partials of W_E and W_B
__global__ void __launch_bounds__(256) em_k5_kernel(Em2dConst c, Em2dBufs b) {
  __shared__ double red[33];
  griddep_wait();
  griddep_launch_dependents();
  k5_block(c, b, blockIdx.x, gridDim.x, red);
}

template <int ORDER, bool CC>
__global__ void __launch_bounds__(256) em_pass_c_kernel(Em2dConst c, Em2dBufs b) {
  constexpr int OI = Orders<ORDER, CC>::I, OH = Orders<ORDER, CC>::H;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < c.n_total;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int s = species_of2(c, p);
    const double x = b.x[p], y = b.y[p];
    const double v[3] = {b.vx[p], b.vy[p], b.vz[p]};
    double vs[3], xh, yh;
    // ESEC2, point shapes: the shape at x* that the previous pass E (or the
    // initial deposit) deposited j^{n,*} with, the same bits as forming it
    Shape2<OI, OH> Sx;
    if (!CC && b.sws)
      Sx.load(b.sws, b.sis, p, c.n_total);
    else
      Sx = shape_at_xstar<OI, OH>(c, b, x, y, v);
    half_push_em<OI, OH>(c, b, s, Sx, x, y, v, vs, xh, yh);
    b.vsx[p] = vs[0];   // pass E forms x^{n+1/2} from v* with the same rounding
    b.vsy[p] = vs[1];
    b.vsz[p] = vs[2];
    const double coef = b.w ? c.q_a[s] * b.w[p] : c.qw_a[s];
    if (CC) {
      for_pieces(c, x, y, c.dt * vs[0], c.dt * vs[1], b.err, [&](double tau, double xm, double ym) {
        const Shape2<OI, OH> S(c, xm, ym);
        deposit_j<OI, OH>(c, b.J2, S, coef * tau, vs);
      });
    } else {
      const Shape2<OI, OH> S(c, xh, yh);
      deposit_j<OI, OH>(c, b.J2, S, coef, vs);
      if (b.sw) S.store(b.sw, b.si, p, c.n_total);  // pass E gathers with it
    }
  }
}

template <int ORDER, bool CC>
__global__ void __launch_bounds__(256) em_pass_e_kernel(Em2dConst c, Em2dBufs b, int slot) {
  constexpr int OI = Orders<ORDER, CC>::I, OH = Orders<ORDER, CC>::H;
  __shared__ double red[33];
  double ke = 0.0;
  unsigned nfb = 0;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < c.n_total;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int s = species_of2(c, p);
    const double x = b.x[p], y = b.y[p];
    const double v[3] = {b.vx[p], b.vy[p], b.vz[p]};
    const double vs[3] = {b.vsx[p], b.vsy[p], b.vsz[p]};
    // the shape at x^{n+1/2} that pass C deposited with (point shapes, loaded:
    // on this FP64-bound pass bytes are cheaper than its arithmetic), else
    // formed again with pass C's rounding
    Shape2<OI, OH> S;
    if (!CC && b.sw) {
      S.load(b.sw, b.si, p, c.n_total);
    } else {
      const double hdt = 0.5 * c.dt;
      const double xh = wrapd(__fma_rn(hdt, vs[0], x), c.Lx, b.err);
      const double yh = wrapd(__fma_rn(hdt, vs[1], y), c.Ly, b.err);
      S = Shape2<OI, OH>(c, xh, yh);
    }
    double e[3], bb[3];
    if (CC) {
      // E^{n+1/2} over the path's pieces with the deposit's fractions and shapes
      gather_eb<OI, OH>(c, nullptr, b.Bp, S, e, bb);
      e[0] = e[1] = e[2] = 0.0;
      for_pieces(c, x, y, c.dt * vs[0], c.dt * vs[1], b.err, [&](double tau, double xm, double ym) {
        const Shape2<OI, OH> Sm(c, xm, ym);
        double ek[3];
        gather_eb<OI, OH>(c, b.Eh, nullptr, Sm, ek, nullptr);
#pragma unroll
        for (int d = 0; d < 3; d++) e[d] += tau * ek[d];
      });
    } else {
      gather_eb<OI, OH>(c, b.Eh, b.Bp, S, e, bb);
    }
    const double k = c.dt * c.qm[s];
    const double vxb[3] = {vs[1] * bb[2] - vs[2] * bb[1], vs[2] * bb[0] - vs[0] * bb[2],
                           vs[0] * bb[1] - vs[1] * bb[0]};
    double vd[3];
#pragma unroll
    for (int d = 0; d < 3; d++) vd[d] = v[d] + k * (e[d] + vxb[d]);
    const double R = v[0] * v[0] + v[1] * v[1] + v[2] * v[2] +
                     2.0 * (vs[0] * (vd[0] - v[0]) + vs[1] * (vd[1] - v[1]) + vs[2] * (vd[2] - v[2]));
    const double vd2 = vd[0] * vd[0] + vd[1] * vd[1] + vd[2] * vd[2];
    double g = 1.0;
    if (c.gamma_on) {
      if (R < 0.0 || vd2 == 0.0)
        nfb++;
      else
        g = sqrt(R / vd2);  // Gamma = sqrt(R) / |v^dag| (one root)
    }
    double vn[3];
#pragma unroll
    for (int d = 0; d < 3; d++) vn[d] = vd[d] * g;
    const double xn = wrapd(x + c.dt * vs[0], c.Lx, b.err);
    const double yn = wrapd(y + c.dt * vs[1], c.Ly, b.err);
    const double wp = b.w ? b.w[p] : 1.0;
    ke += (b.w ? c.half_m[s] * wp : c.half_mw[s]) * (vn[0] * vn[0] + vn[1] * vn[1] + vn[2] * vn[2]);
    if (c.scheme == 2) {
      const Shape2<OI, OH> S2 = shape_at_xstar<OI, OH>(c, b, xn, yn, vn);
      deposit_j<OI, OH>(c, b.J1, S2, b.w ? c.q_a[s] * wp : c.qw_a[s], vn);
      if (!CC && b.sws) S2.store(b.sws, b.sis, p, c.n_total);  // the next pass C's
    }
    b.x[p] = xn;
    b.y[p] = yn;
    b.vx[p] = vn[0];
    b.vy[p] = vn[1];
    b.vz[p] = vn[2];
    if (!isfinite(vn[0] + vn[1] + vn[2])) atomicOr(b.err, kErrNonfinite);
  }
  for (int o = 16; o > 0; o >>= 1) nfb += __shfl_xor_sync(0xffffffffu, nfb, o);
  if ((threadIdx.x & 31) == 0 && nfb) atomicAdd(&b.fallback[slot], (unsigned long long)nfb);
  double t = block_sum2(ke, red);
  if (threadIdx.x == 0) b.ke_part[blockIdx.x] = t;
}

// j^{n,*} of the current state (start-up and after a state change)
template <int ORDER, bool CC>
__global__ void __launch_bounds__(256) em_deposit_initial_kernel(Em2dConst c, Em2dBufs b) {
  constexpr int OI = Orders<ORDER, CC>::I, OH = Orders<ORDER, CC>::H;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < c.n_total;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int s = species_of2(c, p);
    const double v[3] = {b.vx[p], b.vy[p], b.vz[p]};
    const Shape2<OI, OH> S = shape_at_xstar<OI, OH>(c, b, b.x[p], b.y[p], v);
    deposit_j<OI, OH>(c, b.J1, S, b.w ? c.q_a[s] * b.w[p] : c.qw_a[s], v);
    if (!CC && b.sws) S.store(b.sws, b.sis, p, c.n_total);  // pass C gathers with it
  }
}

// Bp = B0 - dt curl E0 (the state's B^{n+1/2})
__global__ void em_bhalf_kernel(Em2dConst c, const double *B, const double *E, double *Bp) {
  const int nc = c.nx * c.ny;
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < 3 * nc; a += gridDim.x * blockDim.x) {
    const int d = a / nc, ij = a % nc, i = ij % c.nx, j = ij / c.nx;
    Bp[a] = B[a] - c.dt * curl_e(c, E, i, j, d);
  }
}

// TE of the step in slot: KE partials + field partials
__global__ void em_finalize_kernel(Em2dConst c, Em2dBufs b, int slot, int nkb, int nfb) {
  __shared__ double red[33];
  griddep_wait();
  griddep_launch_dependents();
  finalize_block(c, b, slot, nkb, nfb, red);
}

__global__ void __launch_bounds__(256) em_kinetic_kernel(Em2dConst c, Em2dBufs b, double *out) {
  __shared__ double red[33];
  const int s = blockIdx.y;
  int64_t beg = s == 0 ? 0 : c.sp_end[s - 1], end = c.sp_end[s];
  double acc = 0.0;
  for (int64_t p = beg + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < end;
       p += (int64_t)gridDim.x * blockDim.x) {
    double v2 = b.vx[p] * b.vx[p] + b.vy[p] * b.vy[p] + b.vz[p] * b.vz[p];
    acc += b.w ? c.half_m[s] * b.w[p] * v2 : c.half_mw[s] * v2;
  }
  double t = block_sum2(acc, red);
  if (threadIdx.x == 0) out[s * gridDim.x + blockIdx.x] = t;
}

}  // namespace

void em2d_k1(const Em2dConst &c, const Em2dBufs &b, LaunchShape lg, cudaStream_t st) {
  em_k1_kernel<<<lg.grid, lg.block, 0, st>>>(c, b);
}

void em2d_pass_c(const Em2dConst &c, const Em2dBufs &b, LaunchShape lp, cudaStream_t st) {
  if (c.cc)
    em_pass_c_kernel<1, true><<<lp.grid, lp.block, 0, st>>>(c, b);
  else if (c.order == 1)
    em_pass_c_kernel<1, false><<<lp.grid, lp.block, 0, st>>>(c, b);
  else
    em_pass_c_kernel<2, false><<<lp.grid, lp.block, 0, st>>>(c, b);
}

void em2d_k3(const Em2dConst &c, const Em2dBufs &b, LaunchShape lg, cudaStream_t st) {
  em_k3_kernel<<<lg.grid, lg.block, 0, st>>>(c, b);
}

void em2d_pass_e(const Em2dConst &c, const Em2dBufs &b, int slot, LaunchShape lp,
                 cudaStream_t st) {
  if (c.cc)
    em_pass_e_kernel<1, true><<<lp.grid, lp.block, 0, st>>>(c, b, slot);
  else if (c.order == 1)
    em_pass_e_kernel<1, false><<<lp.grid, lp.block, 0, st>>>(c, b, slot);
  else
    em_pass_e_kernel<2, false><<<lp.grid, lp.block, 0, st>>>(c, b, slot);
}

void em2d_k5(const Em2dConst &c, const Em2dBufs &b, LaunchShape lg, cudaStream_t st, bool pdl) {
  launch_dependent(em_k5_kernel, LaunchShape{lg.grid, 256}, 0, st, pdl, c, b);
}

void em2d_finalize(const Em2dConst &c, const Em2dBufs &b, int slot, LaunchShape lp,
                   LaunchShape lg, cudaStream_t st, bool pdl) {
  launch_dependent(em_finalize_kernel, LaunchShape{1, 256}, 0, st, pdl, c, b, slot, lp.grid,
                   lg.grid);
}

__global__ void em2d_validate_kernel(const double *x, const double *y, const double *vx,
                                     const double *vy, const double *vz, int64_t n, double Lx,
                                     double Ly, unsigned *err) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    if (!(x[p] >= 0.0 && x[p] < Lx) || !(y[p] >= 0.0 && y[p] < Ly)) atomicOr(err, kErrBounds);
    if (!isfinite(vx[p]) || !isfinite(vy[p]) || !isfinite(vz[p])) atomicOr(err, kErrNonfinite);
  }
}

void em2d_fp64_deposit_initial(const Em2dConst &c, const Em2dBufs &b, LaunchShape lp,
                               cudaStream_t st) {
  if (c.cc)
    em_deposit_initial_kernel<1, true><<<lp.grid, lp.block, 0, st>>>(c, b);
  else if (c.order == 1)
    em_deposit_initial_kernel<1, false><<<lp.grid, lp.block, 0, st>>>(c, b);
  else
    em_deposit_initial_kernel<2, false><<<lp.grid, lp.block, 0, st>>>(c, b);
}

void em2d_fp64_bhalf(const Em2dConst &c, const double *B, const double *E, double *Bp,
                     LaunchShape lg, cudaStream_t st) {
  em_bhalf_kernel<<<lg.grid, lg.block, 0, st>>>(c, B, E, Bp);
}

void em2d_fp64_kinetic(const Em2dConst &c, const Em2dBufs &b, double *out, int nblocks,
                       cudaStream_t st) {
  em_kinetic_kernel<<<dim3(nblocks, c.nsp), 256, 0, st>>>(c, b, out);
}

}  // namespace pic
