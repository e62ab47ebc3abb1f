/*
 * Plain FP64 CPU oracle for the explicit energy-conserving PIC scheme of
 * Ricketson & Hu, "An explicit, energy-conserving particle-in-cell scheme".
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
 * restatement of the paper's particle and field updates that the CUDA
 * library is checked against.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it.  It shares no code, header,
 * table or constant with the CUDA library, and never calls it.
 *
 * Conventions (every function below follows them):
 *   - all arithmetic in IEEE double, compiled with -ffp-contract=off so that
 *     no fused multiply-add changes the rounding;
 *   - plain loops over particles and grid nodes, in the order the paper
 *     writes the steps, no blocking, fusion or reordering;
 *   - per-species charge q and mass m: acceleration (q/m)(E + v x B),
 *     current (1/|h|) sum q w v S, kinetic energy (1/2) m sum w |v|^2
 *     (Sec. 2.1 writes the normalised single-species case q = m = 1; the
 *     energy proofs of Eq. (exp_econs_simple) carry over term by term);
 *   - grid nodes x_i = i h, periodic; E and J collocated on the nodes (1D).
 *
 * Parity status of each function is stated next to it; the pins live in
 * tests/test_oracle_*.py.
 *
 * The checker is built single-threaded (no -fopenmp): every loop then runs in
 * the order written.  The same source built with -fopenmp is used only to
 * time the CPU baseline on all host cores: orc_es1d_step's particle loops are
 * then split over threads, and each thread deposits its markers into a
 * private array that is added to the grid afterwards (a different order of
 * the same sums).  Tests never load that build.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Shape functions (Sec. 2.2: B-spline shapes; tent S(z) = max(0, 1-|z|/h)) */
/* ------------------------------------------------------------------------ */

static long imod(long a, long n) {
  long r = a % n;
  return r < 0 ? r + n : r;
}

/*
 * Weights of the particle at xi = x/h (in cell units) on the nodes it
 * touches.  order 1: the tent function of Sec. 2.2 -> nodes floor(xi) and
 * floor(xi)+1 with weights (1-f, f).  order 2: the quadratic B-spline (the
 * next B-spline, an extension the paper allows but does not test) -> nodes
 * i0-1, i0, i0+1 with i0 = floor(xi + 1/2), d = xi - i0 and weights
 * (1/2 (1/2 - d)^2, 3/4 - d^2, 1/2 (1/2 + d)^2).
 * order 0: the box B0 -> node floor(xi + 1/2) with weight 1 (the shape of
 * the charge-conserving current on a half-node axis, Sec. 3.5).
 * Returns the number of nodes (order + 1); idx is reduced modulo nc.
 * Pinned: partition of unity, linear-field reproduction, symmetry, and the
 * B-spline as the convolution of tents (test_oracle_shapes.py).
 */
int orc_shape_weights(int order, double xi, long nc, long *idx, double *wt) {
  if (order == 0) {
    /* the box B0: weight 1 at the nearest node floor(xi + 1/2) */
    idx[0] = imod((long)floor(xi + 0.5), nc);
    wt[0] = 1.0;
    return 1;
  }
  if (order == 1) {
    double fl = floor(xi);
    double f = xi - fl;
    long i = (long)fl;
    idx[0] = imod(i, nc);
    idx[1] = imod(i + 1, nc);
    wt[0] = 1.0 - f;
    wt[1] = f;
    return 2;
  }
  if (order == 2) {
    double fl = floor(xi + 0.5);
    double d = xi - fl;
    long i0 = (long)fl;
    idx[0] = imod(i0 - 1, nc);
    idx[1] = imod(i0, nc);
    idx[2] = imod(i0 + 1, nc);
    wt[0] = 0.5 * (0.5 - d) * (0.5 - d);
    wt[1] = 0.75 - d * d;
    wt[2] = 0.5 * (0.5 + d) * (0.5 + d);
    return 3;
  }
  return 0;
}

/* Periodic wrap of a position into [0, L). */
static double wrap(double x, double L) {
  double y = x - L * floor(x / L);
  if (y >= L) y -= L;
  if (y < 0.0) y = 0.0;
  return y;
}

/*
 * Deposition, Sec. 2.2: j_h += (1/h) sum_p c_p S(x_h - x_p), where the
 * caller passes c_p = q w_p v_p (current) or c_p = q w_p (charge).
 * Accumulates into J (nc nodes), does not clear it.
 */
void orc_deposit_1d(int order, long nc, double L, long n, const double *x,
                    const double *c, double *J) {
  double h = L / (double)nc;
  for (long p = 0; p < n; p++) {
    long idx[3];
    double wt[3];
    int k = orc_shape_weights(order, x[p] / h, nc, idx, wt);
    for (int j = 0; j < k; j++) J[idx[j]] += c[p] * wt[j] / h;
  }
}

/* Interpolation, Sec. 2.2: E_p = sum_h E_h S(x_p - x_h). */
void orc_gather_1d(int order, long nc, double L, long n, const double *x,
                   const double *E, double *Ep) {
  double h = L / (double)nc;
  for (long p = 0; p < n; p++) {
    long idx[3];
    double wt[3];
    int k = orc_shape_weights(order, x[p] / h, nc, idx, wt);
    double s = 0.0;
    for (int j = 0; j < k; j++) s += E[idx[j]] * wt[j];
    Ep[p] = s;
  }
}

/* ------------------------------------------------------------------------ */
/* 1D1V electrostatic scheme, Ampere form (Secs. 3.2-3.3)                    */
/* ------------------------------------------------------------------------ */

typedef struct {
  long nc;          /* grid nodes */
  double L;         /* periodic length */
  int order;        /* shape order 1 | 2 */
  double dt;
  int scheme;       /* 1 = ESEC1 (Eq. naivetranslation + Eq. PICmodification),
                       2 = ESEC2 (Eq. good_translation) */
  int remove_mean;  /* 1: E -= dt (J - <J>)  (only div j drives E in the
                       Ampere form, Eq. ampere); 0: E -= dt J literally */
  int gamma_on;     /* 1: energy correction of Eq. opt_solution;
                       0: naive scheme, v^{n+1} = v^dagger (ablation) */
  int passes;       /* binomial filter passes F inside the scheme: Ampere uses
                       F j and the gathers F E (0: none) */
} orc_es1d_cfg;

void orc_binomial_filter(long nc, const double *in, double *out);

/* a <- F^passes a (the 1-2-1 filter, periodic), in place */
static void filter_passes(long nc, double *a, int passes) {
  if (passes <= 0) return;
  double *t = (double *)calloc((size_t)nc, sizeof(double));
  for (int k = 0; k < passes; k++) {
    orc_binomial_filter(nc, a, t);
    memcpy(a, t, sizeof(double) * (size_t)nc);
  }
  free(t);
}

typedef struct {
  double q, m;
  long n;
  double *x;        /* [n] positions, updated in place */
  double *v;        /* [n] velocities, updated in place */
  const double *w;  /* [n] weights or NULL for uniform w0 */
  double w0;
} orc_species;

static double weight_of(const orc_species *s, long p) {
  return s->w ? s->w[p] : s->w0;
}

/* Ampere update of the grid field: Eout = Ein - tau (J - <J>) (Eq. ampere;
 * the mean of J is removed when cfg->remove_mean). */
static void ampere_update(const orc_es1d_cfg *cfg, const double *Ein,
                          const double *J, double tau, double *Eout) {
  double mean = 0.0;
  if (cfg->remove_mean) {
    for (long i = 0; i < cfg->nc; i++) mean += J[i];
    mean /= (double)cfg->nc;
  }
  for (long i = 0; i < cfg->nc; i++) Eout[i] = Ein[i] - tau * (J[i] - mean);
}

/* Particle loops split over threads in the OpenMP timing build only (see the
 * header); empty in the checker build. */
#ifdef _OPENMP
#define ORC_PARALLEL_FOR _Pragma("omp parallel for schedule(static)")
#else
#define ORC_PARALLEL_FOR
#endif

/* J += (1/h) sum_p q w_p u_p S(x_h - X_p) over the markers of species s at
 * positions X with velocities U (Sec. 2.2).  Checker build: one loop in marker
 * order.  OpenMP timing build: per-thread private sums, added afterwards. */
static void deposit_current(const orc_es1d_cfg *cfg, const orc_species *s, const double *X,
                            const double *U, double h, double *J) {
  long nc = cfg->nc;
#ifdef _OPENMP
#pragma omp parallel
  {
    double *Jp = (double *)calloc((size_t)nc, sizeof(double));
#pragma omp for schedule(static)
    for (long p = 0; p < s->n; p++) {
      long idx[3];
      double wt[3];
      int k = orc_shape_weights(cfg->order, X[p] / h, nc, idx, wt);
      double c = s->q * weight_of(s, p) * U[p];
      for (int j = 0; j < k; j++) Jp[idx[j]] += c * wt[j] / h;
    }
#pragma omp critical
    for (long i = 0; i < nc; i++) J[i] += Jp[i];
    free(Jp);
  }
#else
  for (long p = 0; p < s->n; p++) {
    long idx[3];
    double wt[3];
    int k = orc_shape_weights(cfg->order, X[p] / h, nc, idx, wt);
    double c = s->q * weight_of(s, p) * U[p];
    for (int j = 0; j < k; j++) J[idx[j]] += c * wt[j] / h;
  }
#endif
}

/*
 * One time step of ESEC1 / ESEC2 (1D1V, B = 0), in the paper's order:
 *
 *   x*      = x^n + dt/2 v^n                                   (both)
 *   j^{n,*} = deposit of v^n at x*;  E* = E^n - dt/2 j^{n,*}   (ESEC2 only,
 *                                                    Eq. doublestardef)
 *   E**_p   = gather of E* at x*  (ESEC1: E^{n,*}_p = gather of E^n at x*)
 *   v*      = v^n + dt/2 (q/m) E**_p
 *   x^{n+1} = x^n + dt v*;   x^{n+1/2} = x^n + dt/2 v*
 *   j^{*,n+1/2} = deposit of v* at x^{n+1/2}
 *   E^{n+1} = E^n - dt j^{*,n+1/2};   E^{n+1/2} = (E^n + E^{n+1})/2
 *   E^{n+1/2}_p = gather of E^{n+1/2} at x^{n+1/2}
 *   v^dag   = v^n + dt (q/m) E^{n+1/2}_p                  (Eq. PICmodification)
 *   R       = |v^n|^2 + 2 v* . (v^dag - v^n)
 *   v^{n+1} = Gamma v^dag, Gamma = sqrt(R) / |v^dag|      (Eq. opt_solution,
 *                                               rearranged form of Sec. 3.2)
 *   If R < 0 (imaginary Gamma) or |v^dag| = 0, Gamma := 1 and the particle is
 *   counted (Sec. 3.2 and Sec. 5.1).
 *
 * With cfg->passes > 0 the binomial filter F (Sec. 5: the paper filters to
 * remove the Nyquist mode) enters energy-consistently: both Ampere updates use
 * F j, and both gathers read F E* and F E^{n+1/2}.  F is symmetric, so
 * sum_h E_h (F j)_h = sum_h (F E)_h j_h and the energy identity stays exact.
 *
 * E is updated in place.  nfallback[s] receives the per-species count.
 * gamma_out: NULL or nsp pointers (each NULL or [n]) receiving Gamma (1 for
 * fallbacks).  Returns 0.
 * Pinned: energy identity Eq. (exp_econs_simple), uniform-field closed form,
 * Gamma = 1 + O(dt^3) / O(dt^4), cold plasma frequency, Landau and
 * two-stream rates, brute force (test_oracle_es1d.py).
 */
int orc_es1d_step_radicand(const orc_es1d_cfg *cfg, orc_species *sp, int nsp, double *E,
                           long *nfallback, double *const *gamma_out,
                           double *const *radicand_out);

int orc_es1d_step(const orc_es1d_cfg *cfg, orc_species *sp, int nsp,
                  double *E, long *nfallback, double *const *gamma_out) {
  return orc_es1d_step_radicand(cfg, sp, nsp, E, nfallback, gamma_out, NULL);
}

/* orc_es1d_step with one more optional output: radicand_out (NULL, or nsp
 * pointers, each NULL or [n]) receives R / |v^dag|^2 of every marker, the
 * scale-free radicand whose sign decides the fallback (NaN where v^dag = 0). */
int orc_es1d_step_radicand(const orc_es1d_cfg *cfg, orc_species *sp, int nsp, double *E,
                           long *nfallback, double *const *gamma_out,
                           double *const *radicand_out) {
  if (nsp <= 0 || cfg->nc <= 0) return -1;
  long nc = cfg->nc;
  double L = cfg->L, dt = cfg->dt, h = L / (double)nc;
  double *Estar = (double *)calloc((size_t)nc, sizeof(double));
  double *J = (double *)calloc((size_t)nc, sizeof(double));
  double *Enew = (double *)calloc((size_t)nc, sizeof(double));
  double *Ehalf = (double *)calloc((size_t)nc, sizeof(double));
  double **xs = (double **)calloc((size_t)nsp, sizeof(double *));
  double **vs = (double **)calloc((size_t)nsp, sizeof(double *));
  double **xh = (double **)calloc((size_t)nsp, sizeof(double *));
  for (int s = 0; s < nsp; s++) {
    xs[s] = (double *)calloc((size_t)sp[s].n + 1, sizeof(double));
    vs[s] = (double *)calloc((size_t)sp[s].n + 1, sizeof(double));
    xh[s] = (double *)calloc((size_t)sp[s].n + 1, sizeof(double));
  }

  /* x* = x^n + dt/2 v^n */
  for (int s = 0; s < nsp; s++) {
    ORC_PARALLEL_FOR
    for (long p = 0; p < sp[s].n; p++)
      xs[s][p] = wrap(sp[s].x[p] + 0.5 * dt * sp[s].v[p], L);
  }

  if (cfg->scheme == 2) {
    /* j^{n,*}: v^n deposited at x*, then E* = E^n - dt/2 j^{n,*} */
    for (long i = 0; i < nc; i++) J[i] = 0.0;
    for (int s = 0; s < nsp; s++) deposit_current(cfg, &sp[s], xs[s], sp[s].v, h, J);
    filter_passes(nc, J, cfg->passes);
    ampere_update(cfg, E, J, 0.5 * dt, Estar);
  } else {
    for (long i = 0; i < nc; i++) Estar[i] = E[i];
  }
  filter_passes(nc, Estar, cfg->passes);   /* the gathered E* is F E* */

  /* v* from the field gathered at x*; then x^{n+1/2} */
  for (int s = 0; s < nsp; s++) {
    double qm = sp[s].q / sp[s].m;
    ORC_PARALLEL_FOR
    for (long p = 0; p < sp[s].n; p++) {
      long idx[3];
      double wt[3];
      int k = orc_shape_weights(cfg->order, xs[s][p] / h, nc, idx, wt);
      double Ess = 0.0;
      for (int j = 0; j < k; j++) Ess += Estar[idx[j]] * wt[j];
      vs[s][p] = sp[s].v[p] + 0.5 * dt * qm * Ess;
      xh[s][p] = wrap(sp[s].x[p] + 0.5 * dt * vs[s][p], L);
    }
  }

  /* j^{*,n+1/2}: v* deposited at x^{n+1/2}; E^{n+1}, E^{n+1/2} */
  for (long i = 0; i < nc; i++) J[i] = 0.0;
  for (int s = 0; s < nsp; s++) deposit_current(cfg, &sp[s], xh[s], vs[s], h, J);
  filter_passes(nc, J, cfg->passes);
  ampere_update(cfg, E, J, dt, Enew);
  for (long i = 0; i < nc; i++) Ehalf[i] = 0.5 * (E[i] + Enew[i]);
  filter_passes(nc, Ehalf, cfg->passes);   /* the gathered E^{n+1/2} is F E^{n+1/2} */

  /* v^dag, Gamma, v^{n+1}; x^{n+1} */
  for (int s = 0; s < nsp; s++) {
    double qm = sp[s].q / sp[s].m;
    long count = 0;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) reduction(+ : count)
#endif
    for (long p = 0; p < sp[s].n; p++) {
      long idx[3];
      double wt[3];
      int k = orc_shape_weights(cfg->order, xh[s][p] / h, nc, idx, wt);
      double Ep = 0.0;
      for (int j = 0; j < k; j++) Ep += Ehalf[idx[j]] * wt[j];
      double vn = sp[s].v[p];
      double vstar = vs[s][p];
      double vdag = vn + dt * qm * Ep;
      double R = vn * vn + 2.0 * vstar * (vdag - vn);
      double vd2 = vdag * vdag;
      double gamma = 1.0;
      if (cfg->gamma_on) {
        if (R < 0.0 || vd2 == 0.0) {
          count++;
        } else {
          gamma = sqrt(R) / sqrt(vd2);
        }
      }
      if (gamma_out && gamma_out[s]) gamma_out[s][p] = gamma;
      if (radicand_out && radicand_out[s]) radicand_out[s][p] = vd2 > 0.0 ? R / vd2 : NAN;
      sp[s].v[p] = gamma == 1.0 ? vdag : vdag * gamma;
      sp[s].x[p] = wrap(sp[s].x[p] + dt * vstar, L);
    }
    if (nfallback) nfallback[s] = count;
  }
  for (long i = 0; i < nc; i++) E[i] = Enew[i];

  for (int s = 0; s < nsp; s++) {
    free(xs[s]);
    free(vs[s]);
    free(xh[s]);
  }
  free(xs);
  free(vs);
  free(xh);
  free(Estar);
  free(J);
  free(Enew);
  free(Ehalf);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Reverse mode of the 1D1V step (for gradients of a final objective)        */
/* ------------------------------------------------------------------------ */

/* Shape weights and their derivatives dS/dxi at xi = x/h (order 1: the tent,
 * piecewise; order 2: the quadratic B-spline, continuously differentiable). */
static int shape_weights_deriv(int order, double xi, long nc, long *idx, double *wt,
                               double *dwt) {
  int k = orc_shape_weights(order, xi, nc, idx, wt);
  if (order == 1) {
    dwt[0] = -1.0;
    dwt[1] = 1.0;
  } else {
    double d = xi - floor(xi + 0.5);
    dwt[0] = -(0.5 - d);
    dwt[1] = -2.0 * d;
    dwt[2] = 0.5 + d;
  }
  return k;
}

/* Adjoint of Eout = Ein - tau (J - <J>): Ein_bar += Eout_bar and the
 * returned Jbar = -tau (Eout_bar - <Eout_bar>) (the mean removal is symmetric). */
static void ampere_adjoint(const orc_es1d_cfg *cfg, const double *Eout_bar, double tau,
                           double *Ein_bar, double *Jbar) {
  double mean = 0.0;
  if (cfg->remove_mean) {
    for (long i = 0; i < cfg->nc; i++) mean += Eout_bar[i];
    mean /= (double)cfg->nc;
  }
  for (long i = 0; i < cfg->nc; i++) {
    Ein_bar[i] += Eout_bar[i];
    Jbar[i] = -tau * (Eout_bar[i] - mean);
  }
}

/*
 * Gradients through nsteps steps of orc_es1d_step, by reverse mode (the
 * adjoint of each operation of the step, taken in the reverse order):
 *   deposit J_h = sum_p c_p S(x_p - x_h)/h  ->  c_bar_p = sum_h J_bar_h S/h,
 *                                              x_bar_p += c_p sum_h J_bar_h S'/h^2
 *   gather  a_p = sum_h E_h S(x_p - x_h)    ->  E_bar_h += a_bar_p S,
 *                                              x_bar_p += a_bar_p sum_h E_h S'/h
 *   Gamma (Sec. 3.2): v^{n+1} = v^dag sqrt(R)/|v^dag| with R = |v^n|^2 +
 *   2 v* (v^dag - v^n); in 1D v^{n+1} = sign(v^dag) sqrt(R), so only R
 *   carries the adjoint: R_bar = v_bar^{n+1} sign(v^dag) / (2 sqrt(R)); a
 *   fallback (Gamma := 1) passes v_bar^{n+1} to v^dag.
 * The periodic wrap has derivative 1.
 * On entry sp and E hold the initial state (unchanged on return), Ebar the
 * adjoint of the final field, xbar[s], vbar[s] the adjoints of the final
 * markers; on return Ebar, xbar, vbar hold the adjoints of the initial state
 * and wbar[s] (if not NULL) the adjoint of each marker's weight (of w0 summed
 * over the markers of a uniformly weighted species).  Returns 0.
 * Pinned by central differences of orc_es1d_run (test_oracle_grad.py).
 */
int orc_es1d_grad(const orc_es1d_cfg *cfg, const orc_species *sp0, int nsp, const double *E0,
                  long nsteps, double *Ebar, double *const *xbar, double *const *vbar,
                  double *const *wbar) {
  if (cfg->passes != 0) return -1;   /* the reverse mode is for the unfiltered scheme */
  long nc = cfg->nc;
  double L = cfg->L, dt = cfg->dt, h = L / (double)nc;
  /* forward, keeping every step's markers and field */
  double **X = (double **)calloc((size_t)nsp * (nsteps + 1), sizeof(double *));
  double **V = (double **)calloc((size_t)nsp * (nsteps + 1), sizeof(double *));
  double *Eh = (double *)calloc((size_t)nc * (nsteps + 1), sizeof(double));
  orc_species *sp = (orc_species *)calloc((size_t)nsp, sizeof(orc_species));
  for (long i = 0; i < nc; i++) Eh[i] = E0[i];
  for (int s = 0; s < nsp; s++) {
    sp[s] = sp0[s];
    X[s] = (double *)calloc((size_t)sp0[s].n + 1, sizeof(double));
    V[s] = (double *)calloc((size_t)sp0[s].n + 1, sizeof(double));
    for (long p = 0; p < sp0[s].n; p++) {
      X[s][p] = sp0[s].x[p];
      V[s][p] = sp0[s].v[p];
    }
  }
  for (long n = 0; n < nsteps; n++) {
    double *En = Eh + (n + 1) * nc;
    for (long i = 0; i < nc; i++) En[i] = Eh[n * nc + i];
    for (int s = 0; s < nsp; s++) {
      double *xn = (double *)calloc((size_t)sp0[s].n + 1, sizeof(double));
      double *vn = (double *)calloc((size_t)sp0[s].n + 1, sizeof(double));
      for (long p = 0; p < sp0[s].n; p++) {
        xn[p] = X[n * nsp + s][p];
        vn[p] = V[n * nsp + s][p];
      }
      X[(n + 1) * nsp + s] = xn;
      V[(n + 1) * nsp + s] = vn;
      sp[s].x = xn;
      sp[s].v = vn;
    }
    orc_es1d_step(cfg, sp, nsp, En, NULL, NULL);
  }

  /* reverse */
  double *Estar = (double *)calloc((size_t)nc, sizeof(double));
  double *J = (double *)calloc((size_t)nc, sizeof(double));
  double *Ehalf = (double *)calloc((size_t)nc, sizeof(double));
  double *Jbar = (double *)calloc((size_t)nc, sizeof(double));
  double *Hbar = (double *)calloc((size_t)nc, sizeof(double));
  double *Esbar = (double *)calloc((size_t)nc, sizeof(double));
  double *Enbar = (double *)calloc((size_t)nc, sizeof(double));
  for (int s = 0; s < nsp; s++)
    if (wbar && wbar[s])
      for (long p = 0; p < (sp0[s].w ? sp0[s].n : 1); p++) wbar[s][p] = 0.0;
  for (long n = nsteps - 1; n >= 0; n--) {
    const double *En = Eh + n * nc, *Enew = Eh + (n + 1) * nc;
    /* recompute the step's grid quantities: E*, E^{n+1/2} */
    if (cfg->scheme == 2) {
      for (long i = 0; i < nc; i++) J[i] = 0.0;
      for (int s = 0; s < nsp; s++)
        for (long p = 0; p < sp0[s].n; p++) {
          long idx[3];
          double wt[3];
          double xs = wrap(X[n * nsp + s][p] + 0.5 * dt * V[n * nsp + s][p], L);
          int k = orc_shape_weights(cfg->order, xs / h, nc, idx, wt);
          double c = sp0[s].q * weight_of(&sp0[s], p) * V[n * nsp + s][p];
          for (int j = 0; j < k; j++) J[idx[j]] += c * wt[j] / h;
        }
      ampere_update(cfg, En, J, 0.5 * dt, Estar);
    } else {
      for (long i = 0; i < nc; i++) Estar[i] = En[i];
    }
    for (long i = 0; i < nc; i++) {
      Ehalf[i] = 0.5 * (En[i] + Enew[i]);
      Hbar[i] = 0.0;
      Esbar[i] = 0.0;
      Enbar[i] = 0.0;
    }
    /* markers, from v^{n+1}, x^{n+1} back to v*, x^{n+1/2}: H_bar and the
     * adjoints of v*, x^{n+1/2} (kept in ub, yb) */
    double **ub = (double **)calloc((size_t)nsp, sizeof(double *));
    double **yb = (double **)calloc((size_t)nsp, sizeof(double *));
    for (int s = 0; s < nsp; s++) {
      double qm = sp0[s].q / sp0[s].m;
      ub[s] = (double *)calloc((size_t)sp0[s].n + 1, sizeof(double));
      yb[s] = (double *)calloc((size_t)sp0[s].n + 1, sizeof(double));
      for (long p = 0; p < sp0[s].n; p++) {
        const double xn = X[n * nsp + s][p], vn = V[n * nsp + s][p];
        long idx[3];
        double wt[3], dwt[3];
        double xs = wrap(xn + 0.5 * dt * vn, L);
        int k = orc_shape_weights(cfg->order, xs / h, nc, idx, wt);
        double a = 0.0;
        for (int j = 0; j < k; j++) a += Estar[idx[j]] * wt[j];
        double u = vn + 0.5 * dt * qm * a;
        double y = wrap(xn + 0.5 * dt * u, L);
        k = shape_weights_deriv(cfg->order, y / h, nc, idx, wt, dwt);
        double b = 0.0, bp = 0.0;
        for (int j = 0; j < k; j++) {
          b += Ehalf[idx[j]] * wt[j];
          bp += Ehalf[idx[j]] * dwt[j];
        }
        double d = vn + dt * qm * b;
        double R = vn * vn + 2.0 * u * (d - vn);
        double vb1 = vbar[s][p], xb1 = xbar[s][p];
        /* x^{n+1} = x^n + dt v* */
        double xb = xb1, ubar = dt * xb1, vb = 0.0, db = 0.0;
        /* v^{n+1} */
        if (cfg->gamma_on && !(R < 0.0 || d * d == 0.0)) {
          double Rb = vb1 * (d > 0.0 ? 1.0 : -1.0) / (2.0 * sqrt(R));
          vb += Rb * (2.0 * vn - 2.0 * u);
          ubar += Rb * 2.0 * (d - vn);
          db += Rb * 2.0 * u;
        } else {
          db += vb1;
        }
        /* v^dag = v^n + dt (q/m) b */
        vb += db;
        double bb = db * dt * qm;
        for (int j = 0; j < k; j++) Hbar[idx[j]] += bb * wt[j];
        double ybar = bb * bp / h;
        xbar[s][p] = xb;
        vbar[s][p] = vb;
        ub[s][p] = ubar;
        yb[s][p] = ybar;
      }
    }
    /* E^{n+1/2} = (E^n + E^{n+1})/2 and E^{n+1} = E^n - dt (j - <j>) */
    for (long i = 0; i < nc; i++) {
      Enbar[i] = Ebar[i] + 0.5 * Hbar[i];  /* adjoint of E^{n+1} */
      Ebar[i] = 0.5 * Hbar[i];             /* adjoint of E^n so far */
    }
    ampere_adjoint(cfg, Enbar, dt, Ebar, Jbar);
    /* j^{*,n+1/2} = deposit of v* at x^{n+1/2}; v* = v^n + dt/2 (q/m) a;
     * x^{n+1/2} = x^n + dt/2 v*; a = gather of E* at x* */
    for (int s = 0; s < nsp; s++) {
      double qm = sp0[s].q / sp0[s].m;
      for (long p = 0; p < sp0[s].n; p++) {
        const double xn = X[n * nsp + s][p], vn = V[n * nsp + s][p];
        const double w = weight_of(&sp0[s], p);
        long idx[3];
        double wt[3], dwt[3];
        double xs = wrap(xn + 0.5 * dt * vn, L);
        int k = shape_weights_deriv(cfg->order, xs / h, nc, idx, wt, dwt);
        double a = 0.0, ap = 0.0;
        for (int j = 0; j < k; j++) {
          a += Estar[idx[j]] * wt[j];
          ap += Estar[idx[j]] * dwt[j];
        }
        double u = vn + 0.5 * dt * qm * a;
        double y = wrap(xn + 0.5 * dt * u, L);
        long idy[3];
        double wy[3], dwy[3];
        int ky = shape_weights_deriv(cfg->order, y / h, nc, idy, wy, dwy);
        double g = 0.0, gp = 0.0;
        for (int j = 0; j < ky; j++) {
          g += Jbar[idy[j]] * wy[j] / h;
          gp += Jbar[idy[j]] * dwy[j] / (h * h);
        }
        double c = sp0[s].q * w * u;
        double ubar = ub[s][p] + sp0[s].q * w * g;
        double ybar = yb[s][p] + c * gp;
        if (wbar && wbar[s]) wbar[s][sp0[s].w ? p : 0] += sp0[s].q * u * g;
        xbar[s][p] += ybar;
        ubar += 0.5 * dt * ybar;
        vbar[s][p] += ubar;
        double abar = 0.5 * dt * qm * ubar;
        for (int j = 0; j < k; j++) Esbar[idx[j]] += abar * wt[j];
        double xsb = abar * ap / h;
        ub[s][p] = xsb;  /* adjoint of x* so far */
      }
    }
    /* E* = E^n - dt/2 (j^{n,*} - <.>) (ESEC2) or E^n (ESEC1) */
    if (cfg->scheme == 2) {
      ampere_adjoint(cfg, Esbar, 0.5 * dt, Ebar, Jbar);
      for (int s = 0; s < nsp; s++)
        for (long p = 0; p < sp0[s].n; p++) {
          const double xn = X[n * nsp + s][p], vn = V[n * nsp + s][p];
          const double w = weight_of(&sp0[s], p);
          long idx[3];
          double wt[3], dwt[3];
          double xs = wrap(xn + 0.5 * dt * vn, L);
          int k = shape_weights_deriv(cfg->order, xs / h, nc, idx, wt, dwt);
          double g = 0.0, gp = 0.0;
          for (int j = 0; j < k; j++) {
            g += Jbar[idx[j]] * wt[j] / h;
            gp += Jbar[idx[j]] * dwt[j] / (h * h);
          }
          if (wbar && wbar[s]) wbar[s][sp0[s].w ? p : 0] += sp0[s].q * vn * g;
          vbar[s][p] += sp0[s].q * w * g;
          ub[s][p] += sp0[s].q * w * vn * gp;
        }
    } else {
      for (long i = 0; i < nc; i++) Ebar[i] += Esbar[i];
    }
    /* x* = x^n + dt/2 v^n */
    for (int s = 0; s < nsp; s++)
      for (long p = 0; p < sp0[s].n; p++) {
        xbar[s][p] += ub[s][p];
        vbar[s][p] += 0.5 * dt * ub[s][p];
      }
    for (int s = 0; s < nsp; s++) {
      free(ub[s]);
      free(yb[s]);
    }
    free(ub);
    free(yb);
  }
  for (long k = 0; k <= nsteps; k++)
    for (int s = 0; s < nsp; s++) {
      free(X[k * nsp + s]);
      free(V[k * nsp + s]);
    }
  free(X);
  free(V);
  free(Eh);
  free(sp);
  free(Estar);
  free(J);
  free(Ehalf);
  free(Jbar);
  free(Hbar);
  free(Esbar);
  free(Enbar);
  return 0;
}

/*
 * Energies of Sec. 5.1: KE_s = (1/2) m_s sum_p w_p v_p^2 per species and
 * W_E = (1/2) h sum_h E_h^2.  Pinned through the energy identity tests.
 */
void orc_es1d_energy(const orc_es1d_cfg *cfg, const orc_species *sp, int nsp,
                     const double *E, double *KE, double *WE) {
  double h = cfg->L / (double)cfg->nc;
  for (int s = 0; s < nsp; s++) {
    double acc = 0.0;
    for (long p = 0; p < sp[s].n; p++)
      acc += weight_of(&sp[s], p) * sp[s].v[p] * sp[s].v[p];
    KE[s] = 0.5 * sp[s].m * acc;
  }
  double we = 0.0;
  for (long i = 0; i < cfg->nc; i++) we += E[i] * E[i];
  *WE = 0.5 * h * we;
}

/*
 * nsteps steps; TE[k] = total energy after k steps (TE[0] initial),
 * nfb[k] = fallback count (all species) of step k.  Returns 0.
 */
int orc_es1d_run(const orc_es1d_cfg *cfg, orc_species *sp, int nsp, double *E,
                 long nsteps, double *TE, double *WE_hist, long *nfb) {
  double *KE = (double *)calloc((size_t)nsp, sizeof(double));
  long *cnt = (long *)calloc((size_t)nsp, sizeof(long));
  double we;
  orc_es1d_energy(cfg, sp, nsp, E, KE, &we);
  double te = we;
  for (int s = 0; s < nsp; s++) te += KE[s];
  if (TE) TE[0] = te;
  if (WE_hist) WE_hist[0] = we;
  for (long k = 0; k < nsteps; k++) {
    orc_es1d_step(cfg, sp, nsp, E, cnt, NULL);
    long c = 0;
    for (int s = 0; s < nsp; s++) c += cnt[s];
    if (nfb) nfb[k] = c;
    if (TE || WE_hist) {
      orc_es1d_energy(cfg, sp, nsp, E, KE, &we);
      te = we;
      for (int s = 0; s < nsp; s++) te += KE[s];
      if (TE) TE[k + 1] = te;
      if (WE_hist) WE_hist[k + 1] = we;
    }
  }
  free(KE);
  free(cnt);
  return 0;
}

/*
 * Initial field from Gauss's law in the Poisson form, Eq. (poisson):
 * dE/dx = rho - rho_background, rho deposited with the same shape.  Solved
 * spectrally (the paper's test code is pseudospectral, Sec. 5): with the
 * discrete Fourier transform rho_k = sum_j rho_j exp(-2 pi i j k / N),
 * E_k = rho_k / (i kappa_k), kappa_k = 2 pi k / L; the k = 0 mode (the
 * neutralising background) and, for even N, the Nyquist mode are zeroed.
 * Plain O(N^2) transform.  Pinned: a single cosine density gives the exact
 * sine field; the discrete derivative of E reproduces rho - <rho>.
 */
static void poisson_spectral(long nc, double L, const double *rho, double *E);

/* Charge density rho_h = (1/h) sum_p q w S(x_h - x_p) of the positions. */
static void deposit_charge(const orc_es1d_cfg *cfg, const orc_species *sp, int nsp,
                           double *rho) {
  long nc = cfg->nc;
  double h = cfg->L / (double)nc;
  for (long j = 0; j < nc; j++) rho[j] = 0.0;
  for (int s = 0; s < nsp; s++)
    for (long p = 0; p < sp[s].n; p++) {
      long idx[3];
      double wt[3];
      int k = orc_shape_weights(cfg->order, sp[s].x[p] / h, nc, idx, wt);
      double c = sp[s].q * weight_of(&sp[s], p);
      for (int j = 0; j < k; j++) rho[idx[j]] += c * wt[j] / h;
    }
}

void orc_poisson_e0_1d(const orc_es1d_cfg *cfg, const orc_species *sp,
                       int nsp, double *E) {
  long nc = cfg->nc;
  double *rho = (double *)calloc((size_t)nc, sizeof(double));
  deposit_charge(cfg, sp, nsp, rho);
  poisson_spectral(nc, cfg->L, rho, E);
  free(rho);
}

/*
 * Charge diagnostics of a 1D1V state (Sec. 2.1: Gauss's law dE/dx = rho - 1 in
 * the paper's units, kept in time by continuity, d rho/dt + dj/dx = 0):
 *   rho_h     = (1/h) sum_p q w_p S(x_h - x_p), the deposit's own shape;
 *   Q_grid    = h sum_h rho_h,   Q_markers = sum_p q w_p;
 *   r         = D E - (rho - <rho>): the residual of Gauss's law with the
 *               spectral derivative D of the initial Poisson solve, on the
 *               Fourier modes m = 1 .. (nc - 1) / 2 (k = 0, the neutralising
 *               background, and the Nyquist mode, which D does not represent,
 *               left out): r_m = i kappa_m E_m - rho_m, kappa_m = 2 pi m / L,
 *               F_m = sum_j F_j exp(-2 pi i m j / nc), and in real space
 *               r_j = (2 / nc) sum_m Re(r_m exp(2 pi i m j / nc));
 *   gauss_l2  = sqrt(h sum_j r_j^2),  rho_l2 = sqrt(h sum_j rhot_j^2) with
 *               rhot the same modes of rho.
 * r and rhot: [nc] or NULL.  Plain O(nc^2) transforms.
 * Pinned (test_oracle_charge1d.py): the residual against numpy's FFT, a single
 * field mode in closed form, zero for the field of the Poisson solve, the
 * charge totals against the markers' charge.
 */
void orc_es1d_charge_diag(const orc_es1d_cfg *cfg, const orc_species *sp, int nsp,
                          const double *E, double *Q_markers, double *Q_grid,
                          double *gauss_l2, double *rho_l2, double *r, double *rhot) {
  const double twopi = 6.283185307179586476925286766559;
  long nc = cfg->nc, M = (nc - 1) / 2;
  double h = cfg->L / (double)nc;
  double *rho = (double *)calloc((size_t)nc, sizeof(double));
  double *rr = (double *)calloc((size_t)nc, sizeof(double));
  double *rt = (double *)calloc((size_t)nc, sizeof(double));
  deposit_charge(cfg, sp, nsp, rho);
  double qm = 0.0, qg = 0.0;
  for (int s = 0; s < nsp; s++)
    for (long p = 0; p < sp[s].n; p++) qm += sp[s].q * weight_of(&sp[s], p);
  for (long j = 0; j < nc; j++) qg += h * rho[j];
  for (long m = 1; m <= M; m++) {
    double er = 0.0, ei = 0.0, pr = 0.0, pi = 0.0;
    for (long j = 0; j < nc; j++) {
      double ang = -twopi * (double)((j * m) % nc) / (double)nc;
      er += E[j] * cos(ang);
      ei += E[j] * sin(ang);
      pr += rho[j] * cos(ang);
      pi += rho[j] * sin(ang);
    }
    double kappa = twopi * (double)m / cfg->L;
    /* r_m = i kappa E_m - rho_m */
    double rre = -kappa * ei - pr, rim = kappa * er - pi;
    for (long j = 0; j < nc; j++) {
      double ang = twopi * (double)((j * m) % nc) / (double)nc;
      rr[j] += 2.0 * (rre * cos(ang) - rim * sin(ang)) / (double)nc;
      rt[j] += 2.0 * (pr * cos(ang) - pi * sin(ang)) / (double)nc;
    }
  }
  double g2 = 0.0, p2 = 0.0;
  for (long j = 0; j < nc; j++) {
    g2 += rr[j] * rr[j];
    p2 += rt[j] * rt[j];
  }
  if (Q_markers) *Q_markers = qm;
  if (Q_grid) *Q_grid = qg;
  if (gauss_l2) *gauss_l2 = sqrt(h * g2);
  if (rho_l2) *rho_l2 = sqrt(h * p2);
  if (r) memcpy(r, rr, sizeof(double) * (size_t)nc);
  if (rhot) memcpy(rhot, rt, sizeof(double) * (size_t)nc);
  free(rho);
  free(rr);
  free(rt);
}

/* E from dE/dx = rho - <rho> as above (k = 0 and the Nyquist mode zeroed). */
static void poisson_spectral(long nc, double L, const double *rho, double *E) {
  const double twopi = 6.283185307179586476925286766559;
  for (long j = 0; j < nc; j++) E[j] = 0.0;
  for (long k = 1; k < nc; k++) {
    if (nc % 2 == 0 && k == nc / 2) continue;
    double re = 0.0, im = 0.0;
    for (long j = 0; j < nc; j++) {
      double ang = -twopi * (double)((j * k) % nc) / (double)nc;
      re += rho[j] * cos(ang);
      im += rho[j] * sin(ang);
    }
    long ks = k < nc - k ? k : k - nc; /* signed frequency */
    double kappa = twopi * (double)ks / L;
    /* E_k = rho_k / (i kappa) = (im - i re) / kappa */
    double ere = im / kappa, eim = -re / kappa;
    for (long j = 0; j < nc; j++) {
      double ang = twopi * (double)((j * k) % nc) / (double)nc;
      E[j] += (ere * cos(ang) - eim * sin(ang)) / (double)nc;
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Standard explicit PIC, the comparator of Sec. 5                          */
/* ------------------------------------------------------------------------ */

/*
 * The paper measures its schemes against Vlasov-Poisson PIC with the
 * classical leapfrog push (in 1D1V the Boris push without B), with binomial
 * filtering of the charge density.  State: x^n, v^{n-1/2} and E^n, the field
 * of the filtered charge of x^n.  One step:
 *   E^n_p     = sum_h E^n_h S(x_h - x_p^n)
 *   v^{n+1/2} = v^{n-1/2} + dt (q/m) E^n_p
 *   x^{n+1}   = x^n + dt v^{n+1/2}
 *   rho^{n+1} = (1/h) sum q w S(x_h - x^{n+1}), `passes` times through the
 *               1-2-1 filter, E^{n+1} from dE/dx = rho - <rho> (spectral)
 * The energy at time n: KE^n = (1/2) m sum w (v^{n-1/2}^2 + v^{n+1/2}^2) / 2 and
 * W_E^n = (h/2) sum (E^n)^2.  It is not conserved (that is the comparison).
 */

/* One pass of the binomial filter out_i = (in_{i-1} + 2 in_i + in_{i+1}) / 4,
 * periodic; its factor on mode k is cos^2(pi k / nc), 0 on the Nyquist mode
 * (pinned against that transfer function). */
void orc_binomial_filter(long nc, const double *in, double *out) {
  for (long i = 0; i < nc; i++)
    out[i] = 0.25 * (in[imod(i - 1, nc)] + 2.0 * in[i] + in[imod(i + 1, nc)]);
}

/* E of the positions: charge, `passes` filter passes, spectral Gauss's law. */
void orc_std_field(const orc_es1d_cfg *cfg, const orc_species *sp, int nsp, int passes,
                   double *E) {
  long nc = cfg->nc;
  double *rho = (double *)calloc((size_t)nc, sizeof(double));
  double *tmp = (double *)calloc((size_t)nc, sizeof(double));
  deposit_charge(cfg, sp, nsp, rho);
  for (int k = 0; k < passes; k++) {
    orc_binomial_filter(nc, rho, tmp);
    memcpy(rho, tmp, sizeof(double) * (size_t)nc);
  }
  poisson_spectral(nc, cfg->L, rho, E);
  free(rho);
  free(tmp);
}

/* Start of the leapfrog from (x^0, v^0): E^0 of x^0 and the usual half kick
 * back, v^{-1/2} = v^0 - dt/2 (q/m) E^0_p, in place in sp[].v. */
void orc_std_start(const orc_es1d_cfg *cfg, orc_species *sp, int nsp, int passes, double *E) {
  orc_std_field(cfg, sp, nsp, passes, E);
  for (int s = 0; s < nsp; s++) {
    double qm = sp[s].q / sp[s].m;
    for (long p = 0; p < sp[s].n; p++) {
      double Ep;
      orc_gather_1d(cfg->order, cfg->nc, cfg->L, 1, &sp[s].x[p], E, &Ep);
      sp[s].v[p] -= 0.5 * cfg->dt * qm * Ep;
    }
  }
}

/* One leapfrog step from (x^n, v^{n-1/2}, E^n) to (x^{n+1}, v^{n+1/2}, E^{n+1})
 * in place; KE (per species) and WE receive the energies at time n. */
int orc_std_step(const orc_es1d_cfg *cfg, orc_species *sp, int nsp, int passes, double *E,
                 double *KE, double *WE) {
  long nc = cfg->nc;
  double dt = cfg->dt, h = cfg->L / (double)nc;
  double we = 0.0;
  for (long j = 0; j < nc; j++) we += E[j] * E[j];
  *WE = 0.5 * h * we;
  for (int s = 0; s < nsp; s++) {
    double qm = sp[s].q / sp[s].m, acc = 0.0;
    for (long p = 0; p < sp[s].n; p++) {
      double Ep;
      orc_gather_1d(cfg->order, nc, cfg->L, 1, &sp[s].x[p], E, &Ep);
      double vold = sp[s].v[p];
      double vnew = vold + dt * qm * Ep;
      acc += weight_of(&sp[s], p) * 0.5 * (vold * vold + vnew * vnew);
      sp[s].v[p] = vnew;
      sp[s].x[p] = wrap(sp[s].x[p] + dt * vnew, cfg->L);
    }
    KE[s] = 0.5 * sp[s].m * acc;
  }
  orc_std_field(cfg, sp, nsp, passes, E);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* 2D3V electromagnetic scheme with the leapfrog / Yee field step (Sec. 4.1) */
/* ------------------------------------------------------------------------ */

/*
 * Yee lattice on a periodic nx x ny grid (Sec. 2.2.2): field components are
 * stored as [ny][nx] arrays; component c of E (and of J) sits at
 * ((i + ox) hx, (j + oy) hy) and component c of B at the face centre:
 *   Ex (1/2, 0)   Ey (0, 1/2)   Ez (0, 0)
 *   Bx (0, 1/2)   By (1/2, 0)   Bz (1/2, 1/2)
 * Gather of E_c and deposit of J_c use the same tensor-product B-spline
 * shape centred on component c's nodes, so the pairing of Eq.
 * (exp_econs_simple) holds component by component.
 */
typedef struct {
  long nx, ny;
  double Lx, Ly;
  int order;   /* 1 | 2 */
  double dt;
  double c;    /* speed of light (dimensionless) */
  int scheme;  /* 1 = ESEC1-type v*, 2 = the j^{n,*} / E* stage of Eq.
                  (EMleapfrog) */
  int gamma_on;
  int charge_conserving;  /* 1: the shapes and path segments below (order 1) */
} orc_em2d_cfg;

typedef struct {
  double q, m;
  long n;
  double *x, *y;          /* [n] */
  double *vx, *vy, *vz;   /* [n] */
  const double *w;
  double w0;
} orc_species2d;

static const double OFFX_E[3] = {0.5, 0.0, 0.0}, OFFY_E[3] = {0.0, 0.5, 0.0};
static const double OFFX_B[3] = {0.0, 0.5, 0.5}, OFFY_B[3] = {0.5, 0.0, 0.5};

/*
 * Tensor-product weights of component with offsets (ox, oy).  Charge-
 * conserving option (Sec. 3.5): the charge uses the bilinear shape (degree 1
 * in x and y, on the nodes (i, j)); for Eq. (detbal) to hold the current
 * component along an axis needs the derivative of that shape, a degree-0 box
 * on the half nodes, so each component takes degree 0 on the axes where it
 * sits on half nodes and degree 1 where it sits on integer nodes: Jx, Ex
 * B0(x) B1(y); Jy, Ey B1(x) B0(y); Jz, Ez B1(x) B1(y) (the B components by the
 * same rule, which no conservation property involves).
 */
static int shape2d(const orc_em2d_cfg *g, double x, double y, double ox,
                   double oy, long *idx, double *wt) {
  long ix[3], iy[3];
  double wx[3], wy[3];
  double hx = g->Lx / (double)g->nx, hy = g->Ly / (double)g->ny;
  int degx = g->charge_conserving ? (ox == 0.5 ? 0 : 1) : g->order;
  int degy = g->charge_conserving ? (oy == 0.5 ? 0 : 1) : g->order;
  int kx = orc_shape_weights(degx, x / hx - ox, g->nx, ix, wx);
  int ky = orc_shape_weights(degy, y / hy - oy, g->ny, iy, wy);
  int k = 0;
  for (int b = 0; b < ky; b++)
    for (int a = 0; a < kx; a++) {
      idx[k] = iy[b] * g->nx + ix[a];
      wt[k] = wx[a] * wy[b];
      k++;
    }
  return k;
}

#define AT(F, i, j) (F)[imod((j), ny) * nx + imod((i), nx)]

/* Discrete curl of E, evaluated on the B locations (Yee differences). */
void orc_yee_curl_e(long nx, long ny, double hx, double hy, const double *Ex,
                    const double *Ey, const double *Ez, double *cx, double *cy,
                    double *cz) {
  for (long j = 0; j < ny; j++)
    for (long i = 0; i < nx; i++) {
      cx[j * nx + i] = (AT(Ez, i, j + 1) - AT(Ez, i, j)) / hy;
      cy[j * nx + i] = -(AT(Ez, i + 1, j) - AT(Ez, i, j)) / hx;
      cz[j * nx + i] = (AT(Ey, i + 1, j) - AT(Ey, i, j)) / hx -
                       (AT(Ex, i, j + 1) - AT(Ex, i, j)) / hy;
    }
}

/* Discrete curl of B, evaluated on the E locations (Yee differences). */
void orc_yee_curl_b(long nx, long ny, double hx, double hy, const double *Bx,
                    const double *By, const double *Bz, double *cx, double *cy,
                    double *cz) {
  for (long j = 0; j < ny; j++)
    for (long i = 0; i < nx; i++) {
      cx[j * nx + i] = (AT(Bz, i, j) - AT(Bz, i, j - 1)) / hy;
      cy[j * nx + i] = -(AT(Bz, i, j) - AT(Bz, i - 1, j)) / hx;
      cz[j * nx + i] = (AT(By, i, j) - AT(By, i - 1, j)) / hx -
                       (AT(Bx, i, j) - AT(Bx, i, j - 1)) / hy;
    }
}
#undef AT

static double wt2d(const orc_species2d *s, long p) {
  return s->w ? s->w[p] : s->w0;
}

/* Deposit q w v_c at (px, py) for the three components into J[3][ncell]. */
static void deposit_em(const orc_em2d_cfg *g, const orc_species2d *s, long n,
                       const double *px, const double *py, const double *ux,
                       const double *uy, const double *uz, double *J) {
  long ncell = g->nx * g->ny;
  double area = (g->Lx / (double)g->nx) * (g->Ly / (double)g->ny);
  for (long p = 0; p < n; p++) {
    const double u[3] = {ux[p], uy[p], uz[p]};
    double qw = s->q * wt2d(s, p);
    for (int c = 0; c < 3; c++) {
      long idx[9];
      double wt[9];
      int k = shape2d(g, px[p], py[p], OFFX_E[c], OFFY_E[c], idx, wt);
      for (int a = 0; a < k; a++) J[c * ncell + idx[a]] += qw * u[c] * wt[a] / area;
    }
  }
}

static void gather3(const orc_em2d_cfg *g, const double *F, const double *ox,
                    const double *oy, double x, double y, double out[3]) {
  long ncell = g->nx * g->ny;
  for (int c = 0; c < 3; c++) {
    long idx[9];
    double wt[9];
    int k = shape2d(g, x, y, ox[c], oy[c], idx, wt);
    double s = 0.0;
    for (int a = 0; a < k; a++) s += F[c * ncell + idx[a]] * wt[a];
    out[c] = s;
  }
}

static int cmp_double(const void *a, const void *b) {
  double u = *(const double *)a, v = *(const double *)b;
  return (u > v) - (u < v);
}

/*
 * The straight path from (x0, y0) to (x0 + dx, y0 + dy) (not wrapped) cut at
 * every grid line x = i hx and y = j hy it crosses (Sec. 3.5: the charge shape
 * is then quadratic along each piece, so Eq. (detbal) holds piece by piece).
 * Returns the number of pieces K and, in *s (malloc'd, K + 1 entries), the
 * path parameters 0 = s_0 <= s_1 <= ... <= s_K = 1 of the cuts.
 */
static int path_cuts(const orc_em2d_cfg *g, double x0, double y0, double dx, double dy,
                     double **s) {
  double hx = g->Lx / (double)g->nx, hy = g->Ly / (double)g->ny;
  long ax0 = (long)floor(x0 / hx), ax1 = (long)floor((x0 + dx) / hx);
  long ay0 = (long)floor(y0 / hy), ay1 = (long)floor((y0 + dy) / hy);
  long nxc = labs(ax1 - ax0), nyc = labs(ay1 - ay0);
  double *t = (double *)malloc(sizeof(double) * (size_t)(nxc + nyc + 2));
  long k = 0;
  t[k++] = 0.0;
  /* the lines between the start and end cells: i = ax0 + 1 .. ax1 moving up,
     i = ax0 .. ax1 + 1 moving down */
  for (long m = 1; m <= nxc; m++) {
    long line = ax1 > ax0 ? ax0 + m : ax0 - m + 1;
    t[k++] = (line * hx - x0) / dx;
  }
  for (long m = 1; m <= nyc; m++) {
    long line = ay1 > ay0 ? ay0 + m : ay0 - m + 1;
    t[k++] = (line * hy - y0) / dy;
  }
  qsort(t + 1, (size_t)(k - 1), sizeof(double), cmp_double);
  t[k] = 1.0;
  *s = t;
  return (int)k;
}

/*
 * Charge-conserving deposit of j^{*,n+1/2} for one marker moving from
 * (x0, y0) by (dx, dy) = dt v*: the sum over the path's pieces of the piece's
 * fraction times the shape at the piece's midpoint.
 */
static void deposit_path(const orc_em2d_cfg *g, double coef, const double u[3], double x0,
                         double y0, double dx, double dy, double *J) {
  long ncell = g->nx * g->ny;
  double *s;
  int K = path_cuts(g, x0, y0, dx, dy, &s);
  for (int k = 0; k < K; k++) {
    double tau = s[k + 1] - s[k], mid = 0.5 * (s[k] + s[k + 1]);
    double mx = wrap(x0 + mid * dx, g->Lx), my = wrap(y0 + mid * dy, g->Ly);
    for (int c = 0; c < 3; c++) {
      long idx[9];
      double wt[9];
      int n = shape2d(g, mx, my, OFFX_E[c], OFFY_E[c], idx, wt);
      for (int a = 0; a < n; a++) J[c * ncell + idx[a]] += coef * u[c] * tau * wt[a];
    }
  }
  free(s);
}

/* The matching gather of E at the same pieces: sum_k tau_k E(midpoint_k). */
static void gather_path(const orc_em2d_cfg *g, const double *F, double x0, double y0,
                        double dx, double dy, double out[3]) {
  double *s;
  int K = path_cuts(g, x0, y0, dx, dy, &s);
  out[0] = out[1] = out[2] = 0.0;
  for (int k = 0; k < K; k++) {
    double tau = s[k + 1] - s[k], mid = 0.5 * (s[k] + s[k + 1]), e[3];
    gather3(g, F, OFFX_E, OFFY_E, wrap(x0 + mid * dx, g->Lx), wrap(y0 + mid * dy, g->Ly), e);
    for (int c = 0; c < 3; c++) out[c] += tau * e[c];
  }
  free(s);
}

static void cross(const double a[3], const double b[3], double r[3]) {
  r[0] = a[1] * b[2] - a[2] * b[1];
  r[1] = a[2] * b[0] - a[0] * b[2];
  r[2] = a[0] * b[1] - a[1] * b[0];
}

/*
 * v* of v* = v^n + dt/2 (q/m)(E** + v* x B): linear in v*; with
 * u = v^n + (q/m)(dt/2) E** and t = (q/m)(dt/2) B the solution is
 * v* = (u + u x t + (u.t) t) / (1 + |t|^2).  Pinned: it satisfies the
 * implicit relation, and with E = 0 the push is the symmetric Boris
 * rotation of Sec. 2.2.1 (test_oracle_em2d.py).
 */
void orc_vstar_solve(const double u[3], const double t[3], double out[3]) {
  double uxt[3];
  cross(u, t, uxt);
  double ut = u[0] * t[0] + u[1] * t[1] + u[2] * t[2];
  double tt = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
  for (int c = 0; c < 3; c++) out[c] = (u[c] + uxt[c] + ut * t[c]) / (1.0 + tt);
}

/*
 * One step of Eq. (EMleapfrog):
 *   x*          = x^n + dt/2 v^n
 *   B^{n+1/2}   = B^{n-1/2} - dt curl_h E^n
 *   E*          = E^n + dt/2 (c^2 curl_h B^{n+1/2} - j^{n,*})   (scheme 2;
 *                 scheme 1 uses E^n)
 *   v*          = v^n + dt/2 (q/m)(E**_p + v* x B^{n+1/2}_p(x*))
 *   x^{n+1}     = x^n + dt v*,   x^{n+1/2} = x^n + dt/2 v*
 *   E^{n+1}     = E^n + dt (c^2 curl_h B^{n+1/2} - j^{*,n+1/2})
 *   v^dag       = v^n + dt (q/m)(E^{n+1/2}_p + v* x B^{n+1/2}_p)
 *   v^{n+1}     = Gamma v^dag  (Eq. opt_solution; fallback Gamma := 1)
 * The B in v^dag is gathered at x^{n+1/2}, as in the electromagnetic
 * schemes of Secs. 3.4 and 4.1.  With charge_conserving the deposit of
 * j^{*,n+1/2} and the gather of E^{n+1/2} run over the pieces of the path
 * x^n -> x^{n+1} (deposit_path, gather_path) with the same fractions and
 * shapes, so the pairing of Eq. (exp_econs_simple) still holds.  E (3 x ncell) and B (3 x ncell, holding
 * B^{n-1/2} on entry and B^{n+1/2} on exit) are updated in place.
 */
int orc_em2d_step(const orc_em2d_cfg *g, orc_species2d *sp, int nsp, double *E,
                  double *B, long *nfallback) {
  if (nsp <= 0 || g->nx <= 0 || g->ny <= 0) return -1;
  long nx = g->nx, ny = g->ny, ncell = nx * ny;
  double dt = g->dt, c2 = g->c * g->c;
  double hx = g->Lx / (double)nx, hy = g->Ly / (double)ny;
  double *cE = (double *)calloc((size_t)(3 * ncell), sizeof(double));
  double *cB = (double *)calloc((size_t)(3 * ncell), sizeof(double));
  double *Bh = (double *)calloc((size_t)(3 * ncell), sizeof(double));
  double *Es = (double *)calloc((size_t)(3 * ncell), sizeof(double));
  double *J = (double *)calloc((size_t)(3 * ncell), sizeof(double));
  double *En = (double *)calloc((size_t)(3 * ncell), sizeof(double));
  double *Eh = (double *)calloc((size_t)(3 * ncell), sizeof(double));

  /* B^{n+1/2} = B^{n-1/2} - dt curl E^n */
  orc_yee_curl_e(nx, ny, hx, hy, E, E + ncell, E + 2 * ncell, cE, cE + ncell,
                 cE + 2 * ncell);
  for (long a = 0; a < 3 * ncell; a++) Bh[a] = B[a] - dt * cE[a];
  orc_yee_curl_b(nx, ny, hx, hy, Bh, Bh + ncell, Bh + 2 * ncell, cB, cB + ncell,
                 cB + 2 * ncell);

  for (int s = 0; s < nsp; s++) {
    orc_species2d *S = &sp[s];
    long n = S->n;
    double qm = S->q / S->m;
    double *xs = (double *)calloc((size_t)n + 1, sizeof(double));
    double *ys = (double *)calloc((size_t)n + 1, sizeof(double));
    (void)qm;
    for (long p = 0; p < n; p++) {
      xs[p] = wrap(S->x[p] + 0.5 * dt * S->vx[p], g->Lx);
      ys[p] = wrap(S->y[p] + 0.5 * dt * S->vy[p], g->Ly);
    }
    if (g->scheme == 2) deposit_em(g, S, n, xs, ys, S->vx, S->vy, S->vz, J);
    free(xs);
    free(ys);
  }
  for (long a = 0; a < 3 * ncell; a++)
    Es[a] = g->scheme == 2 ? E[a] + 0.5 * dt * (c2 * cB[a] - J[a]) : E[a];

  /* per species: v*, x^{n+1/2}, x^{n+1}; deposit j^{*,n+1/2} */
  double **vsx = (double **)calloc((size_t)nsp, sizeof(double *));
  double **vsy = (double **)calloc((size_t)nsp, sizeof(double *));
  double **vsz = (double **)calloc((size_t)nsp, sizeof(double *));
  double **xh = (double **)calloc((size_t)nsp, sizeof(double *));
  double **yh = (double **)calloc((size_t)nsp, sizeof(double *));
  for (long a = 0; a < 3 * ncell; a++) J[a] = 0.0;
  for (int s = 0; s < nsp; s++) {
    orc_species2d *S = &sp[s];
    long n = S->n;
    double qm = S->q / S->m;
    vsx[s] = (double *)calloc((size_t)n + 1, sizeof(double));
    vsy[s] = (double *)calloc((size_t)n + 1, sizeof(double));
    vsz[s] = (double *)calloc((size_t)n + 1, sizeof(double));
    xh[s] = (double *)calloc((size_t)n + 1, sizeof(double));
    yh[s] = (double *)calloc((size_t)n + 1, sizeof(double));
    for (long p = 0; p < n; p++) {
      double xs = wrap(S->x[p] + 0.5 * dt * S->vx[p], g->Lx);
      double ys = wrap(S->y[p] + 0.5 * dt * S->vy[p], g->Ly);
      double Ess[3], Bs[3], u[3], t[3], vst[3];
      gather3(g, Es, OFFX_E, OFFY_E, xs, ys, Ess);
      gather3(g, Bh, OFFX_B, OFFY_B, xs, ys, Bs);
      const double vn[3] = {S->vx[p], S->vy[p], S->vz[p]};
      for (int c = 0; c < 3; c++) {
        u[c] = vn[c] + qm * 0.5 * dt * Ess[c];
        t[c] = qm * 0.5 * dt * Bs[c];
      }
      orc_vstar_solve(u, t, vst);
      vsx[s][p] = vst[0];
      vsy[s][p] = vst[1];
      vsz[s][p] = vst[2];
      xh[s][p] = wrap(S->x[p] + 0.5 * dt * vst[0], g->Lx);
      yh[s][p] = wrap(S->y[p] + 0.5 * dt * vst[1], g->Ly);
    }
    if (g->charge_conserving) {
      double area = hx * hy;
      for (long p = 0; p < n; p++) {
        const double vst[3] = {vsx[s][p], vsy[s][p], vsz[s][p]};
        deposit_path(g, S->q * wt2d(S, p) / area, vst, S->x[p], S->y[p], dt * vst[0],
                     dt * vst[1], J);
      }
    } else {
      deposit_em(g, S, n, xh[s], yh[s], vsx[s], vsy[s], vsz[s], J);
    }
  }
  for (long a = 0; a < 3 * ncell; a++) {
    En[a] = E[a] + dt * (c2 * cB[a] - J[a]);
    Eh[a] = 0.5 * (E[a] + En[a]);
  }

  for (int s = 0; s < nsp; s++) {
    orc_species2d *S = &sp[s];
    double qm = S->q / S->m;
    long count = 0;
    for (long p = 0; p < S->n; p++) {
      double Ep[3], Bp[3], vxb[3], vdag[3];
      if (g->charge_conserving)
        gather_path(g, Eh, S->x[p], S->y[p], dt * vsx[s][p], dt * vsy[s][p], Ep);
      else
        gather3(g, Eh, OFFX_E, OFFY_E, xh[s][p], yh[s][p], Ep);
      gather3(g, Bh, OFFX_B, OFFY_B, xh[s][p], yh[s][p], Bp);
      const double vn[3] = {S->vx[p], S->vy[p], S->vz[p]};
      const double vst[3] = {vsx[s][p], vsy[s][p], vsz[s][p]};
      cross(vst, Bp, vxb);
      for (int c = 0; c < 3; c++) vdag[c] = vn[c] + dt * qm * (Ep[c] + vxb[c]);
      double R = vn[0] * vn[0] + vn[1] * vn[1] + vn[2] * vn[2] +
                 2.0 * (vst[0] * (vdag[0] - vn[0]) + vst[1] * (vdag[1] - vn[1]) +
                        vst[2] * (vdag[2] - vn[2]));
      double vd2 = vdag[0] * vdag[0] + vdag[1] * vdag[1] + vdag[2] * vdag[2];
      double gamma = 1.0;
      if (g->gamma_on) {
        if (R < 0.0 || vd2 == 0.0)
          count++;
        else
          gamma = sqrt(R) / sqrt(vd2);
      }
      S->vx[p] = gamma == 1.0 ? vdag[0] : vdag[0] * gamma;
      S->vy[p] = gamma == 1.0 ? vdag[1] : vdag[1] * gamma;
      S->vz[p] = gamma == 1.0 ? vdag[2] : vdag[2] * gamma;
      S->x[p] = wrap(S->x[p] + dt * vst[0], g->Lx);
      S->y[p] = wrap(S->y[p] + dt * vst[1], g->Ly);
    }
    if (nfallback) nfallback[s] = count;
    free(vsx[s]);
    free(vsy[s]);
    free(vsz[s]);
    free(xh[s]);
    free(yh[s]);
  }
  for (long a = 0; a < 3 * ncell; a++) {
    E[a] = En[a];
    B[a] = Bh[a];
  }
  free(vsx);
  free(vsy);
  free(vsz);
  free(xh);
  free(yh);
  free(cE);
  free(cB);
  free(Bh);
  free(Es);
  free(J);
  free(En);
  free(Eh);
  return 0;
}

/*
 * Energies of Sec. 4.1 for the state (x^n, v^n, E^n, B^{n-1/2}):
 *   KE   = (1/2) m sum w |v|^2 per species,
 *   W_E  = (1/2) |h| sum |E^n|^2,
 *   W_B  = (c^2/2) |h| sum B^{n+1/2} . B^{n-1/2},
 * with B^{n+1/2} = B^{n-1/2} - dt curl_h E^n (the next leapfrog half).
 */
void orc_em2d_energy(const orc_em2d_cfg *g, const orc_species2d *sp, int nsp,
                     const double *E, const double *B, double *KE, double *WE,
                     double *WB) {
  long nx = g->nx, ny = g->ny, ncell = nx * ny;
  double hx = g->Lx / (double)nx, hy = g->Ly / (double)ny, area = hx * hy;
  for (int s = 0; s < nsp; s++) {
    double acc = 0.0;
    for (long p = 0; p < sp[s].n; p++)
      acc += wt2d(&sp[s], p) * (sp[s].vx[p] * sp[s].vx[p] + sp[s].vy[p] * sp[s].vy[p] +
                                sp[s].vz[p] * sp[s].vz[p]);
    KE[s] = 0.5 * sp[s].m * acc;
  }
  double we = 0.0;
  for (long a = 0; a < 3 * ncell; a++) we += E[a] * E[a];
  *WE = 0.5 * area * we;
  double *cE = (double *)calloc((size_t)(3 * ncell), sizeof(double));
  orc_yee_curl_e(nx, ny, hx, hy, E, E + ncell, E + 2 * ncell, cE, cE + ncell,
                 cE + 2 * ncell);
  double wb = 0.0;
  for (long a = 0; a < 3 * ncell; a++) wb += (B[a] - g->dt * cE[a]) * B[a];
  *WB = 0.5 * g->c * g->c * area * wb;
  free(cE);
}

/*
 * Charge density on the nodes (i, j) with the bilinear shape of the
 * charge-conserving option: rho = sum_p q w B1(x/hx - i) B1(y/hy - j) / |h|,
 * and the Gauss's-law residual r = div_h E - rho with the Yee divergence
 * (Ex(i+1/2,j) - Ex(i-1/2,j)) / hx + (Ey(i,j+1/2) - Ey(i,j-1/2)) / hy.  With
 * exact charge conservation (Sec. 3.5) r keeps its initial value.
 */
void orc_em2d_gauss_residual(const orc_em2d_cfg *g, const orc_species2d *sp, int nsp,
                             const double *E, double *rho, double *r) {
  long nx = g->nx, ny = g->ny, ncell = nx * ny;
  double hx = g->Lx / (double)nx, hy = g->Ly / (double)ny, area = hx * hy;
  for (long a = 0; a < ncell; a++) rho[a] = 0.0;
  for (int s = 0; s < nsp; s++)
    for (long p = 0; p < sp[s].n; p++) {
      long ix[2], iy[2];
      double wx[2], wy[2];
      orc_shape_weights(1, sp[s].x[p] / hx, nx, ix, wx);
      orc_shape_weights(1, sp[s].y[p] / hy, ny, iy, wy);
      for (int b = 0; b < 2; b++)
        for (int a = 0; a < 2; a++)
          rho[iy[b] * nx + ix[a]] += sp[s].q * wt2d(&sp[s], p) * wx[a] * wy[b] / area;
    }
  const double *Ex = E, *Ey = E + ncell;
  for (long j = 0; j < ny; j++)
    for (long i = 0; i < nx; i++) {
      long im = imod(i - 1, nx), jm = imod(j - 1, ny);
      double div = (Ex[j * nx + i] - Ex[j * nx + im]) / hx + (Ey[j * nx + i] - Ey[jm * nx + i]) / hy;
      r[j * nx + i] = div - rho[j * nx + i];
    }
}

/* ------------------------------------------------------------------------ */
/* 1D2V electromagnetic schemes with a pseudospectral field solve:          */
/* EMEC(LI), Eq. (EMbasic), and EMEC(PSATD), Eq. (EM_PSATD)                 */
/* ------------------------------------------------------------------------ */

/*
 * Geometry of the paper's Weibel test (Sec. 5): one periodic coordinate y of
 * length L with n collocated nodes y_j = j h; velocities (vx, vy); fields
 * E = (Ex, Ey, 0) and B = (0, 0, Bz).  With only d/dy non-zero the curls are
 *   (curl B)_x = dBz/dy,  (curl B)_y = 0,  (curl E)_z = -dEx/dy,
 * so Maxwell's equations of Eq. (EMbasic) read
 *   dEx/dt = c^2 dBz/dy - jx,   dEy/dt = -jy,   dBz/dt = dEx/dy.
 * d/dy is pseudospectral (Sec. 2.2.3): mode m of the discrete Fourier
 * transform is multiplied by i kk with kk = 2 pi m / L for the signed mode
 * number m in (-n/2, n/2); the Nyquist mode of an even n (which has no real
 * i kk) gets kk = 0.  The matrix of d/dy is then real and antisymmetric, which
 * is the discrete curl identity Eq. (curlIdentity) the energy proofs use.
 * Everything below is a direct O(n^2) discrete Fourier transform.
 */

typedef struct {
  long n;        /* nodes */
  double L;      /* periodic length */
  int order;     /* 1 | 2 */
  double dt;
  double c;      /* speed of light */
  int solver;    /* 1 = CN (Eq. EMbasic), 2 = PSATD (Eq. EM_PSATD) */
  int scheme;    /* 2 = the E*, B* half step with j^{n,*}; 1 = E* = E^n, B* = B^n */
  int gamma_on;
} orc_em1d_cfg;

typedef struct {
  double q, m;
  long n;
  double *y;          /* [n] */
  double *vx, *vy;    /* [n] */
  const double *w;    /* [n] or NULL */
  double w0;
} orc_species1d2v;

/* Signed wavenumber of DFT mode k (0 for the Nyquist mode of an even n). */
static double em1d_kk(long k, long n, double L) {
  long m = k <= n / 2 ? k : k - n;
  if (2 * k == n) m = 0;
  return 2.0 * M_PI * (double)m / L;
}

static void em1d_dft(long n, const double *f, double complex *F) {
  for (long k = 0; k < n; k++) {
    double complex s = 0.0;
    for (long j = 0; j < n; j++) {
      double ang = -2.0 * M_PI * (double)((j * k) % n) / (double)n;
      s += f[j] * (cos(ang) + I * sin(ang));
    }
    F[k] = s;
  }
}

/* Inverse DFT of a Hermitian spectrum; returns the real part. */
static void em1d_idft(long n, const double complex *F, double *f) {
  for (long j = 0; j < n; j++) {
    double complex s = 0.0;
    for (long k = 0; k < n; k++) {
      double ang = 2.0 * M_PI * (double)((j * k) % n) / (double)n;
      s += F[k] * (cos(ang) + I * sin(ang));
    }
    f[j] = creal(s) / (double)n;
  }
}

/* Pseudospectral d/dy of f (pinned against the analytic derivative of band-
 * limited fields and by antisymmetry, test_oracle_em1d.py). */
void orc_spectral_deriv(long n, double L, const double *f, double *df) {
  double complex *F = (double complex *)calloc((size_t)n, sizeof(double complex));
  em1d_dft(n, f, F);
  for (long k = 0; k < n; k++) F[k] *= I * em1d_kk(k, n, L);
  em1d_idft(n, F, df);
  free(F);
}

/*
 * Field advance over tau with the current j held fixed (E = [2][n] as Ex, Ey;
 * B = [n] as Bz; j = [2][n]).  kind:
 *   0 explicit Euler (the E*, B* half step of Eq. EMbasic):
 *       E' = E + tau (c^2 curl B - j),  B' = B - tau curl E;
 *   1 Crank-Nicolson (the full step of Eq. EMbasic):
 *       E' = E + tau (c^2 curl (B + B')/2 - j),  B' = B - tau curl (E + E')/2,
 *     solved exactly mode by mode (a 2 x 2 linear system for Ex, Bz);
 *   2 PSATD (Eq. PSATDformula with Delta t -> tau): the exact solution of
 *     the ODE system Eq. (PSATDconstruction).  Eavg (may be NULL) receives
 *     the time average of E over [0, tau] (the closed form given after Eq.
 *     EM_PSATD).
 * For kind 0 and 1 Eavg, if given, receives (E + E')/2.
 * Pinned: vacuum standing waves against cos(kc t) (PSATD) and the CN phase
 * 2 atan(kc tau/2) per step; a fine Runge-Kutta integration of the ODE with
 * its quadrature of E (PSATD, Eavg); the residual of the CN relations.
 */
void orc_em1d_field_advance(const orc_em1d_cfg *g, int kind, double tau,
                            const double *E, const double *B, const double *j,
                            double *Eout, double *Bout, double *Eavg) {
  long n = g->n;
  double c = g->c, c2 = c * c;
  double complex *Fx = (double complex *)calloc((size_t)n, sizeof(double complex));
  double complex *Fy = (double complex *)calloc((size_t)n, sizeof(double complex));
  double complex *Fb = (double complex *)calloc((size_t)n, sizeof(double complex));
  double complex *Jx = (double complex *)calloc((size_t)n, sizeof(double complex));
  double complex *Jy = (double complex *)calloc((size_t)n, sizeof(double complex));
  double complex *Ox = (double complex *)calloc((size_t)n, sizeof(double complex));
  double complex *Oy = (double complex *)calloc((size_t)n, sizeof(double complex));
  double complex *Ob = (double complex *)calloc((size_t)n, sizeof(double complex));
  double complex *Ax = (double complex *)calloc((size_t)n, sizeof(double complex));
  double complex *Ay = (double complex *)calloc((size_t)n, sizeof(double complex));
  em1d_dft(n, E, Fx);
  em1d_dft(n, E + n, Fy);
  em1d_dft(n, B, Fb);
  em1d_dft(n, j, Jx);
  em1d_dft(n, j + n, Jy);
  for (long k = 0; k < n; k++) {
    double kk = em1d_kk(k, n, g->L);
    if (kind == 0) {
      Ox[k] = Fx[k] + tau * (c2 * I * kk * Fb[k] - Jx[k]);
      Ob[k] = Fb[k] + tau * I * kk * Fx[k];
    } else if (kind == 1) {
      double complex a = I * kk * tau / 2.0;
      double complex r1 = Fx[k] + c2 * a * Fb[k] - tau * Jx[k];
      double complex r2 = Fb[k] + a * Fx[k];
      double complex det = 1.0 - c2 * a * a;
      Ox[k] = (r1 + c2 * a * r2) / det;
      Ob[k] = (r2 + a * r1) / det;
    } else {
      double kabs = fabs(kk), s = kk > 0.0 ? 1.0 : -1.0;
      if (kabs == 0.0) {
        Ox[k] = Fx[k] - tau * Jx[k];
        Ob[k] = Fb[k];
        Ax[k] = Fx[k] - 0.5 * tau * Jx[k];
      } else {
        double C = cos(kabs * c * tau), S = sin(kabs * c * tau);
        Ox[k] = C * Fx[k] + I * s * S * c * Fb[k] - S / (kabs * c) * Jx[k];
        Ob[k] = C * Fb[k] + I * s * (S / c) * Fx[k] - I * s * (1.0 - C) / (kabs * c2) * Jx[k];
        Ax[k] = S / (kabs * c * tau) * Fx[k] + I * s * (1.0 - C) / (kabs * tau) * Fb[k] -
                (1.0 - C) / (kabs * kabs * c2 * tau) * Jx[k];
      }
      Ay[k] = Fy[k] - 0.5 * tau * Jy[k];
    }
    /* the longitudinal component has no curl term in every kind */
    Oy[k] = Fy[k] - tau * Jy[k];
  }
  em1d_idft(n, Ox, Eout);
  em1d_idft(n, Oy, Eout + n);
  em1d_idft(n, Ob, Bout);
  if (Eavg) {
    if (kind == 2) {
      em1d_idft(n, Ax, Eavg);
      em1d_idft(n, Ay, Eavg + n);
    } else {
      for (long a = 0; a < 2 * n; a++) Eavg[a] = 0.5 * (E[a] + Eout[a]);
    }
  }
  free(Fx); free(Fy); free(Fb); free(Jx); free(Jy);
  free(Ox); free(Oy); free(Ob); free(Ax); free(Ay);
}

static double wt1d2v(const orc_species1d2v *s, long p) {
  return s->w ? s->w[p] : s->w0;
}

/* jx, jy += (1/h) q w (ux, uy) S(y_h - y_p) at the positions py. */
static void deposit_1d2v(const orc_em1d_cfg *g, const orc_species1d2v *s,
                         const double *py, const double *ux, const double *uy,
                         double *J) {
  double h = g->L / (double)g->n;
  for (long p = 0; p < s->n; p++) {
    long idx[3];
    double wt[3];
    int k = orc_shape_weights(g->order, py[p] / h, g->n, idx, wt);
    double qw = s->q * wt1d2v(s, p) / h;
    for (int a = 0; a < k; a++) {
      J[idx[a]] += qw * ux[p] * wt[a];
      J[g->n + idx[a]] += qw * uy[p] * wt[a];
    }
  }
}

static double gather_at(const orc_em1d_cfg *g, const double *F, double y) {
  double h = g->L / (double)g->n;
  long idx[3];
  double wt[3];
  int k = orc_shape_weights(g->order, y / h, g->n, idx, wt);
  double s = 0.0;
  for (int a = 0; a < k; a++) s += F[idx[a]] * wt[a];
  return s;
}

/*
 * One step of Eq. (EMbasic) (solver 1) or Eq. (EM_PSATD) (solver 2) for the
 * 1D2V geometry above, E = [2][n] and B = [n] updated in place:
 *   y*          = y^n + dt/2 vy^n
 *   j^{n,*}     = (1/h) sum q w v^n S(y_h - y*)                 (scheme 2)
 *   (E*, B*)    = explicit half step (CN) or PSATD over dt/2 with j^{n,*}
 *                 (scheme 1: E* = E^n, B* = B^n)
 *   v*          = v^n + dt/2 (q/m)(E**_p + v* x B**_p), E**, B** gathered at y*
 *               = (u + u x t)/(1 + t^2) with u = v^n + (q/m)(dt/2) E**_p and
 *                 t = (q/m)(dt/2) B**_p (u . t = 0 in this geometry)
 *   y^{n+1}     = y^n + dt vy*,  y^{n+1/2} = y^n + dt/2 vy*
 *   j^{*,n+1/2} = (1/h) sum q w v* S(y_h - y^{n+1/2})
 *   (E^{n+1}, B^{n+1}) = CN or PSATD over dt with j^{*,n+1/2}
 *   Ebar        = (E^n + E^{n+1})/2 (CN) or the time average <E> (PSATD)
 *   B^{n+1/2}   = (B^n + B^{n+1})/2
 *   v^dag       = v^n + dt (q/m)(Ebar_p + v* x B^{n+1/2}_p) at y^{n+1/2}
 *   v^{n+1}     = Gamma v^dag (Eq. opt_solution; fallback Gamma := 1, counted)
 */
int orc_em1d_step(const orc_em1d_cfg *g, orc_species1d2v *sp, int nsp,
                  double *E, double *B, long *nfallback) {
  if (nsp <= 0 || g->n <= 0 || (g->solver != 1 && g->solver != 2)) return -1;
  long n = g->n;
  double dt = g->dt;
  int full = g->solver == 1 ? 1 : 2;
  double *J = (double *)calloc((size_t)(2 * n), sizeof(double));
  double *Es = (double *)calloc((size_t)(2 * n), sizeof(double));
  double *Bs = (double *)calloc((size_t)n, sizeof(double));
  double *En = (double *)calloc((size_t)(2 * n), sizeof(double));
  double *Bn = (double *)calloc((size_t)n, sizeof(double));
  double *Eb = (double *)calloc((size_t)(2 * n), sizeof(double));
  double *Bh = (double *)calloc((size_t)n, sizeof(double));

  /* j^{n,*} and the half step */
  if (g->scheme == 2) {
    for (int s = 0; s < nsp; s++) {
      orc_species1d2v *S = &sp[s];
      double *ys = (double *)calloc((size_t)S->n + 1, sizeof(double));
      for (long p = 0; p < S->n; p++) ys[p] = wrap(S->y[p] + 0.5 * dt * S->vy[p], g->L);
      deposit_1d2v(g, S, ys, S->vx, S->vy, J);
      free(ys);
    }
    orc_em1d_field_advance(g, full == 1 ? 0 : 2, 0.5 * dt, E, B, J, Es, Bs, NULL);
  } else {
    memcpy(Es, E, sizeof(double) * 2 * n);
    memcpy(Bs, B, sizeof(double) * n);
  }

  /* v*, y^{n+1/2}; deposit j^{*,n+1/2} */
  double **vsx = (double **)calloc((size_t)nsp, sizeof(double *));
  double **vsy = (double **)calloc((size_t)nsp, sizeof(double *));
  double **yh = (double **)calloc((size_t)nsp, sizeof(double *));
  for (long a = 0; a < 2 * n; a++) J[a] = 0.0;
  for (int s = 0; s < nsp; s++) {
    orc_species1d2v *S = &sp[s];
    double qm = S->q / S->m;
    vsx[s] = (double *)calloc((size_t)S->n + 1, sizeof(double));
    vsy[s] = (double *)calloc((size_t)S->n + 1, sizeof(double));
    yh[s] = (double *)calloc((size_t)S->n + 1, sizeof(double));
    for (long p = 0; p < S->n; p++) {
      double ys = wrap(S->y[p] + 0.5 * dt * S->vy[p], g->L);
      double ux = S->vx[p] + qm * 0.5 * dt * gather_at(g, Es, ys);
      double uy = S->vy[p] + qm * 0.5 * dt * gather_at(g, Es + n, ys);
      double t = qm * 0.5 * dt * gather_at(g, Bs, ys);
      vsx[s][p] = (ux + uy * t) / (1.0 + t * t);
      vsy[s][p] = (uy - ux * t) / (1.0 + t * t);
      yh[s][p] = wrap(S->y[p] + 0.5 * dt * vsy[s][p], g->L);
    }
    deposit_1d2v(g, S, yh[s], vsx[s], vsy[s], J);
  }

  /* the full field step */
  orc_em1d_field_advance(g, full, dt, E, B, J, En, Bn, Eb);
  for (long a = 0; a < n; a++) Bh[a] = 0.5 * (B[a] + Bn[a]);

  /* v^dag, Gamma, y^{n+1}, v^{n+1} */
  for (int s = 0; s < nsp; s++) {
    orc_species1d2v *S = &sp[s];
    double qm = S->q / S->m;
    long count = 0;
    for (long p = 0; p < S->n; p++) {
      double y = yh[s][p];
      double ex = gather_at(g, Eb, y), ey = gather_at(g, Eb + n, y);
      double bz = gather_at(g, Bh, y);
      double vx = S->vx[p], vy = S->vy[p], wx = vsx[s][p], wy = vsy[s][p];
      double dx = vx + dt * qm * (ex + wy * bz);
      double dy = vy + dt * qm * (ey - wx * bz);
      double R = vx * vx + vy * vy + 2.0 * (wx * (dx - vx) + wy * (dy - vy));
      double vd2 = dx * dx + dy * dy;
      double gamma = 1.0;
      if (g->gamma_on) {
        if (R < 0.0 || vd2 == 0.0)
          count++;
        else
          gamma = sqrt(R) / sqrt(vd2);
      }
      S->vx[p] = gamma == 1.0 ? dx : dx * gamma;
      S->vy[p] = gamma == 1.0 ? dy : dy * gamma;
      S->y[p] = wrap(S->y[p] + dt * wy, g->L);
    }
    if (nfallback) nfallback[s] = count;
    free(vsx[s]);
    free(vsy[s]);
    free(yh[s]);
  }
  memcpy(E, En, sizeof(double) * 2 * n);
  memcpy(B, Bn, sizeof(double) * n);
  free(vsx); free(vsy); free(yh);
  free(J); free(Es); free(Bs); free(En); free(Bn); free(Eb); free(Bh);
  return 0;
}

/* KE per species, W_E = (h/2) sum (Ex^2 + Ey^2), W_B = (c^2 h/2) sum Bz^2 (the
 * energies of Eq. EM_econs and Eq. PSATDecons). */
void orc_em1d_energy(const orc_em1d_cfg *g, const orc_species1d2v *sp, int nsp,
                     const double *E, const double *B, double *KE, double *WE,
                     double *WB) {
  long n = g->n;
  double h = g->L / (double)n;
  for (int s = 0; s < nsp; s++) {
    double acc = 0.0;
    for (long p = 0; p < sp[s].n; p++)
      acc += wt1d2v(&sp[s], p) * (sp[s].vx[p] * sp[s].vx[p] + sp[s].vy[p] * sp[s].vy[p]);
    KE[s] = 0.5 * sp[s].m * acc;
  }
  double we = 0.0, wb = 0.0;
  for (long a = 0; a < 2 * n; a++) we += E[a] * E[a];
  for (long a = 0; a < n; a++) wb += B[a] * B[a];
  *WE = 0.5 * h * we;
  *WB = 0.5 * g->c * g->c * h * wb;
}
