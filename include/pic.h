/*
 * pic.h -- C ABI of the GB300 library for the explicit, energy-conserving
 * particle-in-cell scheme of Ricketson & Hu ("An explicit, energy-conserving
 * particle-in-cell scheme").
 *
 * What one call of pic_step() computes, per time step (Sec. 3.3, Eq.
 * good_translation; Sec. 4.1, Eq. EMleapfrog):
 *   x*          = x^n + dt/2 v^n
 *   j^{n,*}     = deposit of v^n at x*            (ESEC2 only, Eq. doublestardef)
 *   E*          = E^n - dt/2 j^{n,*}              (ES; EM adds c^2 curl B^{n+1/2})
 *   v*          = v^n + dt/2 (q/m)(E**_p + v* x B)  (E** gathered at x*)
 *   x^{n+1}     = x^n + dt v*,  x^{n+1/2} = x^n + dt/2 v*
 *   j^{*,n+1/2} = deposit of v* at x^{n+1/2}
 *   E^{n+1}     = E^n - dt j^{*,n+1/2}            (Eq. ampere; EM: Eq. EMleapfrog)
 *   v^dag       = v^n + dt (q/m)(E^{n+1/2}_p + v* x B)  (Eq. PICmodification)
 *   v^{n+1}     = Gamma v^dag, Gamma = sqrt(|v^n|^2 + 2 v*.(v^dag - v^n)) / |v^dag|
 *                 (Eq. opt_solution); where the radicand is negative (or
 *                 v^dag = 0) Gamma := 1 and the particle is counted (Sec. 3.2,
 *                 Sec. 5.1).
 * The shape function S is the same B-spline for gather and deposit (Sec. 2.2),
 * of order 1 (the paper's tent) or 2 (quadratic B-spline, an extension).
 *
 * Conventions
 *   - Every function returns an int status: PIC_OK (0) or a negative PIC_ERR_*
 *     code; nothing aborts, throws or exits across this boundary.  After a
 *     nonzero status pic_last_error() describes it (thread-local string).
 *   - Units are the dimensionless ones of Sec. 2.1.  Species have charge q and
 *     mass m: acceleration (q/m)(E + v x B), current (1/|h|) sum q w v S,
 *     kinetic energy (1/2) m sum w |v|^2.  A fixed neutralising background is
 *     implied (it only enters the initial Poisson solve).
 *   - Grid: 1D periodic, nodes x_i = i h, h = L / n[0], E and J collocated on
 *     the nodes (solver PIC_SOLVER_AMPERE_ES, dim_x = dim_v = 1); or 2D periodic
 *     Yee lattice n[0] x n[1] (solver PIC_SOLVER_YEE_LEAPFROG, dim_x = 2,
 *     dim_v = 3) with components Ex (i+1/2, j), Ey (i, j+1/2), Ez (i, j),
 *     Bx (i, j+1/2), By (i+1/2, j), Bz (i+1/2, j+1/2); grid arrays are
 *     component-major [3][n[1]][n[0]]; or 1D periodic with a pseudospectral
 *     field solve (solvers PIC_SOLVER_CN_SPECTRAL / PIC_SOLVER_PSATD,
 *     dim_x = 1, dim_v = 2): the coordinate is y, velocities (vx, vy), fields
 *     E = [2][n] (Ex, Ey) and B = [n] (Bz) on the nodes y_j = j h, n a power
 *     of two in [4, 1024].  d/dy multiplies Fourier mode m by 2 pi i m / L,
 *     and by 0 for the Nyquist mode (Sec. 2.2.3).
 *   - Particle arrays are SoA: x is [dim_x][n], v is [dim_v][n], w is [n].
 *   - Ownership: the library copies everything it is given at pic_init /
 *     pic_set_* and owns all device memory it allocates until pic_free.  Output
 *     pointers are written, never retained.
 *   - Pointers are host pointers unless the config sets ptr_on_device = 1, in
 *     which case every array argument of every call on that handle is a device
 *     pointer on the current device.
 *   - All GPU work is issued on cfg.cuda_stream (a cudaStream_t, or NULL for
 *     the legacy default stream); calls return after that work completes.
 *   - A handle is not thread-safe: one thread at a time per handle.
 */
#ifndef PIC_H
#define PIC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  PIC_OK = 0,
  PIC_ERR_ARG = -1,        /* invalid argument (sizes, enum values, NULL)   */
  PIC_ERR_CUDA = -2,       /* a CUDA runtime call failed                    */
  PIC_ERR_OOM = -3,        /* device allocation failed                      */
  PIC_ERR_NONFINITE = -4,  /* a non-finite value reached the state          */
  PIC_ERR_TIMEOUT = -5,    /* reserved: no kernel waits on another, so this */
                           /* version never returns it                      */
  PIC_ERR_BOUNDS = -6,     /* an input position lies outside [0, L); in the */
                           /* debug-bounds build also a failed index check  */
  PIC_ERR_UNSUPPORTED = -7 /* a valid combination this build does not run   */
};

/* PIC_SOLVER_CN_SPECTRAL: EMEC(LI), the linearly implicit (Crank-Nicolson)
 * Maxwell step of Eq. (EMbasic); PIC_SOLVER_PSATD: EMEC(PSATD), Eq. (EM_PSATD),
 * the analytic Fourier-space step of Eq. (PSATDformula) with the time-averaged
 * E in v^dag.  Both run the 1D2V geometry of the paper's Weibel test (see
 * Conventions) with a pseudospectral d/dy. */
/* PIC_SOLVER_STANDARD_LEAPFROG: not the paper's method but the scheme it is
 * measured against (Sec. 5): Vlasov-Poisson PIC with the leapfrog push and
 * binomial_passes passes of the 1-2-1 filter on the charge, 1D1V, FP64.  Its
 * state is x^n, v^{n-1/2} and E^n (the spectral Gauss's-law field of the
 * filtered charge of x^n): pic_get_particles returns v^{n-1/2};
 * pic_init and pic_set_particles take v^0 (v^n) and start the leapfrog with
 * v^{-1/2} = v^0 - dt/2 (q/m) E^0_p; E0, B0 must be NULL and pic_set_fields is
 * PIC_ERR_UNSUPPORTED (E follows from the charge).  Its energy at step n is
 * (1/2) m sum w (v^{n-1/2}^2 + v^{n+1/2}^2) / 2 + (h/2) sum (E^n)^2, and it is
 * not conserved: that is the comparison.  The scheme, gamma_on and
 * remove_mean fields do not apply; its fallback counts are 0. */
typedef enum {
  PIC_SOLVER_AMPERE_ES = 0,
  PIC_SOLVER_YEE_LEAPFROG = 1,
  PIC_SOLVER_CN_SPECTRAL = 2,
  PIC_SOLVER_PSATD = 3,
  PIC_SOLVER_STANDARD_LEAPFROG = 4
} pic_solver;
/* ESEC1: Eq. (naivetranslation) with the correction of Eq. (PICmodification);
 * ESEC2: Eq. (good_translation), one extra deposit per step, Gamma closer to 1. */
typedef enum { PIC_SCHEME_ESEC1 = 1, PIC_SCHEME_ESEC2 = 2 } pic_scheme;
/* FP64: positions and velocities in double, all arithmetic in double.
 * MIXED: positions as 32-bit fixed point (cell and fraction in one word),
 * velocities as unevaluated float pairs (48-bit significand), shape weights in
 * FP32, current accumulated exactly in 64-bit integers, Gamma from an exact
 * difference; energy reductions in double.  Conserves energy to the same
 * bound (the pairing of Eq. exp_econs_simple is exact by construction).
 * Runs the Ampere solver (1D1V), the Yee solver (2D3V, square domain
 * L[0] == L[1]) and the spectral solvers (1D2V); in the electromagnetic
 * solvers the fields and their update stay FP64 and the magnetic force
 * V* x B is formed in float pairs from the integer v*, so it does no work.
 * One species with a uniform weight, else PIC_ERR_UNSUPPORTED. */
typedef enum { PIC_PREC_FP64 = 0, PIC_PREC_MIXED = 1 } pic_precision;

typedef struct {
  int dim_x;      /* 1 (with dim_v = 1) or 2 (with dim_v = 3)            */
  int dim_v;
  int64_t n[2];   /* nodes per dimension (n[1] ignored when dim_x = 1)  */
  double L[2];    /* periodic lengths                                   */
} pic_grid;

typedef struct {
  double q, m;        /* charge and mass (electrons: -1, 1)                  */
  int64_t n;          /* markers                                             */
  const double *x;    /* [dim_x][n], each coordinate in [0, L)               */
  const double *v;    /* [dim_v][n]                                          */
  const double *w;    /* [n] weights, or NULL for the uniform weight w0      */
  double w0;
} pic_species;

typedef struct {
  pic_grid grid;
  int shape_order;          /* 1 | 2                                          */
  double dt;
  double c;                 /* speed of light (Yee solver only)               */
  pic_solver solver;
  pic_scheme scheme;
  pic_precision precision;
  int sort_period;          /* mixed form: 0 = markers never reordered;       */
                            /* Ampere solver: 1 = kept sorted by (cell, sign  */
                            /* of v) every step, written in key order by the  */
                            /* update pass; P > 1 = counting sort by cell     */
                            /* every P steps.  Yee solver: P >= 1 = the       */
                            /* update pass of every P-th step writes them in  */
                            /* quarter-cell order, and each thread's run of   */
                            /* consecutive markers in one quarter cell sums   */
                            /* its deposits in registers, the runs over the   */
                            /* warp, before the atomics.  Sorting only        */
                            /* reorders markers (pic_get_ids maps them).      */
  int remove_mean;          /* ES: 1 -> E -= dt (J - <J>), 0 -> E -= dt J     */
  int gamma_on;             /* 1 = energy correction; 0 = naive scheme        */
  int ptr_on_device;        /* see Conventions                                */
  void *cuda_stream;        /* cudaStream_t or NULL                           */
  int skip_ids;             /* 1: do not carry marker ids through sorts       */
                            /* (pic_get_ids then fails); 0: keep them         */
  int binomial_passes;      /* 1-2-1 filter passes, 0..8.  Standard solver: on */
                            /* the charge.  Ampere solver, both forms: inside */
                            /* the scheme, energy-consistently (Ampere uses   */
                            /* F j, the gathers F E; F is symmetric, so the   */
                            /* energy identity stays exact), and the initial  */
                            /* Gauss field is that of F rho (ESEC1 then runs  */
                            /* two launches per step).  Other solvers,        */
                            /* batches and the no-alloc entry point: must be  */
                            /* 0.                                             */
  int charge_conserving;    /* Yee solver, FP64, shape_order 1: 1 = exact     */
                            /* charge conservation (Sec. 3.5, Eq. detbal).    */
                            /* With the bilinear charge shape rho, each J/E   */
                            /* component takes the tent on its integer-node   */
                            /* axes and the degree-0 box on its half-node     */
                            /* axes, and the deposit of j^{*,n+1/2} and the   */
                            /* gather of E^{n+1/2} run over the pieces of the */
                            /* path x^n -> x^{n+1} between grid lines; then   */
                            /* div_h E - rho keeps its initial value and the  */
                            /* energy identity is unchanged.  0 = the point   */
                            /* shapes of shape_order.  Other solvers or forms */
                            /* with 1: PIC_ERR_UNSUPPORTED.                   */
  int gamma_fp64;           /* mixed 1D1V form, sort_period 0: 1 = the        */
                            /* correction (t, the R < 0 test and Gamma) in    */
                            /* FP64 for every marker; 0 = FP64 only where     */
                            /* |Gamma - 1| >= 2^-9 or R may be negative, an   */
                            /* FP32 series elsewhere.  The FP64 form computes */
                            /* everything in FP64 (the flag changes nothing); */
                            /* other mixed forms with 1: PIC_ERR_UNSUPPORTED. */
  int separate_passes;      /* mixed 1D1V form, ESEC1, sort_period 0: 0 = one */
                            /* launch per step, the update of step n fused    */
                            /* with the push and deposit of step n+1 (ESEC1  */
                            /* needs no j^{n,*}, so nothing global lies       */
                            /* between them); 1 = two launches per step, as   */
                            /* ESEC2 runs.  Both give the same results bit    */
                            /* for bit.  Other forms: ignored.                */
} pic_config;

typedef struct pic_handle pic_handle;

/*
 * Creates a simulation.  species: nspecies entries (1..8).  E0: initial field,
 * [nodes] (ES), [3][ny][nx] (Yee) or [2][n] (spectral), or NULL: ES solves
 * Gauss's law in the Poisson form (Eq. poisson, dE/dx = rho - <rho>)
 * spectrally from the deposited charge, the electromagnetic solvers start
 * from E = 0.  B0: B^{-1/2} [3][ny][nx] (Yee) or Bz^0 [n] (spectral), or NULL
 * for zero; not allowed for the ES solver.  Positions outside [0, L) -> PIC_ERR_BOUNDS;
 * non-finite input -> PIC_ERR_NONFINITE.  On success *out owns the state.
 */
int pic_init(const pic_config *cfg, const pic_species *species, int nspecies,
             const double *E0, const double *B0, pic_handle **out);

/*
 * Advances nsteps steps (see the header comment).  Optional outputs (host
 * arrays, or device arrays when ptr_on_device), each of length nsteps or
 * NULL: nfallback_per_step[k] = number of particles (all species) whose Gamma
 * fell back to 1 in step k; te_per_step[k] = total energy after step k
 * (KE + W_E + W_B, reduced in double on the device every step).
 * A non-finite total energy stops the call with PIC_ERR_NONFINITE.
 */
int pic_step(pic_handle *h, int nsteps, int64_t *nfallback_per_step, double *te_per_step);

/*
 * Asynchronous form of pic_step: enqueues nsteps steps on the handle's stream
 * and returns without waiting.  The per-step fallback counts and total
 * energies stay on the device (at most 1024 pending steps) until
 * pic_read_stats, which waits for the work, copies them out (arrays of
 * capacity >= pending steps, or NULL), sets *nread to the number of steps
 * read, clears them and reports device-side error flags.  pic_step discards
 * any stats still pending from earlier asynchronous calls.
 */
int pic_step_async(pic_handle *h, int nsteps);
int pic_read_stats(pic_handle *h, int capacity, int64_t *nfallback_per_step, double *te_per_step,
                   int *nread);

/* Number of CUDA kernels this handle has launched so far (all entry points). */
int pic_launch_count(pic_handle *h, int64_t *launches);

/*
 * Per-kernel timing for measurement.  pic_set_profiling(h, 1) clears the
 * totals and brackets every later launch of h with CUDA events on its stream
 * (a few microseconds of overhead per launch); 0 stops.  pic_profile returns
 * the number of launches and their summed device time (ms) of one kind:
 * 0 = pass C (gather at x*, push to v*, deposit of j^{*,n+1/2}),
 * 1 = pass E (gather at x^{n+1/2}, Gamma, state update, next j^{n,*}),
 * 2 = per-step energy/fallback finalisation, 3 = cell sort,
 * 4 = grid field updates (Yee solver), 5 = the fused ESEC1 pass (pass E of a
 * step with pass C of the next, see separate_passes).
 */
int pic_set_profiling(pic_handle *h, int on);
int pic_profile(pic_handle *h, int kind, int64_t *launches, double *total_ms);

/*
 * Energies of the current state (Sec. 5.1; W_B of Sec. 4.1):
 * KE_per_species [nspecies], W_E = (1/2)|h| sum |E|^2,
 * W_B = (c^2/2)|h| sum B^{n+1/2} . B^{n-1/2} (Yee), (c^2/2) h sum Bz^2
 * (spectral solvers, Eq. EM_econs), 0 for the ES solver; TE = sum.
 * Any output may be NULL.  Always host pointers.
 */
int pic_energy(pic_handle *h, double *KE_per_species, double *W_E, double *W_B, double *TE);

/*
 * Charge diagnostics of the current state (Sec. 2.1: Gauss's law, kept in time
 * by continuity when the deposit conserves charge, Sec. 3.5), reduced in FP64
 * on the device:
 *   Q_markers = sum_p q w_p over all species; Q_grid = |h| sum rho_h, with rho
 *   the charge density deposited on the nodes (equal to Q_markers up to
 *   rounding: the shapes are a partition of unity);
 *   the residual r of Gauss's law with the neutralising background:
 *   - Ampere solver (1D): rho with the scheme's own shape (the mixed form's
 *     quantised weights), r = D E^n - (rho - <rho>) with the spectral
 *     derivative D of the initial Poisson solve, on the Fourier modes
 *     1 .. (nodes - 1) / 2 (k = 0 is the background; D does not represent the
 *     Nyquist mode); zero to rounding right after pic_init with E0 = NULL;
 *   - Yee solver (2D): rho with the bilinear shape on the nodes (i, j),
 *     r = div_h E^n - (rho - <rho>) with the Yee divergence
 *     (Ex(i+1/2,j) - Ex(i-1/2,j)) / hx + (Ey(i,j+1/2) - Ey(i,j-1/2)) / hy; with
 *     charge_conserving = 1, r keeps its initial value (Eq. detbal);
 *   gauss_l2 = sqrt(|h| sum r^2); rho_l2 = sqrt(|h| sum (rho - <rho>)^2) over
 *   the same modes (1D) or nodes (2D), its scale.
 * residual: [nodes] (1D) or [ny][nx] (2D), host or device as the handle's
 * pointers, or NULL.  Any output may be NULL.  The spectral solvers and the
 * standard comparator: PIC_ERR_UNSUPPORTED.  The first call allocates the
 * diagnostic's device buffers.
 */
int pic_charge(pic_handle *h, double *Q_markers, double *Q_grid, double *gauss_l2, double *rho_l2,
               double *residual);

/*
 * Resolution of a mixed-form handle (precision PIC_PREC_MIXED, any solver;
 * else PIC_ERR_UNSUPPORTED): *dx = L / 2^32, the step of the fixed-point
 * positions; *dv = the velocity of one unit of the integer v* (the float-pair
 * velocities resolve about 2^-48 of their value in the same units); and
 * *deposit_bits = T: every marker's deposit adds an integer below 2^T, the
 * product of its v* and shape weights rounded to 2^-T of its largest value,
 * so T bounds the relative rounding of each deposited term (the current, and
 * through it the field work of Eq. exp_econs_simple).  Any output may be NULL.
 */
int pic_mixed_resolution(pic_handle *h, double *dx, double *dv, int *deposit_bits);

/* Copies species s out as FP64 SoA ([dim_x][n] positions, [dim_v][n]
 * velocities).  Marker order is the library's current (possibly sorted)
 * order; pic_get_ids returns, for each slot, the marker's index at init.
 * Both return after the data is in place. */
int pic_get_particles(pic_handle *h, int s, double *x, double *v);
int pic_get_ids(pic_handle *h, int s, int64_t *ids);
/* Replaces species s (same n; resets its ids to 0..n-1); returns after the
 * buffers have been read.  The mixed 1D1V form converts buffers that the
 * device can address (device memory, pinned host memory) in one kernel
 * reading them in place, and stages others (pageable host memory) through
 * cudaMemcpy; pic_get_particles writes the same way. */
int pic_set_particles(pic_handle *h, int s, const double *x, const double *v);
/* Fields: E^n and (Yee) B^{n-1/2}; B may be NULL for the ES solver and is
 * required by pic_set_fields for the Yee solver (B^{n+1/2} is then rebuilt as
 * B^{n-1/2} - dt curl E^n). */
int pic_get_fields(pic_handle *h, double *E, double *B);
int pic_set_fields(pic_handle *h, const double *E, const double *B);

/*
 * One-species 1D1V step in the FP64 form on caller-owned device buffers that
 * allocates no device memory (the paper has no counterpart: this is a
 * deployment entry point).  For callers that may not allocate: a framework
 * that owns the whole device heap through its own pool and forbids plugins to
 * call cudaMalloc/cudaFree, or a service whose memory is fixed at start-up.
 * x, v [n] and E [nodes] are device pointers, updated in place over nsteps
 * steps of cfg's scheme (solver PIC_SOLVER_AMPERE_ES, precision
 * PIC_PREC_FP64; uniform weight w0; E is E^n on entry, no Poisson solve).
 * Optional outputs (host or device, length nsteps): per-step fallback counts
 * and total energies, as pic_step.  Limits: at most 8192 nodes and 1024 steps
 * per call, else PIC_ERR_ARG.  Its scratch is one static device array of
 * 352,576 bytes that every GPU which loads the library holds until exit; all
 * calls on a device share it, so calls that overlap on the GPU race and must
 * be serialised.  Every call looks up the array's address on the current
 * device (cudaGetSymbolAddress); no address is kept between calls.  The inputs
 * are checked before the first step: a position outside [0, L) returns
 * PIC_ERR_BOUNDS and a non-finite velocity or field value PIC_ERR_NONFINITE,
 * with x, v and E left as passed.  The call returns after its work on
 * cfg->cuda_stream has completed.
 */
int pic_es1d_step_noalloc(const pic_config *cfg, double q, double m, double w0, int64_t n,
                          double *x, double *v, double *E, int nsteps,
                          int64_t *nfallback_per_step, double *te_per_step);

/* ------------------------------------------------------------ gradients
 * Reverse mode of the FP64 1D form (solver PIC_SOLVER_AMPERE_ES, precision
 * PIC_PREC_FP64, either scheme and shape order): derivatives of an objective
 * of the state after nsteps steps with respect to the state before them.  The
 * paper conserves energy exactly but does not differentiate the scheme; the
 * reverse pass takes the adjoint of every operation of Sec. 3.3 in reverse
 * order (gather and deposit swap roles; Gamma of Sec. 3.2 is differentiated
 * through R, and a fallback through v^dag).
 *
 * pic_grad_forward steps h forward nsteps steps (as pic_step_async; pending
 * stats must have been read) and keeps the markers and field every
 * checkpoint_every steps on the device ((nsteps / checkpoint_every + 1) x
 * (2 N + nodes) doubles).
 *
 * pic_grad_backward takes the adjoints of the state after those steps -
 * Ebar [nodes], xbar [N], vbar [N] (host or device, NULL = zero) - and writes
 * the adjoints of the state before them: Ebar0 [nodes], xbar0, vbar0 and wbar0
 * [N] (the derivative by each marker's weight; for a uniformly weighted
 * species the derivative by its w0 is the sum over its markers), host or
 * device, each may be NULL.  Each segment of checkpoint_every steps is
 * re-run from its checkpoint and reversed; h is left at the state after the
 * forward steps.  The step sequence must not change in between, else
 * PIC_ERR_ARG.
 */
int pic_grad_forward(pic_handle *h, int nsteps, int checkpoint_every);
int pic_grad_backward(pic_handle *h, const double *Ebar, const double *xbar, const double *vbar,
                      double *Ebar0, double *xbar0, double *vbar0, double *wbar0);

/* Number of steps taken since pic_init. */
int pic_step_count(pic_handle *h, int64_t *steps);

/* Releases every resource of h (NULL is a no-op). */
void pic_free(pic_handle *h);

/* Message for the last nonzero status returned on this thread. */
const char *pic_last_error(void);

/* Library version string ("..., debug-bounds)" for the debug-bounds build). */
const char *pic_version(void);

/* The debug-bounds build.  A library compiled with PIC_DEBUG_BOUNDS checks the
 * index arithmetic of the mixed forms where an index is formed (the first
 * node of a marker's shape, the periodic node indices of the 2D shapes, sort
 * keys and sort-on-write slots, the grid nodes a current tile is flushed to):
 * an index outside its range is replaced by 0, so that the access stays in
 * bounds, and recorded; the next call that checks the state's flags
 * (pic_read_stats, pic_step, pic_set_*, pic_batch_read_stats) then returns
 * PIC_ERR_BOUNDS with the check's file and line in pic_last_error().  The
 * records are per process, not per handle.  Results of a run with no failed
 * check are those of the normal build.
 *
 * pic_debug_bounds runs one such check on the device for (index, extent):
 * *flagged = 1 when index lies outside [0, extent) and the check recorded it,
 * 0 when it passed (the record is cleared either way); PIC_ERR_CUDA if the
 * check did not behave so.  In the normal build it returns
 * PIC_ERR_UNSUPPORTED and sets *flagged = -1. */
int pic_debug_bounds(int64_t index, int64_t extent, int *flagged);

/* ---------------------------------------------------------------- batches
 * Many independent 1D runs stepped together (a parameter scan or an ensemble
 * of the scheme of Sec. 3.3 on different problems): each pass of a step is
 * one launch over a work list of (run, block of the run), instead of one
 * launch per run.  The method is unchanged; a batched run gives the same
 * markers, field and fallback counts as the same run stepped alone (its
 * energies agree to round-off: the kinetic sums are blocked differently).
 */
typedef struct pic_batch pic_batch;

/* Creates nruns runs, run r from cfgs[r] and the single species species[r],
 * as pic_init would (E0 from the Poisson solve).  Every run must use
 * PIC_SOLVER_AMPERE_ES, PIC_PREC_MIXED, sort_period 0, at most 512 nodes, the
 * same scheme, the same cuda_stream, gamma_fp64 0 and binomial_passes 0, else
 * PIC_ERR_UNSUPPORTED.  A batch whose runs all have at most 2^15 markers runs
 * blocks of 256 threads, others blocks of 1024.  The batch owns the runs and
 * frees them in pic_batch_free. */
int pic_batch_init(const pic_config *cfgs, const pic_species *species, int nruns,
                   pic_batch **out);

/* Enqueues nsteps steps of every run (asynchronous; at most 1024 steps between
 * pic_batch_read_stats calls, else PIC_ERR_ARG).  With graphs on
 * (pic_batch_set_graph) the launches of a call that starts after stats were
 * read are captured once per (nsteps, step parity) and replayed. */
int pic_batch_step(pic_batch *b, int nsteps);
int pic_batch_set_graph(pic_batch *b, int on);

/* Chooses the blocks per run (about 4, 8 or 16 trips of 4 markers per thread)
 * by timing steps_per_trial steps with each work list (these are real steps
 * of every run: their stats are read with the others), and keeps the fastest.
 * The choice is remembered for this process per (number of runs, total markers
 * rounded to a power of two, largest grid); *trips (may be NULL) receives it. */
int pic_batch_autotune(pic_batch *b, int steps_per_trial, int *trips);

/* Per-step fallback counts and total energies of the steps since the last
 * call, run by run: nfallback[r * capacity + k], te[r * capacity + k] (host
 * arrays, either may be NULL); *nread = steps.  Reports device error flags of
 * any run as pic_read_stats does. */
int pic_batch_read_stats(pic_batch *b, int capacity, int64_t *nfallback, double *te, int *nread);

/* The handle of run r, for its accessors (pic_get_particles, pic_get_fields,
 * pic_energy, pic_step_count, ...).  Do not step it, read its stats or free it
 * directly. */
int pic_batch_run(pic_batch *b, int run, pic_handle **h);

/* Runs, blocks of the work list, and kernels launched so far. */
int pic_batch_info(pic_batch *b, int *nruns, int *nblocks, int64_t *launches);

/* Releases the batch and its runs (NULL is a no-op). */
void pic_batch_free(pic_batch *b);

#ifdef __cplusplus
}
#endif

#endif /* PIC_H */
