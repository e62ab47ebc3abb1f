// Internal declarations shared by the library's translation units (not part of
// the C ABI; the public interface is include/pic.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "ff.cuh"
#include "pic.h"

namespace pic {

constexpr int kMaxSpecies = 8;
constexpr int kMaxNodes1D = 8192;   // 1D grid held whole in shared memory

// Device-side error flags (bit set by kernels, read by the host after a call).
// No kernel of the library waits on another block or launch (every ordering
// is a stream's or a kernel boundary's), so none has a wait that could time
// out: PIC_ERR_TIMEOUT has no flag.
enum : unsigned { kErrNonfinite = 1u, kErrBounds = 2u, kErrVelocityRange = 4u };

#ifdef PIC_DEBUG_BOUNDS
// Records of the index checks of the debug-bounds build, one per translation
// unit with checks: file code << 16 | line of the first failed check, 0 if
// none; each call clears its record.
unsigned bounds_site_es1d_mixed();
unsigned bounds_site_em2d_mixed();
unsigned bounds_site_em1d_spectral();
#endif

struct SpeciesInfo {
  double q, m, w0;
  int64_t n;
  int64_t offset;     // first slot of this species in the concatenated arrays
  bool weighted;
};

// Per-launch constants of the 1D electrostatic kernels.
struct Es1dConst {
  int nc;
  int order;
  int scheme;
  int remove_mean;
  int gamma_on;
  int passes;     // binomial filter passes inside the scheme (FP64 form): F j, F E
  int nsp;
  int64_t n_total;
  double L, h, inv_h, dt;
  // per species
  int64_t sp_end[kMaxSpecies];   // exclusive end slot of species s
  double qm[kMaxSpecies];        // q/m
  double qw_h[kMaxSpecies];      // q w0 / h (uniform weights)
  double q_h[kMaxSpecies];       // q / h (weighted markers: times w_p)
  double half_mw[kMaxSpecies];   // m w0 / 2 (uniform weights)
  double half_m[kMaxSpecies];    // m / 2
};

// Per-launch constants of the 1D mixed-precision kernels (one species, uniform
// weight).  Velocities are stored in "V units": v * cxk.
struct Es1dMixConst {
  int nc;
  int order;
  int scheme;
  int remove_mean;
  int gamma_on;
  int rshift;          // deposit term = round(V* s_k / 2^rshift)
  int split;           // bits b of the low counter of the split current tiles
  unsigned lomask;     // 2^b - 1
  int hishift;         // rshift + b - 32: the signed share from the high word
  int kv;              // one V unit = 2^-kv position units per half step
  int mode;            // 0 unsorted, 1 periodic counting sort, 2 sorted on write every step
  int wide;            // unsorted with nc <= kWideMaxNodes: per-lane tile copies, 1024-thread blocks
  int hround;          // 2^(kv - 1), kv >= 1
  int gamma64;         // 1: the correction in FP64 for every marker (unsorted mode)
  long long rnd;       // 2^(rshift - 1)
  int64_t n;
  double L, h, dt;
  double cxk;          // (dt 2^31 / L) 2^kv
  double jscale;       // J_h = jscale * (integer node sum)
  double ke_scale;     // (m w / 2) / cxk^2
  double e_scale;      // dt/2 (q/m) cxk: E** -> increment of v* in V units
  double kick;         // dt (q/m) cxk: E^{n+1/2} -> v^dag - v^n in V units
  ff kick_jhalf;       // kick dt/2 jscale as a float pair: J units -> kick E units
  ff inv_nc;           // 1 / nc as a float pair
  float c_jstar;       // e_scale dt/2 jscale: J units -> kick-table units of E*
  int passes;          // p passes of the binomial filter inside the scheme (0: none)
};

// One block of a batched launch over several independent runs: block rb of the
// nb blocks that share run `run`.
struct BatchItem {
  int run, rb, nb;
};

// Unsorted mixed form: grids up to this many nodes use 32 copies of the
// current tile and 16 of the field tables per block (one 1024-thread block per
// SM); larger grids one copy (512-thread blocks).
constexpr int kWideMaxNodes = 512;
// Block size of the fused ESEC1 pass in that layout: 768 threads, one block per
// SM.  The fused pass keeps both tables and both shapes of a marker live; at
// 1024 threads its 64 registers spill, at 768 it has 80 and none.
constexpr int kFusedThreads = 768;
// Mixed-form integer node sums J1, J2 hold node i at [i * kJStride]: one node
// per 128-byte line, so the blocks' global atomics spread over the L2 slices.
constexpr int kJStride = 16;

// Buffers of one fused ESEC1 launch (es1d_mix_pass_ec): the current sums and
// grid total it reads (j^{*,n+1/2}), the ones it deposits (j^{*,n+3/2}) and
// the ones it clears (read by the previous launch, written by the next), and
// the block partials of the previous step's energy (for its TE) and of this
// step's.
struct RingIO {
  const long long *Jr, *Tr;
  long long *Jw, *Tw;
  long long *Jc, *Tc;
  const double *ke_prev, *we_prev;
  double *ke_out, *we_out;
};

struct Es1dMixBufs {
  uint32_t *X;              // [N padded to 4] positions, x = X L / 2^32
  float *vh, *vl;           // [N padded to 4] velocity pairs
  int *Vs;                  // [N padded to 4] V* of the current step (pass C -> pass E)
  // sort on write (mode 2): pass E writes the new state in key order here
  uint32_t *Xo;
  float *vho, *vlo;
  int64_t *ids, *ido;       // marker ids (null when not tracked)
  uint32_t *H;              // [2 nc][G] per-block key counts of pass C, then prefixes
  uint32_t *T;              // [2 nc] key totals
  double *E[2];
  float2 *Ek[2];            // [2][nc] kick E (kick = dt (q/m) cxk) as float pairs, same parity as E
  long long *J1[2], *J2[2]; // integer current sums
  long long *Jtot;          // [4] grid totals of J1[0], J1[1], J2[0], J2[1] (for <J>)
  double *ke_part;
  unsigned long long *fallback;
  double *te;
  double *we;
  double *we_part;          // [grid] per-block W_E partials of the newest field
  unsigned *err;
  // passes > 0: the stencils of F^p (2p + 1 weights) and of F^2p (4p + 1) as
  // float pairs (exact: binomial coefficients over powers of 4)
  const float2 *filt;
};

// Per-launch constants of the 2D3V Yee kernels (FP64 form).
struct Em2dConst {
  int nx, ny;
  int order;
  int cc;          // charge-conserving shapes and path pieces (order 1)
  int scheme;
  int gamma_on;
  int nsp;
  int64_t n_total;
  double Lx, Ly, inv_hx, inv_hy, dt, c2, area;
  int64_t sp_end[kMaxSpecies];
  double qm[kMaxSpecies];
  double qw_a[kMaxSpecies];     // q w0 / |h|
  double q_a[kMaxSpecies];      // q / |h| (weighted markers)
  double half_mw[kMaxSpecies];
  double half_m[kMaxSpecies];
};

struct Em2dBufs {
  double *x, *y, *vx, *vy, *vz, *w;   // [N] SoA (w may be null)
  double *E;      // E^n            [3][ny][nx]
  double *En;     // E^{n+1}
  double *Eh;     // E^{n+1/2}
  double *Es;     // E*
  double *B;      // B^{n-1/2}
  double *Bp;     // B^{n+1/2}
  double *Bpp;    // B^{n+3/2} (computed at the end of a step)
  double *J1;     // j^{n,*}
  double *J2;     // j^{*,n+1/2}
  double *vsx, *vsy, *vsz;     // [N] v* of the current step (pass C -> pass E)
  double *sw;     // [weights][N] shape at x^{n+1/2} (point shapes: pass C -> pass E),
  int *si;        // [4][N] its first nodes; both null: pass E forms it again
  double *sws;    // ESEC2, point shapes: the shape at the next step's x* (pass E or
  int *sis;       // the initial deposit -> pass C), as sw / si; null: formed again
  double *ke_part;             // [particle blocks]
  double *wf_part;             // [2 x grid blocks] W_E, W_B partials
  unsigned long long *fallback;
  double *te;
  unsigned *err;
};

// 1D2V electromagnetic path with a pseudospectral field solve (Crank-Nicolson
// or PSATD), FP64; n a power of two in [4, kSpecMaxNodes].
constexpr int kSpecMaxNodes = 1024;
constexpr int kJSlices = 8;                  // slices of the global current (power of two)
constexpr size_t kEm1TileBudget = 96 * 1024; // shared bytes for field tables + tile copies
constexpr int kEm1Coef = 8;                  // per-mode field-advance coefficients

struct Em1dConst {
  int n, log2n;
  int order;
  int scheme;
  int solver;       // 1 Crank-Nicolson, 2 PSATD
  int gamma_on;
  int nsp;
  int rt;           // copies of the shared current tile (power of two, <= 32)
  int64_t n_total;
  double L, h, inv_h, dt, c, c2;
  int64_t sp_end[kMaxSpecies];
  double qm[kMaxSpecies];
  double qw_h[kMaxSpecies];     // q w0 / h
  double q_h[kMaxSpecies];      // q / h (weighted markers)
  double w0[kMaxSpecies];
  double half_m[kMaxSpecies];
};

struct Em1dBufs {
  double *y, *vx, *vy, *w;   // [N] SoA (w may be null)
  double *vsx, *vsy;         // [N] v* of the current step (pass C -> pass E)
  double *sw;                // [order + 1][N] shape weights at y^{n+1/2} and
  int *si;                   // [N] its node (pass C -> pass E), or null (recomputed)
  double *sws;               // ESEC2: the shape at the next step's y* (pass E or the
  int *sis;                  // initial deposit -> pass C), as sw / si; null: formed again
  double *E, *En;            // E^n, E^{n+1}: [2][n] (Ex, Ey); swapped after each step
  double *B, *Bn;            // Bz^n, Bz^{n+1}: [n]
  double *Es, *Bs;           // E*, B* of the half step
  double *Ea, *Bh;           // the E of v^dag (E^{n+1/2} or <E>) and B^{n+1/2}
  double *J1, *J2;           // j^{n,*}, j^{*,n+1/2}: [kJSlices][2][n], summed over slices
  double2 *tw;               // [n/2] FFT twiddles exp(-2 pi i j / n)
  double *coef;              // [2][n/2 + 1][kEm1Coef] per-mode coefficients, full and half step
  double *ke_part;           // [particle blocks]
  unsigned *done;            // [2] arrival counters of pass C and pass E
  unsigned long long *fallback;
  double *te;
  unsigned *err;
};

// Standard explicit PIC (the comparison scheme: leapfrog Vlasov-Poisson with a
// binomially filtered charge), FP64 1D1V; n a power of two in [4, kStdMaxNodes].
constexpr int kStdMaxNodes = 4096;

struct StdConst {
  int n, log2n;
  int order;
  int nsp;
  int rt;           // copies of the shared charge tile (power of two, <= 32)
  int passes;       // 1-2-1 filter passes on the charge
  int64_t n_total;
  double L, h, inv_h, dt;
  int64_t sp_end[kMaxSpecies];
  double qm[kMaxSpecies];
  double qw_h[kMaxSpecies];
  double q_h[kMaxSpecies];
  double w0[kMaxSpecies];
  double half_m[kMaxSpecies];
};

struct StdBufs {
  double *x, *v, *w;     // x^n and v^{n-1/2} [N] (w may be null)
  double *E;             // E^n [n]
  double *rho;           // charge of the next positions [kJSlices][n]
  double2 *tw;           // [n/2] FFT twiddles
  double *g;             // [n/2 + 1] filter gain / |kk| per mode (0: k = 0, Nyquist)
  double *ke_part;       // [particle blocks]
  unsigned *done;        // arrival counter
  unsigned long long *fallback;
  double *te;
  unsigned *err;
};

// Mixed form of the 1D2V spectral path (one species, uniform weight): y as
// 32-bit fixed point (y = Y L / 2^32), (vx, vy) as float pairs in V units
// (v cxk, one V unit moves a marker 2^-kv position units in half a step), v*
// as integers, the currents (jx, jy) as exact integer sums of round(V* s /
// 2^rshift) through per-lane split tiles; the fields and the field solve stay
// FP64 (Em1dBufs), fed with jscale times the integer sums.
struct Em1dMixConst {
  int n, order, scheme, gamma_on;
  int rt;              // copies of the shared current tile
  int kv, hround;      // V units -> half-step position shift: (V + hround) >> kv
  int rshift;          // current term = round(V* s / 2^rshift), rshift in [17, 31]
  long long rnd;       // 2^(rshift - 1)
  int64_t N;
  double L, dt;
  double cxk;          // (dt 2^31 / L) 2^kv
  double jscale;       // J = jscale * (integer node sum)
  double ke_scale;     // (m w / 2) / cxk^2
  double e_half;       // dt/2 (q/m) cxk: E* -> V units
  double t_half;       // dt/2 (q/m): Bz* -> the rotation t of v*
  double kick;         // dt (q/m) cxk: the E of v^dag -> V units
  double m_full;       // dt (q/m): V* x B^{n+1/2} -> V units
};

struct Em1dMixBufs {
  uint32_t *Y;                // [N]
  float *vh[2], *vl[2];       // [N] (vx, vy) pairs in V units
  int *Vs[2];                 // [N] V* (pass C -> pass E)
  long long *J1, *J2;         // [2][n] integer sums of j^{n,*} and j^{*,n+1/2}
};

// Mixed form of the 2D3V Yee path (one species, uniform weight, square
// domain): positions X, Y as 32-bit fixed point (x = X L / 2^32), velocities as
// float pairs in V units (v cxk; one V unit moves a marker 2^-kv position units
// in half a step), v* as integers V*, the currents as exact int64 sums of
// round(V* s_x s_y / 2^rshift) (s: weights in units of 2^-23); the fields stay
// FP64 on the grid, with float tables for the gathers.
struct Em2dMixConst {
  int nx, ny;
  int order, scheme, gamma_on;
  int kv, hround;      // V units -> half-step position shift: (V + hround) >> kv
  int rshift;          // current term = round(V* s_x s_y / 2^rshift), rshift >= 32
  long long rnd;       // 2^(rshift - 1)
  int64_t n;
  double L, dt;
  double cxk;          // (dt 2^31 / L) 2^kv
  double jscale;       // J = jscale * (integer node sum)
  double ke_scale;     // (m w / 2) / cxk^2
  double e_half;       // dt/2 (q/m) cxk: E* -> V units
  double t_half;       // dt/2 (q/m): B -> the rotation vector t of v*
  double kick;         // dt (q/m) cxk: E^{n+1/2} -> V units
  double m_full;       // dt (q/m): (V* x B) -> V units
  int sorted;          // markers kept in quarter-cell order: segmented warp deposits
};

struct Em2dMixBufs {
  uint32_t *X, *Y;                 // [N]
  float *vh[3], *vl[3];            // [N] velocity pairs in V units
  int *Vs[3];                      // [N] V* (pass C -> pass E)
  long long *J1, *J2;              // [3][ny][nx] integer current sums
  float *T1;                       // [6][ny][nx]: e_half E*, then t_half B^{n+1/2}
  float2 *T2;                      // [3][ny][nx]: kick E^{n+1/2} as float pairs
  float *B2;                       // [3][ny][nx]: m_full B^{n+1/2}
  double *ke_part;                 // [particle blocks]
  unsigned long long *fallback;
  unsigned *err;
};

// The quarter-cell sort of the mixed 2D3V markers, written by pass E of the
// step that ends a sort period (off set; null on every other step).
struct Em2dSortIO {
  unsigned *off;            // [4 nx ny] first free slot of each quarter cell
  Em2dMixBufs dst;          // X, Y, vh, vl of the sorted markers
  const int64_t *ids_in;    // [N] marker ids, or null (not carried)
  int64_t *ids_out;         // [N] the ids in the sorted order
};

// Everything the 1D FP64 kernels touch.
struct Es1dFp64Bufs {
  double *x, *v, *w;        // [N] SoA (w may be null)
  double *vs;               // [N] v* of the current step (pass C -> pass E), or null:
                            // pass E then recomputes it (the same bits)
  double *sw;               // [order + 1][N] shape weights at x^{n+1/2} and
  int *si;                  // [N] its node (pass C -> pass E), or null (recomputed)
  double *sws;              // ESEC2: [order + 1][N] shape weights at the next step's
  int *sis;                 // x* and its node (pass E or the initial deposit -> pass
                            // C), or null (recomputed)
  double *E[2];             // ping-pong E^n / E^{n+1}
  double *J1[2];            // j^{n,*} (ESEC2), indexed by step parity
  double *J2[2];            // j^{*,n+1/2}
  double *ke_part;          // [grid] block partials of KE of the step just done
  unsigned long long *fallback;   // [steps_cap] per-step counters
  double *te;               // [steps_cap] total energy after each step
  double *we;               // [1] W_E of the newest field
  unsigned *err;            // device error flags
};

// Reverse mode of the FP64 1D form (es1d_grad.cu): the markers and weights of
// the forward step being reversed, grid scratch and the running adjoints.
struct Es1dGradBufs {
  const double *x, *v;      // [N] markers at the start of the step
  const double *w;          // [N] weights, or null for uniform weights w0[s]
  double w0[kMaxSpecies];
  double *Estar, *H, *J1;   // [nc] E*, E^{n+1/2}, j^{n,*} of the step
  double *Hbar, *Esbar, *Jbar;  // [nc] adjoint scratch
  double *Ebar;             // [nc] adjoint of the field (E^{n+1} in, E^n out)
  double *xbar, *vbar;      // [N] adjoints of the markers (after the step in, before out)
  double *wbar;             // [N] adjoints of the weights, accumulated
  double *ub, *yb;          // [N] marker scratch
  unsigned *err;
};

struct LaunchShape {
  int grid;
  int block;
};

// Sets the message returned by pic_last_error (pic_api.cu).
void set_last_error(const std::string &msg);

// reverse mode of one FP64 1D step, from the step's starting field E and its
// result Enew (es1d_grad.cu)
cudaError_t es1d_grad_prepare(const Es1dConst &c);
void es1d_grad_step(const Es1dConst &c, const Es1dGradBufs &g, const double *E,
                    const double *Enew, LaunchShape ls, cudaStream_t st);

// 1D FP64 path (es1d_fp64.cu)
cudaError_t es1d_fp64_prepare(const Es1dConst &c);
void es1d_fp64_deposit_initial(const Es1dConst &c, const Es1dFp64Bufs &b, int parity,
                               LaunchShape ls, cudaStream_t st);
void es1d_fp64_pass_c(const Es1dConst &c, const Es1dFp64Bufs &b, int64_t step_index,
                      int slot, LaunchShape ls, cudaStream_t st);
void es1d_fp64_pass_e(const Es1dConst &c, const Es1dFp64Bufs &b, int64_t step_index,
                      int slot, LaunchShape ls, cudaStream_t st);
void es1d_fp64_finalize(const Es1dConst &c, const Es1dFp64Bufs &b, int slot, int nblocks,
                        cudaStream_t st);
void es1d_fp64_charge(const Es1dConst &c, const double *x, const double *w, double *rho,
                      LaunchShape ls, cudaStream_t st);
void es1d_fp64_kinetic(const Es1dConst &c, const double *v, const double *w, double *ke_sp,
                       cudaStream_t st);

// 2D3V Yee path (em2d_fp64.cu)
void em2d_k1(const Em2dConst &c, const Em2dBufs &b, LaunchShape lg, cudaStream_t st);
void em2d_pass_c(const Em2dConst &c, const Em2dBufs &b, LaunchShape lp, cudaStream_t st);
void em2d_k3(const Em2dConst &c, const Em2dBufs &b, LaunchShape lg, cudaStream_t st);
void em2d_pass_e(const Em2dConst &c, const Em2dBufs &b, int slot, LaunchShape lp, cudaStream_t st);
// k5 and the finalize kernel wait for the previous kernel with griddep_wait():
// pdl launches them as programmatic dependent launches (the mixed form's chain)
void em2d_k5(const Em2dConst &c, const Em2dBufs &b, LaunchShape lg, cudaStream_t st, bool pdl);
void em2d_finalize(const Em2dConst &c, const Em2dBufs &b, int slot, LaunchShape lp,
                   LaunchShape lg, cudaStream_t st, bool pdl);
void em2d_fp64_deposit_initial(const Em2dConst &c, const Em2dBufs &b, LaunchShape lp,
                               cudaStream_t st);
void em2d_fp64_bhalf(const Em2dConst &c, const double *B, const double *E, double *Bp,
                     LaunchShape lg, cudaStream_t st);
void em2d_fp64_kinetic(const Em2dConst &c, const Em2dBufs &b, double *out, int nblocks,
                       cudaStream_t st);
__global__ void em2d_validate_kernel(const double *x, const double *y, const double *vx,
                                     const double *vy, const double *vz, int64_t n, double Lx,
                                     double Ly, unsigned *err);

// standard-PIC comparator (es1d_standard.cu)
int std_tile_copies(int n);
cudaError_t std_prepare(const StdConst &c, const StdBufs &b, cudaStream_t st);
void std_step(const StdConst &c, const StdBufs &b, int slot, LaunchShape lp, cudaStream_t st);
// E^0 from the charge of x^0, then v^{-1/2} = v^0 - dt/2 (q/m) E^0_p
void std_start(const StdConst &c, const StdBufs &b, LaunchShape lp, cudaStream_t st);
// KE^n partials ke_out [nsp][lp.grid] (v^{n+1/2} formed, not stored) and W_E^n
void std_energy(const StdConst &c, const StdBufs &b, double *ke_out, double *we, LaunchShape lp,
                cudaStream_t st);

// 2D3V Yee path, mixed form (em2d_mixed.cu); the FP64 fields live in Em2dBufs
// and K5 / the finalize kernel of the FP64 form are shared.
// K1 of the mixed form; with fin_slot >= 0 one more block reduces the total
// energy of the step in fin_slot (lp: the passes' shape, lg: the grid's)
void em2dm_k1(const Em2dConst &c, const Em2dMixConst &m, const Em2dMixBufs &mb,
              const Em2dBufs &b, int fin_slot, LaunchShape lp, LaunchShape lg, cudaStream_t st);
void em2dm_k3(const Em2dConst &c, const Em2dMixConst &m, const Em2dMixBufs &mb,
              const Em2dBufs &b, LaunchShape lg, cudaStream_t st);
// pass C; cnt: [4 nx ny] counts of the quarter cells of x^{n+1} (sorted
// markers, the step that ends a sort period) or null
void em2dm_pass_c(const Em2dMixConst &m, const Em2dMixBufs &mb, unsigned *cnt, LaunchShape lp,
                  cudaStream_t st);
// pass E, and K5 of the FP64 fields (c, b) in lg.grid more blocks
void em2dm_pass_e(const Em2dMixConst &m, const Em2dMixBufs &mb, int slot, const Em2dSortIO &so,
                  const Em2dConst &c, const Em2dBufs &b, LaunchShape lp, LaunchShape lg,
                  cudaStream_t st);
// Launch shape of the mixed 2D3V passes C and E (and so the number of kinetic
// partials pass E writes): lp on unsorted markers; on sorted ones one block per
// 256 threads' runs of consecutive markers, so every warp makes one trip.
LaunchShape em2dm_pass_shape(int64_t n, bool sorted, LaunchShape lp);
// Words of the sort's count array: a count per quarter cell, then the totals
// of the scan's tiles.
size_t em2dm_sort_count_words(int nx, int ny);
// offsets off[] of the quarter cells from pass C's counts cnt[], which it
// leaves zero for the next sort
void em2dm_sort_scan(const Em2dMixConst &m, unsigned *cnt, unsigned *off, cudaStream_t st);
// FP64 staging (x, y, vx, vy, vz) <-> the mixed state
void em2dm_from_fp64(const Em2dMixConst &m, const Em2dMixBufs &mb, const Em2dBufs &b,
                     LaunchShape lp, cudaStream_t st);
void em2dm_to_fp64(const Em2dMixConst &m, const Em2dMixBufs &mb, const Em2dBufs &b,
                   LaunchShape lp, cudaStream_t st);
// j^{n,*} of the current state into mb.J1 (cleared first by the caller)
void em2dm_deposit_initial(const Em2dMixConst &m, const Em2dMixBufs &mb, LaunchShape lp,
                           cudaStream_t st);
// kinetic energy block partials (physical units) into out[lp.grid]
void em2dm_kinetic(const Em2dMixConst &m, const Em2dMixBufs &mb, double *out, LaunchShape lp,
                   cudaStream_t st);
// largest |v| component of the FP64 staging velocities (bits of a double)
void em2dm_absmax(const Em2dBufs &b, int64_t n, unsigned long long *out, LaunchShape lp,
                  cudaStream_t st);

// 1D2V spectral path, mixed form (em1d_spectral.cu): the FP64 field side of
// Em1dBufs, the markers of Em1dMixBufs
void em1m_pass_c(const Em1dConst &c, const Em1dBufs &b, const Em1dMixConst &m,
                 const Em1dMixBufs &mb, LaunchShape lp, cudaStream_t st);
void em1m_pass_e(const Em1dConst &c, const Em1dBufs &b, const Em1dMixConst &m,
                 const Em1dMixBufs &mb, int slot, LaunchShape lp, cudaStream_t st);
// j^{0,*} (ESEC2) and the first half step (E*, B*) of the current state
void em1m_start(const Em1dConst &c, const Em1dBufs &b, const Em1dMixConst &m,
                const Em1dMixBufs &mb, LaunchShape lp, cudaStream_t st);
// FP64 staging (y, vx, vy of Em1dBufs) <-> the mixed markers
void em1m_from_fp64(const Em1dConst &c, const Em1dBufs &b, const Em1dMixConst &m,
                    const Em1dMixBufs &mb, LaunchShape lp, cudaStream_t st);
void em1m_to_fp64(const Em1dConst &c, const Em1dBufs &b, const Em1dMixConst &m,
                  const Em1dMixBufs &mb, LaunchShape lp, cudaStream_t st);
// kinetic energy block partials of the mixed markers, and W_E, W_B (em1d_energy's layout)
void em1m_energy(const Em1dConst &c, const Em1dBufs &b, const Em1dMixConst &m,
                 const Em1dMixBufs &mb, double *ke_out, double *wf, LaunchShape lp,
                 cudaStream_t st);
// largest |v| component of the FP64 staging velocities (bits of a double)
void em1m_absmax(const Em1dBufs &b, int64_t n, unsigned long long *out, LaunchShape lp,
                 cudaStream_t st);
// tile copies of the mixed passes: the largest power of two <= 32 whose tile
// and tables fit the budget
int em1m_tile_copies(int n);
cudaError_t em1m_prepare(const Em1dConst &c, const Em1dMixConst &m);

// 1D2V spectral path (em1d_spectral.cu)
// shared-memory opt-in and the twiddle / coefficient tables (b.tw, b.coef)
cudaError_t em1d_prepare(const Em1dConst &c, const Em1dBufs &b, cudaStream_t st);
// copies of the shared current tile for n nodes
int em1d_tile_copies(int n);
void em1d_pass_c(const Em1dConst &c, const Em1dBufs &b, LaunchShape lp, cudaStream_t st);
void em1d_pass_e(const Em1dConst &c, const Em1dBufs &b, int slot, LaunchShape lp, cudaStream_t st);
// j^{0,*} (ESEC2 form) and the first E*, B*
void em1d_start(const Em1dConst &c, const Em1dBufs &b, LaunchShape lp, cudaStream_t st);
// kinetic energy partials ke_out [nsp][lp.grid] and wf = {W_E, W_B}
void em1d_energy(const Em1dConst &c, const Em1dBufs &b, double *ke_out, double *wf,
                 LaunchShape lp, cudaStream_t st);
__global__ void em1d_validate_kernel(const double *y, const double *vx, const double *vy,
                                     int64_t n, double L, unsigned *err);

// 1D mixed path (es1d_mixed.cu)
cudaError_t es1d_mix_prepare(const Es1dMixConst &c);
void es1d_mix_pass_c(const Es1dMixConst &c, const Es1dMixBufs &b, int64_t step_index, int slot,
                     LaunchShape ls, cudaStream_t st);
void es1d_mix_pass_e(const Es1dMixConst &c, const Es1dMixBufs &b, int64_t step_index, int slot,
                     LaunchShape ls, cudaStream_t st);
void es1d_mix_deposit_initial(const Es1dMixConst &c, const Es1dMixBufs &b, int parity,
                              LaunchShape ls, cudaStream_t st);
// ESEC1, unsorted: pass E of step step_index fused with pass C of the next step
void es1d_mix_pass_ec(const Es1dMixConst &c, const Es1dMixBufs &b, const RingIO &io,
                      int64_t step_index, int slot, LaunchShape ls, cudaStream_t st);
void es1d_mix_finalize(const Es1dMixConst &c, const Es1dMixBufs &b, int slot, int nblocks,
                       cudaStream_t st);
void es1d_mix_set_ek(const Es1dMixConst &c, const Es1dMixBufs &b, int parity, cudaStream_t st);
// batched runs (unsorted, nc <= kWideMaxNodes, one scheme): device arrays of the
// runs' constants and buffers and the work list of nitems blocks of `threads`
// (1024, or 256 for batches of small runs)
cudaError_t es1d_batch_prepare(size_t smem, int threads);
// dynamic shared memory of a batch block of `threads` for a run
size_t es1d_batch_smem(const Es1dMixConst &c, int threads);
// prev_slot: stats slot of the previous step to reduce (TE), or -1
void es1d_batch_pass_c(const Es1dMixConst *cs, const Es1dMixBufs *bs, const BatchItem *items,
                       int nitems, int scheme, int threads, size_t smem, int64_t step_index,
                       int prev_slot, cudaStream_t st);
void es1d_batch_pass_e(const Es1dMixConst *cs, const Es1dMixBufs *bs, const BatchItem *items,
                       int nitems, int scheme, int threads, size_t smem, int64_t step_index,
                       int slot, cudaStream_t st);
void es1d_batch_finalize(const Es1dMixConst *cs, const Es1dMixBufs *bs, const int *nblocks,
                         int nruns, int slot, cudaStream_t st);
void es1d_batch_gather_stats(const Es1dMixBufs *bs, int nruns, int n, unsigned long long *fb,
                             double *te, cudaStream_t st);
size_t es1d_mix_smem_max(const Es1dMixConst &c);
void es1d_mix_charge(const Es1dMixConst &c, const Es1dMixBufs &b, long long *count,
                     LaunchShape ls, cudaStream_t st);
void es1d_mix_from_fp64(const Es1dMixConst &c, const double *x, const double *v, Es1dMixBufs &b,
                        LaunchShape ls, cudaStream_t st);
void es1d_mix_to_fp64(const Es1dMixConst &c, const Es1dMixBufs &b, double *x, double *v,
                      LaunchShape ls, cudaStream_t st);
// the same for markers [begin, begin + count) (x, v and the mixed arrays
// indexed from the first marker)
void es1d_mix_from_fp64_part(const Es1dMixConst &c, const double *x, const double *v,
                             Es1dMixBufs &b, int64_t begin, int64_t count, LaunchShape ls,
                             cudaStream_t st);
void es1d_mix_to_fp64_part(const Es1dMixConst &c, const Es1dMixBufs &b, double *x, double *v,
                           int64_t begin, int64_t count, LaunchShape ls, cudaStream_t st);
void es1d_mix_kinetic(const Es1dMixConst &c, const Es1dMixBufs &b, double *part, int nblocks,
                      cudaStream_t st);
void es1d_absmax(const double *v, int64_t n, unsigned long long *out, LaunchShape ls,
                 cudaStream_t st);
int es1d_mix_sort_blocks(const Es1dMixConst &c, int nsm);
void es1d_mix_fused_scan(const Es1dMixConst &c, const Es1dMixBufs &b, int G, cudaStream_t st);
cudaError_t es1d_mix_sort(const Es1dMixConst &c, const Es1dMixBufs &src, const Es1dMixBufs &dst,
                          const int64_t *ids_in, int64_t *ids_out, uint32_t *H, int G,
                          cudaStream_t st);

// charge diagnostics (charge_diag.cu): 1D spectral Gauss residual and the 2D
// Yee one; part receives 3 doubles per block (sum r^2, sum rhot^2, sum rho)
int diag_blocks(int nodes);
void diag_rho_from_counts(const long long *cnt, int nc, double scale, double *rho,
                          cudaStream_t st);
void diag_gauss1d(const double *E, const double *rho, int nc, double L, const double2 *tw,
                  double2 *rm, double2 *pm, double *r, double *part, cudaStream_t st);
void diag_sum_range(const double *a, int64_t n, double *part, int blocks, cudaStream_t st);
void diag_em2d_charge(const Em2dConst &c, const double *x, const double *y, const double *w,
                      double *rho, LaunchShape lp, cudaStream_t st);
void diag_em2d_gauss(const Em2dConst &c, const double *E, const double *rho, double mean,
                     double *r, double *part, cudaStream_t st);

}  // namespace pic
