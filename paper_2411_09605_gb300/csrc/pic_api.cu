// Host runtime behind the C ABI of include/pic.h: argument checks, device
// memory, the per-step launch sequence and the state/energy accessors.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <tuple>
#include <cmath>
#include <string>
#include <vector>

#include "debug_bounds.cuh"
#include "pic_internal.cuh"

using namespace pic;

#ifdef PIC_DEBUG_BOUNDS
namespace pic {
PIC_BOUNDS_READER(bounds_site_pic_api)
}  // namespace pic
#endif

namespace {

thread_local std::string g_last_error;

int fail(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

#define CUDA_TRY(expr)                                                                    \
  do {                                                                                    \
    cudaError_t e_ = (expr);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return fail(e_ == cudaErrorMemoryAllocation ? PIC_ERR_OOM : PIC_ERR_CUDA,           \
                  "%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__,       \
                  __LINE__);                                                              \
  } while (0)

constexpr int kStepsCap = 1024;  // per-step stats slots per chunk of pic_step
constexpr int kXferChunks = 8;   // pieces of a pipelined host transfer of the markers
constexpr int kProfKinds = 8;    // 0 pass C, 1 pass E, 2 stats finalize, 3 sort, 4 field, 5 fused ESEC1 pass

// ids[p] = p for one species' slots (marker ids after pic_set_particles).
__global__ void iota_ids_kernel(int64_t *ids, int64_t n) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x)
    ids[p] = p;
}

// Validates positions in [0, L) and finite velocities of a 1D state.
__global__ void validate_1d_kernel(const double *x, const double *v, int64_t n, double L,
                                   unsigned *err) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    double a = x[p], b = v[p];
    if (!(a >= 0.0 && a < L)) atomicOr(err, kErrBounds);
    if (!isfinite(b)) atomicOr(err, kErrNonfinite);
  }
}

}  // namespace

namespace pic {
// Lets other translation units of the library report through pic_last_error.
void set_last_error(const std::string &msg) { g_last_error = msg; }
}  // namespace pic

struct pic_handle {
  pic_config cfg;
  cudaStream_t st = nullptr;
  int nsp = 0;
  SpeciesInfo sp[kMaxSpecies];
  int64_t N = 0;
  int64_t steps_done = 0;
  int pending = 0;          // asynchronous steps whose stats are not read yet
  bool te_open = false;     // mixed 2D3V: the last pending step's TE is not reduced yet
  int64_t launches = 0;     // kernels launched on behalf of this handle
  bool weighted = false;
  // optional per-launch timing (pic_set_profiling): events around each launch
  bool profiling = false;
  struct Timed { int kind; cudaEvent_t a, b; };
  std::vector<Timed> timed;
  double prof_ms[kProfKinds] = {0};
  int64_t prof_n[kProfKinds] = {0};
  LaunchShape ls{1, 512};
  // 1D FP64 state (in the mixed form x, v serve as FP64 staging for get/set)
  Es1dConst c1{};
  Es1dFp64Bufs b1{};
  // standard-PIC comparator state
  bool stdp = false;
  StdConst cs{};
  StdBufs bs{};
  LaunchShape lsd{1, 256};
  double *std_part = nullptr;  // pic_energy's partials [nsp][lsd.grid] and W_E
  // 1D2V spectral state (Crank-Nicolson or PSATD field solve)
  bool em1 = false;
  Em1dConst c1e{};
  Em1dBufs b1e{};
  LaunchShape le{1, 256};
  double *e1_part = nullptr;  // pic_energy's partials [nsp][le.grid] and W_E, W_B
  // 2D3V Yee state
  bool em = false;
  Em2dConst ce{};
  Em2dBufs be{};
  Em1dMixConst c1m{};   // mixed form of the 1D2V path (em1 && mixed)
  Em1dMixBufs b1m{};
  Em2dMixConst cme{};   // mixed form of the 2D3V path (em && mixed)
  Em2dMixBufs bme{};
  Em2dMixBufs bme_alt{};          // the quarter-cell sort's destination markers
  unsigned *sort2_cnt = nullptr;  // [4 nx ny] counts and offsets of the sort
  unsigned *sort2_off = nullptr;
  LaunchShape lp{1, 256}, lg{1, 256};
  LaunchShape lpm{1, 256};  // passes C and E of the mixed 2D3V form
  // 1D mixed-precision state
  bool mixed = false;
  Es1dMixConst cm{};
  LaunchShape lmix{1, 512};  // passes C and E of the mixed form
  LaunchShape lmix_ec{1, 512};  // the fused ESEC1 pass (same grid)
  double *energy_part = nullptr;  // pic_energy's kinetic partials (ke_part may be in use)
  Es1dMixBufs bm{};
  Es1dMixBufs bm_alt{};     // the counting sort's destination (swapped after a sort)
  int64_t *ids_alt = nullptr;
  uint32_t *sort_hist = nullptr;
  int sort_blocks = 0;
  int nsm = 0;
  // fused ESEC1 (mixed, unsorted): pass C of the next step already ran (its V*
  // and current are in place); the energy partials alternate between two buffers
  bool fused = false, primed = false;
  double *ke_alt = nullptr, *we_alt = nullptr;
  long long *jtot_base = nullptr;  // [8]; bm.Jtot = jtot_base + 4
  int64_t *ids = nullptr;
  // reverse mode (pic_grad_forward / pic_grad_backward), FP64 1D form
  struct Grad {
    int64_t start = -1;       // step count when pic_grad_forward began
    int nsteps = 0, every = 0, nck = 0;
    double *ckpt = nullptr;   // [nck][2N + nc] x, v, E every `every` steps
    double *seg = nullptr;    // [every + 1][2N + nc] the states of one segment
    double *fin = nullptr;    // [2N + nc] the state after the forward steps
    double *grid = nullptr;   // [7][nc] E*, H, J1, H_bar, E*_bar, J_bar, E_bar
    double *mk = nullptr;     // [5][N] x_bar, v_bar, w_bar and marker scratch
    size_t ckpt_cap = 0, seg_cap = 0;
  } grad;
  // charge diagnostics (pic_charge), allocated on first use
  struct Diag {
    double *rho = nullptr;      // [nodes] charge density
    double2 *tw = nullptr;      // [nc] exp(2 pi i t / nc) (1D)
    double2 *rm = nullptr, *pm = nullptr;  // [(nc - 1) / 2] modes of r and rho (1D)
    double *r = nullptr;        // [nodes] residual of Gauss's law
    double *part = nullptr;     // [3 x blocks] block partials; weight sums
    long long *cnt = nullptr;   // [nc] integer charge of the mixed 1D form
    int blocks = 0;
  } diag;
  std::vector<void *> allocs;

  template <typename T>
  int alloc(T **p, size_t count) {
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, sizeof(T) * (count ? count : 1));
    if (e != cudaSuccess)
      return fail(PIC_ERR_OOM, "cudaMalloc of %zu bytes failed: %s", sizeof(T) * count,
                  cudaGetErrorString(e));
    allocs.push_back(q);
    *p = (T *)q;
    return PIC_OK;
  }
  // chunked host transfers of the mixed 1D markers: a copy stream and one
  // event per chunk (plus one), made on first use
  cudaStream_t copy_st = nullptr;
  cudaEvent_t chunk_ev[kXferChunks + 1] = {};
  ~pic_handle() {
    if (copy_st) cudaStreamDestroy(copy_st);
    for (cudaEvent_t e : chunk_ev)
      if (e) cudaEventDestroy(e);
    for (Timed &t : timed) {
      cudaEventDestroy(t.a);
      cudaEventDestroy(t.b);
    }
    for (void *p : allocs) cudaFree(p);
    for (void *p : {(void *)grad.ckpt, (void *)grad.seg, (void *)grad.fin, (void *)grad.grid,
                    (void *)grad.mk})
      if (p) cudaFree(p);
  }
  // Brackets the launches issued by f with timing events when profiling.
  template <typename F>
  cudaError_t timed_launch(int kind, F f) {
    if (!profiling) {
      f();
      return cudaGetLastError();
    }
    Timed t{kind, nullptr, nullptr};
    cudaError_t e = cudaEventCreate(&t.a);
    if (e == cudaSuccess) e = cudaEventCreate(&t.b);
    if (e != cudaSuccess) return e;
    cudaEventRecord(t.a, st);
    f();
    cudaEventRecord(t.b, st);
    timed.push_back(t);
    return cudaGetLastError();
  }
  cudaError_t collect_profile() {
    for (Timed &t : timed) {
      cudaError_t e = cudaEventSynchronize(t.b);
      if (e != cudaSuccess) return e;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, t.a, t.b);
      prof_ms[t.kind] += ms;
      prof_n[t.kind] += 1;
      cudaEventDestroy(t.a);
      cudaEventDestroy(t.b);
    }
    timed.clear();
    return cudaSuccess;
  }
};

namespace {

// The copy stream and its events, made on first use.
cudaError_t ensure_copy_stream(pic_handle *h) {
  if (h->copy_st) return cudaSuccess;
  cudaError_t e = cudaStreamCreateWithFlags(&h->copy_st, cudaStreamNonBlocking);
  for (int k = 0; e == cudaSuccess && k <= kXferChunks; k++)
    e = cudaEventCreateWithFlags(&h->chunk_ev[k], cudaEventDisableTiming);
  return e;
}

// p as the device addresses it: device or managed memory, or host memory that
// is pinned and mapped into the device's address space (kernels then read or
// write it over the host link directly, at the link's rate); null for other
// host memory (pageable), which goes through cudaMemcpy.
template <typename T>
T *device_view(T *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();  // an unknown pointer is not an error here
    return nullptr;
  }
  if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged ||
      a.type == cudaMemoryTypeHost)
    return static_cast<T *>(a.devicePointer);
  return nullptr;
}

// pic_set_particles of the mixed 1D form.  Markers the device can address
// (device memory, pinned host memory) are turned into the mixed state by one
// kernel that reads them where they are.  Other host memory goes into the
// FP64 staging arrays in kXferChunks pieces on the copy stream, and each piece
// is turned into the mixed state on the handle's stream as soon as it has
// arrived, so the conversion overlaps the transfer of the next piece.
cudaError_t upload_mixed_1d(pic_handle *h, const double *x, const double *v) {
  const double *xd = device_view(x), *vd = device_view(v);
  if (xd && vd) {
    es1d_mix_from_fp64_part(h->cm, xd, vd, h->bm, 0, h->N, h->ls, h->st);
    return cudaGetLastError();
  }
  cudaError_t e = ensure_copy_stream(h);
  Es1dFp64Bufs &b = h->b1;
  const int64_t n = h->N, chunk = (n + kXferChunks - 1) / kXferChunks;
  // earlier work on the handle's stream may still read the staging arrays
  if (e == cudaSuccess) e = cudaEventRecord(h->chunk_ev[kXferChunks], h->st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(h->copy_st, h->chunk_ev[kXferChunks], 0);
  for (int k = 0; e == cudaSuccess && k < kXferChunks && k * chunk < n; k++) {
    const int64_t b0 = k * chunk, cnt = std::min(chunk, n - b0);
    e = cudaMemcpyAsync(b.x + b0, x + b0, sizeof(double) * cnt, cudaMemcpyDefault, h->copy_st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(b.v + b0, v + b0, sizeof(double) * cnt, cudaMemcpyDefault, h->copy_st);
    if (e == cudaSuccess) e = cudaEventRecord(h->chunk_ev[k], h->copy_st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->st, h->chunk_ev[k], 0);
    if (e == cudaSuccess) {
      es1d_mix_from_fp64_part(h->cm, b.x, b.v, h->bm, b0, cnt, h->ls, h->st);
      e = cudaGetLastError();
    }
  }
  return e;
}

// pic_get_particles of the mixed 1D form: written by one kernel straight into
// memory the device can address; otherwise each piece is converted to FP64 on
// the handle's stream and copied out on the copy stream while the next piece
// converts.  Returns after the last write.
cudaError_t download_mixed_1d(pic_handle *h, double *x, double *v) {
  double *xd = x ? device_view(x) : nullptr, *vd = v ? device_view(v) : nullptr;
  if (x && v && xd && vd) {
    es1d_mix_to_fp64_part(h->cm, h->bm, xd, vd, 0, h->N, h->ls, h->st);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? cudaStreamSynchronize(h->st) : e;
  }
  cudaError_t e = ensure_copy_stream(h);
  Es1dFp64Bufs &b = h->b1;
  const int64_t n = h->N, chunk = (n + kXferChunks - 1) / kXferChunks;
  for (int k = 0; e == cudaSuccess && k < kXferChunks && k * chunk < n; k++) {
    const int64_t b0 = k * chunk, cnt = std::min(chunk, n - b0);
    es1d_mix_to_fp64_part(h->cm, h->bm, b.x, b.v, b0, cnt, h->ls, h->st);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(h->chunk_ev[k], h->st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->copy_st, h->chunk_ev[k], 0);
    if (e == cudaSuccess && x)
      e = cudaMemcpyAsync(x + b0, b.x + b0, sizeof(double) * cnt, cudaMemcpyDefault, h->copy_st);
    if (e == cudaSuccess && v)
      e = cudaMemcpyAsync(v + b0, b.v + b0, sizeof(double) * cnt, cudaMemcpyDefault, h->copy_st);
  }
  if (e == cudaSuccess) e = cudaEventRecord(h->chunk_ev[kXferChunks], h->copy_st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(h->st, h->chunk_ev[kXferChunks], 0);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
  return e;
}

// Marker ids 0..n-1 of species S, set on the device (no host array).
cudaError_t reset_ids(pic_handle *h, const SpeciesInfo &S) {
  if (S.n == 0) return cudaSuccess;
  const int grid = (int)std::min<int64_t>((S.n + 255) / 256, 4096);
  iota_ids_kernel<<<grid, 256, 0, h->st>>>(h->ids + S.offset, S.n);
  h->launches += 1;
  return cudaGetLastError();
}

int check_flags(pic_handle *h, const char *where) {
  unsigned flags = 0;
  CUDA_TRY(cudaMemcpyAsync(&flags, h->b1.err, sizeof flags, cudaMemcpyDeviceToHost, h->st));
  CUDA_TRY(cudaStreamSynchronize(h->st));
#ifdef PIC_DEBUG_BOUNDS
  // a failed index check comes first: the flags after it may be its effects
  // (the records are per process, not per handle)
  const struct {
    unsigned (*read)();
    const char *unit;
  } units[] = {{bounds_site_es1d_mixed, "es1d_mixed.cu"},
               {bounds_site_em2d_mixed, "em2d_mixed.cu"},
               {bounds_site_em1d_spectral, "em1d_spectral.cu"}};
  for (const auto &u : units)
    if (const unsigned site = u.read()) {
      if (flags) CUDA_TRY(cudaMemsetAsync(h->b1.err, 0, sizeof(unsigned), h->st));
      return fail(PIC_ERR_BOUNDS, "%s: index check failed at %s:%u (a kernel of %s)", where,
                  bounds_file_name(site), site & 0xFFFFu, u.unit);
    }
#endif
  if (flags) {
    CUDA_TRY(cudaMemsetAsync(h->b1.err, 0, sizeof(unsigned), h->st));
    if (flags & kErrNonfinite) return fail(PIC_ERR_NONFINITE, "%s: non-finite value in the state", where);
    if (flags & kErrBounds)
      return fail(PIC_ERR_BOUNDS, "%s: a position left [0, L) (input out of range, or a "
                                  "particle crossed more than one period in a step)", where);
    if (flags & kErrVelocityRange)
      return fail(PIC_ERR_BOUNDS, "%s: a velocity left the mixed form's fixed-point range "
                                  "(8 times the largest initial speed)", where);
    return fail(PIC_ERR_CUDA, "%s: device error flags 0x%x", where, flags);
  }
  return PIC_OK;
}

// Spectral solve of dE/dx = rho - <rho> on the 1D grid (Eq. poisson in field
// form): E_k = rho_k / (i kappa_k), k = 0 and (even n) the Nyquist mode set to 0.
void poisson_1d_host(const std::vector<double> &rho, double L, std::vector<double> &E) {
  const int n = (int)rho.size();
  const double twopi = 6.283185307179586476925286766559;
  std::vector<double> cs(n), sn(n);
  for (int j = 0; j < n; j++) {
    cs[j] = cos(twopi * j / n);
    sn[j] = sin(twopi * j / n);
  }
  E.assign(n, 0.0);
  for (int k = 1; k < n; k++) {
    if (n % 2 == 0 && k == n / 2) continue;
    double re = 0.0, im = 0.0;
    for (int j = 0; j < n; j++) {
      int t = (int)(((int64_t)j * k) % n);
      re += rho[j] * cs[t];
      im -= rho[j] * sn[t];
    }
    int ks = k < n - k ? k : k - n;
    double kappa = twopi * ks / L;
    double er = im / kappa, ei = -re / kappa;  // rho_k / (i kappa)
    for (int j = 0; j < n; j++) {
      int t = (int)(((int64_t)j * k) % n);
      E[j] += (er * cs[t] - ei * sn[t]) / n;
    }
  }
}

void wire_sorted_output(pic_handle *h);

// Cell-sorts the mixed-form markers (and their ids) into the alternate
// buffers and swaps them in.
int sort_mixed(pic_handle *h) {
  CUDA_TRY(h->timed_launch(3, [&] {
    es1d_mix_sort(h->cm, h->bm, h->bm_alt, h->ids, h->ids_alt, h->sort_hist, h->sort_blocks,
                  h->st);
  }));
  h->launches += 3;
  std::swap(h->bm.X, h->bm_alt.X);
  std::swap(h->bm.vh, h->bm_alt.vh);
  std::swap(h->bm.vl, h->bm_alt.vl);
  std::swap(h->ids, h->ids_alt);
  wire_sorted_output(h);
  return PIC_OK;
}

// Sort on write: pass E writes into the alternate arrays, which are swapped in
// after every step.
void wire_sorted_output(pic_handle *h) {
  Es1dMixBufs &bm = h->bm;
  if (h->cm.mode != 2) return;
  bm.Xo = h->bm_alt.X;
  bm.vho = h->bm_alt.vh;
  bm.vlo = h->bm_alt.vl;
  bm.ids = h->cfg.skip_ids ? nullptr : h->ids;
  bm.ido = h->cfg.skip_ids ? nullptr : h->ids_alt;
}

void swap_sorted_output(pic_handle *h) {
  Es1dMixBufs &bm = h->bm;
  std::swap(h->bm.X, h->bm_alt.X);
  std::swap(h->bm.vh, h->bm_alt.vh);
  std::swap(h->bm.vl, h->bm_alt.vl);
  if (!h->cfg.skip_ids) std::swap(h->ids, h->ids_alt);
  wire_sorted_output(h);
  (void)bm;
}

// Markers a tile copy of the mixed 1D passes takes in one launch on grids of up
// to kWideMaxNodes nodes: those of one wave of the wide launch (one
// 1024-thread block per SM, 32 copies a block, 4 markers per thread and
// trip, or kFusedThreads-thread blocks for the fused ESEC1 pass on the same
// grid, whichever is more), at least 2048.  Every launch of such a handle
// keeps to it, whatever its scheme, so that all modes round alike.
int64_t mixed_wide_pcnt(int64_t N, int nsm) {
  const int64_t ngroups = (N + 3) / 4;
  const int64_t grid = std::max<int64_t>(1, std::min<int64_t>((ngroups + 1023) / 1024, nsm));
  const int64_t trips = (ngroups + grid * 1024 - 1) / (grid * 1024);
  const int64_t trips_ec = (ngroups + grid * kFusedThreads - 1) / (grid * kFusedThreads);
  return std::max<int64_t>(2048, std::max(trips * 128, trips_ec * (kFusedThreads / 8)));
}

// Mixed form: constants, integer/float-pair state converted from the FP64
// staging arrays, j^{n,*} of the initial state.
int init_mixed(pic_handle *h, bool solve_e0) {
  const Es1dConst &c = h->c1;
  const SpeciesInfo &S = h->sp[0];
  const Es1dFp64Bufs &b = h->b1;
  Es1dMixConst &m = h->cm;
  m.nc = c.nc;
  m.order = c.order;
  m.scheme = c.scheme;
  m.remove_mean = c.remove_mean;
  m.gamma_on = c.gamma_on;
  m.n = h->N;
  m.L = c.L;
  m.h = c.h;
  m.dt = c.dt;
  // velocity scale: V units of (dt 2^31 / L) 2^kv, with room for 8x the
  // largest initial speed inside the 31-bit range
  unsigned long long *mx = nullptr;
  int rc;
  if ((rc = h->alloc(&mx, 1))) return rc;
  CUDA_TRY(cudaMemsetAsync(mx, 0, sizeof(unsigned long long), h->st));
  es1d_absmax(b.v, h->N, mx, h->ls, h->st);
  CUDA_TRY(cudaGetLastError());
  unsigned long long bits = 0;
  CUDA_TRY(cudaMemcpyAsync(&bits, mx, sizeof bits, cudaMemcpyDeviceToHost, h->st));
  CUDA_TRY(cudaStreamSynchronize(h->st));
  double vmax;
  memcpy(&vmax, &bits, sizeof vmax);
  double cx = c.dt * 2147483648.0 / c.L;
  double vcap = std::max(8.0 * vmax, 1e-6 * c.L / c.dt);
  int kv = (int)std::floor(std::log2(1073741824.0 / (cx * vcap)));
  // kv >= 1 keeps the half-step shift a plain rounded shift (the range check
  // on every V* reports speeds that no longer fit 31 bits)
  m.kv = std::min(24, std::max(1, kv));
  m.hround = 1 << (m.kv - 1);
  m.cxk = std::ldexp(cx, m.kv);
  m.mode = h->cfg.sort_period == 1 ? 2 : (h->cfg.sort_period > 1 ? 1 : 0);
  m.gamma64 = h->cfg.gamma_fp64;
  m.wide = m.mode == 0 && c.nc <= kWideMaxNodes;
  const int64_t ngroups = (h->N + 3) / 4;
  if (m.wide) {
    // one wave of 1024-thread blocks, one per SM (the per-copy marker count is
    // checked against the counters' bound below)
    const int64_t want = std::min<int64_t>((ngroups + 1023) / 1024, h->nsm);
    h->lmix = LaunchShape{(int)std::max<int64_t>(1, want), 1024};
    h->lmix_ec = LaunchShape{h->lmix.grid, kFusedThreads};
  } else {
    h->lmix = h->ls;
    h->lmix_ec = h->ls;
  }
  // ESEC1 in one launch per step (the fused pass) on this handle
  const bool fused = m.scheme == 1 && m.mode == 0 && !h->cfg.separate_passes && c.passes == 0;
  // Terms round(V* s / 2^r) are below 2^T = 2^(54 - r).  At most pcnt markers
  // add into one tile copy of a block in a launch.  Its split counters hold the
  // low b = 32 - lg bits of each term (lg = ceil(log2 pcnt): pcnt 2^b <= 2^32)
  // and the signed rest (pcnt 2^(T-b) <= 2^31), so T <= 63 - 2 lg; the signed
  // share comes from the high word of V* s (r + b >= 32: T <= 22 + b); the
  // sorted modes' warp sums take 4 terms a lane in 20-bit halves (T <= 44);
  // the int64 grid sums need N 2^T < 2^62.  Every launch of a handle keeps to
  // the same pcnt: on grids of up to kWideMaxNodes nodes the markers a copy
  // takes in one wave of the wide launch (mixed_wide_pcnt, at least 2048; the
  // batched launch takes at most 16 trips of 128 markers a copy, the sorted
  // modes' single-copy launch pcnt markers a 512-thread block), on larger
  // grids the markers of a 512-thread block of the single-copy launch.  One r
  // and b for every mode keep the results independent of the marker order.
  int64_t pcnt;
  if (c.nc <= kWideMaxNodes) {
    pcnt = mixed_wide_pcnt(h->N, h->nsm);
  } else {
    const int64_t threads = (int64_t)h->ls.grid * 512;
    const int64_t trips = (ngroups + threads - 1) / threads;
    pcnt = std::max<int64_t>(2048, trips * 512 * 4);
  }
  if (m.wide) {
    const int64_t wthreads = (int64_t)h->lmix.grid * 1024;
    const int64_t ethreads = (int64_t)h->lmix_ec.grid * kFusedThreads;
    if (((ngroups + wthreads - 1) / wthreads) * 128 > pcnt ||
        ((ngroups + ethreads - 1) / ethreads) * (kFusedThreads / 8) > pcnt)
      return fail(PIC_ERR_UNSUPPORTED, "pic_init: internal launch size of the wide passes");
  } else if (c.nc <= kWideMaxNodes && h->lmix.grid * pcnt < 4 * ngroups) {
    return fail(PIC_ERR_UNSUPPORTED, "pic_init: internal launch size for the sorted modes");
  }
  int lg = 0;
  while (((int64_t)1 << lg) < pcnt) lg++;
  m.split = 32 - lg;
  int T = std::min(std::min(63 - 2 * lg, 22 + m.split), 44);
  int bitlen = 0;
  while (bitlen < 62 && ((int64_t)1 << bitlen) <= h->N) bitlen++;
  T = std::min(T, 62 - bitlen);
  m.rshift = 54 - T;
  if (m.rshift > 31 || m.rshift + m.split < 32)
    return fail(PIC_ERR_UNSUPPORTED, "pic_init: %lld markers need a deposit shift of %d",
                (long long)h->N, m.rshift);
  m.rnd = 1ll << (m.rshift - 1);
  m.lomask = (1u << m.split) - 1u;
  m.hishift = m.rshift + m.split - 32;
  m.jscale = S.q * S.w0 * std::ldexp(1.0, m.rshift) / (c.h * m.cxk * 8388608.0);
  m.ke_scale = 0.5 * S.m * S.w0 / (m.cxk * m.cxk);
  m.e_scale = 0.5 * c.dt * S.q / S.m * m.cxk;
  m.kick = c.dt * S.q / S.m * m.cxk;
  m.kick_jhalf = ff_from_double(m.kick * 0.5 * c.dt * m.jscale);
  m.inv_nc = ff_from_double(1.0 / c.nc);
  m.c_jstar = (float)(m.e_scale * 0.5 * c.dt * m.jscale);
  m.passes = c.passes;
  CUDA_TRY(es1d_mix_prepare(m));
  Es1dMixBufs &bm = h->bm;
  bm.filt = nullptr;
  if (m.passes > 0) {
    // the stencils of F^p and F^2p: C(2p, p + k) / 4^p, C(4p, 2p + k) / 16^p
    // (exact doubles, exact float pairs)
    std::vector<float2> w;
    for (int n : {2 * m.passes, 4 * m.passes}) {
      double cnk = 1.0;
      const double scale = std::ldexp(1.0, -n);
      for (int k = 0; k <= n; k++) {
        const ff f = ff_from_double(cnk * scale);
        w.push_back(make_float2(f.hi, f.lo));
        cnk = cnk * (n - k) / (k + 1);
      }
    }
    float2 *filt = nullptr;
    if ((rc = h->alloc(&filt, w.size()))) return rc;
    CUDA_TRY(cudaMemcpyAsync(filt, w.data(), sizeof(float2) * w.size(), cudaMemcpyHostToDevice,
                             h->st));
    CUDA_TRY(cudaStreamSynchronize(h->st));
    bm.filt = filt;
  }
  size_t npad = (size_t)((h->N + 3) / 4 * 4);
  if ((rc = h->alloc(&bm.X, npad)) || (rc = h->alloc(&bm.vh, npad)) || (rc = h->alloc(&bm.vl, npad)) ||
      (rc = h->alloc(&bm.Vs, npad)))
    return rc;
  for (int k = 0; k < 2; k++)
    if ((rc = h->alloc(&bm.J1[k], (size_t)c.nc * kJStride)) ||
        (rc = h->alloc(&bm.J2[k], (size_t)c.nc * kJStride)))
      return rc;
  CUDA_TRY(cudaMemsetAsync(bm.X, 0, sizeof(uint32_t) * npad, h->st));
  CUDA_TRY(cudaMemsetAsync(bm.vh, 0, sizeof(float) * npad, h->st));
  CUDA_TRY(cudaMemsetAsync(bm.vl, 0, sizeof(float) * npad, h->st));
  for (int k = 0; k < 2; k++) {
    bm.E[k] = b.E[k];
    if ((rc = h->alloc(&bm.Ek[k], (size_t)c.nc))) return rc;
    CUDA_TRY(cudaMemsetAsync(bm.J1[k], 0, sizeof(long long) * c.nc * kJStride, h->st));
    CUDA_TRY(cudaMemsetAsync(bm.J2[k], 0, sizeof(long long) * c.nc * kJStride, h->st));
  }
  bm.ke_part = b.ke_part;
  bm.fallback = b.fallback;
  bm.te = b.te;
  bm.we = b.we;
  // grid totals: [4] for J1[0], J1[1], J2[0], J2[1], with room on either side
  // (a fused ESEC1 step addresses the totals of its three current buffers)
  if ((rc = h->alloc(&h->jtot_base, 8))) return rc;
  CUDA_TRY(cudaMemsetAsync(h->jtot_base, 0, sizeof(long long) * 8, h->st));
  bm.Jtot = h->jtot_base + 4;
  h->fused = fused;
  h->primed = false;
  if (h->fused && ((rc = h->alloc(&h->ke_alt, (size_t)h->ls.grid)) ||
                   (rc = h->alloc(&h->we_alt, (size_t)h->ls.grid))))
    return rc;
  if ((rc = h->alloc(&bm.we_part, (size_t)h->ls.grid))) return rc;
  CUDA_TRY(cudaMemsetAsync(bm.we_part, 0, sizeof(double) * h->ls.grid, h->st));
  bm.err = b.err;
  if (h->cfg.sort_period > 0) {
    Es1dMixBufs &alt = h->bm_alt;
    alt = bm;
    if ((rc = h->alloc(&alt.X, npad)) || (rc = h->alloc(&alt.vh, npad)) ||
        (rc = h->alloc(&alt.vl, npad)) || (rc = h->alloc(&h->ids_alt, (size_t)h->N)))
      return rc;
    CUDA_TRY(cudaMemsetAsync(alt.X, 0, sizeof(uint32_t) * npad, h->st));
    CUDA_TRY(cudaMemsetAsync(alt.vh, 0, sizeof(float) * npad, h->st));
    CUDA_TRY(cudaMemsetAsync(alt.vl, 0, sizeof(float) * npad, h->st));
    h->sort_blocks = es1d_mix_sort_blocks(m, h->nsm);
    if ((rc = h->alloc(&h->sort_hist, (size_t)c.nc * (h->sort_blocks + 1)))) return rc;
    if (m.mode == 2) {
      // sort on write: pass E's destination is the alternate set; key counts
      // are kept per pass block
      if ((rc = h->alloc(&bm.H, (size_t)2 * c.nc * h->ls.grid)) || (rc = h->alloc(&bm.T, 2 * (size_t)c.nc)))
        return rc;
    }
  }
  es1d_mix_from_fp64(m, b.x, b.v, bm, h->ls, h->st);
  CUDA_TRY(cudaGetLastError());
  if (solve_e0) {
    // Gauss's law from the exact integer charge of the stored markers (the
    // same weights every later deposit uses; independent of marker order)
    long long *cnt = bm.J2[1];
    es1d_mix_charge(m, bm, cnt, h->ls, h->st);
    CUDA_TRY(cudaGetLastError());
    std::vector<long long> ci(c.nc);
    CUDA_TRY(cudaMemcpyAsync(ci.data(), cnt, sizeof(long long) * c.nc, cudaMemcpyDeviceToHost, h->st));
    CUDA_TRY(cudaStreamSynchronize(h->st));
    std::vector<double> r(c.nc), e, t(c.nc);
    for (int i = 0; i < c.nc; i++) r[i] = S.q * S.w0 / c.h * std::ldexp((double)ci[i], -23);
    // with the filter inside the scheme, Gauss's law of the filtered charge
    for (int k = 0; k < m.passes; k++) {
      for (int i = 0; i < c.nc; i++)
        t[i] = 0.25 * (r[(i + c.nc - 1) % c.nc] + 2.0 * r[i] + r[(i + 1) % c.nc]);
      r.swap(t);
    }
    poisson_1d_host(r, c.L, e);
    CUDA_TRY(cudaMemcpyAsync(b.E[0], e.data(), sizeof(double) * c.nc, cudaMemcpyHostToDevice, h->st));
    CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(long long) * c.nc, h->st));
    CUDA_TRY(cudaStreamSynchronize(h->st));
  }
  if (h->cfg.sort_period > 0) {
    if ((rc = sort_mixed(h))) return rc;
  }
  wire_sorted_output(h);
  es1d_mix_set_ek(m, bm, (int)(h->steps_done & 1), h->st);
  if (m.scheme == 2) {
    es1d_mix_deposit_initial(m, bm, (int)(h->steps_done & 1), m.wide ? h->lmix : h->ls, h->st);
    CUDA_TRY(cudaGetLastError());
  }
  return PIC_OK;
}

int init_es1d(pic_handle *h, const pic_species *species, const double *E0) {
  const pic_config &cfg = h->cfg;
  int nc = (int)cfg.grid.n[0];
  Es1dConst &c = h->c1;
  c.nc = nc;
  c.order = cfg.shape_order;
  c.scheme = cfg.scheme;
  c.remove_mean = cfg.remove_mean;
  c.gamma_on = cfg.gamma_on;
  c.passes = cfg.binomial_passes;
  c.nsp = h->nsp;
  c.n_total = h->N;
  c.L = cfg.grid.L[0];
  c.h = c.L / nc;
  c.inv_h = nc / c.L;
  c.dt = cfg.dt;
  for (int s = 0; s < h->nsp; s++) {
    const SpeciesInfo &S = h->sp[s];
    c.sp_end[s] = S.offset + S.n;
    c.qm[s] = S.q / S.m;
    c.qw_h[s] = S.q * S.w0 / c.h;
    c.q_h[s] = S.q / c.h;
    c.half_mw[s] = 0.5 * S.m * S.w0;
    c.half_m[s] = 0.5 * S.m;
  }
  for (int s = h->nsp; s < kMaxSpecies; s++) c.sp_end[s] = h->N;

  CUDA_TRY(es1d_fp64_prepare(c));
  Es1dFp64Bufs &b = h->b1;
  int rc;
  if ((rc = h->alloc(&b.x, h->N)) || (rc = h->alloc(&b.v, h->N)) ||
      (!h->mixed && (rc = h->alloc(&b.vs, h->N))))
    return rc;
  b.sw = nullptr;
  b.si = nullptr;
  b.sws = nullptr;
  b.sis = nullptr;
  if (!h->mixed && ((rc = h->alloc(&b.sw, (size_t)(c.order + 1) * h->N)) ||
                    (rc = h->alloc(&b.si, h->N))))
    return rc;
  // ESEC2: the shape at x* from pass E (or the initial deposit) to pass C
  if (!h->mixed && c.scheme == 2 &&
      ((rc = h->alloc(&b.sws, (size_t)(c.order + 1) * h->N)) || (rc = h->alloc(&b.sis, h->N))))
    return rc;
  b.w = nullptr;
  if (h->weighted && (rc = h->alloc(&b.w, h->N))) return rc;
  for (int k = 0; k < 2; k++)
    if ((rc = h->alloc(&b.E[k], nc)) || (rc = h->alloc(&b.J1[k], nc)) ||
        (rc = h->alloc(&b.J2[k], nc)))
      return rc;
  if ((rc = h->alloc(&b.ke_part, h->ls.grid)) || (rc = h->alloc(&h->energy_part, h->ls.grid)) ||
      (rc = h->alloc(&b.fallback, kStepsCap)) ||
      (rc = h->alloc(&b.te, kStepsCap)) || (rc = h->alloc(&b.we, 1)) ||
      (rc = h->alloc(&b.err, 1)) || (rc = h->alloc(&h->ids, h->N)))
    return rc;
  CUDA_TRY(cudaMemsetAsync(b.err, 0, sizeof(unsigned), h->st));
  for (int s = 0; s < h->nsp; s++) {
    const SpeciesInfo &S = h->sp[s];
    const pic_species &in = species[s];
    CUDA_TRY(cudaMemcpyAsync(b.x + S.offset, in.x, sizeof(double) * S.n, cudaMemcpyDefault, h->st));
    CUDA_TRY(cudaMemcpyAsync(b.v + S.offset, in.v, sizeof(double) * S.n, cudaMemcpyDefault, h->st));
    if (h->weighted) {
      if (in.w) {
        CUDA_TRY(cudaMemcpyAsync(b.w + S.offset, in.w, sizeof(double) * S.n, cudaMemcpyDefault, h->st));
      } else {
        std::vector<double> tmp((size_t)S.n, S.w0);
        CUDA_TRY(cudaMemcpyAsync(b.w + S.offset, tmp.data(), sizeof(double) * S.n,
                                 cudaMemcpyHostToDevice, h->st));
        CUDA_TRY(cudaStreamSynchronize(h->st));
      }
    }
  }
  std::vector<int64_t> ids((size_t)h->N);
  for (int64_t s = 0; s < h->nsp; s++)
    for (int64_t p = 0; p < h->sp[s].n; p++) ids[(size_t)(h->sp[s].offset + p)] = p;
  CUDA_TRY(cudaMemcpyAsync(h->ids, ids.data(), sizeof(int64_t) * h->N, cudaMemcpyHostToDevice, h->st));
  validate_1d_kernel<<<h->ls.grid, 256, 0, h->st>>>(b.x, b.v, h->N, c.L, b.err);
  CUDA_TRY(cudaGetLastError());
  if ((rc = check_flags(h, "pic_init"))) return rc;

  for (int k = 0; k < 2; k++) {
    CUDA_TRY(cudaMemsetAsync(b.J1[k], 0, sizeof(double) * nc, h->st));
    CUDA_TRY(cudaMemsetAsync(b.J2[k], 0, sizeof(double) * nc, h->st));
    CUDA_TRY(cudaMemsetAsync(b.E[k], 0, sizeof(double) * nc, h->st));
  }
  if (E0 || h->mixed) {
    std::vector<double> e(nc, 0.0);
    if (E0) {
    CUDA_TRY(cudaMemcpyAsync(e.data(), E0, sizeof(double) * nc, cudaMemcpyDefault, h->st));
    CUDA_TRY(cudaStreamSynchronize(h->st));
    for (int i = 0; i < nc; i++)
      if (!std::isfinite(e[i])) return fail(PIC_ERR_NONFINITE, "pic_init: E0[%d] is not finite", i);
    }
    CUDA_TRY(cudaMemcpyAsync(b.E[0], e.data(), sizeof(double) * nc, cudaMemcpyHostToDevice, h->st));
  } else {
    double *rho = b.J2[1];  // scratch, cleared again below
    es1d_fp64_charge(c, b.x, b.w, rho, h->ls, h->st);
    CUDA_TRY(cudaGetLastError());
    std::vector<double> r(nc), e, t(nc);
    CUDA_TRY(cudaMemcpyAsync(r.data(), rho, sizeof(double) * nc, cudaMemcpyDeviceToHost, h->st));
    CUDA_TRY(cudaStreamSynchronize(h->st));
    // with filtering inside the scheme, Gauss's law of the filtered charge
    // (the field the filtered Ampere updates keep consistent)
    for (int k = 0; k < c.passes; k++) {
      for (int i = 0; i < nc; i++)
        t[i] = 0.25 * (r[(i + nc - 1) % nc] + 2.0 * r[i] + r[(i + 1) % nc]);
      r.swap(t);
    }
    poisson_1d_host(r, c.L, e);
    CUDA_TRY(cudaMemcpyAsync(b.E[0], e.data(), sizeof(double) * nc, cudaMemcpyHostToDevice, h->st));
    CUDA_TRY(cudaMemsetAsync(rho, 0, sizeof(double) * nc, h->st));
  }
  if (h->mixed) {
    if ((rc = init_mixed(h, E0 == nullptr))) return rc;
  } else if (c.scheme == 2) {
    es1d_fp64_deposit_initial(c, b, 0, h->ls, h->st);
    CUDA_TRY(cudaGetLastError());
  }
  CUDA_TRY(cudaStreamSynchronize(h->st));
  return check_flags(h, "pic_init");
}

// Copies the FP64 1D state (x, v and E of the current step) to or from a
// packed [2N + nc] device buffer.
cudaError_t state_copy(pic_handle *h, double *buf, bool save) {
  const size_t N = (size_t)h->N, nc = (size_t)h->c1.nc;
  double *E = h->b1.E[h->steps_done & 1];
  double *dst[3] = {buf, buf + N, buf + 2 * N}, *src[3] = {h->b1.x, h->b1.v, E};
  const size_t cnt[3] = {N, N, nc};
  for (int k = 0; k < 3; k++) {
    cudaError_t e = save ? cudaMemcpyAsync(dst[k], src[k], sizeof(double) * cnt[k],
                                           cudaMemcpyDeviceToDevice, h->st)
                         : cudaMemcpyAsync(src[k], dst[k], sizeof(double) * cnt[k],
                                           cudaMemcpyDeviceToDevice, h->st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Re-establishes the invariants of the step sequence after a state change:
// zero currents and, for ESEC2, j^{n,*} of the new state.
int restart_es1d(pic_handle *h, bool particles_changed) {
  Es1dFp64Bufs &b = h->b1;
  int par = (int)(h->steps_done & 1);
  if (h->mixed) {
    Es1dMixBufs &bm = h->bm;
    for (int k = 0; k < 2; k++) {
      CUDA_TRY(cudaMemsetAsync(bm.J1[k], 0, sizeof(long long) * h->cm.nc * kJStride, h->st));
      CUDA_TRY(cudaMemsetAsync(bm.J2[k], 0, sizeof(long long) * h->cm.nc * kJStride, h->st));
    }
    CUDA_TRY(cudaMemsetAsync(h->jtot_base, 0, sizeof(long long) * 8, h->st));
    h->primed = false;
    // the FP64 staging arrays hold the new markers only after pic_set_particles
    if (particles_changed) es1d_mix_from_fp64(h->cm, b.x, b.v, bm, h->ls, h->st);
    es1d_mix_set_ek(h->cm, bm, par, h->st);
    if (h->cm.scheme == 2)
      es1d_mix_deposit_initial(h->cm, bm, par, h->cm.wide ? h->lmix : h->ls, h->st);
    CUDA_TRY(cudaGetLastError());
    return check_flags(h, "pic_set_*");
  }
  for (int k = 0; k < 2; k++) {
    CUDA_TRY(cudaMemsetAsync(b.J1[k], 0, sizeof(double) * h->c1.nc, h->st));
    CUDA_TRY(cudaMemsetAsync(b.J2[k], 0, sizeof(double) * h->c1.nc, h->st));
  }
  if (h->c1.scheme == 2) es1d_fp64_deposit_initial(h->c1, b, par, h->ls, h->st);
  CUDA_TRY(cudaGetLastError());
  validate_1d_kernel<<<h->ls.grid, 256, 0, h->st>>>(b.x, b.v, h->N, h->c1.L, b.err);
  CUDA_TRY(cudaGetLastError());
  return check_flags(h, "pic_set_*");
}

// Yee state change: validate markers, B^{n+1/2} from (E^n, B^{n-1/2}), j^{n,*}.
// The mixed form takes its markers from the FP64 staging arrays only when
// they changed (markers_changed); otherwise its own state stays as it is.
int restart_em2d(pic_handle *h, bool markers_changed = true) {
  Em2dBufs &b = h->be;
  const int64_t nc3 = 3 * (int64_t)h->ce.nx * h->ce.ny;
  if (markers_changed || !h->mixed) {
    em2d_validate_kernel<<<h->lp.grid, 256, 0, h->st>>>(b.x, b.y, b.vx, b.vy, b.vz, h->N,
                                                         h->ce.Lx, h->ce.Ly, b.err);
    CUDA_TRY(cudaGetLastError());
  }
  em2d_fp64_bhalf(h->ce, b.B, b.E, b.Bp, h->lg, h->st);
  if (h->mixed) {
    Em2dMixBufs &mb = h->bme;
    if (markers_changed) em2dm_from_fp64(h->cme, mb, b, h->lp, h->st);
    CUDA_TRY(cudaMemsetAsync(mb.J1, 0, sizeof(long long) * nc3, h->st));
    CUDA_TRY(cudaMemsetAsync(mb.J2, 0, sizeof(long long) * nc3, h->st));
    if (h->ce.scheme == 2) em2dm_deposit_initial(h->cme, mb, h->lp, h->st);
  } else {
    CUDA_TRY(cudaMemsetAsync(b.J1, 0, sizeof(double) * nc3, h->st));
    CUDA_TRY(cudaMemsetAsync(b.J2, 0, sizeof(double) * nc3, h->st));
    if (h->ce.scheme == 2) em2d_fp64_deposit_initial(h->ce, b, h->lp, h->st);
  }
  CUDA_TRY(cudaGetLastError());
  return check_flags(h, "pic_init/pic_set_*");
}

// Mixed form of the 2D3V path: the velocity scale from the largest initial
// speed, the deposit shift from the marker count, the per-marker state and
// the float tables (the FP64 staging arrays hold the initial markers).
int init_em2d_mixed(pic_handle *h) {
  const Em2dConst &c = h->ce;
  const SpeciesInfo &S = h->sp[0];
  Em2dMixConst &m = h->cme;
  Em2dMixBufs &mb = h->bme;
  m.nx = c.nx;
  m.ny = c.ny;
  m.order = c.order;
  m.scheme = c.scheme;
  m.gamma_on = c.gamma_on;
  m.n = h->N;
  m.L = c.Lx;
  m.dt = c.dt;
  unsigned long long *mx = nullptr;
  int rc;
  if ((rc = h->alloc(&mx, 1))) return rc;
  CUDA_TRY(cudaMemsetAsync(mx, 0, sizeof(unsigned long long), h->st));
  em2dm_absmax(h->be, h->N, mx, h->lp, h->st);
  CUDA_TRY(cudaGetLastError());
  unsigned long long bits = 0;
  CUDA_TRY(cudaMemcpyAsync(&bits, mx, sizeof bits, cudaMemcpyDeviceToHost, h->st));
  CUDA_TRY(cudaStreamSynchronize(h->st));
  double vmax;
  memcpy(&vmax, &bits, sizeof vmax);
  // V units of (dt 2^31 / L) 2^kv, with room for 8x the largest initial speed
  // inside the 31-bit range; kv >= 1 keeps the half-step shift a rounded shift
  const double cx = c.dt * 2147483648.0 / m.L;
  const double vcap = std::max(8.0 * vmax, 1e-6 * m.L / c.dt);
  const int kv = (int)std::floor(std::log2(1073741824.0 / (cx * vcap)));
  m.kv = std::min(24, std::max(1, kv));
  m.hround = 1 << (m.kv - 1);
  m.cxk = std::ldexp(cx, m.kv);
  // terms round(V* s_x s_y / 2^r) are below 2^(77 - r); with N < 2^bitlen
  // markers every node sum stays below 2^62 for r = bitlen + 15 (and r >= 32
  // for the split product in the kernels)
  int bitlen = 0;
  while (bitlen < 62 && ((int64_t)1 << bitlen) <= h->N) bitlen++;
  m.rshift = std::max(32, bitlen + 15);
  m.rnd = 1ll << (m.rshift - 1);
  const double qm = S.q / S.m;
  m.jscale = S.q * S.w0 * std::ldexp(1.0, m.rshift - 46) / (c.area * m.cxk);
  m.ke_scale = 0.5 * S.m * S.w0 / (m.cxk * m.cxk);
  m.e_half = 0.5 * c.dt * qm * m.cxk;
  m.t_half = 0.5 * c.dt * qm;
  m.kick = c.dt * qm * m.cxk;
  m.m_full = c.dt * qm;
  const size_t n = (size_t)h->N, nc3 = 3 * (size_t)c.nx * c.ny;
  if ((rc = h->alloc(&mb.X, n)) || (rc = h->alloc(&mb.Y, n)) || (rc = h->alloc(&mb.J1, nc3)) ||
      (rc = h->alloc(&mb.J2, nc3)) || (rc = h->alloc(&mb.T1, 2 * nc3)) ||
      (rc = h->alloc(&mb.T2, nc3)) || (rc = h->alloc(&mb.B2, nc3)))
    return rc;
  for (int d = 0; d < 3; d++)
    if ((rc = h->alloc(&mb.vh[d], n)) || (rc = h->alloc(&mb.vl[d], n)) ||
        (rc = h->alloc(&mb.Vs[d], n)))
      return rc;
  mb.ke_part = h->be.ke_part;
  mb.fallback = h->be.fallback;
  mb.err = h->be.err;
  m.sorted = h->cfg.sort_period > 0;
  if (m.sorted) {
    // markers written in quarter-cell order every sort_period steps (ids
    // follow them); the counts stay zero between sorts
    Em2dMixBufs &alt = h->bme_alt;
    alt = mb;
    const size_t ncnt = em2dm_sort_count_words(c.nx, c.ny);
    if ((rc = h->alloc(&alt.X, n)) || (rc = h->alloc(&alt.Y, n)) ||
        (rc = h->alloc(&h->ids_alt, n)) || (rc = h->alloc(&h->sort2_cnt, ncnt)) ||
        (rc = h->alloc(&h->sort2_off, 4 * (size_t)c.nx * c.ny)))
      return rc;
    for (int d = 0; d < 3; d++)
      if ((rc = h->alloc(&alt.vh[d], n)) || (rc = h->alloc(&alt.vl[d], n))) return rc;
    CUDA_TRY(cudaMemsetAsync(h->sort2_cnt, 0, sizeof(unsigned) * ncnt, h->st));
  }
  return PIC_OK;
}

// After pass E wrote the mixed 2D markers (and their ids) in quarter-cell
// order into the alternate arrays: swaps them in.
void swap_em2d_sorted(pic_handle *h) {
  Em2dMixBufs &a = h->bme, &b = h->bme_alt;
  std::swap(a.X, b.X);
  std::swap(a.Y, b.Y);
  for (int d = 0; d < 3; d++) {
    std::swap(a.vh[d], b.vh[d]);
    std::swap(a.vl[d], b.vl[d]);
  }
  if (!h->cfg.skip_ids) std::swap(h->ids, h->ids_alt);
}

// 2D3V Yee: constants, SoA markers, fields E^0, B^{-1/2} and B^{1/2}, j^{0,*}.
int init_em2d(pic_handle *h, const pic_species *species, const double *E0, const double *B0) {
  const pic_config &cfg = h->cfg;
  Em2dConst &c = h->ce;
  Em2dBufs &b = h->be;
  c.nx = (int)cfg.grid.n[0];
  c.ny = (int)cfg.grid.n[1];
  c.order = cfg.shape_order;
  c.cc = cfg.charge_conserving;
  c.scheme = cfg.scheme;
  c.gamma_on = cfg.gamma_on;
  c.nsp = h->nsp;
  c.n_total = h->N;
  c.Lx = cfg.grid.L[0];
  c.Ly = cfg.grid.L[1];
  c.inv_hx = c.nx / c.Lx;
  c.inv_hy = c.ny / c.Ly;
  c.dt = cfg.dt;
  c.c2 = cfg.c * cfg.c;
  c.area = (c.Lx / c.nx) * (c.Ly / c.ny);
  for (int s = 0; s < h->nsp; s++) {
    const SpeciesInfo &S = h->sp[s];
    c.sp_end[s] = S.offset + S.n;
    c.qm[s] = S.q / S.m;
    c.qw_a[s] = S.q * S.w0 / c.area;
    c.q_a[s] = S.q / c.area;
    c.half_mw[s] = 0.5 * S.m * S.w0;
    c.half_m[s] = 0.5 * S.m;
  }
  for (int s = h->nsp; s < kMaxSpecies; s++) c.sp_end[s] = h->N;
  const int64_t nc3 = 3 * (int64_t)c.nx * c.ny;
  h->lp.block = 256;
  h->lp.grid = (int)std::max<int64_t>(1, std::min<int64_t>((h->N + 255) / 256, (int64_t)h->nsm * 4));
  h->lg.block = 256;
  h->lg.grid = (int)std::max<int64_t>(1, std::min<int64_t>((nc3 + 255) / 256, (int64_t)h->nsm * 4));
  int rc;
  if ((rc = h->alloc(&b.x, h->N)) || (rc = h->alloc(&b.y, h->N)) || (rc = h->alloc(&b.vx, h->N)) ||
      (rc = h->alloc(&b.vy, h->N)) || (rc = h->alloc(&b.vz, h->N)))
    return rc;
  if (!h->mixed && ((rc = h->alloc(&b.vsx, h->N)) || (rc = h->alloc(&b.vsy, h->N)) ||
                    (rc = h->alloc(&b.vsz, h->N))))
    return rc;
  // the point-shape FP64 passes hand the shape at x^{n+1/2} from pass C to pass
  // E: 4 first nodes and 4 (order + 1) weights a marker
  b.sw = nullptr;
  b.si = nullptr;
  b.sws = nullptr;
  b.sis = nullptr;
  if (!h->mixed && !cfg.charge_conserving &&
      ((rc = h->alloc(&b.sw, (size_t)4 * (cfg.shape_order + 1) * h->N)) ||
       (rc = h->alloc(&b.si, (size_t)4 * h->N))))
    return rc;
  // ESEC2: the shape at x* from pass E (or the initial deposit) to pass C
  if (!h->mixed && !cfg.charge_conserving && cfg.scheme == 2 &&
      ((rc = h->alloc(&b.sws, (size_t)4 * (cfg.shape_order + 1) * h->N)) ||
       (rc = h->alloc(&b.sis, (size_t)4 * h->N))))
    return rc;
  b.w = nullptr;
  if (h->weighted && (rc = h->alloc(&b.w, h->N))) return rc;
  double **fields[] = {&b.E, &b.En, &b.Eh, &b.Es, &b.B, &b.Bp, &b.Bpp, &b.J1, &b.J2};
  for (double **f : fields)
    if ((rc = h->alloc(f, nc3))) return rc;
  // the mixed passes on sorted markers launch a block per 256 runs of markers
  h->lpm = h->mixed ? em2dm_pass_shape(h->N, cfg.sort_period > 0, h->lp) : h->lp;
  const size_t nke = std::max((size_t)h->lp.grid * kMaxSpecies, (size_t)h->lpm.grid);
  if ((rc = h->alloc(&b.ke_part, nke)) ||
      (rc = h->alloc(&h->energy_part, (size_t)h->lp.grid * kMaxSpecies)) ||
      (rc = h->alloc(&b.wf_part, 2 * (size_t)h->lg.grid)) || (rc = h->alloc(&b.fallback, kStepsCap)) ||
      (rc = h->alloc(&b.te, kStepsCap)) || (rc = h->alloc(&b.err, 1)) ||
      (rc = h->alloc(&h->ids, h->N)))
    return rc;
  // the 1D bookkeeping fields shared by the step/stats/error paths
  h->b1.err = b.err;
  h->b1.fallback = b.fallback;
  h->b1.te = b.te;
  CUDA_TRY(cudaMemsetAsync(b.err, 0, sizeof(unsigned), h->st));
  for (int s = 0; s < h->nsp; s++) {
    const SpeciesInfo &S = h->sp[s];
    const pic_species &in = species[s];
    double *dst[5] = {b.x, b.y, b.vx, b.vy, b.vz};
    for (int d = 0; d < 2; d++)
      CUDA_TRY(cudaMemcpyAsync(dst[d] + S.offset, in.x + d * S.n, sizeof(double) * S.n,
                               cudaMemcpyDefault, h->st));
    for (int d = 0; d < 3; d++)
      CUDA_TRY(cudaMemcpyAsync(dst[2 + d] + S.offset, in.v + d * S.n, sizeof(double) * S.n,
                               cudaMemcpyDefault, h->st));
    if (h->weighted) {
      if (in.w) {
        CUDA_TRY(cudaMemcpyAsync(b.w + S.offset, in.w, sizeof(double) * S.n, cudaMemcpyDefault, h->st));
      } else {
        std::vector<double> tmp((size_t)S.n, S.w0);
        CUDA_TRY(cudaMemcpyAsync(b.w + S.offset, tmp.data(), sizeof(double) * S.n,
                                 cudaMemcpyHostToDevice, h->st));
        CUDA_TRY(cudaStreamSynchronize(h->st));
      }
    }
  }
  std::vector<int64_t> ids((size_t)h->N);
  for (int s = 0; s < h->nsp; s++)
    for (int64_t p = 0; p < h->sp[s].n; p++) ids[(size_t)(h->sp[s].offset + p)] = p;
  CUDA_TRY(cudaMemcpyAsync(h->ids, ids.data(), sizeof(int64_t) * h->N, cudaMemcpyHostToDevice, h->st));
  CUDA_TRY(cudaMemsetAsync(b.E, 0, sizeof(double) * nc3, h->st));
  CUDA_TRY(cudaMemsetAsync(b.B, 0, sizeof(double) * nc3, h->st));
  if (E0) CUDA_TRY(cudaMemcpyAsync(b.E, E0, sizeof(double) * nc3, cudaMemcpyDefault, h->st));
  if (B0) CUDA_TRY(cudaMemcpyAsync(b.B, B0, sizeof(double) * nc3, cudaMemcpyDefault, h->st));
  CUDA_TRY(cudaStreamSynchronize(h->st));
  if (h->mixed && (rc = init_em2d_mixed(h))) return rc;
  return restart_em2d(h);
}

// Standard-PIC state change: validate markers, E^n from the charge and the
// half kick back to v^{n-1/2} (the velocities given are v^n).
int restart_std(pic_handle *h) {
  StdBufs &b = h->bs;
  validate_1d_kernel<<<h->lsd.grid, 256, 0, h->st>>>(b.x, b.v, h->N, h->cs.L, b.err);
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaMemsetAsync(b.rho, 0, sizeof(double) * kJSlices * h->cs.n, h->st));
  CUDA_TRY(cudaMemsetAsync(b.done, 0, sizeof(unsigned), h->st));
  std_start(h->cs, b, h->lsd, h->st);
  CUDA_TRY(cudaGetLastError());
  h->launches += 3;
  return check_flags(h, "pic_init/pic_set_*");
}

// Standard PIC, 1D1V: constants, SoA markers, tables, E^0 and v^{-1/2}.
int init_std(pic_handle *h, const pic_species *species) {
  const pic_config &cfg = h->cfg;
  StdConst &c = h->cs;
  StdBufs &b = h->bs;
  c.n = (int)cfg.grid.n[0];
  c.log2n = 0;
  while ((1 << c.log2n) < c.n) c.log2n++;
  c.order = cfg.shape_order;
  c.nsp = h->nsp;
  c.rt = std_tile_copies(c.n);
  c.passes = cfg.binomial_passes;
  c.n_total = h->N;
  c.L = cfg.grid.L[0];
  c.h = c.L / c.n;
  c.inv_h = c.n / c.L;
  c.dt = cfg.dt;
  for (int s = 0; s < h->nsp; s++) {
    const SpeciesInfo &S = h->sp[s];
    c.sp_end[s] = S.offset + S.n;
    c.qm[s] = S.q / S.m;
    c.qw_h[s] = S.q * S.w0 / c.h;
    c.q_h[s] = S.q / c.h;
    c.w0[s] = S.w0;
    c.half_m[s] = 0.5 * S.m;
  }
  for (int s = h->nsp; s < kMaxSpecies; s++) c.sp_end[s] = h->N;
  h->lsd.block = 256;
  h->lsd.grid = (int)std::max<int64_t>(1, std::min<int64_t>((h->N + 255) / 256, (int64_t)h->nsm * 2));
  const size_t n = (size_t)c.n;
  int rc;
  if ((rc = h->alloc(&b.x, h->N)) || (rc = h->alloc(&b.v, h->N))) return rc;
  b.w = nullptr;
  if (h->weighted && (rc = h->alloc(&b.w, h->N))) return rc;
  if ((rc = h->alloc(&b.E, n)) || (rc = h->alloc(&b.rho, kJSlices * n)) ||
      (rc = h->alloc(&b.tw, n / 2)) || (rc = h->alloc(&b.g, n / 2 + 1)) ||
      (rc = h->alloc(&b.ke_part, (size_t)h->lsd.grid)) || (rc = h->alloc(&b.done, 1)) ||
      (rc = h->alloc(&b.fallback, kStepsCap)) || (rc = h->alloc(&b.te, kStepsCap)) ||
      (rc = h->alloc(&b.err, 1)) || (rc = h->alloc(&h->ids, h->N)) ||
      (rc = h->alloc(&h->std_part, (size_t)h->lsd.grid * h->nsp + 1)))
    return rc;
  h->b1.err = b.err;
  h->b1.fallback = b.fallback;
  h->b1.te = b.te;
  CUDA_TRY(cudaMemsetAsync(b.err, 0, sizeof(unsigned), h->st));
  CUDA_TRY(std_prepare(c, b, h->st));
  h->launches += 1;
  for (int s = 0; s < h->nsp; s++) {
    const SpeciesInfo &S = h->sp[s];
    const pic_species &in = species[s];
    CUDA_TRY(cudaMemcpyAsync(b.x + S.offset, in.x, sizeof(double) * S.n, cudaMemcpyDefault, h->st));
    CUDA_TRY(cudaMemcpyAsync(b.v + S.offset, in.v, sizeof(double) * S.n, cudaMemcpyDefault, h->st));
    if (h->weighted) {
      if (in.w) {
        CUDA_TRY(cudaMemcpyAsync(b.w + S.offset, in.w, sizeof(double) * S.n, cudaMemcpyDefault, h->st));
      } else {
        std::vector<double> tmp((size_t)S.n, S.w0);
        CUDA_TRY(cudaMemcpyAsync(b.w + S.offset, tmp.data(), sizeof(double) * S.n,
                                 cudaMemcpyHostToDevice, h->st));
        CUDA_TRY(cudaStreamSynchronize(h->st));
      }
    }
  }
  std::vector<int64_t> ids((size_t)h->N);
  for (int s = 0; s < h->nsp; s++)
    for (int64_t p = 0; p < h->sp[s].n; p++) ids[(size_t)(h->sp[s].offset + p)] = p;
  CUDA_TRY(cudaMemcpyAsync(h->ids, ids.data(), sizeof(int64_t) * h->N, cudaMemcpyHostToDevice, h->st));
  CUDA_TRY(cudaStreamSynchronize(h->st));
  return restart_std(h);
}

// 1D2V spectral state change: validate markers, j^{n,*} and the half step.
// 1D2V state change: validate markers, j^{n,*} and the half step (E*, B*).
// The mixed form takes its markers from the FP64 staging arrays only when
// they changed.
int restart_em1d(pic_handle *h, bool markers_changed = true) {
  Em1dBufs &b = h->b1e;
  const int n = h->c1e.n;
  if (markers_changed || !h->mixed) {
    em1d_validate_kernel<<<h->le.grid, 256, 0, h->st>>>(b.y, b.vx, b.vy, h->N, h->c1e.L, b.err);
    CUDA_TRY(cudaGetLastError());
  }
  CUDA_TRY(cudaMemsetAsync(b.J1, 0, sizeof(double) * kJSlices * 2 * n, h->st));
  CUDA_TRY(cudaMemsetAsync(b.J2, 0, sizeof(double) * kJSlices * 2 * n, h->st));
  CUDA_TRY(cudaMemsetAsync(b.done, 0, sizeof(unsigned) * 2, h->st));
  if (h->mixed) {
    const Em1dMixBufs &mb = h->b1m;
    CUDA_TRY(cudaMemsetAsync(mb.J1, 0, sizeof(long long) * 2 * n, h->st));
    CUDA_TRY(cudaMemsetAsync(mb.J2, 0, sizeof(long long) * 2 * n, h->st));
    if (markers_changed) em1m_from_fp64(h->c1e, b, h->c1m, mb, h->le, h->st);
    em1m_start(h->c1e, b, h->c1m, mb, h->le, h->st);
    h->launches += 1 + (markers_changed ? 2 : 1) + 2 * (h->c1e.scheme == 2);
  } else {
    em1d_start(h->c1e, b, h->le, h->st);
    h->launches += 2 + (h->c1e.scheme == 2);
  }
  CUDA_TRY(cudaGetLastError());
  return check_flags(h, "pic_init/pic_set_*");
}

// Mixed form of the 1D2V path: the velocity scale from the largest initial
// speed, the deposit shift from the markers per tile copy, the per-marker
// state (the FP64 staging arrays hold the initial markers).
int init_em1d_mixed(pic_handle *h) {
  const Em1dConst &c = h->c1e;
  const SpeciesInfo &S = h->sp[0];
  Em1dMixConst &m = h->c1m;
  Em1dMixBufs &mb = h->b1m;
  m.n = c.n;
  m.order = c.order;
  m.scheme = c.scheme;
  m.gamma_on = c.gamma_on;
  m.rt = em1m_tile_copies(c.n);
  m.N = h->N;
  m.L = c.L;
  m.dt = c.dt;
  unsigned long long *mx = nullptr;
  int rc;
  if ((rc = h->alloc(&mx, 1))) return rc;
  CUDA_TRY(cudaMemsetAsync(mx, 0, sizeof(unsigned long long), h->st));
  em1m_absmax(h->b1e, h->N, mx, h->le, h->st);
  CUDA_TRY(cudaGetLastError());
  unsigned long long bits = 0;
  CUDA_TRY(cudaMemcpyAsync(&bits, mx, sizeof bits, cudaMemcpyDeviceToHost, h->st));
  CUDA_TRY(cudaStreamSynchronize(h->st));
  double vmax;
  memcpy(&vmax, &bits, sizeof vmax);
  // V units of (dt 2^31 / L) 2^kv, with room for 8x the largest initial speed
  // inside the 31-bit range; kv >= 1 keeps the half-step shift a rounded shift
  const double cx = c.dt * 2147483648.0 / c.L;
  const double vcap = std::max(8.0 * vmax, 1e-6 * c.L / c.dt);
  const int kv = (int)std::floor(std::log2(1073741824.0 / (cx * vcap)));
  m.kv = std::min(24, std::max(1, kv));
  m.hround = 1 << (m.kv - 1);
  m.cxk = std::ldexp(cx, m.kv);
  // Terms round(V* s / 2^r) are below 2^T = 2^(54 - r).  pcnt markers add into
  // one tile copy (the threads that share it, each over its grid-stride
  // trips): its split counters need pcnt 2^16 < 2^32 and pcnt 2^(T-16) < 2^31,
  // so T = 47 - ceil(log2 pcnt); the int64 sums need N 2^T < 2^63.
  const int64_t threads = (int64_t)h->le.grid * 256;
  const int64_t trips = ((h->N + 3) / 4 + threads - 1) / threads;   // 4 markers a trip
  const int64_t pcnt = std::max<int64_t>(1, 4 * trips * (256 / m.rt));
  int lg = 0;
  while (((int64_t)1 << lg) < pcnt) lg++;
  int bitlen = 0;
  while (bitlen < 62 && ((int64_t)1 << bitlen) <= h->N) bitlen++;
  const int T = std::min(37, std::min(47 - lg, 62 - bitlen));
  m.rshift = 54 - T;
  if (m.rshift < 17 || m.rshift > 31)
    return fail(PIC_ERR_UNSUPPORTED, "pic_init: %lld markers need a deposit shift of %d (17..31)",
                (long long)h->N, m.rshift);
  m.rnd = 1ll << (m.rshift - 1);
  const double qm = S.q / S.m;
  m.jscale = S.q * S.w0 * std::ldexp(1.0, m.rshift) / (c.h * m.cxk * 8388608.0);
  m.ke_scale = 0.5 * S.m * S.w0 / (m.cxk * m.cxk);
  m.e_half = 0.5 * c.dt * qm * m.cxk;
  m.t_half = 0.5 * c.dt * qm;
  m.kick = c.dt * qm * m.cxk;
  m.m_full = c.dt * qm;
  const size_t N = (size_t)(h->N + 3) / 4 * 4;   // padded: the passes move 4 markers at a time
  if ((rc = h->alloc(&mb.Y, N)) || (rc = h->alloc(&mb.J1, 2 * (size_t)c.n)) ||
      (rc = h->alloc(&mb.J2, 2 * (size_t)c.n)))
    return rc;
  for (int d = 0; d < 2; d++)
    if ((rc = h->alloc(&mb.vh[d], N)) || (rc = h->alloc(&mb.vl[d], N)) ||
        (rc = h->alloc(&mb.Vs[d], N)))
      return rc;
  CUDA_TRY(em1m_prepare(c, m));
  return PIC_OK;
}

// 1D2V with a spectral field solve: constants, SoA markers (y, vx, vy), fields.
int init_em1d(pic_handle *h, const pic_species *species, const double *E0, const double *B0) {
  const pic_config &cfg = h->cfg;
  Em1dConst &c = h->c1e;
  Em1dBufs &b = h->b1e;
  c.n = (int)cfg.grid.n[0];
  c.log2n = 0;
  while ((1 << c.log2n) < c.n) c.log2n++;
  c.order = cfg.shape_order;
  c.scheme = cfg.scheme;
  c.solver = cfg.solver == PIC_SOLVER_CN_SPECTRAL ? 1 : 2;
  c.gamma_on = cfg.gamma_on;
  c.nsp = h->nsp;
  c.rt = em1d_tile_copies(c.n);
  c.n_total = h->N;
  c.L = cfg.grid.L[0];
  c.h = c.L / c.n;
  c.inv_h = c.n / c.L;
  c.dt = cfg.dt;
  c.c = cfg.c;
  c.c2 = cfg.c * cfg.c;
  for (int s = 0; s < h->nsp; s++) {
    const SpeciesInfo &S = h->sp[s];
    c.sp_end[s] = S.offset + S.n;
    c.qm[s] = S.q / S.m;
    c.qw_h[s] = S.q * S.w0 / c.h;
    c.q_h[s] = S.q / c.h;
    c.w0[s] = S.w0;
    c.half_m[s] = 0.5 * S.m;
  }
  for (int s = h->nsp; s < kMaxSpecies; s++) c.sp_end[s] = h->N;
  h->le.block = 256;
  // the FP64 passes are bound by the FP64 pipe (two blocks per SM keep it
  // busy); the mixed passes need the latency hiding of four (at 64 registers
  // a thread, four 256-thread blocks fill an SM's register file)
  const int64_t per_sm = h->mixed ? 4 : 2;
  h->le.grid = (int)std::max<int64_t>(1, std::min<int64_t>((h->N + 255) / 256, (int64_t)h->nsm * per_sm));
  const size_t n = (size_t)c.n;
  int rc;
  if ((rc = h->alloc(&b.y, h->N)) || (rc = h->alloc(&b.vx, h->N)) || (rc = h->alloc(&b.vy, h->N)))
    return rc;
  if (!h->mixed && ((rc = h->alloc(&b.vsx, h->N)) || (rc = h->alloc(&b.vsy, h->N)))) return rc;
  // the FP64 passes hand the shape at y^{n+1/2} from pass C to pass E and,
  // with ESEC2, the shape at the next y* from pass E to pass C
  b.sw = nullptr;
  b.si = nullptr;
  b.sws = nullptr;
  b.sis = nullptr;
  if (!h->mixed && ((rc = h->alloc(&b.sw, (size_t)(cfg.shape_order + 1) * h->N)) ||
                    (rc = h->alloc(&b.si, h->N))))
    return rc;
  if (!h->mixed && cfg.scheme == 2 &&
      ((rc = h->alloc(&b.sws, (size_t)(cfg.shape_order + 1) * h->N)) ||
       (rc = h->alloc(&b.sis, h->N))))
    return rc;
  b.w = nullptr;
  if (h->weighted && (rc = h->alloc(&b.w, h->N))) return rc;
  double **e2[] = {&b.E, &b.En, &b.Es, &b.Ea};
  for (double **f : e2)
    if ((rc = h->alloc(f, 2 * n))) return rc;
  if ((rc = h->alloc(&b.J1, kJSlices * 2 * n)) || (rc = h->alloc(&b.J2, kJSlices * 2 * n)) ||
      (rc = h->alloc(&b.tw, n / 2)) || (rc = h->alloc(&b.coef, 2 * kEm1Coef * (n / 2 + 1))))
    return rc;
  double **e1[] = {&b.B, &b.Bn, &b.Bs, &b.Bh};
  for (double **f : e1)
    if ((rc = h->alloc(f, n))) return rc;
  if ((rc = h->alloc(&b.ke_part, (size_t)h->le.grid)) || (rc = h->alloc(&b.done, 2)) ||
      (rc = h->alloc(&b.fallback, kStepsCap)) || (rc = h->alloc(&b.te, kStepsCap)) ||
      (rc = h->alloc(&b.err, 1)) || (rc = h->alloc(&h->ids, h->N)) ||
      (rc = h->alloc(&h->e1_part, (size_t)h->le.grid * h->nsp + 2)))
    return rc;
  h->b1.err = b.err;
  h->b1.fallback = b.fallback;
  h->b1.te = b.te;
  CUDA_TRY(em1d_prepare(c, b, h->st));
  h->launches += 1;
  CUDA_TRY(cudaMemsetAsync(b.err, 0, sizeof(unsigned), h->st));
  for (int s = 0; s < h->nsp; s++) {
    const SpeciesInfo &S = h->sp[s];
    const pic_species &in = species[s];
    CUDA_TRY(cudaMemcpyAsync(b.y + S.offset, in.x, sizeof(double) * S.n, cudaMemcpyDefault, h->st));
    CUDA_TRY(cudaMemcpyAsync(b.vx + S.offset, in.v, sizeof(double) * S.n, cudaMemcpyDefault, h->st));
    CUDA_TRY(cudaMemcpyAsync(b.vy + S.offset, in.v + S.n, sizeof(double) * S.n, cudaMemcpyDefault,
                             h->st));
    if (h->weighted) {
      if (in.w) {
        CUDA_TRY(cudaMemcpyAsync(b.w + S.offset, in.w, sizeof(double) * S.n, cudaMemcpyDefault, h->st));
      } else {
        std::vector<double> tmp((size_t)S.n, S.w0);
        CUDA_TRY(cudaMemcpyAsync(b.w + S.offset, tmp.data(), sizeof(double) * S.n,
                                 cudaMemcpyHostToDevice, h->st));
        CUDA_TRY(cudaStreamSynchronize(h->st));
      }
    }
  }
  std::vector<int64_t> ids((size_t)h->N);
  for (int s = 0; s < h->nsp; s++)
    for (int64_t p = 0; p < h->sp[s].n; p++) ids[(size_t)(h->sp[s].offset + p)] = p;
  CUDA_TRY(cudaMemcpyAsync(h->ids, ids.data(), sizeof(int64_t) * h->N, cudaMemcpyHostToDevice, h->st));
  CUDA_TRY(cudaMemsetAsync(b.E, 0, sizeof(double) * 2 * n, h->st));
  CUDA_TRY(cudaMemsetAsync(b.B, 0, sizeof(double) * n, h->st));
  if (E0) CUDA_TRY(cudaMemcpyAsync(b.E, E0, sizeof(double) * 2 * n, cudaMemcpyDefault, h->st));
  if (B0) CUDA_TRY(cudaMemcpyAsync(b.B, B0, sizeof(double) * n, cudaMemcpyDefault, h->st));
  CUDA_TRY(cudaStreamSynchronize(h->st));
  if (h->mixed && (rc = init_em1d_mixed(h))) return rc;
  return restart_em1d(h);
}

#ifdef PIC_DEBUG_BOUNDS
// one index check of the debug-bounds build, run on the device
__global__ void bounds_probe_kernel(long long i, long long n, long long *out) {
  *out = PIC_INDEX(i, n);
}
#endif

}  // namespace

extern "C" {

const char *pic_last_error(void) { return g_last_error.c_str(); }

#ifdef PIC_DEBUG_BOUNDS
const char *pic_version(void) { return "gb300-ecpic 0.1 (sm_103a, debug-bounds)"; }
#else
const char *pic_version(void) { return "gb300-ecpic 0.1 (sm_103a)"; }
#endif

int pic_debug_bounds(int64_t index, int64_t extent, int *flagged) {
  if (!flagged) return fail(PIC_ERR_ARG, "pic_debug_bounds: flagged is NULL");
  *flagged = -1;
#ifdef PIC_DEBUG_BOUNDS
  long long *d = nullptr, got = -1;
  cudaError_t e = cudaMalloc(&d, sizeof *d);
  if (e == cudaSuccess) {
    bounds_probe_kernel<<<1, 1>>>((long long)index, (long long)extent, d);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(&got, d, sizeof got, cudaMemcpyDeviceToHost);
  if (d) cudaFree(d);
  if (e != cudaSuccess) return fail(PIC_ERR_CUDA, "pic_debug_bounds: %s", cudaGetErrorString(e));
  const unsigned site = bounds_site_pic_api();
  const bool in_range = index >= 0 && index < extent;
  // the check yields the index when it passes, 0 when it records a failure
  if ((site != 0) == in_range || got != (in_range ? (long long)index : 0ll))
    return fail(PIC_ERR_CUDA, "pic_debug_bounds: check of %lld in [0, %lld) gave %lld, record 0x%x",
                (long long)index, (long long)extent, got, site);
  *flagged = site != 0;
  return PIC_OK;
#else
  (void)index;
  (void)extent;
  return fail(PIC_ERR_UNSUPPORTED, "pic_debug_bounds: library built without PIC_DEBUG_BOUNDS");
#endif
}

int pic_init(const pic_config *cfg, const pic_species *species, int nspecies, const double *E0,
             const double *B0, pic_handle **out) {
  if (!out) return fail(PIC_ERR_ARG, "pic_init: out is NULL");
  *out = nullptr;
  if (!cfg || !species) return fail(PIC_ERR_ARG, "pic_init: cfg or species is NULL");
  if (nspecies < 1 || nspecies > kMaxSpecies)
    return fail(PIC_ERR_ARG, "pic_init: nspecies must be in [1, %d]", kMaxSpecies);
  if (cfg->shape_order != 1 && cfg->shape_order != 2)
    return fail(PIC_ERR_ARG, "pic_init: shape_order must be 1 or 2");
  if (cfg->scheme != PIC_SCHEME_ESEC1 && cfg->scheme != PIC_SCHEME_ESEC2)
    return fail(PIC_ERR_ARG, "pic_init: scheme must be PIC_SCHEME_ESEC1 or PIC_SCHEME_ESEC2");
  if (!(cfg->dt > 0.0) || !std::isfinite(cfg->dt)) return fail(PIC_ERR_ARG, "pic_init: dt must be > 0");
  if (cfg->precision != PIC_PREC_FP64 && cfg->precision != PIC_PREC_MIXED)
    return fail(PIC_ERR_ARG, "pic_init: unknown precision");
  if (cfg->binomial_passes < 0 || cfg->binomial_passes > 8)
    return fail(PIC_ERR_ARG, "pic_init: binomial_passes must be in [0, 8]");
  if (cfg->sort_period < 0) return fail(PIC_ERR_ARG, "pic_init: sort_period must be >= 0");
  if (cfg->sort_period > 0 &&
      ((cfg->solver != PIC_SOLVER_AMPERE_ES && cfg->solver != PIC_SOLVER_YEE_LEAPFROG) ||
       cfg->precision != PIC_PREC_MIXED))
    return fail(PIC_ERR_UNSUPPORTED, "pic_init: sort_period is an option of the mixed form of "
                                     "the Ampere and Yee solvers");
  if (cfg->charge_conserving != 0 && cfg->charge_conserving != 1)
    return fail(PIC_ERR_ARG, "pic_init: charge_conserving must be 0 or 1");
  if (cfg->gamma_fp64 != 0 && cfg->gamma_fp64 != 1)
    return fail(PIC_ERR_ARG, "pic_init: gamma_fp64 must be 0 or 1");
  if (cfg->separate_passes != 0 && cfg->separate_passes != 1)
    return fail(PIC_ERR_ARG, "pic_init: separate_passes must be 0 or 1");
  if (cfg->gamma_fp64 && cfg->precision == PIC_PREC_MIXED &&
      (cfg->solver != PIC_SOLVER_AMPERE_ES || cfg->sort_period != 0 || cfg->binomial_passes != 0))
    return fail(PIC_ERR_UNSUPPORTED, "pic_init: gamma_fp64 is built for the mixed form of the "
                                     "Ampere solver with sort_period 0 and no filter");
  if (cfg->charge_conserving &&
      (cfg->solver != PIC_SOLVER_YEE_LEAPFROG || cfg->precision != PIC_PREC_FP64 ||
       cfg->shape_order != 1))
    return fail(PIC_ERR_UNSUPPORTED, "pic_init: charge_conserving runs the Yee solver in the FP64 "
                                     "form with shape_order 1");
  if (cfg->binomial_passes != 0 &&
      !(cfg->solver == PIC_SOLVER_STANDARD_LEAPFROG || cfg->solver == PIC_SOLVER_AMPERE_ES))
    return fail(PIC_ERR_UNSUPPORTED, "pic_init: binomial_passes is for the standard and the "
                                     "Ampere solvers");
  if (cfg->solver == PIC_SOLVER_AMPERE_ES) {
    if (cfg->grid.dim_x != 1 || cfg->grid.dim_v != 1)
      return fail(PIC_ERR_ARG, "pic_init: the Ampere solver runs 1D1V (dim_x = dim_v = 1)");
    if (cfg->grid.n[0] < 4 || cfg->grid.n[0] > kMaxNodes1D)
      return fail(PIC_ERR_ARG, "pic_init: 1D grid needs 4..%d nodes", kMaxNodes1D);
    if (!(cfg->grid.L[0] > 0.0)) return fail(PIC_ERR_ARG, "pic_init: L must be > 0");
    if (B0) return fail(PIC_ERR_ARG, "pic_init: B0 given for the electrostatic solver");
  } else if (cfg->solver == PIC_SOLVER_STANDARD_LEAPFROG) {
    if (cfg->grid.dim_x != 1 || cfg->grid.dim_v != 1)
      return fail(PIC_ERR_ARG, "pic_init: the standard solver runs 1D1V (dim_x = dim_v = 1)");
    const int64_t n = cfg->grid.n[0];
    if (n < 4 || n > kStdMaxNodes || (n & (n - 1)))
      return fail(PIC_ERR_ARG, "pic_init: the standard solver needs a power of two in [4, %d] nodes",
                  kStdMaxNodes);
    if (!(cfg->grid.L[0] > 0.0)) return fail(PIC_ERR_ARG, "pic_init: L must be > 0");
    if (cfg->binomial_passes < 0 || cfg->binomial_passes > 8)
      return fail(PIC_ERR_ARG, "pic_init: binomial_passes must be in [0, 8]");
    if (E0 || B0) return fail(PIC_ERR_ARG, "pic_init: the standard solver takes E from the charge");
    if (cfg->precision == PIC_PREC_MIXED)
      return fail(PIC_ERR_UNSUPPORTED, "pic_init: the standard solver runs in the FP64 form");
  } else if (cfg->solver == PIC_SOLVER_CN_SPECTRAL || cfg->solver == PIC_SOLVER_PSATD) {
    if (cfg->grid.dim_x != 1 || cfg->grid.dim_v != 2)
      return fail(PIC_ERR_ARG, "pic_init: the spectral solvers run 1D2V (dim_x = 1, dim_v = 2)");
    const int64_t n = cfg->grid.n[0];
    if (n < 4 || n > kSpecMaxNodes || (n & (n - 1)))
      return fail(PIC_ERR_ARG, "pic_init: the spectral solvers need a power of two in [4, %d] nodes",
                  kSpecMaxNodes);
    if (!(cfg->grid.L[0] > 0.0) || !(cfg->c > 0.0) || !std::isfinite(cfg->c))
      return fail(PIC_ERR_ARG, "pic_init: the spectral solvers need L > 0 and c > 0");

  } else if (cfg->solver == PIC_SOLVER_YEE_LEAPFROG) {
    if (cfg->grid.dim_x != 2 || cfg->grid.dim_v != 3)
      return fail(PIC_ERR_ARG, "pic_init: the Yee solver runs 2D3V (dim_x = 2, dim_v = 3)");
    if (cfg->grid.n[0] < 4 || cfg->grid.n[1] < 4 || cfg->grid.n[0] > 8192 || cfg->grid.n[1] > 8192)
      return fail(PIC_ERR_ARG, "pic_init: Yee grid needs 4..8192 nodes per dimension");
    if (!(cfg->grid.L[0] > 0.0) || !(cfg->grid.L[1] > 0.0) || !(cfg->c > 0.0))
      return fail(PIC_ERR_ARG, "pic_init: Yee solver needs L > 0 and c > 0");
    if (cfg->precision == PIC_PREC_MIXED && cfg->grid.L[0] != cfg->grid.L[1])
      return fail(PIC_ERR_UNSUPPORTED, "pic_init: the mixed form of the Yee solver needs a "
                                       "square domain (L[0] == L[1])");
  } else {
    return fail(PIC_ERR_ARG, "pic_init: unknown solver");
  }
  int64_t N = 0;
  bool weighted = false;
  for (int s = 0; s < nspecies; s++) {
    const pic_species &S = species[s];
    if (S.n < 0) return fail(PIC_ERR_ARG, "pic_init: species %d has n < 0", s);
    if (S.n > 0 && (!S.x || !S.v)) return fail(PIC_ERR_ARG, "pic_init: species %d x or v is NULL", s);
    if (!(S.m > 0.0) || !std::isfinite(S.q)) return fail(PIC_ERR_ARG, "pic_init: species %d needs m > 0 and finite q", s);
    if (S.w) weighted = true;
    N += S.n;
  }
  if (N > ((int64_t)1 << 40)) return fail(PIC_ERR_ARG, "pic_init: too many markers");
  if (cfg->precision == PIC_PREC_MIXED && (nspecies != 1 || weighted))
    return fail(PIC_ERR_UNSUPPORTED, "pic_init: the mixed form runs one species with a uniform "
                                     "weight (use PIC_PREC_FP64 for several species or weighted markers)");

  pic_handle *h = new pic_handle();
  h->cfg = *cfg;
  h->st = (cudaStream_t)cfg->cuda_stream;
  h->nsp = nspecies;
  h->weighted = weighted;
  h->mixed = cfg->precision == PIC_PREC_MIXED;
  int64_t off = 0;
  for (int s = 0; s < nspecies; s++) {
    h->sp[s] = SpeciesInfo{species[s].q, species[s].m, species[s].w0, species[s].n, off,
                           species[s].w != nullptr};
    off += species[s].n;
  }
  h->N = N;
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) {
    delete h;
    return fail(PIC_ERR_CUDA, "pic_init: no usable CUDA device: %s", cudaGetErrorString(e));
  }
  int64_t want = (N + 511) / 512;
  h->ls.block = 512;
  h->ls.grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)nsm * 2));
  if (cfg->precision == PIC_PREC_MIXED) {
    // at most 16 grid-stride trips of 4 markers per thread (32768 per block),
    // the bound the split integer tile is sized for
    const int64_t need = ((N + 3) / 4 + 512 * 16 - 1) / (512 * 16);
    h->ls.grid = (int)std::max<int64_t>(h->ls.grid, need);
    // the sorted 1D modes on grids of up to kWideMaxNodes nodes: at most the
    // wide launch's per-copy count of markers per 512-thread block (the tile
    // bound of that grid size)
    if (cfg->solver == PIC_SOLVER_AMPERE_ES && cfg->sort_period > 0 &&
        cfg->grid.n[0] <= kWideMaxNodes) {
      const int64_t pc = mixed_wide_pcnt(N, nsm);
      h->ls.grid = (int)std::max<int64_t>(h->ls.grid, (4 * ((N + 3) / 4) + pc - 1) / pc);
    }
  }
  h->nsm = nsm;
  h->em = cfg->solver == PIC_SOLVER_YEE_LEAPFROG;
  h->em1 = cfg->solver == PIC_SOLVER_CN_SPECTRAL || cfg->solver == PIC_SOLVER_PSATD;
  h->stdp = cfg->solver == PIC_SOLVER_STANDARD_LEAPFROG;
  int rc = h->em     ? init_em2d(h, species, E0, B0)
           : h->em1  ? init_em1d(h, species, E0, B0)
           : h->stdp ? init_std(h, species)
                     : init_es1d(h, species, E0);
  if (rc) {
    std::string msg = g_last_error;
    delete h;
    g_last_error = msg;
    return rc;
  }
  *out = h;
  return PIC_OK;
}

int pic_step_async(pic_handle *h, int nsteps) {
  if (!h) return fail(PIC_ERR_ARG, "pic_step_async: NULL handle");
  if (nsteps < 0) return fail(PIC_ERR_ARG, "pic_step_async: nsteps < 0");
  if (h->pending + nsteps > kStepsCap)
    return fail(PIC_ERR_ARG, "pic_step_async: more than %d steps pending; call pic_read_stats",
                kStepsCap);
  Es1dFp64Bufs &b = h->b1;
  if (h->pending == 0 && nsteps > 0) {
    CUDA_TRY(cudaMemsetAsync(b.fallback, 0, sizeof(unsigned long long) * kStepsCap, h->st));
  }
  for (int k = 0; k < nsteps && h->stdp; k++) {
    const int slot = h->pending;
    CUDA_TRY(h->timed_launch(1, [&] { std_step(h->cs, h->bs, slot, h->lsd, h->st); }));
    h->launches += 1;
    h->steps_done++;
    h->pending++;
  }
  for (int k = 0; k < nsteps && h->em1; k++) {
    Em1dBufs &e = h->b1e;
    const int slot = h->pending;
    if (h->mixed) {
      CUDA_TRY(h->timed_launch(0, [&] { em1m_pass_c(h->c1e, e, h->c1m, h->b1m, h->le, h->st); }));
      CUDA_TRY(h->timed_launch(1, [&] {
        em1m_pass_e(h->c1e, e, h->c1m, h->b1m, slot, h->le, h->st);
      }));
    } else {
      CUDA_TRY(h->timed_launch(0, [&] { em1d_pass_c(h->c1e, e, h->le, h->st); }));
      CUDA_TRY(h->timed_launch(1, [&] { em1d_pass_e(h->c1e, e, slot, h->le, h->st); }));
    }
    h->launches += 2;
    std::swap(e.E, e.En);
    std::swap(e.B, e.Bn);
    h->steps_done++;
    h->pending++;
  }
  for (int k = 0; k < nsteps && h->em; k++) {
    Em2dBufs &e = h->be;
    const int slot = h->pending;
    if (h->mixed) {
      // sorted markers: pass E of every sort_period-th step writes them in
      // quarter-cell order (from pass C's counts and their scan)
      const bool sort_now = h->cme.sorted && (h->steps_done + 1) % h->cfg.sort_period == 0;
      const Em2dMixBufs &mb = h->bme;
      Em2dSortIO so{};
      if (sort_now) {
        so.off = h->sort2_off;
        so.dst = h->bme_alt;
        so.ids_in = h->cfg.skip_ids ? nullptr : h->ids;
        so.ids_out = h->cfg.skip_ids ? nullptr : h->ids_alt;
      }
      unsigned *cnt = sort_now ? h->sort2_cnt : nullptr;
      // K1 also reduces the previous step's TE; pass E also runs K5
      const int fin = (h->te_open && slot > 0) ? slot - 1 : -1;
      CUDA_TRY(h->timed_launch(4, [&] {
        em2dm_k1(h->ce, h->cme, mb, e, fin, h->lpm, h->lg, h->st);
      }));
      CUDA_TRY(h->timed_launch(0, [&] { em2dm_pass_c(h->cme, mb, cnt, h->lpm, h->st); }));
      if (sort_now) {
        CUDA_TRY(h->timed_launch(3, [&] {
          em2dm_sort_scan(h->cme, h->sort2_cnt, h->sort2_off, h->st);
        }));
        h->launches += 2;
      }
      CUDA_TRY(h->timed_launch(4, [&] { em2dm_k3(h->ce, h->cme, mb, e, h->lg, h->st); }));
      CUDA_TRY(h->timed_launch(1, [&] {
        em2dm_pass_e(h->cme, mb, slot, so, h->ce, e, h->lpm, h->lg, h->st);
      }));
      if (sort_now) swap_em2d_sorted(h);
      h->te_open = true;
      h->launches += 4;
    } else {
      CUDA_TRY(h->timed_launch(4, [&] { em2d_k1(h->ce, e, h->lg, h->st); }));
      CUDA_TRY(h->timed_launch(0, [&] { em2d_pass_c(h->ce, e, h->lp, h->st); }));
      CUDA_TRY(h->timed_launch(4, [&] { em2d_k3(h->ce, e, h->lg, h->st); }));
      CUDA_TRY(h->timed_launch(1, [&] { em2d_pass_e(h->ce, e, slot, h->lp, h->st); }));
      CUDA_TRY(h->timed_launch(4, [&] { em2d_k5(h->ce, e, h->lg, h->st, false); }));
      CUDA_TRY(h->timed_launch(2, [&] {
        em2d_finalize(h->ce, e, slot, h->lp, h->lg, h->st, false);
      }));
      h->launches += 6;
    }
    std::swap(e.E, e.En);
    double *old = e.B;
    e.B = e.Bp;
    e.Bp = e.Bpp;
    e.Bpp = old;
    h->steps_done++;
    h->pending++;
  }
  for (int k = 0; k < nsteps && !h->em && !h->em1 && !h->stdp; k++) {
    if (h->mixed) {
      if (h->cm.mode == 1 && h->steps_done > 0 && h->steps_done % h->cfg.sort_period == 0) {
        int rc = sort_mixed(h);
        if (rc) return rc;
      }
      if (h->fused) {
        // ESEC1 in one launch per step.  The currents rotate through J2[0],
        // J2[1], J1[0] (ESEC1 has no j^{n,*}): step n reads buffer n mod 3.
        Es1dMixBufs &bm = h->bm;
        long long *ring[3] = {bm.J2[0], bm.J2[1], bm.J1[0]};
        long long *tot[3] = {bm.Jtot + 2, bm.Jtot + 3, bm.Jtot + 0};
        const int64_t n = h->steps_done;
        const int r0 = (int)(n % 3), r1 = (int)((n + 1) % 3), r2 = (int)((n + 2) % 3);
        if (!h->primed) {
          // pass C of step n alone, depositing into buffer n mod 3
          Es1dMixBufs bp = bm;
          const int par = (int)(n & 1);
          if (par) bp.J2[1] = ring[r0]; else bp.J2[0] = ring[r0];
          bp.Jtot = tot[r0] - 2 - par;
          CUDA_TRY(h->timed_launch(0, [&] {
            es1d_mix_pass_c(h->cm, bp, n, h->pending, h->lmix, h->st);
          }));
          h->launches += 1;
          h->primed = true;
        }
        const RingIO io{ring[r0], tot[r0], ring[r1], tot[r1], ring[r2], tot[r2],
                        bm.ke_part, bm.we_part, h->ke_alt, h->we_alt};
        CUDA_TRY(h->timed_launch(5, [&] {
          es1d_mix_pass_ec(h->cm, bm, io, n, h->pending, h->lmix_ec, h->st);
        }));
        std::swap(bm.ke_part, h->ke_alt);
        std::swap(bm.we_part, h->we_alt);
        h->launches += 1;
        h->steps_done++;
        h->pending++;
        continue;
      }
      CUDA_TRY(h->timed_launch(0, [&] {
        es1d_mix_pass_c(h->cm, h->bm, h->steps_done, h->pending, h->lmix, h->st);
      }));
      if (h->cm.mode == 2) {
        CUDA_TRY(h->timed_launch(3, [&] { es1d_mix_fused_scan(h->cm, h->bm, h->lmix.grid, h->st); }));
        h->launches += 1;
      }
      CUDA_TRY(h->timed_launch(1, [&] {
        es1d_mix_pass_e(h->cm, h->bm, h->steps_done, h->pending, h->lmix, h->st);
      }));
      if (h->cm.mode == 2) swap_sorted_output(h);
    } else {
      CUDA_TRY(h->timed_launch(0, [&] {
        es1d_fp64_pass_c(h->c1, b, h->steps_done, h->pending, h->ls, h->st);
      }));
      CUDA_TRY(h->timed_launch(1, [&] {
        es1d_fp64_pass_e(h->c1, b, h->steps_done, h->pending, h->ls, h->st);
      }));
    }
    h->launches += 2;
    h->steps_done++;
    h->pending++;
  }
  return PIC_OK;
}

int pic_read_stats(pic_handle *h, int capacity, int64_t *nfallback_per_step, double *te_per_step,
                   int *nread) {
  if (!h) return fail(PIC_ERR_ARG, "pic_read_stats: NULL handle");
  int n = h->pending;
  if (nread) *nread = n;
  if (n == 0) return check_flags(h, "pic_read_stats");
  if ((nfallback_per_step || te_per_step) && capacity < n)
    return fail(PIC_ERR_ARG, "pic_read_stats: %d steps pending, capacity %d", n, capacity);
  Es1dFp64Bufs &b = h->b1;
  if (h->em && h->mixed && h->te_open) {
    CUDA_TRY(h->timed_launch(2, [&] {
      em2d_finalize(h->ce, h->be, n - 1, h->lpm, h->lg, h->st, false);
    }));
    h->launches += 1;
  }
  h->te_open = false;
  if (!h->em && !h->em1 && !h->stdp) {
    CUDA_TRY(h->timed_launch(2, [&] {
      if (h->mixed)
        es1d_mix_finalize(h->cm, h->bm, n - 1, h->lmix.grid, h->st);
      else
        es1d_fp64_finalize(h->c1, b, n - 1, h->ls.grid, h->st);
    }));
    h->launches += 1;
  }
  std::vector<unsigned long long> fb(n);
  std::vector<double> te(n);
  CUDA_TRY(cudaMemcpyAsync(fb.data(), b.fallback, sizeof(unsigned long long) * n,
                           cudaMemcpyDeviceToHost, h->st));
  CUDA_TRY(cudaMemcpyAsync(te.data(), b.te, sizeof(double) * n, cudaMemcpyDeviceToHost, h->st));
  CUDA_TRY(cudaStreamSynchronize(h->st));
  h->pending = 0;
  if (nfallback_per_step) {
    std::vector<int64_t> f64(fb.begin(), fb.end());
    CUDA_TRY(cudaMemcpyAsync(nfallback_per_step, f64.data(), sizeof(int64_t) * n,
                             cudaMemcpyDefault, h->st));
  }
  if (te_per_step)
    CUDA_TRY(cudaMemcpyAsync(te_per_step, te.data(), sizeof(double) * n, cudaMemcpyDefault, h->st));
  CUDA_TRY(cudaStreamSynchronize(h->st));
  return check_flags(h, "pic_read_stats");
}

int pic_step(pic_handle *h, int nsteps, int64_t *nfallback_per_step, double *te_per_step) {
  if (!h) return fail(PIC_ERR_ARG, "pic_step: NULL handle");
  if (nsteps < 0) return fail(PIC_ERR_ARG, "pic_step: nsteps < 0");
  int rc = PIC_OK;
  if (h->pending) {  // stats of earlier asynchronous steps are discarded
    if ((rc = pic_read_stats(h, 0, nullptr, nullptr, nullptr))) return rc;
  }
  int done = 0;
  while (done < nsteps) {
    int chunk = std::min(kStepsCap, nsteps - done);
    if ((rc = pic_step_async(h, chunk))) return rc;
    if ((rc = pic_read_stats(h, chunk, nfallback_per_step ? nfallback_per_step + done : nullptr,
                             te_per_step ? te_per_step + done : nullptr, nullptr)))
      return rc;
    done += chunk;
  }
  return PIC_OK;
}

int pic_set_profiling(pic_handle *h, int on) {
  if (!h) return fail(PIC_ERR_ARG, "pic_set_profiling: NULL handle");
  CUDA_TRY(h->collect_profile());
  for (int k = 0; k < kProfKinds; k++) {
    h->prof_ms[k] = 0.0;
    h->prof_n[k] = 0;
  }
  h->profiling = on != 0;
  return PIC_OK;
}

int pic_profile(pic_handle *h, int kind, int64_t *launches, double *total_ms) {
  if (!h || kind < 0 || kind >= kProfKinds) return fail(PIC_ERR_ARG, "pic_profile: bad arguments");
  CUDA_TRY(h->collect_profile());
  if (launches) *launches = h->prof_n[kind];
  if (total_ms) *total_ms = h->prof_ms[kind];
  return PIC_OK;
}

int pic_launch_count(pic_handle *h, int64_t *launches) {
  if (!h || !launches) return fail(PIC_ERR_ARG, "pic_launch_count: bad arguments");
  *launches = h->launches;
  return PIC_OK;
}

static int energy_em2d(pic_handle *h, double *KE_per_species, double *W_E, double *W_B, double *TE) {
  const Em2dConst &c = h->ce;
  Em2dBufs &b = h->be;
  const int nb = h->lp.grid;
  // own partials: the mixed form keeps the last step's in ke_part until the
  // next step (or pic_read_stats) has reduced them
  double *part_d = h->energy_part;
  if (h->mixed)
    em2dm_kinetic(h->cme, h->bme, part_d, h->lp, h->st);
  else
    em2d_fp64_kinetic(c, b, part_d, nb, h->st);
  CUDA_TRY(cudaGetLastError());
  const size_t nc3 = 3 * (size_t)c.nx * c.ny;
  std::vector<double> part((size_t)nb * h->nsp), e(nc3), bo(nc3), bp(nc3);
  CUDA_TRY(cudaMemcpyAsync(part.data(), part_d, sizeof(double) * part.size(),
                           cudaMemcpyDeviceToHost, h->st));
  CUDA_TRY(cudaMemcpyAsync(e.data(), b.E, sizeof(double) * nc3, cudaMemcpyDeviceToHost, h->st));
  CUDA_TRY(cudaMemcpyAsync(bo.data(), b.B, sizeof(double) * nc3, cudaMemcpyDeviceToHost, h->st));
  CUDA_TRY(cudaMemcpyAsync(bp.data(), b.Bp, sizeof(double) * nc3, cudaMemcpyDeviceToHost, h->st));
  CUDA_TRY(cudaStreamSynchronize(h->st));
  double te = 0.0;
  for (int s = 0; s < h->nsp; s++) {
    double k = 0.0;
    for (int i = 0; i < nb; i++) k += part[(size_t)s * nb + i];
    if (KE_per_species) KE_per_species[s] = k;
    te += k;
  }
  double we = 0.0, wb = 0.0;
  for (size_t a = 0; a < nc3; a++) {
    we += e[a] * e[a];
    wb += bp[a] * bo[a];
  }
  we *= 0.5 * c.area;
  wb *= 0.5 * c.c2 * c.area;  // W_B^n = (c^2/2)|h| sum B^{n+1/2} . B^{n-1/2}
  te += we + wb;
  if (W_E) *W_E = we;
  if (W_B) *W_B = wb;
  if (TE) *TE = te;
  if (!std::isfinite(te)) return fail(PIC_ERR_NONFINITE, "pic_energy: non-finite energy");
  return PIC_OK;
}

static int energy_em1d(pic_handle *h, double *KE_per_species, double *W_E, double *W_B, double *TE) {
  const int nb = h->le.grid;
  double *ke = h->e1_part, *wf = h->e1_part + (size_t)nb * h->nsp;
  if (h->mixed)
    em1m_energy(h->c1e, h->b1e, h->c1m, h->b1m, ke, wf, h->le, h->st);
  else
    em1d_energy(h->c1e, h->b1e, ke, wf, h->le, h->st);
  CUDA_TRY(cudaGetLastError());
  h->launches += 1;
  std::vector<double> part((size_t)nb * h->nsp + 2);
  CUDA_TRY(cudaMemcpyAsync(part.data(), h->e1_part, sizeof(double) * part.size(),
                           cudaMemcpyDeviceToHost, h->st));
  CUDA_TRY(cudaStreamSynchronize(h->st));
  double te = 0.0;
  for (int s = 0; s < h->nsp; s++) {
    double k = 0.0;
    for (int i = 0; i < nb; i++) k += part[(size_t)s * nb + i];
    if (KE_per_species) KE_per_species[s] = k;
    te += k;
  }
  const double we = part[(size_t)nb * h->nsp], wb = part[(size_t)nb * h->nsp + 1];
  te += we + wb;
  if (W_E) *W_E = we;
  if (W_B) *W_B = wb;
  if (TE) *TE = te;
  if (!std::isfinite(te)) return fail(PIC_ERR_NONFINITE, "pic_energy: non-finite energy");
  return PIC_OK;
}

static int energy_std(pic_handle *h, double *KE_per_species, double *W_E, double *W_B, double *TE) {
  const int nb = h->lsd.grid;
  double *ke = h->std_part, *we = h->std_part + (size_t)nb * h->nsp;
  std_energy(h->cs, h->bs, ke, we, h->lsd, h->st);
  CUDA_TRY(cudaGetLastError());
  h->launches += 1;
  std::vector<double> part((size_t)nb * h->nsp + 1);
  CUDA_TRY(cudaMemcpyAsync(part.data(), h->std_part, sizeof(double) * part.size(),
                           cudaMemcpyDeviceToHost, h->st));
  CUDA_TRY(cudaStreamSynchronize(h->st));
  double te = 0.0;
  for (int s = 0; s < h->nsp; s++) {
    double k = 0.0;
    for (int i = 0; i < nb; i++) k += part[(size_t)s * nb + i];
    if (KE_per_species) KE_per_species[s] = k;
    te += k;
  }
  const double wev = part[(size_t)nb * h->nsp];
  te += wev;
  if (W_E) *W_E = wev;
  if (W_B) *W_B = 0.0;
  if (TE) *TE = te;
  if (!std::isfinite(te)) return fail(PIC_ERR_NONFINITE, "pic_energy: non-finite energy");
  return PIC_OK;
}

int pic_energy(pic_handle *h, double *KE_per_species, double *W_E, double *W_B, double *TE) {
  if (!h) return fail(PIC_ERR_ARG, "pic_energy: NULL handle");
  if (h->stdp) return energy_std(h, KE_per_species, W_E, W_B, TE);
  if (h->em) return energy_em2d(h, KE_per_species, W_E, W_B, TE);
  if (h->em1) return energy_em1d(h, KE_per_species, W_E, W_B, TE);
  const Es1dConst &c = h->c1;
  // own partials: the stepping kernels keep the last step's partials in ke_part
  // until the next step (or pic_read_stats) has reduced them
  double *ke_d = h->energy_part;
  if (h->ls.grid < h->nsp) return fail(PIC_ERR_ARG, "pic_energy: internal size");
  std::vector<double> ke(h->nsp), e(c.nc);
  if (h->mixed) {
    es1d_mix_kinetic(h->cm, h->bm, ke_d, h->ls.grid, h->st);
    CUDA_TRY(cudaGetLastError());
    std::vector<double> part(h->ls.grid);
    CUDA_TRY(cudaMemcpyAsync(part.data(), ke_d, sizeof(double) * h->ls.grid, cudaMemcpyDeviceToHost,
                             h->st));
    CUDA_TRY(cudaStreamSynchronize(h->st));
    double acc = 0.0;
    for (double p : part) acc += p;
    ke[0] = acc;
  } else {
    es1d_fp64_kinetic(c, h->b1.v, h->b1.w, ke_d, h->st);
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaMemcpyAsync(ke.data(), ke_d, sizeof(double) * h->nsp, cudaMemcpyDeviceToHost, h->st));
  }
  CUDA_TRY(cudaMemcpyAsync(e.data(), h->b1.E[h->steps_done & 1], sizeof(double) * c.nc,
                           cudaMemcpyDeviceToHost, h->st));
  CUDA_TRY(cudaStreamSynchronize(h->st));
  double we = 0.0;
  for (int i = 0; i < c.nc; i++) we += e[i] * e[i];
  we *= 0.5 * c.h;
  double te = we;
  for (int s = 0; s < h->nsp; s++) {
    te += ke[s];
    if (KE_per_species) KE_per_species[s] = ke[s];
  }
  if (W_E) *W_E = we;
  if (W_B) *W_B = 0.0;
  if (TE) *TE = te;
  if (!std::isfinite(te)) return fail(PIC_ERR_NONFINITE, "pic_energy: non-finite energy");
  return PIC_OK;
}

int pic_get_particles(pic_handle *h, int s, double *x, double *v) {
  if (!h || s < 0 || s >= h->nsp) return fail(PIC_ERR_ARG, "pic_get_particles: bad handle or species");
  const SpeciesInfo &S = h->sp[s];
  if (h->stdp) {
    if (x) CUDA_TRY(cudaMemcpyAsync(x, h->bs.x + S.offset, sizeof(double) * S.n, cudaMemcpyDefault,
                                    h->st));
    if (v) CUDA_TRY(cudaMemcpyAsync(v, h->bs.v + S.offset, sizeof(double) * S.n, cudaMemcpyDefault,
                                    h->st));
    CUDA_TRY(cudaStreamSynchronize(h->st));
    return PIC_OK;
  }
  if (h->em1) {
    if (h->mixed) {
      em1m_to_fp64(h->c1e, h->b1e, h->c1m, h->b1m, h->le, h->st);
      CUDA_TRY(cudaGetLastError());
    }
    if (x) CUDA_TRY(cudaMemcpyAsync(x, h->b1e.y + S.offset, sizeof(double) * S.n, cudaMemcpyDefault,
                                    h->st));
    if (v) {
      CUDA_TRY(cudaMemcpyAsync(v, h->b1e.vx + S.offset, sizeof(double) * S.n, cudaMemcpyDefault,
                               h->st));
      CUDA_TRY(cudaMemcpyAsync(v + S.n, h->b1e.vy + S.offset, sizeof(double) * S.n,
                               cudaMemcpyDefault, h->st));
    }
    CUDA_TRY(cudaStreamSynchronize(h->st));
    return PIC_OK;
  }
  if (h->em) {
    if (h->mixed) {
      em2dm_to_fp64(h->cme, h->bme, h->be, h->lp, h->st);
      CUDA_TRY(cudaGetLastError());
    }
    const double *src[5] = {h->be.x, h->be.y, h->be.vx, h->be.vy, h->be.vz};
    for (int d = 0; d < 2 && x; d++)
      CUDA_TRY(cudaMemcpyAsync(x + d * S.n, src[d] + S.offset, sizeof(double) * S.n,
                               cudaMemcpyDefault, h->st));
    for (int d = 0; d < 3 && v; d++)
      CUDA_TRY(cudaMemcpyAsync(v + d * S.n, src[2 + d] + S.offset, sizeof(double) * S.n,
                               cudaMemcpyDefault, h->st));
    CUDA_TRY(cudaStreamSynchronize(h->st));
    return PIC_OK;
  }
  if (h->mixed) {   // one species: the pieces cover the species
    CUDA_TRY(download_mixed_1d(h, x, v));
    return PIC_OK;
  }
  if (x) CUDA_TRY(cudaMemcpyAsync(x, h->b1.x + S.offset, sizeof(double) * S.n, cudaMemcpyDefault, h->st));
  if (v) CUDA_TRY(cudaMemcpyAsync(v, h->b1.v + S.offset, sizeof(double) * S.n, cudaMemcpyDefault, h->st));
  CUDA_TRY(cudaStreamSynchronize(h->st));
  return PIC_OK;
}

int pic_get_ids(pic_handle *h, int s, int64_t *ids) {
  if (!h || s < 0 || s >= h->nsp || !ids) return fail(PIC_ERR_ARG, "pic_get_ids: bad arguments");
  if (h->cfg.skip_ids && h->mixed && h->cfg.sort_period > 0)
    return fail(PIC_ERR_ARG, "pic_get_ids: marker ids are not kept (skip_ids = 1)");
  const SpeciesInfo &S = h->sp[s];
  CUDA_TRY(cudaMemcpyAsync(ids, h->ids + S.offset, sizeof(int64_t) * S.n, cudaMemcpyDefault, h->st));
  CUDA_TRY(cudaStreamSynchronize(h->st));
  return PIC_OK;
}

int pic_set_particles(pic_handle *h, int s, const double *x, const double *v) {
  if (!h || s < 0 || s >= h->nsp || !x || !v) return fail(PIC_ERR_ARG, "pic_set_particles: bad arguments");
  const SpeciesInfo &S = h->sp[s];
  if (h->stdp) {
    CUDA_TRY(cudaMemcpyAsync(h->bs.x + S.offset, x, sizeof(double) * S.n, cudaMemcpyDefault, h->st));
    CUDA_TRY(cudaMemcpyAsync(h->bs.v + S.offset, v, sizeof(double) * S.n, cudaMemcpyDefault, h->st));
    CUDA_TRY(reset_ids(h, S));
    return restart_std(h);
  }
  if (h->em1) {
    CUDA_TRY(cudaMemcpyAsync(h->b1e.y + S.offset, x, sizeof(double) * S.n, cudaMemcpyDefault, h->st));
    CUDA_TRY(cudaMemcpyAsync(h->b1e.vx + S.offset, v, sizeof(double) * S.n, cudaMemcpyDefault, h->st));
    CUDA_TRY(cudaMemcpyAsync(h->b1e.vy + S.offset, v + S.n, sizeof(double) * S.n, cudaMemcpyDefault,
                             h->st));
    CUDA_TRY(reset_ids(h, S));
    return restart_em1d(h);
  }
  if (h->em) {
    double *dst[5] = {h->be.x, h->be.y, h->be.vx, h->be.vy, h->be.vz};
    for (int d = 0; d < 2; d++)
      CUDA_TRY(cudaMemcpyAsync(dst[d] + S.offset, x + d * S.n, sizeof(double) * S.n,
                               cudaMemcpyDefault, h->st));
    for (int d = 0; d < 3; d++)
      CUDA_TRY(cudaMemcpyAsync(dst[2 + d] + S.offset, v + d * S.n, sizeof(double) * S.n,
                               cudaMemcpyDefault, h->st));
    CUDA_TRY(reset_ids(h, S));
    return restart_em2d(h);
  }
  if (h->mixed) {   // one species; the pieces are converted as they arrive
    CUDA_TRY(upload_mixed_1d(h, x, v));
    CUDA_TRY(reset_ids(h, S));
    return restart_es1d(h, false);
  }
  CUDA_TRY(cudaMemcpyAsync(h->b1.x + S.offset, x, sizeof(double) * S.n, cudaMemcpyDefault, h->st));
  CUDA_TRY(cudaMemcpyAsync(h->b1.v + S.offset, v, sizeof(double) * S.n, cudaMemcpyDefault, h->st));
  CUDA_TRY(reset_ids(h, S));
  return restart_es1d(h, true);
}

int pic_get_fields(pic_handle *h, double *E, double *B) {
  if (!h) return fail(PIC_ERR_ARG, "pic_get_fields: NULL handle");
  if (h->stdp) {
    if (B) return fail(PIC_ERR_ARG, "pic_get_fields: B given for an electrostatic solver");
    if (E) CUDA_TRY(cudaMemcpyAsync(E, h->bs.E, sizeof(double) * h->cs.n, cudaMemcpyDefault, h->st));
    CUDA_TRY(cudaStreamSynchronize(h->st));
    return PIC_OK;
  }
  if (h->em1) {
    const size_t n = (size_t)h->c1e.n;
    if (E) CUDA_TRY(cudaMemcpyAsync(E, h->b1e.E, sizeof(double) * 2 * n, cudaMemcpyDefault, h->st));
    if (B) CUDA_TRY(cudaMemcpyAsync(B, h->b1e.B, sizeof(double) * n, cudaMemcpyDefault, h->st));
    CUDA_TRY(cudaStreamSynchronize(h->st));
    return PIC_OK;
  }
  if (h->em) {
    const size_t nc3 = 3 * (size_t)h->ce.nx * h->ce.ny;
    if (E) CUDA_TRY(cudaMemcpyAsync(E, h->be.E, sizeof(double) * nc3, cudaMemcpyDefault, h->st));
    if (B) CUDA_TRY(cudaMemcpyAsync(B, h->be.B, sizeof(double) * nc3, cudaMemcpyDefault, h->st));
    CUDA_TRY(cudaStreamSynchronize(h->st));
    return PIC_OK;
  }
  (void)B;
  if (E)
    CUDA_TRY(cudaMemcpyAsync(E, h->b1.E[h->steps_done & 1], sizeof(double) * h->c1.nc,
                             cudaMemcpyDefault, h->st));
  CUDA_TRY(cudaStreamSynchronize(h->st));
  return PIC_OK;
}

int pic_set_fields(pic_handle *h, const double *E, const double *B) {
  if (!h || !E) return fail(PIC_ERR_ARG, "pic_set_fields: bad arguments");
  if (h->stdp)
    return fail(PIC_ERR_UNSUPPORTED, "pic_set_fields: the standard solver's E follows from the "
                                     "charge (Gauss's law)");
  if (h->em1) {
    if (!B) return fail(PIC_ERR_ARG, "pic_set_fields: the spectral solvers need Bz");
    const size_t n = (size_t)h->c1e.n;
    CUDA_TRY(cudaMemcpyAsync(h->b1e.E, E, sizeof(double) * 2 * n, cudaMemcpyDefault, h->st));
    CUDA_TRY(cudaMemcpyAsync(h->b1e.B, B, sizeof(double) * n, cudaMemcpyDefault, h->st));
    CUDA_TRY(cudaStreamSynchronize(h->st));
    return restart_em1d(h, false);
  }
  if (h->em) {
    if (!B) return fail(PIC_ERR_ARG, "pic_set_fields: the Yee solver needs B^{n-1/2}");
    const size_t nc3 = 3 * (size_t)h->ce.nx * h->ce.ny;
    CUDA_TRY(cudaMemcpyAsync(h->be.E, E, sizeof(double) * nc3, cudaMemcpyDefault, h->st));
    CUDA_TRY(cudaMemcpyAsync(h->be.B, B, sizeof(double) * nc3, cudaMemcpyDefault, h->st));
    CUDA_TRY(cudaStreamSynchronize(h->st));
    return restart_em2d(h, false);
  }
  if (B) return fail(PIC_ERR_ARG, "pic_set_fields: B given for the electrostatic solver");
  CUDA_TRY(cudaMemcpyAsync(h->b1.E[h->steps_done & 1], E, sizeof(double) * h->c1.nc,
                           cudaMemcpyDefault, h->st));
  CUDA_TRY(cudaStreamSynchronize(h->st));
  return restart_es1d(h, false);
}

int pic_grad_forward(pic_handle *h, int nsteps, int checkpoint_every) {
  if (!h || nsteps <= 0 || checkpoint_every <= 0)
    return fail(PIC_ERR_ARG, "pic_grad_forward: bad arguments");
  if (h->em || h->em1 || h->stdp || h->mixed || h->c1.passes != 0)
    return fail(PIC_ERR_UNSUPPORTED, "pic_grad_forward: the reverse mode is built for the FP64 "
                                     "1D form");
  if (h->pending) return fail(PIC_ERR_ARG, "pic_grad_forward: read the pending stats first");
  if (checkpoint_every > kStepsCap) checkpoint_every = kStepsCap;
  pic_handle::Grad &g = h->grad;
  const size_t N = (size_t)h->N, nc = (size_t)h->c1.nc, len = 2 * N + nc;
  const int nck = (nsteps + checkpoint_every - 1) / checkpoint_every;
  if ((size_t)nck * len > g.ckpt_cap) {
    if (g.ckpt) cudaFree(g.ckpt);
    g.ckpt = nullptr;
    g.ckpt_cap = 0;
    CUDA_TRY(cudaMalloc(&g.ckpt, sizeof(double) * nck * len));
    g.ckpt_cap = (size_t)nck * len;
  }
  g.start = h->steps_done;
  g.nsteps = nsteps;
  g.every = checkpoint_every;
  g.nck = nck;
  for (int k = 0; k < nsteps; k++) {
    if (k % checkpoint_every == 0)
      CUDA_TRY(state_copy(h, g.ckpt + (size_t)(k / checkpoint_every) * len, true));
    if (h->pending == kStepsCap) {
      int rc = pic_read_stats(h, 0, nullptr, nullptr, nullptr);
      if (rc) return rc;
    }
    int rc = pic_step_async(h, 1);
    if (rc) return rc;
  }
  return PIC_OK;
}

int pic_grad_backward(pic_handle *h, const double *Ebar, const double *xbar, const double *vbar,
                      double *Ebar0, double *xbar0, double *vbar0, double *wbar0) {
  if (!h) return fail(PIC_ERR_ARG, "pic_grad_backward: NULL handle");
  pic_handle::Grad &g = h->grad;
  if (g.start < 0 || h->steps_done != g.start + g.nsteps)
    return fail(PIC_ERR_ARG, "pic_grad_backward: no pic_grad_forward ends at the current step");
  int rc = pic_read_stats(h, 0, nullptr, nullptr, nullptr);
  if (rc) return rc;
  const size_t N = (size_t)h->N, nc = (size_t)h->c1.nc, len = 2 * N + nc;
  const int every = g.every;
  if (!g.fin) {
    CUDA_TRY(cudaMalloc(&g.fin, sizeof(double) * len));
    CUDA_TRY(cudaMalloc(&g.grid, sizeof(double) * 7 * nc));
    CUDA_TRY(cudaMalloc(&g.mk, sizeof(double) * 5 * N));
  }
  if ((size_t)(every + 1) * len > g.seg_cap) {
    if (g.seg) cudaFree(g.seg);
    g.seg = nullptr;
    g.seg_cap = 0;
    CUDA_TRY(cudaMalloc(&g.seg, sizeof(double) * (every + 1) * len));
    g.seg_cap = (size_t)(every + 1) * len;
  }
  CUDA_TRY(es1d_grad_prepare(h->c1));
  Es1dGradBufs gb{};
  gb.w = h->b1.w;
  for (int s = 0; s < h->nsp; s++) gb.w0[s] = h->sp[s].w0;
  gb.Estar = g.grid;
  gb.H = g.grid + nc;
  gb.J1 = g.grid + 2 * nc;
  gb.Hbar = g.grid + 3 * nc;
  gb.Esbar = g.grid + 4 * nc;
  gb.Jbar = g.grid + 5 * nc;
  gb.Ebar = g.grid + 6 * nc;
  gb.xbar = g.mk;
  gb.vbar = g.mk + N;
  gb.wbar = g.mk + 2 * N;
  gb.ub = g.mk + 3 * N;
  gb.yb = g.mk + 4 * N;
  gb.err = h->b1.err;
  // adjoints of the final state (NULL = 0)
  CUDA_TRY(cudaMemsetAsync(g.mk, 0, sizeof(double) * 5 * N, h->st));
  CUDA_TRY(cudaMemsetAsync(g.grid, 0, sizeof(double) * 7 * nc, h->st));
  if (Ebar) CUDA_TRY(cudaMemcpyAsync(gb.Ebar, Ebar, sizeof(double) * nc, cudaMemcpyDefault, h->st));
  if (xbar) CUDA_TRY(cudaMemcpyAsync(gb.xbar, xbar, sizeof(double) * N, cudaMemcpyDefault, h->st));
  if (vbar) CUDA_TRY(cudaMemcpyAsync(gb.vbar, vbar, sizeof(double) * N, cudaMemcpyDefault, h->st));
  CUDA_TRY(state_copy(h, g.fin, true));
  const int64_t fin_step = h->steps_done;
  for (int seg = g.nck - 1; seg >= 0; seg--) {
    const int s0 = seg * every, s1 = std::min(g.nsteps, s0 + every);
    // re-run the segment from its checkpoint, keeping every step's state
    h->steps_done = g.start + s0;
    CUDA_TRY(state_copy(h, g.ckpt + (size_t)seg * len, false));
    if ((rc = restart_es1d(h, false))) return rc;
    for (int k = s0; k < s1; k++) {
      CUDA_TRY(state_copy(h, g.seg + (size_t)(k - s0) * len, true));
      if ((rc = pic_step_async(h, 1))) return rc;
    }
    CUDA_TRY(state_copy(h, g.seg + (size_t)(s1 - s0) * len, true));
    if ((rc = pic_read_stats(h, 0, nullptr, nullptr, nullptr))) return rc;
    // reverse the segment's steps
    for (int k = s1 - 1; k >= s0; k--) {
      const double *st = g.seg + (size_t)(k - s0) * len, *nx = st + len;
      gb.x = st;
      gb.v = st + N;
      es1d_grad_step(h->c1, gb, st + 2 * N, nx + 2 * N, h->ls, h->st);
      CUDA_TRY(cudaGetLastError());
      h->launches += h->c1.scheme == 2 ? 7 : 6;
    }
  }
  // adjoints of the initial state
  if (Ebar0) CUDA_TRY(cudaMemcpyAsync(Ebar0, gb.Ebar, sizeof(double) * nc, cudaMemcpyDefault, h->st));
  if (xbar0) CUDA_TRY(cudaMemcpyAsync(xbar0, gb.xbar, sizeof(double) * N, cudaMemcpyDefault, h->st));
  if (vbar0) CUDA_TRY(cudaMemcpyAsync(vbar0, gb.vbar, sizeof(double) * N, cudaMemcpyDefault, h->st));
  if (wbar0) CUDA_TRY(cudaMemcpyAsync(wbar0, gb.wbar, sizeof(double) * N, cudaMemcpyDefault, h->st));
  // back to the state after the forward steps
  h->steps_done = fin_step;
  CUDA_TRY(state_copy(h, g.fin, false));
  if ((rc = restart_es1d(h, false))) return rc;
  CUDA_TRY(cudaStreamSynchronize(h->st));
  return check_flags(h, "pic_grad_backward");
}

// Sum over the species of q sum_p w_p (uniform species: q w0 n; weighted ones
// through a device reduction of their weights).
static int markers_charge(pic_handle *h, const double *w, double *Q) {
  double q = 0.0;
  for (int s = 0; s < h->nsp; s++) {
    const SpeciesInfo &S = h->sp[s];
    if (!S.weighted || !w) {
      q += S.q * S.w0 * (double)S.n;
      continue;
    }
    const int nb = std::max(1, std::min(h->diag.blocks, (int)((S.n + 255) / 256)));
    diag_sum_range(w + S.offset, S.n, h->diag.part, nb, h->st);
    CUDA_TRY(cudaGetLastError());
    std::vector<double> part(nb);
    CUDA_TRY(cudaMemcpyAsync(part.data(), h->diag.part, sizeof(double) * nb,
                             cudaMemcpyDeviceToHost, h->st));
    CUDA_TRY(cudaStreamSynchronize(h->st));
    double sw = 0.0;
    for (double v : part) sw += v;
    q += S.q * sw;
  }
  *Q = q;
  return PIC_OK;
}

int pic_charge(pic_handle *h, double *Q_markers, double *Q_grid, double *gauss_l2, double *rho_l2,
               double *residual) {
  if (!h) return fail(PIC_ERR_ARG, "pic_charge: NULL handle");
  if (h->stdp || h->em1)
    return fail(PIC_ERR_UNSUPPORTED, "pic_charge: built for the Ampere and Yee solvers");
  int rc;
  const int nodes = h->em ? h->ce.nx * h->ce.ny : h->c1.nc;
  auto &D = h->diag;
  if (!D.rho) {
    D.blocks = std::max(diag_blocks(nodes), 1024);
    if ((rc = h->alloc(&D.rho, (size_t)nodes)) || (rc = h->alloc(&D.r, (size_t)nodes)) ||
        (rc = h->alloc(&D.part, 3 * (size_t)D.blocks)))
      return rc;
    if (!h->em) {
      const int nc = h->c1.nc, M = std::max(1, (nc - 1) / 2);
      if ((rc = h->alloc(&D.tw, (size_t)nc)) || (rc = h->alloc(&D.rm, (size_t)M)) ||
          (rc = h->alloc(&D.pm, (size_t)M)) || (rc = h->alloc(&D.cnt, (size_t)nc)))
        return rc;
      std::vector<double2> tw(nc);
      const double twopi = 6.283185307179586476925286766559;
      for (int t = 0; t < nc; t++) tw[t] = make_double2(cos(twopi * t / nc), sin(twopi * t / nc));
      CUDA_TRY(cudaMemcpyAsync(D.tw, tw.data(), sizeof(double2) * nc, cudaMemcpyHostToDevice, h->st));
    }
  }
  double qm = 0.0, area = 0.0, mean = 0.0;
  const double *E = nullptr;
  if (h->em) {
    const Em2dConst &c = h->ce;
    if (h->mixed) {
      em2dm_to_fp64(h->cme, h->bme, h->be, h->lp, h->st);
      CUDA_TRY(cudaGetLastError());
    }
    if ((rc = markers_charge(h, h->be.w, &qm))) return rc;
    area = (c.Lx / c.nx) * (c.Ly / c.ny);
    mean = qm / (c.Lx * c.Ly);
    CUDA_TRY(cudaMemsetAsync(D.rho, 0, sizeof(double) * nodes, h->st));
    diag_em2d_charge(c, h->be.x, h->be.y, h->be.w, D.rho, h->lp, h->st);
    diag_em2d_gauss(c, h->be.E, D.rho, mean, D.r, D.part, h->st);
  } else {
    const Es1dConst &c = h->c1;
    area = c.h;
    if ((rc = markers_charge(h, h->b1.w, &qm))) return rc;
    if (h->mixed) {
      // the mixed form's own charge: its quantised weights summed exactly
      CUDA_TRY(cudaMemsetAsync(D.cnt, 0, sizeof(long long) * c.nc, h->st));
      es1d_mix_charge(h->cm, h->bm, D.cnt, h->ls, h->st);
      const SpeciesInfo &S = h->sp[0];
      diag_rho_from_counts(D.cnt, c.nc, S.q * S.w0 / c.h * std::ldexp(1.0, -23), D.rho, h->st);
    } else {
      CUDA_TRY(cudaMemsetAsync(D.rho, 0, sizeof(double) * nodes, h->st));
      es1d_fp64_charge(c, h->b1.x, h->b1.w, D.rho, h->ls, h->st);
    }
    E = h->b1.E[h->steps_done & 1];
    diag_gauss1d(E, D.rho, c.nc, c.L, D.tw, D.rm, D.pm, D.r, D.part, h->st);
  }
  CUDA_TRY(cudaGetLastError());
  const int nb = diag_blocks(nodes);
  std::vector<double> part(3 * (size_t)nb);
  CUDA_TRY(cudaMemcpyAsync(part.data(), D.part, sizeof(double) * part.size(),
                           cudaMemcpyDeviceToHost, h->st));
  if (residual)
    CUDA_TRY(cudaMemcpyAsync(residual, D.r, sizeof(double) * nodes, cudaMemcpyDefault, h->st));
  CUDA_TRY(cudaStreamSynchronize(h->st));
  double r2 = 0.0, p2 = 0.0, rs = 0.0;
  for (int b = 0; b < nb; b++) {
    r2 += part[3 * b];
    p2 += part[3 * b + 1];
    rs += part[3 * b + 2];
  }
  if (Q_markers) *Q_markers = qm;
  if (Q_grid) *Q_grid = area * rs;
  if (gauss_l2) *gauss_l2 = std::sqrt(area * r2);
  if (rho_l2) *rho_l2 = std::sqrt(area * p2);
  return PIC_OK;
}

int pic_mixed_resolution(pic_handle *h, double *dx, double *dv, int *deposit_bits) {
  if (!h) return fail(PIC_ERR_ARG, "pic_mixed_resolution: NULL handle");
  if (!h->mixed) return fail(PIC_ERR_UNSUPPORTED, "pic_mixed_resolution: not a mixed-form handle");
  double L, cxk;
  int T;
  if (h->em) {
    L = h->cme.L;
    cxk = h->cme.cxk;
    T = 77 - h->cme.rshift;   // V* (31 bits) times two 23-bit weights
  } else if (h->em1) {
    L = h->c1m.L;
    cxk = h->c1m.cxk;
    T = 54 - h->c1m.rshift;
  } else {
    L = h->cm.L;
    cxk = h->cm.cxk;
    T = 54 - h->cm.rshift;
  }
  if (dx) *dx = L / 4294967296.0;
  if (dv) *dv = 1.0 / cxk;
  if (deposit_bits) *deposit_bits = T;
  return PIC_OK;
}

int pic_step_count(pic_handle *h, int64_t *steps) {
  if (!h || !steps) return fail(PIC_ERR_ARG, "pic_step_count: bad arguments");
  *steps = h->steps_done;
  return PIC_OK;
}

void pic_free(pic_handle *h) {
  if (!h) return;
  if (h->st) cudaStreamSynchronize(h->st);
  else cudaDeviceSynchronize();
  delete h;
}

}  // extern "C"

// ------------------------------------------------------------------ batches
// Independent 1D runs of the mixed form stepped together: one launch per pass
// for all runs, over a work list of (run, block of the run).  The runs are
// ordinary handles (their accessors work); only their stepping and stats go
// through the batch.
struct pic_batch {
  std::vector<pic_handle *> runs;
  cudaStream_t st = nullptr;
  cudaStream_t own = nullptr;  // created when the runs were given no stream
  int scheme = 2;
  size_t smem = 0;
  int nitems = 0;
  int trips = 8;  // target 4-marker trips per block of a run
  int threads = 1024;  // block size of the passes (256 for batches of small runs)
  bool prev_closed = false;  // the last pending step's TE was reduced already
  Es1dMixConst *d_c = nullptr;
  Es1dMixBufs *d_b = nullptr;
  BatchItem *d_items = nullptr;
  int *d_nb = nullptr;
  unsigned long long *d_fb = nullptr;  // [runs][kStepsCap] gathered counts
  double *d_te = nullptr;              // [runs][kStepsCap] gathered energies
  int64_t steps_done = 0;
  int pending = 0;
  int64_t launches = 0;
  bool use_graph = false;
  struct Graph {
    int steps, parity;
    cudaGraphExec_t exec;
  };
  std::vector<Graph> graphs;
  ~pic_batch() {
    if (st) cudaStreamSynchronize(st);
    for (Graph &g : graphs) cudaGraphExecDestroy(g.exec);
    for (void *p : {(void *)d_c, (void *)d_b, (void *)d_items, (void *)d_nb, (void *)d_fb,
                    (void *)d_te})
      if (p) cudaFree(p);
    for (pic_handle *h : runs) pic_free(h);
    if (own) cudaStreamDestroy(own);
  }
  // The launches of nsteps steps from the current step count, on st.
  void enqueue(int nsteps, int first_slot) {
    for (int k = 0; k < nsteps; k++) {
      const int64_t step = steps_done + k;
      const int prev = (k == 0 && prev_closed) ? -1 : first_slot + k - 1;
      es1d_batch_pass_c(d_c, d_b, d_items, nitems, scheme, threads, smem, step, prev, st);
      es1d_batch_pass_e(d_c, d_b, d_items, nitems, scheme, threads, smem, step, first_slot + k,
                        st);
    }
    if (nsteps > 0) prev_closed = false;
  }
};

namespace {
// Blocks per run: about `trips` 4-marker trips each (at most 16, the bound the
// runs' integer tiles are sized for).
constexpr int kBatchTrips = 8;
// A batch whose runs all have at most this many markers runs 256-thread blocks.
constexpr int64_t kBatchSmallRun = 1 << 15;

// trips of a run of ngroups 4-marker groups over nb blocks of `threads`
int64_t batch_trips(int64_t ngroups, int nb, int threads) {
  return (ngroups + (int64_t)nb * threads - 1) / ((int64_t)nb * threads);
}

// Work list of a batch for a trip target; returns the blocks per run.
std::vector<int> batch_items(const std::vector<pic_handle *> &runs, int trips, int threads,
                             std::vector<BatchItem> &items) {
  std::vector<int> nbs;
  items.clear();
  for (int r = 0; r < (int)runs.size(); r++) {
    const pic_handle *h = runs[r];
    const int64_t ngroups = (h->N + 3) / 4;
    int nb = (int)std::max<int64_t>(1, (ngroups + (int64_t)threads * trips - 1) /
                                           ((int64_t)threads * trips));
    nb = std::min(nb, h->ls.grid);  // the run's per-block partials hold ls.grid entries
    while (batch_trips(ngroups, nb, threads) > 16 && nb < h->ls.grid) nb++;
    nbs.push_back(nb);
    for (int k = 0; k < nb; k++) items.push_back(BatchItem{r, k, nb});
  }
  return nbs;
}

// Tuned trip targets, per (runs, log2 of all markers, largest grid) in this process.
std::map<std::tuple<int, int, int>, int> g_batch_tuned;
}  // namespace

extern "C" {

int pic_batch_init(const pic_config *cfgs, const pic_species *species, int nruns,
                   pic_batch **out) {
  if (!cfgs || !species || !out || nruns <= 0)
    return fail(PIC_ERR_ARG, "pic_batch_init: bad arguments");
  *out = nullptr;
  for (int r = 0; r < nruns; r++) {
    const pic_config &c = cfgs[r];
    if (c.solver != PIC_SOLVER_AMPERE_ES || c.precision != PIC_PREC_MIXED || c.sort_period != 0 ||
        c.grid.n[0] > kWideMaxNodes || c.scheme != cfgs[0].scheme ||
        c.cuda_stream != cfgs[0].cuda_stream || c.gamma_fp64 != 0 || c.binomial_passes != 0)
      return fail(PIC_ERR_UNSUPPORTED,
                  "pic_batch_init: run %d: batches take unsorted mixed-form 1D runs with at most "
                  "%d nodes, one scheme, one stream, gamma_fp64 = 0 and no filter", r,
                  kWideMaxNodes);
  }
  pic_batch *b = new pic_batch();
  b->scheme = cfgs[0].scheme;
  b->threads = 256;
  for (int r = 0; r < nruns; r++)
    if (species[r].n > kBatchSmallRun) b->threads = 1024;
  std::vector<Es1dMixConst> hc(nruns);
  std::vector<Es1dMixBufs> hb(nruns);
  std::vector<BatchItem> items;
  std::vector<int> nbs(nruns);
  for (int r = 0; r < nruns; r++) {
    pic_handle *h = nullptr;
    int rc = pic_init(&cfgs[r], &species[r], 1, nullptr, nullptr, &h);
    if (rc) {
      std::string msg = g_last_error;
      delete b;
      return fail(rc, "pic_batch_init: run %d: %s", r, msg.c_str());
    }
    b->runs.push_back(h);
    if (!h->cm.wide) {
      delete b;
      return fail(PIC_ERR_UNSUPPORTED, "pic_batch_init: run %d is not in the wide layout", r);
    }
    b->st = h->st;
    hc[r] = h->cm;
    hb[r] = h->bm;
    b->smem = std::max(b->smem, es1d_batch_smem(h->cm, b->threads));
  }
  b->trips = kBatchTrips;
  nbs = batch_items(b->runs, b->trips, b->threads, items);
  for (int r = 0; r < nruns; r++) {
    const int64_t ngroups = (b->runs[r]->N + 3) / 4;
    if (batch_trips(ngroups, nbs[r], b->threads) > 16) {
      delete b;
      return fail(PIC_ERR_UNSUPPORTED, "pic_batch_init: run %d is too large for a batch", r);
    }
  }
  b->nitems = (int)items.size();
  if (!cfgs[0].cuda_stream) {
    // the legacy default stream cannot be captured into a graph: the batch and
    // its runs move to a stream of their own
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->own, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      delete b;
      return fail(PIC_ERR_CUDA, "pic_batch_init: %s", cudaGetErrorString(e));
    }
    b->st = b->own;
    for (pic_handle *h : b->runs) h->st = b->own;
  }
  auto up = [&](auto **dst, const auto &v) -> cudaError_t {
    cudaError_t e = cudaMalloc((void **)dst, sizeof(v[0]) * v.size());
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(*dst, v.data(), sizeof(v[0]) * v.size(), cudaMemcpyHostToDevice, b->st);
    return e;
  };
  cudaError_t e = up(&b->d_c, hc);
  if (e == cudaSuccess) e = up(&b->d_b, hb);
  if (e == cudaSuccess) e = up(&b->d_items, items);
  if (e == cudaSuccess) e = up(&b->d_nb, nbs);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_fb, sizeof(unsigned long long) * kStepsCap * nruns);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_te, sizeof(double) * kStepsCap * nruns);
  if (e == cudaSuccess) e = es1d_batch_prepare(b->smem, b->threads);
  for (int r = 0; r < nruns && e == cudaSuccess; r++)
    e = cudaMemsetAsync(hb[r].fallback, 0, sizeof(unsigned long long) * kStepsCap, b->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);
  if (e != cudaSuccess) {
    delete b;
    return fail(e == cudaErrorMemoryAllocation ? PIC_ERR_OOM : PIC_ERR_CUDA,
                "pic_batch_init: %s", cudaGetErrorString(e));
  }
  *out = b;
  return PIC_OK;
}

// Replaces the work list for a new trip target (the graphs captured with the
// old list are dropped).
static int batch_retarget(pic_batch *b, int trips) {
  std::vector<BatchItem> items;
  std::vector<int> nbs = batch_items(b->runs, trips, b->threads, items);
  for (int r = 0; r < (int)b->runs.size(); r++) {
    const int64_t ngroups = (b->runs[r]->N + 3) / 4;
    if (batch_trips(ngroups, nbs[r], b->threads) > 16) return PIC_OK;
  }
  CUDA_TRY(cudaStreamSynchronize(b->st));
  if (b->pending && !b->prev_closed) {
    // the energy of the last pending step is reduced over the old work list's
    // block partials now, and not again by the next step's pass C
    es1d_batch_finalize(b->d_c, b->d_b, b->d_nb, (int)b->runs.size(), b->pending - 1, b->st);
    CUDA_TRY(cudaGetLastError());
    b->prev_closed = true;
  }
  cudaFree(b->d_items);
  cudaFree(b->d_nb);
  b->d_items = nullptr;
  b->d_nb = nullptr;
  CUDA_TRY(cudaMalloc(&b->d_items, sizeof(BatchItem) * items.size()));
  CUDA_TRY(cudaMalloc(&b->d_nb, sizeof(int) * nbs.size()));
  CUDA_TRY(cudaMemcpy(b->d_items, items.data(), sizeof(BatchItem) * items.size(),
                      cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(b->d_nb, nbs.data(), sizeof(int) * nbs.size(), cudaMemcpyHostToDevice));
  for (auto &g : b->graphs) cudaGraphExecDestroy(g.exec);
  b->graphs.clear();
  b->nitems = (int)items.size();
  b->trips = trips;
  return PIC_OK;
}

int pic_batch_set_graph(pic_batch *b, int on) {
  if (!b) return fail(PIC_ERR_ARG, "pic_batch_set_graph: NULL batch");
  b->use_graph = on != 0;
  return PIC_OK;
}

int pic_batch_autotune(pic_batch *b, int steps_per_trial, int *trips) {
  if (!b || steps_per_trial <= 0) return fail(PIC_ERR_ARG, "pic_batch_autotune: bad arguments");
  int64_t markers = 0;
  int ncmax = 0;
  for (pic_handle *h : b->runs) {
    markers += h->N;
    ncmax = std::max(ncmax, h->cm.nc);
  }
  int lg = 0;
  while (((int64_t)1 << lg) < markers) lg++;
  const auto key = std::make_tuple((int)b->runs.size(), lg, ncmax);
  auto it = g_batch_tuned.find(key);
  int best = b->trips;
  if (it != g_batch_tuned.end()) {
    best = it->second;
  } else {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CUDA_TRY(cudaEventCreate(&e0));
    CUDA_TRY(cudaEventCreate(&e1));
    float best_ms = 1e30f;
    for (int t : {4, 8, 16}) {
      if (b->pending + steps_per_trial > kStepsCap) break;
      int rc = batch_retarget(b, t);
      if (rc) return rc;
      if (b->trips != t) continue;  // this target would break the tiles' bound
      CUDA_TRY(cudaEventRecord(e0, b->st));
      b->enqueue(steps_per_trial, b->pending);
      CUDA_TRY(cudaEventRecord(e1, b->st));
      CUDA_TRY(cudaEventSynchronize(e1));
      float ms = 0.f;
      CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
      b->launches += 2 * steps_per_trial;
      b->steps_done += steps_per_trial;
      b->pending += steps_per_trial;
      for (pic_handle *h : b->runs) h->steps_done += steps_per_trial;
      if (ms < best_ms) {
        best_ms = ms;
        best = t;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    g_batch_tuned[key] = best;
  }
  int rc = batch_retarget(b, best);
  if (rc) return rc;
  if (trips) *trips = b->trips;
  return PIC_OK;
}

int pic_batch_step(pic_batch *b, int nsteps) {
  if (!b || nsteps < 0) return fail(PIC_ERR_ARG, "pic_batch_step: bad arguments");
  if (b->pending + nsteps > kStepsCap)
    return fail(PIC_ERR_ARG, "pic_batch_step: %d steps pending, at most %d before "
                             "pic_batch_read_stats", b->pending + nsteps, kStepsCap);
  if (nsteps == 0) return PIC_OK;
  const int parity = (int)(b->steps_done & 1);
  if (b->use_graph && b->pending == 0) {
    // the same launches for the same step count and parity replay one graph
    cudaGraphExec_t exec = nullptr;
    for (auto &g : b->graphs)
      if (g.steps == nsteps && g.parity == parity) exec = g.exec;
    if (!exec) {
      cudaGraph_t graph = nullptr;
      CUDA_TRY(cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal));
      b->enqueue(nsteps, 0);
      cudaError_t e = cudaStreamEndCapture(b->st, &graph);
      if (e == cudaSuccess) e = cudaGetLastError();
      if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
      if (graph) cudaGraphDestroy(graph);
      CUDA_TRY(e);
      b->graphs.push_back({nsteps, parity, exec});
    }
    CUDA_TRY(cudaGraphLaunch(exec, b->st));
  } else {
    b->enqueue(nsteps, b->pending);
    CUDA_TRY(cudaGetLastError());
  }
  b->launches += 2 * nsteps;
  b->steps_done += nsteps;
  b->pending += nsteps;
  for (pic_handle *h : b->runs) h->steps_done += nsteps;
  return PIC_OK;
}

int pic_batch_read_stats(pic_batch *b, int capacity, int64_t *nfallback, double *te, int *nread) {
  if (!b) return fail(PIC_ERR_ARG, "pic_batch_read_stats: NULL batch");
  const int n = b->pending, nruns = (int)b->runs.size();
  if (nread) *nread = n;
  if (n > 0) {
    if ((nfallback || te) && capacity < n)
      return fail(PIC_ERR_ARG, "pic_batch_read_stats: %d steps pending, capacity %d", n,
                  capacity);
    if (!b->prev_closed) es1d_batch_finalize(b->d_c, b->d_b, b->d_nb, nruns, n - 1, b->st);
    b->prev_closed = false;
    es1d_batch_gather_stats(b->d_b, nruns, n, b->d_fb, b->d_te, b->st);
    CUDA_TRY(cudaGetLastError());
    b->launches += 2;
    std::vector<unsigned long long> fb((size_t)n * nruns);
    std::vector<double> tv((size_t)n * nruns);
    CUDA_TRY(cudaMemcpyAsync(fb.data(), b->d_fb, sizeof(unsigned long long) * fb.size(),
                             cudaMemcpyDeviceToHost, b->st));
    CUDA_TRY(cudaMemcpyAsync(tv.data(), b->d_te, sizeof(double) * tv.size(),
                             cudaMemcpyDeviceToHost, b->st));
    CUDA_TRY(cudaStreamSynchronize(b->st));
    for (int r = 0; r < nruns; r++)
      for (int k = 0; k < n; k++) {
        if (nfallback) nfallback[(size_t)r * capacity + k] = (int64_t)fb[(size_t)r * n + k];
        if (te) te[(size_t)r * capacity + k] = tv[(size_t)r * n + k];
      }
    b->pending = 0;
  }
  for (pic_handle *h : b->runs) {
    int rc = check_flags(h, "pic_batch_read_stats");
    if (rc) return rc;
  }
  return PIC_OK;
}

int pic_batch_run(pic_batch *b, int run, pic_handle **h) {
  if (!b || !h || run < 0 || run >= (int)b->runs.size())
    return fail(PIC_ERR_ARG, "pic_batch_run: bad arguments");
  *h = b->runs[run];
  return PIC_OK;
}

int pic_batch_info(pic_batch *b, int *nruns, int *nblocks, int64_t *launches) {
  if (!b) return fail(PIC_ERR_ARG, "pic_batch_info: NULL batch");
  if (nruns) *nruns = (int)b->runs.size();
  if (nblocks) *nblocks = b->nitems;
  if (launches) *launches = b->launches;
  return PIC_OK;
}

void pic_batch_free(pic_batch *b) { delete b; }

}  // extern "C"
