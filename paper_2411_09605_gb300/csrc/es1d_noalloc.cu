// pic_es1d_step_noalloc: the 1D1V FP64 step on caller-owned device buffers,
// with every piece of scratch memory taken from one fixed, file-scope device
// array instead of cudaMalloc.
//
// Some callers cannot let a library allocate device memory: a host framework
// that owns the whole device heap through its own pool and forbids plugins from
// calling cudaMalloc/cudaFree (those calls would also synchronise the device),
// or a long-running service whose memory budget is fixed when it starts.  This
// entry point runs the same pass C / pass E kernels as pic_step with all of
// their scratch (currents, the alternate field buffer, block partials, per-step
// counters, error flags) carved out of g_noalloc_scratch.
//
// The array is a static device object: every GPU that loads the library holds
// kNoallocScratchBytes of it until the process exits, and every call on a
// device shares it (the contents of the last call remain; what must start at
// zero is cleared at the start of each call).  Calls that overlap on the GPU
// (two streams, or two host threads) race on it and must be serialised by the
// caller.  Host code cannot use the array's name as a device address, so every
// call looks the address up (cudaGetSymbolAddress) on the current device; no
// address is kept between calls, so a call made after the device's context was
// reset sees the array of the new context.
//
// The inputs are checked before any step runs: a position outside [0, L) or a
// non-finite velocity or field value returns an error with x, v and E as the
// caller passed them.
#include <cuda_runtime.h>

#include <string>

#include "pic_internal.cuh"

namespace pic {
namespace {

// Scratch layout (bytes): E_alt, J1[2], J2[2] (8192 doubles each), block
// partials (1024 doubles), per-step energies (1024 doubles), W_E (1 double),
// per-step fallback counters (1024 x u64), device error flags.  v* is not
// kept between the passes (that would take N doubles): the buffer's v* array
// stays null and pass E recomputes v* from the same E* table.
constexpr int kNoallocMaxNodes = kMaxNodes1D;
constexpr int kNoallocMaxSteps = 1024;
constexpr int kNoallocMaxBlocks = 1024;
constexpr size_t kNoallocScratchBytes =
    sizeof(double) * (5 * (size_t)kNoallocMaxNodes + kNoallocMaxBlocks + kNoallocMaxSteps + 8) +
    sizeof(unsigned long long) * kNoallocMaxSteps + 256;

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

int noalloc_fail(int code, const char *msg, cudaError_t e = cudaSuccess) {
  std::string m = msg;
  if (e != cudaSuccess) {
    m += ": ";
    m += cudaGetErrorString(e);
  }
  set_last_error(m);
  return code;
}

// Flags positions outside [0, L) and non-finite velocities and field values.
__global__ void noalloc_validate_kernel(const double *x, const double *v, int64_t n,
                                        const double *E, int nc, double L, unsigned *err) {
  unsigned bad = 0;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    double a = x[p], b = v[p];
    if (!(a >= 0.0 && a < L)) bad |= kErrBounds;
    if (!isfinite(b)) bad |= kErrNonfinite;
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += gridDim.x * blockDim.x)
    if (!isfinite(E[i])) bad |= kErrNonfinite;
  if (bad) atomicOr(err, bad);
}

bool is_device_pointer(const void *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace
}  // namespace pic

using namespace pic;

extern "C" int pic_es1d_step_noalloc(const pic_config *cfg, double q, double m, double w0,
                                     int64_t n, double *x, double *v, double *E, int nsteps,
                                     int64_t *nfallback_per_step, double *te_per_step) {
  if (!cfg) return noalloc_fail(PIC_ERR_ARG, "pic_es1d_step_noalloc: cfg is NULL");
  if (cfg->solver != PIC_SOLVER_AMPERE_ES || cfg->grid.dim_x != 1 || cfg->grid.dim_v != 1 ||
      cfg->precision != PIC_PREC_FP64 || cfg->binomial_passes != 0 || cfg->charge_conserving != 0)
    return noalloc_fail(PIC_ERR_ARG,
                        "pic_es1d_step_noalloc: needs the 1D1V Ampere solver in FP64 form, "
                        "without filtering (binomial_passes = 0, charge_conserving = 0)");
  const int64_t nc = cfg->grid.n[0];
  if (nc < 4 || nc > kNoallocMaxNodes)
    return noalloc_fail(PIC_ERR_ARG, "pic_es1d_step_noalloc: grid must have 4..8192 nodes "
                                     "(the fixed scratch holds at most 8192)");
  if (nsteps < 0 || nsteps > kNoallocMaxSteps)
    return noalloc_fail(PIC_ERR_ARG, "pic_es1d_step_noalloc: nsteps must be in 0..1024 "
                                     "(the fixed scratch keeps at most 1024 per-step records)");
  if (cfg->shape_order != 1 && cfg->shape_order != 2)
    return noalloc_fail(PIC_ERR_ARG, "pic_es1d_step_noalloc: shape_order must be 1 or 2");
  if (cfg->scheme != PIC_SCHEME_ESEC1 && cfg->scheme != PIC_SCHEME_ESEC2)
    return noalloc_fail(PIC_ERR_ARG, "pic_es1d_step_noalloc: unknown scheme");
  if (!(cfg->dt > 0.0) || !(cfg->grid.L[0] > 0.0) || !(m > 0.0) || n < 0)
    return noalloc_fail(PIC_ERR_ARG, "pic_es1d_step_noalloc: needs dt > 0, L > 0, m > 0, n >= 0");
  if (!E || (n > 0 && (!x || !v)))
    return noalloc_fail(PIC_ERR_ARG, "pic_es1d_step_noalloc: x, v and E are required");
  if (!is_device_pointer(E) || (n > 0 && (!is_device_pointer(x) || !is_device_pointer(v))))
    return noalloc_fail(PIC_ERR_ARG, "pic_es1d_step_noalloc: x, v and E must be device memory");
  if (nsteps == 0) return PIC_OK;

  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return noalloc_fail(PIC_ERR_CUDA, "pic_es1d_step_noalloc: device query", e);
  // the array's address in the current device's context, looked up on every
  // call (nothing is cached across calls or devices)
  void *ptr = nullptr;
  e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
  if (e != cudaSuccess || !ptr)
    return noalloc_fail(PIC_ERR_CUDA, "pic_es1d_step_noalloc: cudaGetSymbolAddress", e);
  unsigned char *base = (unsigned char *)ptr;

  Es1dConst c{};
  c.nc = (int)nc;
  c.order = cfg->shape_order;
  c.scheme = cfg->scheme;
  c.remove_mean = cfg->remove_mean;
  c.gamma_on = cfg->gamma_on;
  c.nsp = 1;
  c.n_total = n;
  c.L = cfg->grid.L[0];
  c.h = c.L / (double)nc;
  c.inv_h = (double)nc / c.L;
  c.dt = cfg->dt;
  for (int s = 0; s < kMaxSpecies; s++) c.sp_end[s] = n;
  c.qm[0] = q / m;
  c.qw_h[0] = q * w0 / c.h;
  c.q_h[0] = q / c.h;
  c.half_mw[0] = 0.5 * m * w0;
  c.half_m[0] = 0.5 * m;

  LaunchShape ls;
  ls.block = 512;
  int64_t want = (n + 511) / 512;
  ls.grid = (int)(want < 1 ? 1 : (want < (int64_t)nsm * 2 ? want : (int64_t)nsm * 2));
  if (ls.grid > kNoallocMaxBlocks) ls.grid = kNoallocMaxBlocks;

  double *d = (double *)base;
  Es1dFp64Bufs b{};
  b.x = x;
  b.v = v;
  b.w = nullptr;
  b.E[0] = E;
  b.E[1] = d;
  b.J1[0] = d + 1 * kNoallocMaxNodes;
  b.J1[1] = d + 2 * kNoallocMaxNodes;
  b.J2[0] = d + 3 * kNoallocMaxNodes;
  b.J2[1] = d + 4 * kNoallocMaxNodes;
  b.ke_part = d + 5 * kNoallocMaxNodes;
  b.te = b.ke_part + kNoallocMaxBlocks;
  b.we = b.te + kNoallocMaxSteps;
  b.fallback = (unsigned long long *)(b.we + 8);
  b.err = (unsigned *)(b.fallback + kNoallocMaxSteps);

  cudaStream_t st = (cudaStream_t)cfg->cuda_stream;
  e = es1d_fp64_prepare(c);
  if (e != cudaSuccess) return noalloc_fail(PIC_ERR_CUDA, "pic_es1d_step_noalloc: kernel setup", e);
  // clear what must start at zero: currents, counters, flags
  e = cudaMemsetAsync(b.J1[0], 0, sizeof(double) * 4 * kNoallocMaxNodes, st);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(b.fallback, 0, sizeof(unsigned long long) * kNoallocMaxSteps, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(b.err, 0, sizeof(unsigned), st);
  if (e != cudaSuccess) return noalloc_fail(PIC_ERR_CUDA, "pic_es1d_step_noalloc: clear scratch", e);
  // validate before stepping: a bad input returns with x, v and E untouched
  {
    noalloc_validate_kernel<<<ls.grid, 256, 0, st>>>(x, v, n, E, (int)nc, c.L, b.err);
    unsigned pre = 0;
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&pre, b.err, sizeof pre, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return noalloc_fail(PIC_ERR_CUDA, "pic_es1d_step_noalloc: validation", e);
    if (pre & kErrNonfinite)
      return noalloc_fail(PIC_ERR_NONFINITE,
                          "pic_es1d_step_noalloc: non-finite velocity or field on input");
    if (pre & kErrBounds)
      return noalloc_fail(PIC_ERR_BOUNDS, "pic_es1d_step_noalloc: a position is outside [0, L)");
  }
  if (c.scheme == 2) es1d_fp64_deposit_initial(c, b, 0, ls, st);
  for (int k = 0; k < nsteps; k++) {
    es1d_fp64_pass_c(c, b, k, k, ls, st);
    es1d_fp64_pass_e(c, b, k, k, ls, st);
  }
  es1d_fp64_finalize(c, b, nsteps - 1, ls.grid, st);
  e = cudaGetLastError();
  if (e != cudaSuccess) return noalloc_fail(PIC_ERR_CUDA, "pic_es1d_step_noalloc: launch", e);
  if (nsteps & 1) {  // E^{n+nsteps} sits in the alternate buffer
    e = cudaMemcpyAsync(E, b.E[1], sizeof(double) * nc, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return noalloc_fail(PIC_ERR_CUDA, "pic_es1d_step_noalloc: copy E", e);
  }
  if (nfallback_per_step)
    e = cudaMemcpyAsync(nfallback_per_step, b.fallback, sizeof(int64_t) * nsteps,
                        cudaMemcpyDefault, st);
  if (e == cudaSuccess && te_per_step)
    e = cudaMemcpyAsync(te_per_step, b.te, sizeof(double) * nsteps, cudaMemcpyDefault, st);
  unsigned flags = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&flags, b.err, sizeof flags, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return noalloc_fail(PIC_ERR_CUDA, "pic_es1d_step_noalloc: readback", e);
  if (flags & kErrNonfinite)
    return noalloc_fail(PIC_ERR_NONFINITE, "pic_es1d_step_noalloc: non-finite value in the state");
  if (flags & kErrBounds)
    return noalloc_fail(PIC_ERR_BOUNDS, "pic_es1d_step_noalloc: a position is outside [0, L)");
  return PIC_OK;
}
