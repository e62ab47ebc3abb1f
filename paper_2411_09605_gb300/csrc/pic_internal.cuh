// Internal declarations shared by the library's translation units (not part of
// the C ABI; the public interface is include/pic.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "pic.h"

namespace pic {

constexpr int kMaxSpecies = 8;
constexpr int kMaxNodes1D = 8192;   // 1D grid held whole in shared memory

// Device-side error flags (bit set by kernels, read by the host after a call).
enum : unsigned { kErrNonfinite = 1u, kErrBounds = 2u, kErrVelocityRange = 4u, kErrTimeout = 8u };

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

// Everything the 1D FP64 kernels touch.
struct Es1dFp64Bufs {
  double *x, *v, *w;        // [N] SoA (w may be null)
  double *E[2];             // ping-pong E^n / E^{n+1}
  double *J1[2];            // j^{n,*} (ESEC2), indexed by step parity
  double *J2[2];            // j^{*,n+1/2}
  double *ke_part;          // [grid] block partials of KE of the step just done
  unsigned long long *fallback;   // [steps_cap] per-step counters
  double *te;               // [steps_cap] total energy after each step
  double *we;               // [1] W_E of the newest field
  unsigned *err;            // device error flags
};

struct LaunchShape {
  int grid;
  int block;
};

// Sets the message returned by pic_last_error (pic_api.cu).
void set_last_error(const std::string &msg);

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

}  // namespace pic
