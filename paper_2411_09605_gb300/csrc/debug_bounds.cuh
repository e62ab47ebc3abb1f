// Index checks of the debug-bounds build.
//
// The mixed forms index shared-memory tiles, grid arrays and sort slots with
// arithmetic whose range follows from invariants rather than from a test on
// the index: a 32-bit fixed-point position puts the first node of a shape in
// a known range, the one-sided periodic wraps of the 2D shapes cover exactly
// the nodes that can leave [0, n), the slots of a sort on write are counts
// taken in an earlier pass.  A library compiled with -DPIC_DEBUG_BOUNDS checks
// these ranges where the index is formed: PIC_INDEX(i, n) yields i when
// 0 <= i < n and otherwise records the check's file and line and yields 0, so
// that the access it feeds stays in bounds (the result is then wrong, and
// flagged).  Each translation unit keeps its own record (a device variable of
// internal linkage, as the library is not compiled with relocatable device
// code) and exports a host function that reads and clears it; the library's
// flag checks collect them and turn a record into PIC_ERR_BOUNDS with the
// file and line in pic_last_error().  Without the macro PIC_INDEX(i, n) is i
// and the kernels are the normal build's.
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

namespace pic {

// the files that hold checks (index 0: none recorded)
constexpr const char *kBoundsFiles[] = {"", "mixed_common.cuh", "es1d_mixed.cu",
                                        "em2d_mixed.cu", "em1d_spectral.cu", "pic_api.cu"};
constexpr int kBoundsNumFiles = (int)(sizeof kBoundsFiles / sizeof kBoundsFiles[0]);

constexpr bool bounds_ends_with(const char *s, const char *t) {
  int ns = 0, nt = 0;
  while (s[ns]) ns++;
  while (t[nt]) nt++;
  if (nt > ns) return false;
  for (int i = 0; i < nt; i++)
    if (s[ns - nt + i] != t[i]) return false;
  return nt > 0 && (ns == nt || s[ns - nt - 1] == '/' || s[ns - nt - 1] == '\\');
}
constexpr unsigned bounds_file_code(const char *path) {
  for (int i = 1; i < kBoundsNumFiles; i++)
    if (bounds_ends_with(path, kBoundsFiles[i])) return (unsigned)i;
  return 0u;
}
// a record: file code in the high 16 bits, line in the low 16
inline const char *bounds_file_name(unsigned site) {
  const unsigned f = site >> 16;
  return f < (unsigned)kBoundsNumFiles && f > 0 ? kBoundsFiles[f] : "?";
}

#ifdef PIC_DEBUG_BOUNDS
// first failed check of this unit (0: none)
static __device__ unsigned g_bounds_site;

static __device__ __noinline__ void bounds_fail(unsigned site) {
  atomicCAS(&g_bounds_site, 0u, site);
}

template <typename I>
static __device__ __forceinline__ I bounds_index(I i, long long n, unsigned site) {
  if ((long long)i >= 0 && (long long)i < n) return i;
  bounds_fail(site);
  return I(0);
}

#define PIC_BOUNDS_SITE \
  ((std::integral_constant<unsigned, ::pic::bounds_file_code(__FILE__)>::value << 16) | \
   ((unsigned)__LINE__ & 0xFFFFu))
#define PIC_INDEX(i, n) ::pic::bounds_index((i), (long long)(n), PIC_BOUNDS_SITE)
// host function NAME() returning this unit's record (0: none) and clearing it
#define PIC_BOUNDS_READER(NAME)                                              \
  unsigned NAME() {                                                          \
    unsigned v = 0;                                                          \
    if (cudaMemcpyFromSymbol(&v, g_bounds_site, sizeof v) != cudaSuccess) v = 0; \
    if (v) {                                                                 \
      const unsigned z = 0;                                                  \
      cudaMemcpyToSymbol(g_bounds_site, &z, sizeof z);                       \
    }                                                                        \
    return v;                                                                \
  }
#else
#define PIC_INDEX(i, n) (i)
#define PIC_BOUNDS_READER(NAME)
#endif

}  // namespace pic
