// Programmatic dependent launch.  A kernel launched with launch_dependent may
// be scheduled while the previous kernel in the stream is still running: it
// calls griddep_wait() before it reads or writes anything the previous kernels
// touch (the wait returns once they have completed and their writes are
// visible), and griddep_launch_dependents() lets the next such kernel be
// scheduled.  In a kernel launched the ordinary way both are no-ops.
#pragma once

#include <cuda_runtime.h>

#include "pic_internal.cuh"

namespace pic {

__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Launches kern with programmatic stream serialization when pdl is set, the
// ordinary way otherwise; errors surface in cudaGetLastError.
template <typename... P, typename... A>
void launch_dependent(void (*kern)(P...), LaunchShape ls, size_t smem, cudaStream_t st, bool pdl,
                      A... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(ls.grid);
  cfg.blockDim = dim3(ls.block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl ? 1 : 0;
  cudaLaunchKernelEx(&cfg, kern, args...);
}

}  // namespace pic
