// Programmatic dependent launch for the kernels of the solver loops (Krylov iterations, refinement
// residuals) and of the FNO.
//
// A kernel launched with launch_pdl may be scheduled before the kernel ahead of it on the stream
// has fully retired (the driver overlaps the two launches' set-up).  Its first statement is
// pdl_enter(): griddepcontrol.wait blocks until that predecessor has completed and its memory is
// visible (it returns at once after a plain launch), so nothing is read or written early.  The
// kernels do not release their dependents explicitly (griddepcontrol.launch_dependents at entry
// measured slower: the next kernel's waiting CTAs took SM slots from the running one's tail), so
// the release is the implicit one at block exit.
#pragma once
#include <cuda_runtime.h>

#include <utility>

__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}
