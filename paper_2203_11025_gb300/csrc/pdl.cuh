// Programmatic dependent launch for the kernels of one solve chain.
//
// A kernel launched by launch_pdl may be scheduled while the previous kernel in the
// stream is still running; it must call griddep_wait() before it reads or writes global
// memory (the wait returns once that kernel has completed and its writes are visible; it
// is a no-op for a plain launch).  griddep_launch() lets the next kernel of the chain be
// scheduled once every CTA of this grid has issued it or exited, so that the next
// launch and prologue overlap this kernel's tail.  Captured into CUDA graphs as
// programmatic dependency edges.
#pragma once

#include <cuda_runtime.h>

#include <utility>

namespace helm {

__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void griddep_launch() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }

// Launch with programmatic stream serialisation; a plain launch when the attribute is
// refused.
template <typename... P, typename... A>
void launch_pdl(void (*k)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, A&&... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if (cudaLaunchKernelEx(&cfg, k, std::forward<A>(args)...) != cudaSuccess) {
    cudaGetLastError();
    k<<<grid, block, smem, s>>>(std::forward<A>(args)...);
  }
}

}  // namespace helm
