// Programmatic dependent launch, shared by the single-domain and batched
// step kernels.  A step kernel lets the next launch in the stream start (its
// CTAs become resident while this grid drains) and, before touching any
// population, waits for the previous grid's completion and memory.  Without
// the launch attribute both instructions have no effect.  Each kernel waits
// on its immediate predecessor only; since that one waited on its own, the
// wait covers every earlier launch in the stream.
#pragma once

#include <cuda_runtime.h>

#include <utility>

namespace lbm {

__device__ __forceinline__ void pdl_release() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void pdl_acquire() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Launch with the programmatic-stream-serialization attribute when pdl.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, bool pdl, cudaStream_t st,
                       Args&&... args) {
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

}  // namespace lbm
