// Programmatic dependent launch: a kernel launched with launch_pdl may start
// while the previous kernel on its stream is still finishing. Such a kernel
// must call pdl_wait() before it reads anything an earlier kernel writes or
// writes anything an earlier kernel reads; work before that point (index
// arithmetic, twiddle and constant loads from the context's tables) overlaps
// the previous kernel's tail and the launch latency. pdl_trigger() lets the
// next kernel be scheduled once every block of this one has passed it.
#pragma once
#include <cuda_runtime.h>

#include <utility>

namespace ckks {

__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// on = 0 launches without the attribute (plain stream order; pdl_wait is
// then a no-op).
template <typename... KArgs, typename... Args>
inline void launch_pdl(int on, void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = on ? 1 : 0;
  cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

}  // namespace ckks
