// Programmatic dependent launch.  A kernel launched with pdl_launch may begin
// while the kernel before it on the stream is still running: it can set up
// shared memory, barriers, tensor memory and read data that no kernel of the
// current sequence writes (tables, bands, factorizations), but it must call
// pdl_wait() before it reads or writes any buffer that the previous kernels
// use.  pdl_wait() returns once those kernels have completed and their
// memory is visible; for a kernel launched the ordinary way it returns at
// once.  pdl_trigger() lets the next kernel on the stream be scheduled as
// soon as every block of this one has started.
#pragma once
#include <cuda_runtime.h>
#include <utility>

__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
cudaError_t pdl_launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args &&...args) {
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
