// Programmatic dependent launch: a kernel launched with pdl_launch may be scheduled while
// the kernel before it in the stream is still running, so its CTAs take SMs as that
// kernel's last CTAs retire instead of after a full drain and a new launch.  Every kernel
// launched this way starts with TAT_GRID_DEPENDENCY(): it lets its own dependents be
// scheduled (once all of its CTAs are running) and then waits until the previous kernel
// has completed and its memory is visible, before touching any global memory.  Launched
// without the attribute, both instructions do nothing.  While the stream is being captured
// into a CUDA graph the attribute is left off: graph replays already start kernels back to
// back, and measured with programmatic edges they ran slower (learned primal-dual step
// 4.92 ms against 4.71 ms; eager launches 5.09 ms against 5.79 ms).
#pragma once

#include <cuda_runtime.h>

#include <utility>

#define TAT_GRID_DEPENDENCY()                                                 \
  do {                                                                        \
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");         \
    asm volatile("griddepcontrol.wait;\n" ::: "memory");                      \
  } while (0)

namespace tat {

// `enable` false launches without the attribute (the operators choose per plan: with their
// large kernels at n = 512 the early-scheduled CTAs cost more than the overlap gains).
template <typename... KArgs, typename... Args>
inline cudaError_t pdl_launch(bool enable, void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  const bool plain = cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone;
  cfg.attrs = attr;
  cfg.numAttrs = plain || !enable ? 0 : 1;
  return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

}  // namespace tat
