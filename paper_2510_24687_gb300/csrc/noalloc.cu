// tat_forward_noalloc: the forward operator with its scratch in a static
// device buffer instead of a caller-provided workspace.
//
// Some callers cannot allocate device memory at the point where they need A:
// a serving process that has handed the rest of the GPU to a pool it manages
// and may not grow beyond it, or a latency-critical host loop in which the
// implicit device synchronisation of cudaMalloc/cudaFree is not acceptable.
// For them this entry point runs the same five kernels as tat_forward, using
// a file-scope buffer of kNoAllocScratchBytes that every GPU loading this
// library holds until the process exits.  No call here allocates.
#include <cstdint>
#include <cstdio>

#include "plan.hpp"

namespace {

constexpr size_t kNoAllocScratchBytes = 16u << 20;  // 16 MiB: n = 512, 1024 x 1024 data, batch 1

// Device-side storage.  In host code this name is only a stand-in for the
// symbol: its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Looks up the buffer's device address on the current device.  Done on every
// call (cudaGetSymbolAddress allocates nothing), so that a device reset or a
// new primary context never leaves a stale address behind.
tat_status scratch_address(void** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p) {
    fprintf(stderr, "tat_forward_noalloc: cudaGetSymbolAddress failed: %s\n", cudaGetErrorString(e));
    cudaGetLastError();
    return TAT_ERR_CUDA;
  }
  *out = p;
  return TAT_OK;
}

}  // namespace

extern "C" tat_status tat_forward_noalloc(tat_plan_t plan, const float* f, float* g, tat_stream_t stream) {
  if (!plan || !f || !g) return TAT_ERR_INVALID_ARG;
  // the kernels read f and write g as 4-byte floats
  if (reinterpret_cast<uintptr_t>(f) % 4 || reinterpret_cast<uintptr_t>(g) % 4) return TAT_ERR_INVALID_ARG;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return TAT_ERR_CUDA;
  }
  if (dev != plan->device) return TAT_ERR_INVALID_ARG;
  const size_t need = (plan->ws_x + plan->ws_y) * sizeof(float2);
  if (need > kNoAllocScratchBytes) {
    fprintf(stderr, "tat_forward_noalloc: this plan needs %zu bytes of scratch; the static buffer holds %zu\n",
            need, kNoAllocScratchBytes);
    return TAT_ERR_UNSUPPORTED;
  }
  void* scratch = nullptr;
  const tat_status s = scratch_address(&scratch);
  if (s != TAT_OK) return s;
  // Every scratch element the five stages read is written earlier in the same
  // call, so nothing needs clearing between calls.
  const tat::DevPlan& d = plan->d;
  return tat::launch_forward(plan, 1, f, (long long)d.n * d.n, g, (long long)d.n_det * d.n_t, scratch,
                             static_cast<cudaStream_t>(stream));
}
