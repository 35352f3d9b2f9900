// Fixed device scratch for the allocation-free adjoint entry point
// (mg_step_backward_noalloc in mg_runtime.cpp).
//
// Some callers cannot allocate device memory while they run the backward
// pass: a host framework that owns every byte of the device through its own
// pool, a process whose memory budget is already committed, or a loop that
// must not take cudaMalloc's implicit device synchronisation. For them the
// segment-recompute scratch of the adjoint lives in this file-scope array,
// which every GPU that loads the library holds until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "mg_internal.h"

namespace mg {

// 32 MiB of floats: (ckpt_every * K + 1) * 21 * n_slots must fit.
constexpr size_t kNoAllocScratchFloats = size_t(8) << 20;

static __device__ __align__(256) float g_noalloc_scratch[kNoAllocScratchFloats];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_mu;
float* g_ptr[kMaxDevices] = {};
}  // namespace

// Device address of the scratch array on the current device. In host code
// the array's name is only a host-side stand-in, so the address is looked up
// once per device (with that device current) and cached.
cudaError_t noalloc_scratch(float** ptr, size_t* capacity_floats) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_ptr[dev] = static_cast<float*>(p);
  }
  *ptr = g_ptr[dev];
  *capacity_floats = kNoAllocScratchFloats;
  return cudaSuccess;
}

}  // namespace mg
