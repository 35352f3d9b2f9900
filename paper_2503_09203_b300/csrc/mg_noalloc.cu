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
struct Cached {
  void* ctx = nullptr;   // context the address belongs to
  float* ptr = nullptr;
};
Cached g_cache[kMaxDevices];

// The current driver context (null if it cannot be read). Reached through the
// runtime's driver entry point, so the library does not link the driver
// library directly (it still loads on machines without a GPU driver).
void* current_context() {
  using Fn = int (*)(void**);
  static Fn fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      f = nullptr;
    return reinterpret_cast<Fn>(f);
  }();
  void* ctx = nullptr;
  if (!fn || fn(&ctx) != 0) return nullptr;
  return ctx;
}
}  // namespace

// Device address of the scratch array on the current device. In host code
// the array's name is only a host-side stand-in, so the address is looked up
// with the device current and cached together with the context it belongs
// to; a new context on the same device (after cudaDeviceReset, or after the
// primary context was released and created again, which reloads the module)
// makes the next call look it up again.
cudaError_t noalloc_scratch(float** ptr, size_t* capacity_floats) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  void* ctx = current_context();
  Cached& c = g_cache[dev];
  if (!c.ptr || !ctx || ctx != c.ctx) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    c.ptr = static_cast<float*>(p);
    c.ctx = current_context();   // the lookup may have made the primary context current
  }
  *ptr = c.ptr;
  *capacity_floats = kNoAllocScratchFloats;
  return cudaSuccess;
}

}  // namespace mg
