// Allocation-free variant of the dressing step (qflow_dress_device_static).
//
// Some callers cannot call cudaMalloc: an application whose device memory is owned by another
// allocator (an arena or pool that must see every allocation), code that must not trigger the
// implicit device synchronisation an allocation can cause, or a service with a fixed, pre-
// reserved memory budget.  This entry point runs exactly the same kernels as
// qflow_dress_device, but its scratch lives in a file-scope device array that is part of the
// library image, so the call itself allocates nothing.  The array is held by every GPU that
// loads this library until the process exits.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "qflow_internal.h"

namespace {

constexpr size_t kStaticScratchBytes = (size_t)QFLOW_STATIC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_dress_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};  // device address of g_dress_scratch, per device

// Device address of the scratch array on the current device (set up on first use: the host
// name of the array is only a stand-in and must never be passed to a kernel).
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_dress_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" int qflow_dress_device_static(const double* h, const double* eri, const double* t1, const double* t2,
                                         int32_t n, int32_t nocc, double* e0, double* F, double* W, void* stream) {
  if (!h || !eri || !t1 || !t2 || !e0 || !F || !W || n < 2 || n > 128 || nocc < 1 || nocc >= n)
    return QFLOW_ERR_ARG;
  const size_t need = qf::dress_workspace_bytes(n, nocc);
  if (need > kStaticScratchBytes) return QFLOW_ERR_TOO_LARGE;
  void* scratch = nullptr;
  cudaError_t e = scratch_address(&scratch);
  if (e != cudaSuccess) return QFLOW_ERR_CUDA;
  // Every scratch element is written by a kernel of this call before it is read, so nothing
  // left from an earlier call needs clearing.
  e = qf::launch_dress(h, eri, t1, t2, n, nocc, e0, F, W, scratch, kStaticScratchBytes, (cudaStream_t)stream);
  return (e == cudaSuccess) ? QFLOW_OK : QFLOW_ERR_CUDA;
}

extern "C" size_t qflow_static_scratch_bytes(void) { return kStaticScratchBytes; }
