// Allocation-free variant of the dressing step (qflow_dress_device_static).
//
// Some callers cannot call cudaMalloc: an application whose device memory is owned by another
// allocator (an arena or pool that must see every allocation), code that must not trigger the
// implicit device synchronisation an allocation can cause, or a service with a fixed, pre-
// reserved memory budget.  This entry point runs exactly the same kernels as
// qflow_dress_device, but its scratch lives in a file-scope device array that is part of the
// library image, so the call itself allocates nothing.  The array is held by every GPU that
// loads this library until the process exits.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "qflow_internal.h"
#include "scratch_cache.h"

namespace {

constexpr size_t kStaticScratchBytes = (size_t)QFLOW_STATIC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_dress_scratch[kStaticScratchBytes];

qf::ScratchAddressCache g_cache;  // device address of g_dress_scratch per (device, context)

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

// Driver entry points through the runtime (no link against libcuda); nullptr if unavailable.
template <class Fn>
Fn driver_fn(const char* name, int version) {
  void* f = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion(name, &f, version, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess)
    return nullptr;
  return reinterpret_cast<Fn>(f);
}

// Identifier of the calling thread's current context (unique for the life of the process).
cudaError_t current_context_id(unsigned long long* id) {
  static const CtxGetCurrentFn get_current = driver_fn<CtxGetCurrentFn>("cuCtxGetCurrent", 4000);
  static const CtxGetIdFn get_id = driver_fn<CtxGetIdFn>("cuCtxGetId", 12000);
  if (!get_current || !get_id) return cudaErrorNotSupported;
  CUcontext ctx = nullptr;
  if (get_current(&ctx) != CUDA_SUCCESS || !ctx) return cudaErrorDeviceUninitialized;
  return get_id(ctx, id) == CUDA_SUCCESS ? cudaSuccess : cudaErrorDeviceUninitialized;
}

// Device address of the scratch array in the current context.  The host name of the array is
// only a stand-in and must never be passed to a kernel; the address is looked up with the
// device current, once per context (again after a device reset).  A lookup is refused while
// `stream` is capturing: it may load the module, which is not a capturable operation.
int scratch_address(cudaStream_t stream, void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return qf::cuda_status(e);
  if (dev < 0 || dev >= qf::ScratchAddressCache::kMaxDevices) return QFLOW_ERR_CUDA;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  e = cudaStreamIsCapturing(stream, &cap);  // also makes the device's primary context current
  if (e != cudaSuccess) return qf::cuda_status(e);
  unsigned long long ctx = 0;
  e = current_context_id(&ctx);
  if (e != cudaSuccess) return qf::cuda_status(e);
  if (void* p = g_cache.find(dev, ctx)) {
    *out = p;
    return QFLOW_OK;
  }
  if (cap != cudaStreamCaptureStatusNone) return QFLOW_ERR_STATE;
  void* p = nullptr;
  e = cudaGetSymbolAddress(&p, g_dress_scratch);
  if (e != cudaSuccess) return qf::cuda_status(e);
  g_cache.put(dev, ctx, p);
  *out = p;
  return QFLOW_OK;
}

}  // namespace

extern "C" int qflow_dress_device_static(const double* h, const double* eri, const double* t1, const double* t2,
                                         int32_t n, int32_t nocc, double* e0, double* F, double* W, void* stream) {
  if (!h || !eri || !t1 || !t2 || !e0 || !F || !W || n < 2 || n > 128 || nocc < 1 || nocc >= n)
    return QFLOW_ERR_ARG;
  const size_t need = qf::dress_workspace_bytes(n, nocc);
  if (need > kStaticScratchBytes) return QFLOW_ERR_TOO_LARGE;
  void* scratch = nullptr;
  const int rc = scratch_address((cudaStream_t)stream, &scratch);
  if (rc != QFLOW_OK) return rc;
  // Every scratch element is written by a kernel of this call before it is read, so nothing
  // left from an earlier call needs clearing.
  return qf::cuda_status(
      qf::launch_dress(h, eri, t1, t2, n, nocc, e0, F, W, scratch, kStaticScratchBytes, (cudaStream_t)stream));
}

extern "C" size_t qflow_static_scratch_bytes(void) { return kStaticScratchBytes; }
