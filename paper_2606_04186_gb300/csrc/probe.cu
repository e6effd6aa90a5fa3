// FMA throughput probe: the measured FP32 and FP64 peaks that the solver's roofline divides by.
//
// Every thread runs eight independent chains x <- x * a + b (fma) for `iters` steps; the grid
// fills every SM with as many 256-thread blocks as fit, so the pipes see enough independent
// work to stay busy.  Flops per launch = 2 * 8 * iters * threads; the rate is that over the
// launch's CUDA-event duration, best of three timed launches after one warm-up launch.  The
// chains stay finite (|a| < 1, so x tends to b / (1 - a)) and every thread writes its sum, so
// no chain is optimised away.
#include <cuda_runtime.h>
#include <stdint.h>

#include "qflow_internal.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kThreads) fma_chains(T* out, int iters, T a, T b) {
  T x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
#pragma unroll 1
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 16; ++r)
#pragma unroll
      for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  T s = (T)0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
cudaError_t time_chains(int iters, cudaStream_t st, double* tflops) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_chains<T>, kThreads, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  const int grid = sms * per_sm;
  T* out = nullptr;
  e = cudaMallocAsync(&out, (size_t)grid * kThreads * sizeof(T), st);
  if (e != cudaSuccess) return e;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  e = cudaEventCreate(&ev[0]);
  if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
  double best_ms = 0.0;
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {  // rep 0 is the warm-up
    e = cudaEventRecord(ev[0], st);
    if (e != cudaSuccess) break;
    fma_chains<T><<<grid, kThreads, 0, st>>>(out, iters, (T)0.999, (T)1e-3);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(ev[1], st);
    if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
    if (e == cudaSuccess && rep > 0 && (best_ms == 0.0 || ms < best_ms)) best_ms = ms;
  }
  for (cudaEvent_t x : ev)
    if (x) cudaEventDestroy(x);
  cudaFreeAsync(out, st);
  if (e != cudaSuccess) return e;
  const double flops = 2.0 * kChains * 16.0 * (double)iters * (double)grid * kThreads;
  *tflops = (best_ms > 0.0) ? flops / (best_ms * 1e-3) / 1e12 : 0.0;
  return cudaStreamSynchronize(st);
}

}  // namespace

extern "C" int qflow_fma_peak(int32_t precision, double* tflops, void* stream) {
  if (!tflops || (precision != QFLOW_PREC_FP64 && precision != QFLOW_PREC_MIXED)) return QFLOW_ERR_ARG;
  const cudaStream_t st = (cudaStream_t)stream;
  // about 30 ms per launch at the expected rates (FP32 ~70 TFLOP/s, FP64 ~1.2 TFLOP/s)
  const cudaError_t e = (precision == QFLOW_PREC_FP64) ? time_chains<double>(400, st, tflops)
                                                       : time_chains<float>(25000, st, tflops);
  return qf::cuda_status(e);
}
