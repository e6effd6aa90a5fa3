// Device-level entry point of the tensor-core GEMM (the engine of the dressing contractions),
// on plain row-major operands: C[m][n] = sum_k A[m][k] B[n][k].
#include <cuda_runtime.h>
#include <stdint.h>

#include "qflow_internal.h"
#include "tc_gemm.cuh"

namespace {

struct RowMajor {
  const float* p;
  int ld;
  __device__ float operator()(int r, int k) const { return p[(size_t)r * ld + k]; }
};

struct StoreRowMajor {
  float* p;
  int ld;
  __device__ void operator()(int m, int n, float v) const { p[(size_t)m * ld + n] = v; }
  __device__ void run(int m, int n, const float (&v)[32], int cnt) const {
    float* q = p + (size_t)m * ld + n;
#pragma unroll
    for (int j = 0; j < 32; ++j)
      if (j < cnt) q[j] = v[j];
  }
};

}  // namespace

extern "C" int qflow_gemm_tf32x3_device(int32_t M, int32_t N, int32_t K, const float* A, int32_t lda, const float* B,
                                        int32_t ldb, float* C, int32_t ldc, int32_t* err, void* stream) {
  if (M < 0 || N < 0 || K < 0 || !err || lda < K || ldb < K || ldc < N) return QFLOW_ERR_ARG;
  if (M == 0 || N == 0) return QFLOW_OK;
  if (!A || !B || !C) return QFLOW_ERR_ARG;
  cudaError_t e = qf::tc::gemm_tf32x3<128>(M, N, K, RowMajor{A, lda}, RowMajor{B, ldb}, StoreRowMajor{C, ldc}, err,
                                           (cudaStream_t)stream);
  return e == cudaSuccess ? QFLOW_OK : QFLOW_ERR_CUDA;
}
