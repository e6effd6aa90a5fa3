// Internal declarations shared by the library's translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/qflow.h"

#define QFLOW_DIIS_MAX 8

namespace qf {

// Per-space solver status codes written by the solve kernels.
enum SpaceStatus : int32_t { kSpaceOk = 0, kSpaceNoConv = 1, kSpaceRoot = 2, kSpaceNonFinite = 3, kSpaceInvalid = 4 };

struct SolveArgs {
  int32_t n, nocc, nvir;
  const double* e0;
  const double* F;
  const double* W;
  const qflow_space* spaces;
  int64_t nspaces;
  int64_t space_base;
  const int64_t* sorted_index;  // nullable: sorted index of spaces[s]; else space_base + s
  const int32_t* owner1;
  const int32_t* owner2;
  const double* t1_old;
  const double* t2_old;
  double* t1_new;
  double* t2_new;
  double* energy;
  int32_t* status;
  int32_t* iters;
  const float* W32;  // nullable FP32 copy of W (mixed path)
  void* guess;  // start vectors / saved roots: double (FP64 path) or float (mixed path)
  int32_t save_root;
  int32_t max_iter;
  double tol;
};

// Launch the batched solver for spaces of size class k (1, 2 or 3) in the given precision.
cudaError_t launch_solve(int k, int precision, const SolveArgs& a, cudaStream_t st);
// Warp-per-space mixed-precision solvers (solve_warp.cu).  W32: optional FP32 copy of W (same
// layout); NULL reads and converts the FP64 W.  ctas_per_sm: 0 = as many as fit.
cudaError_t launch_solve_warp(int k, const SolveArgs& a, const float* W32, const float* guess_in, float* guess_out,
                              int ctas_per_sm, cudaStream_t st);
// One persistent launch over every size class (cls[k], k = 1..3; guesses from cls[k].guess):
// warps take `chunk` work items per atomic from `queue` (zeroed by the call), 6e6o first.
cudaError_t launch_solve_persistent(const SolveArgs* cls, const float* W32, unsigned long long* queue, int chunk,
                                    int ctas_per_sm, cudaStream_t st);
// FP32 copy of the dressed two-body integrals for the mixed-precision solver.
cudaError_t launch_to_f32(const double* W, float* W32, size_t count, cudaStream_t st);

// Dressing (step a) on caller-provided device buffers; returns a CUDA error code.
size_t dress_workspace_bytes(int n, int nocc);
int dress_launch_count(int n, int nocc, bool mixed);  // kernels one launch_dress issues
// g32: NULL for FP64 contractions; else n^4 floats of scratch, and the T2 terms are contracted
// in FP32 (mixed precision).
cudaError_t launch_dress(const double* h, const double* eri, const double* t1, const double* t2, int n, int nocc,
                         double* e0, double* F, double* W, void* work, size_t work_bytes, cudaStream_t st,
                         float* g32 = nullptr);

// Sweep reductions (step c): out4 = [mean E, max |t_new - t_old|, failed spaces, worst status].
size_t mean_maxdiff_workspace(int64_t nspaces, int64_t nt);
cudaError_t launch_reduce(const double* energy, const int32_t* status, int64_t nspaces, const double* t_old,
                          const double* t_new, int64_t nt, double* out4, void* work, cudaStream_t st);

// Pool DIIS (diis.cu): workspace size for a ring of m vectors of length N, the per-sweep step
// (t_new is replaced by the extrapolation once two vectors are stored) and the history reset.
size_t diis_workspace_bytes(int m, int64_t N);
cudaError_t launch_diis(void* work, int m, const double* t_old, double* t_new, int64_t N, cudaStream_t st);
cudaError_t diis_reset(void* work, int m, int64_t N, cudaStream_t st);

}  // namespace qf
