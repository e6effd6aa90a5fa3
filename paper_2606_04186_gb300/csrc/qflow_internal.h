// Internal declarations shared by the library's translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/qflow.h"

#define QFLOW_DIIS_MAX 8

namespace qf {

// Library error code of a failed CUDA runtime call: an allocation failure is QFLOW_ERR_OOM,
// every other failure QFLOW_ERR_CUDA.
inline int cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return QFLOW_OK;
  if (e == cudaErrorMemoryAllocation) return QFLOW_ERR_OOM;
  return QFLOW_ERR_CUDA;
}

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
  const int64_t* items;         // nullable: item i of a launch is space items[i]; else space i
  const int32_t* owner1;
  const int32_t* owner2;
  const uint8_t* owns;  // nullable: owns[s] != 0 iff spaces[s] owns an amplitude (the mixed
                        // solver forms no increment for a space that owns none)
  const double* t1_old;
  const double* t2_old;
  double* t1_new;
  double* t2_new;
  double* energy;
  int32_t* status;
  int32_t* iters;
  const float* W32;  // nullable FP32 copy of W (mixed path)
  const float* F32;  // nullable FP32 copy of F (mixed path; else F is converted per element)
  const unsigned long long* count_dev;  // nullable: the launch covers items [0, *count_dev) instead
  const double* ducc_eri;  // non-null: DUCC form (FP64 solver): bare integrals (pq|rs), n^4
  const double* ducc_F0;   // and the bare Fock matrix, n^2; the solver subtracts the space's
                           // internal part from the gathered G block and replaces owned amplitudes
  const void* guess;  // nullable start vectors: double (FP64 path) or float (mixed path)
  void* root_out;     // nullable: receives converged roots (Phi coefficient 1), same type/layout
  int32_t max_iter;
  double tol;
};

// Launch the batched solver for spaces of size class k (1, 2 or 3) in the given precision.
cudaError_t launch_solve(int k, int precision, const SolveArgs& a, cudaStream_t st);
// Warp-per-space mixed-precision solvers (solve_warp.cu).  W32: optional FP32 copy of W (same
// layout); NULL reads and converts the FP64 W.
// Iteration cap of the warp solver's pass in the mixed path: spaces still unconverged after it
// (a few hard spaces whose Phi-dominant root has lower roots close by) are solved again by the
// FP64 solver, whose larger subspace converges on them, within max_iter steps.
constexpr int kWarpIterCap = 16;

// The FP64 solver on the spaces of class k that a previous solve left with status kSpaceNoConv:
// their positions are collected into items (device, a.nspaces entries) with the count in
// *count (device); then the solver runs on that list.  Start vectors and saved roots are not
// used.  Three launches (count reset, collection, solve); graph-capturable.
cudaError_t launch_solve_rescue(int k, const SolveArgs& a, int64_t* items, unsigned long long* count,
                                cudaStream_t st);

// Warp solver launches: `warps` spaces (warps) per CTA, 1..15 (0 = 15); one CTA per SM.
cudaError_t launch_solve_warp(int k, const SolveArgs& a, const float* W32, const float* guess_in, float* guess_out,
                              int warps, cudaStream_t st);
// One persistent launch over every size class (cls[k], k = 1..3; guesses from cls[k].guess):
// warps take `chunk` work items per atomic from `queue` (zeroed by the call), 6e6o first.
cudaError_t launch_solve_persistent(const SolveArgs* cls, const float* W32, unsigned long long* queue, int chunk,
                                    int warps, cudaStream_t st);
// FP32 copy of the dressed two-body integrals for the mixed-precision solver.
cudaError_t launch_to_f32(const double* W, float* W32, size_t count, cudaStream_t st);

// Dressing (step a) on caller-provided device buffers; returns a CUDA error code.
size_t dress_workspace_bytes(int n, int nocc);
size_t dress_workspace_bytes_mixed(int n, int nocc);  // + FP32 GEMM scratch of the mixed path
int dress_launch_count(int n, int nocc, bool mixed);  // kernels one launch_dress issues
// g32: NULL for FP64 contractions; else n^4 floats of scratch, and the T2 terms are contracted
// in FP32 (mixed precision); the mixed form adds the T2 term of the vvvv block only where at most
// three of its four virtual indices differ (all a (k, k) space with k <= 3 reads), the other
// vvvv elements keep their T1-transformed values.
// ladder_bn: tile width (32, 64 or 128 columns) of the mixed path's ladder + oooo product; 0 = 64.
cudaError_t launch_dress(const double* h, const double* eri, const double* t1, const double* t2, int n, int nocc,
                         double* e0, double* F, double* W, void* work, size_t work_bytes, cudaStream_t st,
                         float* g32 = nullptr, int ladder_bn = 0);
// Times the ladder + oooo product at each tile width on the workspace of a mixed dressing that
// has run (scratch overwritten; synchronises the stream): *best = the fastest, ms[3] = the times
// of 32, 64 and 128 columns.
cudaError_t tune_ladder(int n, int nocc, const float* g32, void* work, size_t work_bytes, cudaStream_t st, int* best,
                        float* ms);

// Step (a) in the Hermitian (DUCC) form (ducc.cu): e0, F, W of the part G common to every space,
// and F0 = the bare Fock matrix (the per-space part needs it).  FP64.
size_t ducc_workspace_bytes(int n, int nocc);
int ducc_launch_count(int n, int nocc);
cudaError_t launch_dress_ducc(const double* h, const double* eri, const double* t1, const double* t2, int n, int nocc,
                              double* e0, double* F, double* W, double* F0, void* work, size_t work_bytes,
                              cudaStream_t st);

// Sweep reductions (step c): out4 = [mean E, max |t_new - t_old|, failed spaces, worst status].
size_t mean_maxdiff_workspace(int64_t nspaces, int64_t nt);
cudaError_t launch_reduce(const double* energy, const int32_t* status, int64_t nspaces, const double* t_old,
                          const double* t_new, int64_t nt, double* out4, void* work, cudaStream_t st);

// Exchange vector of a sharded sweep, [pool | energy | status | iterations] in FP64, entries the
// shard did not produce set to -0.0 (pack); after the element-wise sum over ranks, owned pool
// entries and every per-space entry are taken from it (unpack).
cudaError_t launch_exchange_pack(const double* pool_new, const uint8_t* pool_mask, int64_t np, const double* energy,
                                 const int32_t* status, const int32_t* iters, const uint8_t* space_mask, int64_t ns,
                                 double* x, cudaStream_t st);
cudaError_t launch_exchange_unpack(const double* x, const int32_t* own1, int64_t n1, const int32_t* own2, int64_t n2,
                                   double* pool_new, double* energy, int32_t* status, int32_t* iters, int64_t ns,
                                   cudaStream_t st);

// Pool DIIS (diis.cu): workspace size for a ring of m vectors of length N, the per-sweep step
// (t_new is replaced by the extrapolation once two vectors are stored) and the history reset.
size_t diis_workspace_bytes(int m, int64_t N);
cudaError_t launch_diis(void* work, int m, const double* t_old, double* t_new, int64_t N, cudaStream_t st);
cudaError_t diis_reset(void* work, int m, int64_t N, cudaStream_t st);

// Warm-start network (mlp.cu).  Parameters packed W1, b1, W2, b2, W3, b3 (W [fan_in][fan_out]).
int64_t mlp_param_count(int I, int H, int O);
size_t mlp_workspace_bytes(int I, int H, int O, int64_t rows);
cudaError_t mlp_forward(int I, int H, int O, const float* params, const float* x, int64_t rows, float* y, void* work,
                        cudaStream_t st);
cudaError_t mlp_loss_grad(int I, int H, int O, const float* params, const float* x, const float* t,
                          const uint8_t* mask, int64_t rows, float* grad, float* loss, void* work, cudaStream_t st);
cudaError_t mlp_adam(int64_t n, float* p, const float* g, float* m, float* v, int step, float lr, float b1, float b2,
                     float eps, cudaStream_t st);
// features[s][708] of (3,3) spaces spaces[s * stride]; standardised as (x - mu) * sc when mu
// is given
cudaError_t mlp_features(int n, const double* F, const double* W, const qflow_space* spaces, int64_t nspaces,
                         int64_t stride, const float* mu, const float* sc, float* out, cudaStream_t st);
// targets[r][54] (+ mask[r]) from roots (double when fp64, else float) of class positions
// r * stride; status/sorted_index/mask nullable (then every row counts)
cudaError_t mlp_targets(const void* roots, bool fp64, int64_t rows, int64_t stride, const int64_t* sorted_index,
                        const int32_t* status, float* targets, uint8_t* mask, cudaStream_t st);
// targets[r][54] = the pool's internal amplitudes of spaces[r * stride] (mask set to 1)
cudaError_t mlp_pool_targets(const double* pool, const qflow_space* spaces, int64_t rows, int64_t stride, int nocc,
                             int nvir, float* targets, uint8_t* mask, cudaStream_t st);
// pool <- mu + sd * pred for the amplitudes each space (class position r, sorted index
// sorted_index[r]) owns
cudaError_t mlp_pool_from_pred(const float* pred, const float* mu, const float* sd, const qflow_space* spaces,
                               const int64_t* sorted_index, int64_t rows, int nocc, int nvir, const int32_t* owner1,
                               const int32_t* owner2, double* pool, cudaStream_t st);
// The spaces of one class list (rows records with their sorted indices) that own an amplitude,
// gathered into out_sp / out_idx with their count (device); flag: nspaces bytes of scratch.
cudaError_t mlp_owner_spaces(const int32_t* owner1, int64_t n1, const int32_t* owner2, int64_t n2, int64_t nspaces,
                             const qflow_space* spaces, const int64_t* sorted_index, int64_t rows, uint8_t* flag,
                             qflow_space* out_sp, int64_t* out_idx, unsigned long long* count, cudaStream_t st);
// out[i] = 1 / sd[i] (0 where sd[i] <= 0)
cudaError_t mlp_invert(const float* sd, int n, float* out, cudaStream_t st);
// start vectors guess[r][400] (double when fp64, else float) from outputs pred[r][54];
// increment = mu + sd * pred when mu is given
cudaError_t mlp_guess(const float* pred, int64_t rows, const float* mu, const float* sd, void* guess, bool fp64,
                      cudaStream_t st);
size_t mlp_stats_workspace_bytes(int64_t rows, int cols);
// column mean (mu) and 1/sd (inverse) or sd of X over rows with mask set (count of them)
cudaError_t mlp_col_stats(const float* X, int64_t rows, int cols, const uint8_t* mask, int64_t count, int inverse,
                          float* mu, float* scale, void* work, cudaStream_t st);
// out[r] = (X[order[r]] - mu) * sc (order, mu nullable); copies masks when mask_out is given
cudaError_t mlp_rows(const float* X, int64_t rows, int cols, const int64_t* order, const float* mu, const float* sc,
                     float* out, const uint8_t* mask_in, uint8_t* mask_out, cudaStream_t st);

}  // namespace qf
