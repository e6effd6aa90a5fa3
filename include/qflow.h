/*
 * qflow.h -- C ABI of the GB300-native singles-and-doubles Quantum Flow sweep.
 *
 * The paper (arXiv 2606.04186) defines one flow cycle as: downfold the Hamiltonian into every
 * active space with the current global amplitude pool (Eqs. 5-8, N = 1), solve each space,
 * write the amplitudes each space owns back into the pool, barrier (Numerical
 * Implementation).  This library runs that cycle on one GPU:
 *   (a) dressing: H-bar = e^{-T} H e^{T} (SES-CC reading of the flow's sigma), normal ordered
 *       with respect to the closed-shell reference, truncated to <= two-body: E0, F[n][n],
 *       W[n][n][n][n] with W[p][q][r][s] = coefficient of {E_pq E_rs}/2 (creators p, r;
 *       annihilators q, s; pair symmetry W[p][q][r][s] = W[r][s][p][q]);
 *   (b) per space: gather the active block of (E0, F, W), fold the active occupied orbitals
 *       (rewrite relative to the space's vacuum), find the Phi-dominant right eigenpair of the
 *       determinant operator (Sz = 0) with a batched Davidson solver;
 *   (c) per space: increment X1 = C1, X2 = C2 - C1*C1 from the normalised CI vector; every
 *       amplitude takes t_old + X from its owner space only (first space in ascending
 *       Delta-eps order that contains all its indices; Jacobi sweep); E_QFlow = mean E(i).
 *
 * Conventions used by every entry point
 *   n       spatial orbitals (1 <= n <= 128), orbitals 0..nocc-1 doubly occupied.
 *   h       [n][n] row-major FP64 core Hamiltonian.
 *   eri     [n][n][n][n] row-major FP64 two-electron integrals (pq|rs), chemists' order.
 *   t1      [nocc][nvir] FP64, t1[i][a] = t_i^a (a counted from nocc).
 *   t2      [nocc][nocc][nvir][nvir] FP64 alpha-beta amplitude t_ij^ab = t2[i][j][a][b];
 *           the library keeps t2[i][j][a][b] == t2[j][i][b][a].
 *   spaces  qflow_space[nspaces]; (no, nv) in {(1,1), (2,2), (3,3)}; orb[] holds the no
 *           occupied then the nv virtual absolute orbital indices, each group strictly
 *           ascending; unused slots are -1.
 *
 * Errors: every int-returning call returns QFLOW_OK (0) or a negative qflow_status; nothing
 * throws across the ABI.  QFLOW_WARN_UNCOVERED (a positive bit) is or-ed into the return of
 * qflow_init / qflow_plan when some amplitude has no owner (it keeps its value).
 * Ownership: the library copies every input at the call; output buffers are owned by the
 * caller.  A handle owns all its device memory and one CUDA stream; it is not thread safe.
 */
#ifndef QFLOW_H
#define QFLOW_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  QFLOW_OK = 0,
  QFLOW_ERR_ARG = -1,        /* invalid argument (sizes, space list, null pointer)        */
  QFLOW_ERR_CUDA = -2,       /* a CUDA runtime call failed                                 */
  QFLOW_ERR_OOM = -3,        /* device allocation failed                                   */
  QFLOW_ERR_NOCONV = -4,     /* some space's Davidson solver hit its iteration limit       */
  QFLOW_ERR_ROOT = -5,       /* selected root complex or |c_Phi| < 1e-3                    */
  QFLOW_ERR_NONFINITE = -6,  /* NaN/Inf in an energy or amplitude                          */
  QFLOW_ERR_STATE = -7,      /* call out of order (e.g. energy before the first sweep)     */
  QFLOW_ERR_TOO_LARGE = -8,  /* problem needs more scratch than qflow_dress_device_static has */
  QFLOW_WARN_UNCOVERED = 1   /* bit: some amplitudes have no owner space                   */
} qflow_status;

typedef enum {
  QFLOW_PREC_FP64 = 0,   /* plain: every step in FP64                                        */
  QFLOW_PREC_MIXED = 1   /* dressing: FP64 integrals with FP32 T1 correction sums, reference
                            energy and Fock-like sums in FP64, T2 contractions as tensor-core
                            GEMMs (three-term TF32, FP32 accumulation) added to FP64 bases;
                            solver: FP32 gather/fold/set-up, sigma and Davidson vectors;
                            Rayleigh-Ritz matrix, projected root and Gram-Schmidt coefficients
                            to FP64 accuracy (double-float); FP64 energy, amplitude update,
                            DIIS and reductions.  Spaces the FP32 warp pass leaves unconverged
                            after 16 steps are re-solved by the FP64 solver in the same sweep */
} qflow_precision;

typedef struct {
  int32_t no, nv;
  int32_t orb[6];
} qflow_space;

/* Downfolding form of a space's effective Hamiltonian (Eqs. 1-8 with N = 1).
 *   QFLOW_FORM_SESCC: sigma read as the cluster operator T (SES-CC); H-bar = e^{-T} H e^{T}
 *     truncated to <= two-body, one dressing for every space, increments X added to the pool.
 *   QFLOW_FORM_DUCC: the paper's anti-Hermitian sigma = T - T^+ (DUCC); a space's operator is
 *     [H + [H, s] + 1/2 [[F, s], s]]_(<=2), s = sigma_ext = the pool's amplitudes with an index
 *     outside the space, F the Fock operator (all terms through second order; each commutator
 *     normal ordered with respect to Phi and kept to <= two-body: the paper leaves the truncation
 *     open).  Computed as a part common to every space (eight FP64 dressings per sweep) minus the
 *     space's internal part (per space, in the solver).  The operator is Hermitian; the root's
 *     cluster amplitudes (C1, C2 - C1^2 / 2) replace the owned amplitudes.  Requires
 *     QFLOW_PREC_FP64; no network guesses; no wave-ordered sweeps (QFLOW_ERR_STATE). */
typedef enum {
  QFLOW_FORM_SESCC = 0,
  QFLOW_FORM_DUCC = 1
} qflow_form;

typedef enum {
  QFLOW_SCHED_AUTO = 0,       /* mixed precision: the first sweep runs the persistent queue;
                                 at the second sweep the autotuner times its candidates, items
                                 per fetch (1, 2, 4, 8) x warps per CTA (15, 12), on a
                                 calibration subset and keeps the fastest                      */
  QFLOW_SCHED_PER_CLASS = 1,  /* one grid-stride launch per size class                        */
  QFLOW_SCHED_PERSISTENT = 2  /* one persistent launch; warps take spaces of every class from a
                                 single work queue, 6e6o first                                 */
} qflow_schedule_kind;

typedef struct {
  int32_t precision;          /* qflow_precision                                            */
  int32_t max_iter;           /* Davidson iteration limit per space (default 60); mixed:
                                 the warp pass stops at 16, later steps run in FP64         */
  double tol;                 /* Davidson residual 2-norm (default 1e-9 fp64, 1e-6 mixed)   */
  int32_t diis;               /* 0 = off, else Pulay DIIS on the pool with a history of 2..8
                                 sweeps (FP64, on the device; not in the paper: it accelerates
                                 the sweep iteration without moving its fixed point).  The
                                 history restarts at qflow_set_amplitudes.                  */
  int32_t guess;              /* 0 = Phi, 1 = previous sweep's root of the same space (keeps
                                 one CI vector per space on the device: 400 x 4 B per 6e6o
                                 space in mixed precision, x 8 B in FP64).  In a flow the pool
                                 absorbs each root's increment, so Phi is usually the closer
                                 start; 1 pays off when the pool is held fixed.
                                 2 = warm-start network (QFLOW_GUESS_NETWORK below): 6e6o
                                 roots are kept like 1, but sweeps start from Phi except the
                                 first sweep after a model is set or trained, which starts the
                                 6e6o spaces from the network's guess.                       */
  int32_t schedule;           /* qflow_schedule_kind (mixed precision; FP64 uses per-class
                                 launches)                                                   */
  int32_t graph;              /* 1 = once the schedule is fixed (mixed: from the third sweep,
                                 FP64: from the second), capture the sweep's device work in a
                                 CUDA graph and replay it (default 1)                        */
  int32_t form;               /* qflow_form: the downfolding form (default QFLOW_FORM_SESCC)  */
  int32_t warps;              /* mixed precision: spaces (warps) per CTA of the solver, 1..15;
                                 0 = chosen by the autotuner (QFLOW_SCHED_AUTO) or 15        */
  int32_t chunk;              /* mixed precision, persistent queue: consecutive spaces a warp
                                 takes per fetch, 1..16; 0 = chosen by the autotuner
                                 (QFLOW_SCHED_AUTO) or 1                                     */
  int32_t ladder_bn;          /* mixed precision, SES-CC form: tile width (columns) of the
                                 dressing's ladder + oooo tensor-core product, 32, 64 or 128;
                                 0 = chosen by the autotuner (QFLOW_SCHED_AUTO) or 64.  Every
                                 width gives the same products bit for bit.                  */
  int32_t reserved[2];
} qflow_options;

/* Fill *opt with the defaults above for the given precision. */
void qflow_default_options(qflow_options* opt, int32_t precision);

/* ---- host-only planning (no GPU needed) ------------------------------------------------- */

/* Order and ownership of a space list (Algorithm 1's final sort; owner rule of the Numerical
 * Implementation).  eps_p = h_pp + sum_{k<nocc} [2 (pp|kk) - (pk|kp)] summed k ascending;
 * Delta-eps = (sum eps_v, ascending) - (sum eps_o, ascending); ties broken by size class,
 * occupied tuple, virtual tuple, input position.
 *   perm[nspaces]                      out: sorted position -> input index
 *   owner1[nocc*nvir]                  out: sorted index of the owner of t1[i][a], or -1
 *   owner2[nocc*nocc*nvir*nvir]        out: owner of t2[i][j][a][b] (== owner of t2[j][i][b][a])
 *   n_uncovered                        out (nullable): amplitudes with no owner
 * Any output pointer may be NULL except perm. */
int qflow_plan(const double* h, const double* eri, int32_t n, int32_t nocc, const qflow_space* spaces,
               int64_t nspaces, int64_t* perm, int32_t* owner1, int32_t* owner2, int64_t* n_uncovered);

/* Coverage-driven active-space sampling (Numerical Implementation, Algorithm 1), host only.
 * Candidates draw `no` of the nocc occupied and `nv` of the nvir virtual orbitals uniformly
 * without replacement; a candidate is kept when it covers at least one (o1 < o2, v1 < v2) tuple
 * no earlier kept candidate covered; sampling stops when every tuple is covered; the kept spaces
 * are returned sorted by ascending Delta-eps (sum eps_v - sum eps_o, each sum in ascending
 * orbital order; ties keep the sampling order).  Random numbers: SplitMix64 from state `seed`; a
 * draw of k of m is a partial Fisher-Yates shuffle of 0..m-1 restarted from the identity, element
 * i swapped with i + (u mod (m - i)); occupied orbitals are drawn first.
 *   eps[nocc + nvir]   orbital energies (host), finite
 *   no, nv             2 <= no <= min(3, nocc), 2 <= nv <= min(3, nvir)
 *   out[capacity]      host records (no, nv, absolute orbitals, unused slots -1);
 *                      capacity C(nocc,2) C(nvir,2) always suffices (every kept space covers a
 *                      new tuple); NULL allowed with capacity 0 to ask for the count
 *   count              out: spaces in the cycle;  draws (nullable) out: candidates drawn
 * Errors: QFLOW_ERR_ARG; QFLOW_ERR_TOO_LARGE when capacity < count (count is still set). */
int qflow_sample_spaces(int32_t nocc, int32_t nvir, int32_t no, int32_t nv, const double* eps, uint64_t seed,
                        qflow_space* out, int64_t capacity, int64_t* count, int64_t* draws);

/* Shard `rank` of `nranks` of a space list, for sweeps split over several processes (one GPU
 * each; the paper's cycles run in process groups that meet at a barrier after every cycle,
 * Numerical Implementation).  The device order of the list is grouped by size class and, within
 * a class, in orbital-tuple order (occupied tuple, then virtual tuple); rank r takes positions
 * [floor(r c_k / R), floor((r+1) c_k / R)) of every class k (c_k spaces, R ranks).
 *   space_mask[nspaces]   out (nullable): 1 for the sorted positions the shard solves, else 0
 *   pool_mask[nocc*nvir + nocc^2*nvir^2]  out (nullable): 1 for the amplitudes (t1 then t2)
 *                          whose owner space the shard solves, else 0
 * Over all ranks the space masks partition the list and the pool masks the owned amplitudes.
 * Errors: QFLOW_ERR_ARG (bad rank / nranks or invalid problem), QFLOW_ERR_OOM. */
int qflow_shard_plan(const double* h, const double* eri, int32_t n, int32_t nocc, const qflow_space* spaces,
                     int64_t nspaces, int32_t rank, int32_t nranks, uint8_t* space_mask, uint8_t* pool_mask);

/* ---- handle API: one flow on one GPU ---------------------------------------------------- */

typedef struct qflow_ctx* qflow_handle;

/* Copy h, eri (host pointers) and the space list to the current CUDA device, plan the sweep,
 * start from an empty pool.  opt may be NULL (plain FP64, Jacobi, no DIIS, Phi guess). */
int qflow_init(qflow_handle* out, const double* h, const double* eri, int32_t n, int32_t nocc,
               const qflow_space* spaces, int64_t nspaces, const qflow_options* opt);

/* One sweep (barrier to barrier).  Outputs (nullable): change of E_QFlow since the previous
 * sweep (+inf after the first), max |t_new - t_old| over the pool, number of spaces whose
 * solver did not finish with status 0.  Returns QFLOW_ERR_NOCONV / ROOT / NONFINITE when some
 * space failed (its owned amplitudes then keep their old value). */
int qflow_sweep(qflow_handle hnd, double* d_e, double* max_dt, int32_t* nfailed);

/* One sweep in waves of `wave` spaces in Delta-eps order: every wave is downfolded with the pool
 * the waves before it left, and its owned amplitudes are updated before the next wave starts
 * (the paper's pool is populated progressively as the process groups traverse the sorted list,
 * Numerical Implementation; the spaces of one wave run together).  Energies, max|t_new - t_old|
 * (over the whole sweep) and failures as qflow_sweep; DIIS (if on) acts on the sweep's start and
 * end pools.  wave >= nspaces is qflow_sweep (Jacobi).  Each wave runs the full dressing, so a
 * sweep costs about nspaces / wave dressings.  Wave sweeps run plain launches, do not apply the
 * network's start vectors and keep the current launch schedule.  Errors: QFLOW_ERR_ARG
 * (wave < 1), QFLOW_ERR_STATE (sharded handle). */
int qflow_sweep_waves(qflow_handle hnd, int64_t wave, double* d_e, double* max_dt, int32_t* nfailed);

/* ---- sharded sweeps: every rank holds a handle of the whole problem ----------------------
 * After qflow_set_shard(h, rank, nranks) a sweep is three calls: qflow_sweep_shard_begin
 * dresses (replicated: every rank dresses the same pool), solves the shard's spaces (see
 * qflow_shard_plan) and writes the exchange vector; the caller sums the exchange vectors of all
 * ranks element-wise (an allreduce with sum, e.g. NCCL on the device buffers) into each rank's
 * buffer; qflow_sweep_shard_end merges it and runs DIIS and the reductions.  Every rank then
 * holds the same pool, per-space energies and statistics, bitwise equal to an unsharded sweep:
 * each owned amplitude (owner rule: one owner space) and each per-space value is produced by
 * exactly one rank, and the other ranks contribute -0.0, which leaves any value unchanged under
 * addition.  qflow_sweep returns QFLOW_ERR_STATE on a sharded handle; sharded sweeps run plain
 * launches (no graph replay).  nranks = 1 makes the three-call form cover the whole list. */
int qflow_set_shard(qflow_handle hnd, int32_t rank, int32_t nranks);

/* Length (FP64 elements) of the exchange vector: pool (nocc*nvir + nocc^2*nvir^2), then the
 * energy and a code per space (2 * nspaces, sorted order), code = status * 2^20 + Davidson
 * iterations (an exact integer in FP64). */
int64_t qflow_exchange_size(qflow_handle hnd);

/* Dressing + this shard's solves; fills exchange[qflow_exchange_size] (device pointer, caller
 * owned, 8-byte aligned) and synchronises the handle's stream before returning.  Errors:
 * QFLOW_ERR_STATE without qflow_set_shard or while a sharded sweep is open. */
int qflow_sweep_shard_begin(qflow_handle hnd, double* exchange);

/* Merge of the summed exchange vector (device pointer; must be complete on the device when the
 * call is made), DIIS, reductions.  Outputs and return codes as qflow_sweep.  Errors:
 * QFLOW_ERR_STATE without a preceding qflow_sweep_shard_begin.  Between begin and end the
 * handle refuses qflow_set_amplitudes, qflow_dressed and the network's pool calls. */
int qflow_sweep_shard_end(qflow_handle hnd, const double* exchange, double* d_e, double* max_dt,
                          int32_t* nfailed);

/* E_QFlow of the last sweep and (nullable) the per-space energies in sorted order. */
int qflow_energy(qflow_handle hnd, double* e_mean, double* e_per_space);

/* Copy the pool to host buffers t1[nocc*nvir], t2[nocc*nocc*nvir*nvir]. */
int qflow_amplitudes(qflow_handle hnd, double* t1, double* t2);

/* Overwrite the pool from host buffers (warm start, fixed-point tests). */
int qflow_set_amplitudes(qflow_handle hnd, const double* t1, const double* t2);

/* Sorted position -> caller's input index (int64[nspaces]). */
int qflow_space_order(qflow_handle hnd, int64_t* perm);

/* Per-space solver diagnostics of the last sweep, sorted order (nullable outputs):
 * Davidson iterations and status (0 ok, 1 no convergence, 2 root, 3 non-finite,
 * 4 invalid space). */
int qflow_space_stats(qflow_handle hnd, int32_t* iterations, int32_t* status);

/* The dressed integrals of the current pool (what the next sweep will use): e0 (1),
 * F[n*n], W[n^4] copied to host buffers (any may be NULL).  With QFLOW_PREC_MIXED the vvvv
 * block of W is dressed only where at most three of its four virtual indices differ (every
 * element a (k, k) space with k <= 3 reads); its other elements hold the T1-transformed
 * integrals.  qflow_dress_device dresses every element. */
int qflow_dressed(qflow_handle hnd, double* e0, double* F, double* W);

/* Timing of the last sweep from CUDA events recorded on the handle's stream:
 * phase_ms[3] = dressing, per-space solve, merge reductions (milliseconds); and the number
 * of kernels the sweep launched.  Either output may be NULL. */
int qflow_last_sweep_info(qflow_handle hnd, double* phase_ms, int64_t* kernel_launches);

/* Launch schedule in use (tuned at the second sweep): persistent queue or per-class launches,
 * items per queue fetch, warps (spaces) per CTA of the solver (one CTA per SM), whether sweeps
 * replay a CUDA graph, and the autotuner's calibration times (milliseconds per candidate, up to
 * QFLOW_TUNE_MAX; 0 for a candidate a fixed warps option skipped; the count is 0 before the
 * calibration, when the schedule was fixed, or when it came from the per-process cache).  Any
 * output may be NULL. */
#define QFLOW_TUNE_MAX 8
int qflow_schedule(qflow_handle hnd, int32_t* persistent, int32_t* chunk, int32_t* warps_per_cta, int32_t* graph,
                   float* candidate_ms, int32_t* n_candidates);

/* Tile width in use for the mixed dressing's ladder + oooo product (QFLOW_SCHED_AUTO times
 * 32, 64 and 128 columns at the second sweep, beside the solver's candidates) and the times of
 * those three candidates in milliseconds (count 0 when the width was fixed, came from the
 * per-process cache, or before the calibration).  Any output may be NULL. */
#define QFLOW_LADDER_TUNE_MAX 3
int qflow_dress_schedule(qflow_handle hnd, int32_t* ladder_bn, float* candidate_ms, int32_t* n_candidates);

/* Stream the handle works on (a cudaStream_t). */
void* qflow_stream(qflow_handle hnd);

void qflow_destroy(qflow_handle hnd);
const char* qflow_strerror(int code);

/* ---- device-level steps (device pointers, caller-allocated, stream-ordered) --------------
 * These run one step of the sweep on buffers the caller owns.  All pointers are device
 * pointers except where noted; `stream` is a cudaStream_t (NULL = default stream).  The
 * calls are asynchronous; errors of the launch are returned, errors of the kernels surface at
 * the next synchronisation.                                                                 */

/* Scratch bytes qflow_dress_device needs for n orbitals. */
size_t qflow_dress_workspace(int32_t n, int32_t nocc);

/* Step (a): e0[1], F[n*n], W[n^4] of H-bar_<=2 for the pool (t1, t2); FP64.
 * work: qflow_dress_workspace(n, nocc) bytes of device scratch. */
int qflow_dress_device(const double* h, const double* eri, const double* t1, const double* t2, int32_t n,
                       int32_t nocc, double* e0, double* F, double* W, void* work, size_t work_bytes,
                       void* stream);

/* Steps (b)+(c) for a list of spaces of one size class (all (k,k), k = size_class in 1..3)
 * given dressed integrals (e0, F, W) on the device:
 *   spaces    qflow_space[nspaces] on the device (already in sorted order); a space whose
 *             (no, nv) is not (k, k) or whose orbitals are out of range gets status 4 and is
 *             skipped
 *   owner1/2  int32 owner maps (sorted indices, see qflow_plan), device; may be NULL, then no
 *             amplitude is written
 *   space_base  sorted index of spaces[0] (owners are compared with space_base + k)
 *   t1_old/t2_old  pool read by every space; t1_new/t2_new receive t_old + X for owned
 *             amplitudes (the caller initialises them, e.g. with a copy of the old pool)
 *   energy[nspaces], status[nspaces], iters[nspaces]: outputs (iters may be NULL)
 *   guess     NULL or device [nspaces][C(2k,k)^2] start vectors in the path's working
 *             precision (double for QFLOW_PREC_FP64, float for QFLOW_PREC_MIXED), any scale.
 *             FP64: the solver starts from the guess (an all-zero vector means Phi).  Mixed:
 *             the solver first tests Phi (converged there: done), else starts from the span
 *             of Phi and the guess, whose sigma counts as one iteration.  Receives the
 *             converged root (Phi coefficient 1) when save_root != 0
 *   precision qflow_precision; max_iter, tol as in qflow_options.
 * Mixed: the warp solver runs at most min(max_iter, 16) Davidson steps; when max_iter > 16 the
 * spaces it leaves unconverged are then solved by the FP64 solver (start from Phi, max_iter
 * steps), which needs 8 bytes of device scratch per space: the call allocates and frees it
 * on `stream` (cudaMallocAsync / cudaFreeAsync). */
int qflow_solve_device(int32_t n, int32_t nocc, const double* e0, const double* F, const double* W,
                       int32_t size_class, const qflow_space* spaces, int64_t nspaces, int64_t space_base, const int32_t* owner1,
                       const int32_t* owner2, const double* t1_old, const double* t2_old, double* t1_new,
                       double* t2_new, double* energy, int32_t* status, int32_t* iters, void* guess,
                       int32_t save_root, int32_t precision, int32_t max_iter, double tol, void* stream);

/* Tensor-core GEMM engine of the dressing contractions (tcgen05, kind::tf32 with three-term
 * hi/lo operand splits, FP32 accumulation in tensor memory): C[m][n] = sum_k A[m][k] B[n][k]
 * for row-major FP32 device arrays (leading dimensions lda >= K, ldb >= K, ldc >= N).  Each
 * product is accurate to about 2^-21 relative; accumulation is FP32.  err: device int, set to 1 when a tile gave up
 * waiting for its tensor-core work (it then leaves its C block unwritten); the caller zeroes
 * it.  Asynchronous on `stream`. */
int qflow_gemm_tf32x3_device(int32_t M, int32_t N, int32_t K, const float* A, int32_t lda, const float* B,
                             int32_t ldb, float* C, int32_t ldc, int32_t* err, void* stream);

/* ---- measurement: FMA peaks -------------------------------------------------------------
 * The paper has no counterpart; the solver's roofline divides by these rates.  Measures the
 * FMA throughput of this GPU in FP64 (precision QFLOW_PREC_FP64) or FP32 (QFLOW_PREC_MIXED):
 * every SM runs as many 256-thread blocks as fit, each thread eight independent fma chains;
 * *tflops = 2 x FMAs / CUDA-event time of the launch, best of three after a warm-up (about
 * 30 ms per launch).  Allocates a small output buffer on `stream` (stream-ordered) and
 * synchronises `stream` before returning.  Errors: QFLOW_ERR_ARG, QFLOW_ERR_CUDA. */
int qflow_fma_peak(int32_t precision, double* tflops, void* stream);

/* ---- allocation-free dressing ---------------------------------------------------------------
 * The paper has no counterpart to this entry point; it exists for callers that cannot call
 * cudaMalloc: applications whose device memory belongs to another allocator (an arena or pool
 * that must account for every byte), code that must not risk the implicit device
 * synchronisation an allocation may cause, or services with a fixed pre-reserved budget.
 *
 * qflow_dress_device_static computes exactly what qflow_dress_device computes (same kernels,
 * same arguments except the workspace) but takes its scratch from a static device array of
 * QFLOW_STATIC_SCRATCH_BYTES bytes inside the library, so the call allocates nothing (no
 * cudaMalloc, no cudaFree, no allocating library routine).  The array is held by every GPU
 * that loads the library until the process exits.
 *   - Limit: the call returns QFLOW_ERR_TOO_LARGE when qflow_dress_workspace(n, nocc) exceeds
 *     QFLOW_STATIC_SCRATCH_BYTES (4 MiB, e.g. 40 orbitals with 6 occupied fit, 82 do not).
 *   - Set-up: the first call on a device looks up the device address of the array on that
 *     device (with it current) and keeps it for that device's current context; make that first
 *     call before any stream capture.  A call that would do the look-up while `stream` is
 *     capturing returns QFLOW_ERR_STATE and enqueues nothing.  After a device reset (or any
 *     re-creation of the context) the kept address is dropped and looked up again.
 *   - Sharing: every call on a device uses the same array, which keeps the last call's data;
 *     the kernels write every scratch element before reading it, so nothing needs clearing.
 *     Calls whose work overlaps on the GPU (other streams, other threads) race on the array:
 *     order them on one stream or serialise them.
 * Other arguments, layouts and errors: as qflow_dress_device (QFLOW_ERR_OOM for an allocation
 * failure reported by the runtime, QFLOW_ERR_CUDA for any other CUDA failure). */
#define QFLOW_STATIC_SCRATCH_BYTES (4u * 1024u * 1024u)
int qflow_dress_device_static(const double* h, const double* eri, const double* t1, const double* t2, int32_t n,
                              int32_t nocc, double* e0, double* F, double* W, void* stream);
/* Size of that static scratch array in bytes. */
size_t qflow_static_scratch_bytes(void);

/* ---- warm-start network (not in the paper) -----------------------------------------------
 * The paper mentions learning only for choosing active spaces.  This optional network
 * predicts the CI -> CC increment of a 6e6o space from its folded integrals, and the first
 * sweep after a model is loaded starts those spaces' Davidson solvers from the prediction
 * instead of Phi.  The solver still converges every space to its own tolerance, so energies
 * and amplitudes do not depend on the network; only the iteration count does.
 *
 * Features of a (3,3) space (QFLOW_MLP_NIN = 708 floats): the vacuum-ordered one-body block
 * h[p][q] = F[p][q] - sum_{k occupied} (2 W[p][q][k][k] - W[p][k][k][q]) over the six local
 * orbitals (occupied first; 36, row-major), W[p][q][r][s] once per index-pair pair
 * P = 6p+q <= R = 6r+s (666, row-major over (P, R)), F[p][p] of the six orbitals (6).
 * Targets (QFLOW_MLP_NOUT = 54): X1[i][a] (9, row-major) and X2[i][j][a][b] once per
 * P = 3i+a <= R = 3j+b (45, row-major over (P, R)), local indices.
 * Start vector (400 determinants, the solver's layout: alpha string * 20 + beta string,
 * strings by increasing bit mask over the local orbitals): Phi + X1 Phi + (X2 + X1^2/2) Phi.
 * Network: H1 = tanh(x W1 + b1), H2 = tanh(H1 W2 + b2), y = H2 W3 + b3, FP32, W stored
 * [fan_in][fan_out] row-major; parameters packed as W1, b1, W2, b2, W3, b3
 * (qflow_mlp_param_count).  Loss: 1/(2 rows) sum (y - t)^2 over rows whose mask is set.
 * Adam: m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2, p -= lr (m/(1-b1^k)) / (sqrt(v/(1-b2^k)) + eps).
 * A model (qflow_mlp_model_size floats) is the parameters followed by the standardisation
 * mu_x[708], s_x[708] (network input = (x - mu_x) * s_x) and mu_y[54], sd_y[54]
 * (increment = mu_y + sd_y * network output). */
#define QFLOW_MLP_NIN 708
#define QFLOW_MLP_NOUT 54
#define QFLOW_GUESS_NETWORK 2

int64_t qflow_mlp_param_count(int32_t n_in, int32_t hidden, int32_t n_out);
int64_t qflow_mlp_model_size(int32_t hidden);

/* Load a model for the handle (host floats, qflow_mlp_model_size(hidden)); hidden in 1..1024.
 * has_stats = 0: the standardisation is computed from the training set at the next
 * qflow_mlp_train (the stored one is ignored).  Resets the Adam state.  In guess mode 2 the
 * next sweep starts 6e6o spaces from the model's prediction (an increment model). */
int qflow_mlp_set_model(qflow_handle hnd, int32_t hidden, const float* model, int32_t has_stats);
/* Copy the handle's model to a host buffer of qflow_mlp_model_size(hidden) floats. */
int qflow_mlp_get_model(qflow_handle hnd, float* model);

/* Append training pairs for every 6e6o space at class position p = k * stride (the class
 * position of a 6e6o space is its rank in lexicographic order of orb[0..5], ties by Delta-eps
 * position).  Two kinds of pair, one kind per handle:
 *   QFLOW_MLP_TARGET_INCREMENT: features from the last sweep's dressed integrals, target the
 *     increment of the space's converged root (guess mode 2, right after a sweep; spaces whose
 *     solve failed enter with a cleared mask).  A model trained on these gives Davidson guesses.
 *   QFLOW_MLP_TARGET_POOL: features from the bare integrals (the dressing of the zero pool),
 *     target the space's internal amplitudes in the current pool, e.g. after the flow has
 *     converged.  A model trained on these initialises a new flow's pool (qflow_mlp_warm_pool).
 * The call re-dresses for POOL pairs (the next sweep dresses again).  The first call fixes the
 * capacity (max_pairs rows); later calls append until it is full.  n_pairs (nullable) receives
 * the number of stored pairs. */
#define QFLOW_MLP_TARGET_INCREMENT 0
#define QFLOW_MLP_TARGET_POOL 1
int qflow_mlp_collect(qflow_handle hnd, int32_t target, int64_t stride, int64_t max_pairs, int64_t* n_pairs);

/* Warm start of the flow: the pool is set to the model's prediction, from the bare integrals,
 * of every 6e6o space's internal amplitudes, each amplitude taken from its owner space (the
 * owner rule of the merge); amplitudes no 6e6o space owns start at zero.  Needs a model with
 * standardisation (trained on QFLOW_MLP_TARGET_POOL pairs).  The sweeps that follow are the
 * plain flow, so its fixed point does not depend on the model; only the number of sweeps to
 * reach it does.  Resets the DIIS history. */
int qflow_mlp_warm_pool(qflow_handle hnd);

/* Train the loaded model on the stored pairs: `epochs` passes of mini-batches of `batch` rows
 * in the order given by order[n_pairs] (host, nullable = stored order), one Adam step
 * (b1 0.9, b2 0.999, eps 1e-8, learning rate lr) per batch.  loss (host, nullable,
 * `epochs` floats) receives each epoch's mean batch loss on standardised targets. */
int qflow_mlp_train(qflow_handle hnd, int32_t epochs, int32_t batch, float lr, const int64_t* order,
                    float* loss);

/* Device-level network steps (device pointers, stream-ordered, see the device-level section).
 * Workspace: qflow_mlp_workspace(n_in, hidden, n_out, rows) bytes. */
size_t qflow_mlp_workspace(int32_t n_in, int32_t hidden, int32_t n_out, int64_t rows);
/* y[rows][n_out] = network(x[rows][n_in]). */
int qflow_mlp_forward_device(int32_t n_in, int32_t hidden, int32_t n_out, const float* params, const float* x,
                             int64_t rows, float* y, void* work, void* stream);
/* loss[1] and grad[param_count] of the loss above; mask[rows] nullable (all rows count). */
int qflow_mlp_grad_device(int32_t n_in, int32_t hidden, int32_t n_out, const float* params, const float* x,
                          const float* target, const uint8_t* mask, int64_t rows, float* grad, float* loss,
                          void* work, void* stream);
/* One Adam step on n parameters; step counts from 1. */
int qflow_mlp_adam_device(int64_t n, float* params, const float* grad, float* m, float* v, int32_t step, float lr,
                          float beta1, float beta2, float eps, void* stream);
/* features[nspaces][708] of (3,3) spaces (device list) from dressed F, W (no standardisation). */
int qflow_mlp_features_device(int32_t n, const double* F, const double* W, const qflow_space* spaces,
                              int64_t nspaces, float* features, void* stream);
/* targets[rows][54] from CI vectors roots[rows][400] (Phi coefficient 1, float). */
int qflow_mlp_targets_device(const float* roots, int64_t rows, float* targets, void* stream);
/* Start vectors guess[rows][400] (float) from increments y[rows][54]. */
int qflow_mlp_guess_device(const float* y, int64_t rows, float* guess, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* QFLOW_H */
