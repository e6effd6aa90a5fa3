// C ABI of the flow: planning (ordering + ownership), the handle that owns one flow's device
// state, and the device-level step entry points.  Declarations and contracts: include/qflow.h.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <array>
#include <map>
#include <mutex>
#include <limits>
#include <new>
#include <numeric>
#include <vector>

#include "qflow_internal.h"

using qf::SolveArgs;
using qf::cuda_status;

namespace {

// ---- validation and planning -------------------------------------------------------------

int validate(const double* h, const double* eri, int32_t n, int32_t nocc, const qflow_space* sp, int64_t ns) {
  if (!h || !eri || !sp || n < 2 || n > 128 || nocc < 1 || nocc >= n || ns < 0) return QFLOW_ERR_ARG;
  for (int64_t k = 0; k < ns; ++k) {
    const qflow_space& s = sp[k];
    if (s.no != s.nv || s.no < 1 || s.no > 3 || s.no > nocc || s.nv > n - nocc) return QFLOW_ERR_ARG;
    for (int t = 0; t < s.no + s.nv; ++t) {
      const int o = s.orb[t];
      const bool occ = t < s.no;
      if (occ && (o < 0 || o >= nocc)) return QFLOW_ERR_ARG;
      if (!occ && (o < nocc || o >= n)) return QFLOW_ERR_ARG;
      if (t > 0 && t != s.no && s.orb[t - 1] >= o) return QFLOW_ERR_ARG;
    }
  }
  return QFLOW_OK;
}

// eps_p = h_pp + sum_k [2 (pp|kk) - (pk|kp)], k ascending (no contraction: -ffp-contract=off).
std::vector<double> fock_diagonal(const double* h, const double* eri, int n, int nocc) {
  std::vector<double> e(n);
  const size_t n1 = n, n2 = n1 * n1, n3 = n2 * n1;
  for (int p = 0; p < n; ++p) {
    double acc = h[(size_t)p * n + p];
    for (int k = 0; k < nocc; ++k) {
      const double j = eri[p * n3 + p * n2 + (size_t)k * n1 + k];
      const double x = eri[p * n3 + (size_t)k * n2 + (size_t)k * n1 + p];
      volatile double t = 2.0 * j;  // keep the FP64 rounding sequence of the definition
      acc = acc + (t - x);
    }
    e[p] = acc;
  }
  return e;
}

struct Plan {
  std::vector<int64_t> perm;
  std::vector<int32_t> own1, own2;
  int64_t uncovered = 0;
};

void make_plan(const double* h, const double* eri, int n, int nocc, const qflow_space* sp, int64_t ns, Plan* pl,
               bool want_owners) {
  const int nv = n - nocc;
  std::vector<double> eps = fock_diagonal(h, eri, n, nocc);
  std::vector<double> de(ns);
  for (int64_t k = 0; k < ns; ++k) {
    double sv = 0.0, so = 0.0;
    for (int t = 0; t < sp[k].nv; ++t) sv = sv + eps[sp[k].orb[sp[k].no + t]];
    for (int t = 0; t < sp[k].no; ++t) so = so + eps[sp[k].orb[t]];
    de[k] = sv - so;
  }
  pl->perm.resize(ns);
  std::iota(pl->perm.begin(), pl->perm.end(), (int64_t)0);
  std::sort(pl->perm.begin(), pl->perm.end(), [&](int64_t a, int64_t b) {
    if (de[a] != de[b]) return de[a] < de[b];
    const qflow_space &x = sp[a], &y = sp[b];
    if (x.no != y.no) return x.no < y.no;
    for (int t = 0; t < x.no; ++t)
      if (x.orb[t] != y.orb[t]) return x.orb[t] < y.orb[t];
    for (int t = 0; t < x.nv; ++t)
      if (x.orb[x.no + t] != y.orb[y.no + t]) return x.orb[x.no + t] < y.orb[y.no + t];
    return a < b;
  });
  if (!want_owners) return;
  pl->own1.assign((size_t)nocc * nv, -1);
  pl->own2.assign((size_t)nocc * nocc * nv * nv, -1);
  int64_t left = (int64_t)pl->own1.size() + (int64_t)pl->own2.size();
  for (int64_t s = 0; s < ns && left > 0; ++s) {
    const qflow_space& q = sp[pl->perm[s]];
    for (int i = 0; i < q.no; ++i)
      for (int a = 0; a < q.nv; ++a) {
        int32_t& o = pl->own1[(size_t)q.orb[i] * nv + (q.orb[q.no + a] - nocc)];
        if (o < 0) {
          o = (int32_t)s;
          --left;
        }
      }
    for (int i = 0; i < q.no; ++i)
      for (int j = 0; j < q.no; ++j)
        for (int a = 0; a < q.nv; ++a)
          for (int b = 0; b < q.nv; ++b) {
            const int I = q.orb[i], J = q.orb[j], A = q.orb[q.no + a] - nocc, B = q.orb[q.no + b] - nocc;
            int32_t& o = pl->own2[(((size_t)I * nocc + J) * nv + A) * nv + B];
            if (o < 0) {
              o = (int32_t)s;
              --left;
            }
          }
  }
  pl->uncovered = 0;
  for (int32_t o : pl->own1) pl->uncovered += (o < 0);
  for (int32_t o : pl->own2) pl->uncovered += (o < 0);
}

// Device order of a planned list: grouped by size class (k = 1, 2, 3), and within a class in
// orbital-tuple order (occupied tuple, then virtual tuple) so that warps running at the same time
// gather overlapping rows of W from L2.  gidx[d] = Delta-eps (sorted) position of device slot d.
void group_spaces(const qflow_space* spaces, int64_t ns, const Plan& pl, std::vector<qflow_space>* grouped,
                  std::vector<int64_t>* gidx, int64_t cls_count[4], int64_t cls_off[4]) {
  grouped->assign((size_t)ns, qflow_space{});
  gidx->assign((size_t)ns, 0);
  for (int k = 0; k < 4; ++k) cls_count[k] = 0;
  for (int64_t s = 0; s < ns; ++s) cls_count[spaces[pl.perm[s]].no]++;
  cls_off[0] = 0;
  cls_off[1] = 0;
  cls_off[2] = cls_count[1];
  cls_off[3] = cls_count[1] + cls_count[2];
  int64_t fill[4] = {0, cls_off[1], cls_off[2], cls_off[3]};
  for (int64_t s = 0; s < ns; ++s) {
    const qflow_space& q = spaces[pl.perm[s]];
    (*grouped)[fill[q.no]] = q;
    (*gidx)[fill[q.no]] = s;
    fill[q.no]++;
  }
  for (int k = 1; k <= 3; ++k) {
    const int64_t b = cls_off[k], e = b + cls_count[k];
    std::vector<int64_t> ord((size_t)(e - b));
    std::iota(ord.begin(), ord.end(), b);
    std::stable_sort(ord.begin(), ord.end(), [&](int64_t x, int64_t y) {
      for (int t = 0; t < 2 * k; ++t)
        if ((*grouped)[x].orb[t] != (*grouped)[y].orb[t]) return (*grouped)[x].orb[t] < (*grouped)[y].orb[t];
      return (*gidx)[x] < (*gidx)[y];
    });
    std::vector<qflow_space> gs(ord.size());
    std::vector<int64_t> gi(ord.size());
    for (size_t t = 0; t < ord.size(); ++t) {
      gs[t] = (*grouped)[ord[t]];
      gi[t] = (*gidx)[ord[t]];
    }
    std::copy(gs.begin(), gs.end(), grouped->begin() + b);
    std::copy(gi.begin(), gi.end(), gidx->begin() + b);
  }
}

// Shard `rank` of `nranks`: in every size class the class positions [lo[k], hi[k]) of the device
// order (equal shares, the first ranks one smaller when the count does not divide).
void shard_ranges(const int64_t cls_count[4], int rank, int nranks, int64_t lo[4], int64_t hi[4]) {
  for (int k = 0; k < 4; ++k) {
    lo[k] = cls_count[k] * rank / nranks;
    hi[k] = cls_count[k] * (rank + 1) / nranks;
  }
}

// Exchange masks of shard `rank`: space_mask[s] = 1 for the Delta-eps positions s the shard
// solves; pool_mask[x] = 1 for the amplitudes (t1 then t2) whose owner space it solves.
void shard_masks(const std::vector<int64_t>& gidx, const int64_t cls_count[4], const int64_t cls_off[4],
                 const int32_t* own1, int64_t n1, const int32_t* own2, int64_t n2, int rank, int nranks,
                 uint8_t* space_mask, uint8_t* pool_mask) {
  int64_t lo[4], hi[4];
  shard_ranges(cls_count, rank, nranks, lo, hi);
  std::vector<uint8_t> sm(gidx.size(), 0);
  for (int k = 1; k <= 3; ++k)
    for (int64_t d = cls_off[k] + lo[k]; d < cls_off[k] + hi[k]; ++d) sm[(size_t)gidx[(size_t)d]] = 1;
  if (space_mask) std::copy(sm.begin(), sm.end(), space_mask);
  if (pool_mask) {
    for (int64_t x = 0; x < n1; ++x) pool_mask[x] = (own1[x] >= 0) ? sm[(size_t)own1[x]] : 0;
    for (int64_t x = 0; x < n2; ++x) pool_mask[n1 + x] = (own2[x] >= 0) ? sm[(size_t)own2[x]] : 0;
  }
}

}  // namespace

// ---- handle --------------------------------------------------------------------------------

struct qflow_ctx {
  int32_t n = 0, nocc = 0, nvir = 0;
  int64_t nspaces = 0;
  qflow_options opt{};
  cudaStream_t stream = nullptr;
  std::vector<int64_t> perm;
  int64_t cls_count[4] = {0, 0, 0, 0};  // spaces per size class k = 1..3 (grouped on device)
  int64_t cls_off[4] = {0, 0, 0, 0};
  // device buffers
  double *h = nullptr, *eri = nullptr;
  double *pool = nullptr, *pool_new = nullptr;  // [t1 | t2]
  double *e0 = nullptr, *F = nullptr, *W = nullptr;
  double* energy = nullptr;
  int32_t *status = nullptr, *iters = nullptr;
  int32_t *own1 = nullptr, *own2 = nullptr;
  uint8_t* owns = nullptr;  // [device slot]: 1 if the space there owns an amplitude
  qflow_space* spaces = nullptr;  // grouped by class, sorted within a class
  int64_t* sorted_index = nullptr;
  void* dwork = nullptr;
  size_t dwork_bytes = 0;
  void* rwork = nullptr;
  double* red = nullptr;  // [4] reduction results
  double* red_host = nullptr;  // pinned
  double e_mean = 0.0;
  bool have_energy = false;
  int64_t n_t1 = 0, n_t2 = 0;
  void* guess[4] = {nullptr, nullptr, nullptr, nullptr};  // previous roots per size class (opt.guess == 1)
  void* diis = nullptr;                                   // DIIS ring (opt.diis > 0)
  float* W32 = nullptr;  // FP32 copies of W (n^4) and F (n^2, after W) for the mixed-precision solver
  unsigned long long* queue = nullptr;                    // persistent-launch work counter
  double* F0 = nullptr;  // DUCC form: the bare Fock matrix (the per-space part of the operator needs it)
  int64_t* rescue_items = nullptr;  // mixed path: positions of spaces the warp pass left unconverged
  unsigned long long* rescue_count = nullptr;  // and their count (device)
  // launch schedule of the mixed-precision solver: persistent queue or one launch per class
  int sched_persistent = 1, sched_chunk = 1, sched_warps = 15;  // items per fetch, warps (spaces) per CTA
  bool tuned = false;
  int64_t sweeps = 0;  // sweeps run so far
  float tune_ms[QFLOW_TUNE_MAX] = {0};
  int tune_count = 0;
  // tile width of the mixed dressing's ladder + oooo product (0 = the default until tuned) and
  // the tuner's times for 32, 64 and 128 columns
  int ladder_bn = 0;
  float ladder_ms[QFLOW_LADDER_TUNE_MAX] = {0};
  int ladder_count = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  int64_t graph_launches = 0;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};  // phase marks of the last sweep
  int64_t last_launches = 0;                                  // kernels launched by the last sweep
  // warm-start network (opt.guess == 2): model = parameters + standardisation (device)
  int mlp_hidden = 0;
  int64_t mlp_nparam = 0;
  float* mlp_model = nullptr;
  float *mlp_grad = nullptr, *mlp_m = nullptr, *mlp_v = nullptr;  // Adam state
  int mlp_step = 0;
  bool mlp_has_stats = false;
  bool mlp_pending = false;    // the next sweep starts 6e6o spaces from the network
  bool mlp_guess_now = false;  // set while such a sweep is enqueued
  bool fw_of_last_sweep = false;  // F, W still hold the dressing of the last sweep
  int64_t mlp_cap = 0, mlp_n = 0;  // training pairs: capacity, stored
  int mlp_target = 0;              // kind of the stored pairs (QFLOW_MLP_TARGET_*)
  float *mlp_X = nullptr, *mlp_T = nullptr;
  uint8_t* mlp_mask = nullptr;
  // sharded sweeps (qflow_set_shard): this rank solves class positions [lo[k], hi[k]) of class k
  int shard_rank = 0, shard_n = 1;
  int64_t shard_lo[4] = {0, 0, 0, 0}, shard_hi[4] = {0, 0, 0, 0};
  uint8_t *space_mask = nullptr, *pool_mask = nullptr;  // device, see shard_masks
  bool shard_open = false;  // between qflow_sweep_shard_begin and _end
  bool shard_warm = false;  // that sweep started from the network's guesses
  // wave-ordered sweeps: class positions of each class sorted by Delta-eps position (device),
  // and those positions' sorted indices (host, ascending) to cut a wave into per-class ranges
  int64_t* wave_items = nullptr;
  std::vector<int64_t> wave_sidx[4];
  double* pool_start = nullptr;  // the pool at the start of a wave-ordered sweep
};

namespace {

template <typename T>
cudaError_t dalloc(T** p, size_t count) {
  return cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T) + 16);
}

void free_ctx(qflow_ctx* c) {
  if (!c) return;
  void* ptrs[] = {c->h, c->eri, c->pool, c->pool_new, c->e0, c->F, c->W, c->energy, c->status, c->iters,
                  c->own1, c->own2, c->owns, c->spaces, c->sorted_index, c->dwork, c->rwork, c->red};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  for (void* p : c->guess)
    if (p) cudaFree(p);
  if (c->diis) cudaFree(c->diis);
  if (c->W32) cudaFree(c->W32);
  if (c->queue) cudaFree(c->queue);
  if (c->rescue_items) cudaFree(c->rescue_items);
  if (c->F0) cudaFree(c->F0);
  if (c->rescue_count) cudaFree(c->rescue_count);
  void* mptrs[] = {c->mlp_model, c->mlp_grad, c->mlp_m, c->mlp_v, c->mlp_X, c->mlp_T, c->mlp_mask,
                   c->space_mask, c->pool_mask, c->wave_items, c->pool_start};
  for (void* p : mptrs)
    if (p) cudaFree(p);
  if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
  if (c->graph) cudaGraphDestroy(c->graph);
  if (c->red_host) cudaFreeHost(c->red_host);
  for (cudaEvent_t e : c->ev)
    if (e) cudaEventDestroy(e);
  if (c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

}  // namespace

extern "C" {

void qflow_default_options(qflow_options* opt, int32_t precision) {
  if (!opt) return;
  memset(opt, 0, sizeof(*opt));
  opt->precision = precision;
  opt->max_iter = 60;
  opt->tol = (precision == QFLOW_PREC_MIXED) ? 1e-6 : 1e-9;
  opt->diis = 0;
  opt->guess = 0;
  opt->schedule = QFLOW_SCHED_AUTO;
  opt->graph = 1;
  opt->form = QFLOW_FORM_SESCC;
  opt->warps = 0;
}

int qflow_plan(const double* h, const double* eri, int32_t n, int32_t nocc, const qflow_space* spaces,
               int64_t nspaces, int64_t* perm, int32_t* owner1, int32_t* owner2, int64_t* n_uncovered) {
  if (!perm) return QFLOW_ERR_ARG;
  int v = validate(h, eri, n, nocc, spaces, nspaces);
  if (v != QFLOW_OK) return v;
  Plan pl;
  try {
    make_plan(h, eri, n, nocc, spaces, nspaces, &pl, owner1 || owner2 || n_uncovered);
  } catch (const std::bad_alloc&) {
    return QFLOW_ERR_OOM;
  }
  memcpy(perm, pl.perm.data(), sizeof(int64_t) * (size_t)nspaces);
  if (owner1) memcpy(owner1, pl.own1.data(), sizeof(int32_t) * pl.own1.size());
  if (owner2) memcpy(owner2, pl.own2.data(), sizeof(int32_t) * pl.own2.size());
  if (n_uncovered) *n_uncovered = pl.uncovered;
  return (pl.uncovered > 0) ? QFLOW_WARN_UNCOVERED : QFLOW_OK;
}

int qflow_shard_plan(const double* h, const double* eri, int32_t n, int32_t nocc, const qflow_space* spaces,
                     int64_t nspaces, int32_t rank, int32_t nranks, uint8_t* space_mask, uint8_t* pool_mask) {
  if (nranks < 1 || rank < 0 || rank >= nranks) return QFLOW_ERR_ARG;
  int v = validate(h, eri, n, nocc, spaces, nspaces);
  if (v != QFLOW_OK) return v;
  try {
    Plan pl;
    make_plan(h, eri, n, nocc, spaces, nspaces, &pl, true);
    std::vector<qflow_space> grouped;
    std::vector<int64_t> gidx;
    int64_t cnt[4], off[4];
    group_spaces(spaces, nspaces, pl, &grouped, &gidx, cnt, off);
    shard_masks(gidx, cnt, off, pl.own1.data(), (int64_t)pl.own1.size(), pl.own2.data(), (int64_t)pl.own2.size(),
                rank, nranks, space_mask, pool_mask);
  } catch (const std::bad_alloc&) {
    return QFLOW_ERR_OOM;
  }
  return QFLOW_OK;
}

int qflow_init(qflow_handle* out, const double* h, const double* eri, int32_t n, int32_t nocc,
               const qflow_space* spaces, int64_t nspaces, const qflow_options* opt) {
  if (!out) return QFLOW_ERR_ARG;
  *out = nullptr;
  int v = validate(h, eri, n, nocc, spaces, nspaces);
  if (v != QFLOW_OK) return v;
  qflow_ctx* c = new (std::nothrow) qflow_ctx();
  if (!c) return QFLOW_ERR_OOM;
  if (opt) c->opt = *opt; else qflow_default_options(&c->opt, QFLOW_PREC_FP64);
  if (c->opt.precision != QFLOW_PREC_FP64 && c->opt.precision != QFLOW_PREC_MIXED) {
    delete c;
    return QFLOW_ERR_ARG;
  }
  if (c->opt.warps < 0 || c->opt.warps > 15) {
    delete c;
    return QFLOW_ERR_ARG;
  }
  if (c->opt.warps > 0) c->sched_warps = c->opt.warps;
  if (c->opt.chunk < 0 || c->opt.chunk > 16) {
    delete c;
    return QFLOW_ERR_ARG;
  }
  if (c->opt.chunk > 0) c->sched_chunk = c->opt.chunk;
  if (c->opt.ladder_bn != 0 && c->opt.ladder_bn != 32 && c->opt.ladder_bn != 64 && c->opt.ladder_bn != 128) {
    delete c;
    return QFLOW_ERR_ARG;
  }
  c->ladder_bn = c->opt.ladder_bn;
  if (c->opt.form != QFLOW_FORM_SESCC && c->opt.form != QFLOW_FORM_DUCC) {
    delete c;
    return QFLOW_ERR_ARG;
  }
  if (c->opt.form == QFLOW_FORM_DUCC && (c->opt.precision != QFLOW_PREC_FP64 || c->opt.guess == QFLOW_GUESS_NETWORK)) {
    delete c;
    return QFLOW_ERR_ARG;
  }
  if (c->opt.max_iter <= 0) c->opt.max_iter = 60;
  if (c->opt.diis < 0 || c->opt.diis > QFLOW_DIIS_MAX || c->opt.diis == 1 || c->opt.guess < 0 ||
      c->opt.guess > QFLOW_GUESS_NETWORK) {
    delete c;
    return QFLOW_ERR_ARG;
  }
  if (!(c->opt.tol > 0.0)) c->opt.tol = (c->opt.precision == QFLOW_PREC_MIXED) ? 1e-6 : 1e-9;
  c->n = n;
  c->nocc = nocc;
  c->nvir = n - nocc;
  c->nspaces = nspaces;
  c->n_t1 = (int64_t)nocc * c->nvir;
  c->n_t2 = (int64_t)nocc * nocc * c->nvir * c->nvir;
  Plan pl;
  try {
    make_plan(h, eri, n, nocc, spaces, nspaces, &pl, true);
  } catch (const std::bad_alloc&) {
    delete c;
    return QFLOW_ERR_OOM;
  }
  c->perm = pl.perm;
  std::vector<qflow_space> grouped;
  std::vector<int64_t> gidx;
  group_spaces(spaces, nspaces, pl, &grouped, &gidx, c->cls_count, c->cls_off);
  const size_t n1 = n, n4 = n1 * n1 * n1 * n1;
  cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
  c->dwork_bytes = (c->opt.precision == QFLOW_PREC_MIXED) ? qf::dress_workspace_bytes_mixed(n, nocc)
                   : (c->opt.form == QFLOW_FORM_DUCC)      ? qf::ducc_workspace_bytes(n, nocc)
                                                          : qf::dress_workspace_bytes(n, nocc);
  const size_t npool = (size_t)(c->n_t1 + c->n_t2);
  if (e == cudaSuccess) e = dalloc(&c->h, n1 * n1);
  if (e == cudaSuccess) e = dalloc(&c->eri, n4);
  if (e == cudaSuccess) e = dalloc(&c->pool, npool);
  if (e == cudaSuccess) e = dalloc(&c->pool_new, npool);
  if (e == cudaSuccess) e = dalloc(&c->e0, 1);
  if (e == cudaSuccess) e = dalloc(&c->F, n1 * n1);
  if (e == cudaSuccess) e = dalloc(&c->W, n4);
  if (e == cudaSuccess) e = dalloc(&c->energy, (size_t)std::max<int64_t>(nspaces, 1));
  if (e == cudaSuccess) e = dalloc(&c->status, (size_t)std::max<int64_t>(nspaces, 1));
  if (e == cudaSuccess) e = dalloc(&c->iters, (size_t)std::max<int64_t>(nspaces, 1));
  if (e == cudaSuccess) e = dalloc(&c->own1, (size_t)c->n_t1);
  if (e == cudaSuccess) e = dalloc(&c->own2, (size_t)c->n_t2);
  if (e == cudaSuccess) e = dalloc(&c->owns, (size_t)std::max<int64_t>(nspaces, 1));
  if (e == cudaSuccess) e = dalloc(&c->spaces, (size_t)std::max<int64_t>(nspaces, 1));
  if (e == cudaSuccess) e = dalloc(&c->sorted_index, (size_t)std::max<int64_t>(nspaces, 1));
  if (e == cudaSuccess) e = cudaMalloc(&c->dwork, c->dwork_bytes);
  if (e == cudaSuccess) e = cudaMalloc(&c->rwork, qf::mean_maxdiff_workspace(nspaces, (int64_t)npool));
  if (e == cudaSuccess) e = dalloc(&c->red, 4);
  if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&c->red_host), 4 * sizeof(double));
  for (int k = 0; k < 4 && e == cudaSuccess; ++k) e = cudaEventCreate(&c->ev[k]);
  if (c->opt.precision == QFLOW_PREC_MIXED && e == cudaSuccess) e = dalloc(&c->W32, n4 + n1 * n1);
  if (c->opt.form == QFLOW_FORM_DUCC && e == cudaSuccess) e = dalloc(&c->F0, n1 * n1);
  if (e == cudaSuccess) e = dalloc(&c->queue, 1);
  if (c->opt.precision == QFLOW_PREC_MIXED && e == cudaSuccess) {
    int64_t most = 1;
    for (int k = 1; k <= 3; ++k) most = std::max(most, c->cls_count[k]);
    e = dalloc(&c->rescue_items, (size_t)most);
    if (e == cudaSuccess) e = dalloc(&c->rescue_count, 1);
  }
  if (c->opt.schedule == QFLOW_SCHED_PER_CLASS) {
    c->sched_persistent = 0;
    c->tuned = true;
  } else if (c->opt.schedule == QFLOW_SCHED_PERSISTENT) {
    c->sched_persistent = 1;
    c->tuned = true;
  }
  if (c->opt.diis > 0 && e == cudaSuccess) {
    e = cudaMalloc(&c->diis, qf::diis_workspace_bytes(c->opt.diis, (int64_t)npool));
    if (e == cudaSuccess) e = qf::diis_reset(c->diis, c->opt.diis, (int64_t)npool, c->stream);
  }
  if (c->opt.guess == 1 || c->opt.guess == QFLOW_GUESS_NETWORK) {  // roots of every class (1) or 6e6o (2)
    const size_t ndet[4] = {0, 4, 36, 400};
    const size_t esz = (c->opt.precision == QFLOW_PREC_MIXED) ? sizeof(float) : sizeof(double);
    for (int k = (c->opt.guess == 1 ? 1 : 3); k <= 3 && e == cudaSuccess; ++k) {
      if (c->cls_count[k] == 0) continue;
      const size_t bytes = (size_t)c->cls_count[k] * ndet[k] * esz;
      e = cudaMalloc(&c->guess[k], bytes);
      if (e == cudaSuccess) e = cudaMemsetAsync(c->guess[k], 0, bytes, c->stream);  // zero = start from Phi
    }
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->h, h, sizeof(double) * n1 * n1, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->eri, eri, sizeof(double) * n4, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->pool, 0, sizeof(double) * npool, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->own1, pl.own1.data(), sizeof(int32_t) * pl.own1.size(), cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->own2, pl.own2.data(), sizeof(int32_t) * pl.own2.size(), cudaMemcpyHostToDevice, c->stream);
  // owner flags by device slot (the solver reads them beside the space record, without waiting
  // for the sorted index)
  std::vector<uint8_t> owns_s((size_t)std::max<int64_t>(nspaces, 1), 0), owns((size_t)std::max<int64_t>(nspaces, 1), 0);
  for (int32_t o : pl.own1)
    if (o >= 0) owns_s[(size_t)o] = 1;
  for (int32_t o : pl.own2)
    if (o >= 0) owns_s[(size_t)o] = 1;
  for (int64_t d = 0; d < nspaces; ++d) owns[(size_t)d] = owns_s[(size_t)gidx[(size_t)d]];
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->owns, owns.data(), owns.size(), cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess && nspaces > 0)
    e = cudaMemcpyAsync(c->spaces, grouped.data(), sizeof(qflow_space) * (size_t)nspaces, cudaMemcpyHostToDevice,
                        c->stream);
  if (e == cudaSuccess && nspaces > 0)
    e = cudaMemcpyAsync(c->sorted_index, gidx.data(), sizeof(int64_t) * (size_t)nspaces, cudaMemcpyHostToDevice,
                        c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    free_ctx(c);
    return cuda_status(e);
  }
  *out = c;
  return (pl.uncovered > 0) ? QFLOW_WARN_UNCOVERED : QFLOW_OK;
}

}  // extern "C"

namespace {

qf::SolveArgs solve_args(qflow_ctx* c, int k) {
  SolveArgs a{};
  a.n = c->n;
  a.nocc = c->nocc;
  a.nvir = c->nvir;
  a.e0 = c->e0;
  a.F = c->F;
  a.W = c->W;
  const int64_t lo = (c->shard_n > 1) ? c->shard_lo[k] : 0;
  a.spaces = c->spaces + c->cls_off[k] + lo;
  a.nspaces = (c->shard_n > 1) ? c->shard_hi[k] - lo : c->cls_count[k];
  a.space_base = 0;
  a.sorted_index = c->sorted_index + c->cls_off[k] + lo;
  a.owner1 = c->own1;
  a.owner2 = c->own2;
  a.owns = c->owns + c->cls_off[k] + lo;
  a.t1_old = c->pool;
  a.t2_old = c->pool + c->n_t1;
  a.t1_new = c->pool_new;
  a.t2_new = c->pool_new + c->n_t1;
  a.energy = c->energy;
  a.status = c->status;
  a.iters = c->iters;
  a.W32 = c->W32;
  a.F32 = c->W32 ? c->W32 + (size_t)c->n * c->n * c->n * c->n : nullptr;
  // guess mode 1: start from and keep the previous roots; mode 2: keep 6e6o roots, start from
  // them only on a warm-start sweep (where the network has just written them)
  const size_t ndet[4] = {0, 4, 36, 400};
  const size_t esz = (c->opt.precision == QFLOW_PREC_MIXED) ? sizeof(float) : sizeof(double);
  void* roots = c->guess[k] ? static_cast<char*>(c->guess[k]) + (size_t)lo * ndet[k] * esz : nullptr;
  a.guess = (c->opt.guess == 1 || c->mlp_guess_now) ? roots : nullptr;
  a.root_out = roots;
  a.max_iter = c->opt.max_iter;
  a.tol = c->opt.tol;
  if (c->opt.form == QFLOW_FORM_DUCC) {
    a.ducc_eri = c->eri;
    a.ducc_F0 = c->F0;
  }
  return a;
}

// Phase marker k.  Inside a stream capture the record becomes an event node of the graph, so
// every replay records it again (a plain record would only take part in the capture).
cudaError_t mark(qflow_ctx* c, int k) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(c->stream, &cs);
  if (e != cudaSuccess) return e;
  return cudaEventRecordWithFlags(c->ev[k], c->stream,
                                  cs == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : cudaEventRecordDefault);
}

// e0, F, W of the operator every space gathers, for the pool (t1, t2): the SES-CC dressing, or the
// common part G of the DUCC form (which also leaves the bare Fock matrix in F0).
cudaError_t dress_pool(qflow_ctx* c, const double* t1, const double* t2) {
  if (c->opt.form == QFLOW_FORM_DUCC)
    return qf::launch_dress_ducc(c->h, c->eri, t1, t2, c->n, c->nocc, c->e0, c->F, c->W, c->F0, c->dwork,
                                 c->dwork_bytes, c->stream);
  return qf::launch_dress(c->h, c->eri, t1, t2, c->n, c->nocc, c->e0, c->F, c->W, c->dwork, c->dwork_bytes, c->stream,
                          c->W32, c->ladder_bn);
}

int dress_pool_launches(const qflow_ctx* c) {
  return (c->opt.form == QFLOW_FORM_DUCC) ? qf::ducc_launch_count(c->n, c->nocc)
                                          : qf::dress_launch_count(c->n, c->nocc, c->W32 != nullptr);
}

// Step (a): dressing (+ the FP32 copy of W for the mixed solver).
cudaError_t enqueue_dress(qflow_ctx* c, int64_t* launches) {
  cudaError_t e = mark(c, 0);
  if (e == cudaSuccess) e = dress_pool(c, c->pool, c->pool + c->n_t1);
  *launches += dress_pool_launches(c);
  if (e == cudaSuccess && c->W32) {
    const size_t n4 = (size_t)c->n * c->n * c->n * c->n;
    e = qf::launch_to_f32(c->W, c->W32, n4, c->stream);
    if (e == cudaSuccess) e = qf::launch_to_f32(c->F, c->W32 + n4, (size_t)c->n * c->n, c->stream);
    *launches += 2;
  }
  if (e == cudaSuccess) e = mark(c, 1);
  return e;
}

// The per-space solves with a given schedule; `count` > 0 limits every class to its first
// `count` spaces (autotuner calibration).
cudaError_t enqueue_solve_cls(qflow_ctx* c, SolveArgs* cls, int persistent, int chunk, int warps, int64_t* launches,
                              bool calibrating);

cudaError_t enqueue_solve(qflow_ctx* c, int persistent, int chunk, int warps, int64_t count, int64_t* launches) {
  SolveArgs cls[4];
  for (int k = 1; k <= 3; ++k) {
    cls[k] = solve_args(c, k);
    if (count > 0) {  // calibration: a prefix of each class, no saved roots
      if (cls[k].nspaces > count) cls[k].nspaces = count;
      cls[k].guess = nullptr;
      cls[k].root_out = nullptr;
    }
  }
  return enqueue_solve_cls(c, cls, persistent, chunk, warps, launches, count > 0);
}

// The solves of the given per-class arguments (cls[1..3]) with a given schedule.  In the mixed
// path the warp solver's pass stops at qf::kWarpIterCap steps; unless `calibrating`, the spaces it
// leaves unconverged are then solved again by the FP64 solver within max_iter steps.
cudaError_t enqueue_solve_cls(qflow_ctx* c, SolveArgs* cls, int persistent, int chunk, int warps, int64_t* launches,
                              bool calibrating) {
  if (c->opt.precision != QFLOW_PREC_MIXED) {
    cudaError_t e = cudaSuccess;
    for (int k = 1; k <= 3 && e == cudaSuccess; ++k) {
      if (cls[k].nspaces == 0) continue;
      e = qf::launch_solve(k, c->opt.precision, cls[k], c->stream);
      ++*launches;
    }
    return e;
  }
  SolveArgs warp[4];
  for (int k = 1; k <= 3; ++k) {
    warp[k] = cls[k];
    if (warp[k].max_iter > qf::kWarpIterCap) warp[k].max_iter = qf::kWarpIterCap;
  }
  cudaError_t e = cudaSuccess;
  if (persistent) {
    *launches += 2;  // queue reset + kernel
    e = qf::launch_solve_persistent(warp, c->W32, c->queue, chunk, warps, c->stream);
  } else {
    for (int k = 3; k >= 1 && e == cudaSuccess; --k) {
      if (warp[k].nspaces == 0) continue;
      e = qf::launch_solve_warp(k, warp[k], c->W32, static_cast<const float*>(warp[k].guess),
                                static_cast<float*>(warp[k].root_out), warps, c->stream);
      ++*launches;
    }
  }
  for (int k = 3; k >= 1 && e == cudaSuccess && !calibrating; --k) {
    if (cls[k].nspaces == 0 || cls[k].max_iter <= qf::kWarpIterCap) continue;
    e = qf::launch_solve_rescue(k, cls[k], c->rescue_items, c->rescue_count, c->stream);
    *launches += 3;
  }
  return e;
}

// Step (b): pool_new <- pool, then the solves write t_old + X into pool_new for owned amplitudes.
cudaError_t enqueue_solve_phase(qflow_ctx* c, int64_t* launches) {
  const size_t npool = (size_t)(c->n_t1 + c->n_t2);
  cudaError_t e = cudaMemcpyAsync(c->pool_new, c->pool, sizeof(double) * npool, cudaMemcpyDeviceToDevice, c->stream);
  if (e == cudaSuccess) e = enqueue_solve(c, c->sched_persistent, c->sched_chunk, c->sched_warps, 0, launches);
  return e;
}

// Step (c) after the solves: DIIS, phase mark 2 (unless already set), reductions,
// pool_new -> pool, phase mark 3, scalars to the host.
cudaError_t enqueue_merge_phase(qflow_ctx* c, bool mark2, int64_t* launches) {
  const size_t npool = (size_t)(c->n_t1 + c->n_t2);
  cudaError_t e = cudaSuccess;
  if (c->diis) {
    e = qf::launch_diis(c->diis, c->opt.diis, c->pool, c->pool_new, (int64_t)npool, c->stream);
    *launches += 4;
  }
  if (e == cudaSuccess && mark2) e = mark(c, 2);
  if (e == cudaSuccess)
    e = qf::launch_reduce(c->energy, c->status, c->nspaces, c->pool, c->pool_new, (int64_t)npool, c->red, c->rwork,
                          c->stream);
  *launches += 2;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->pool, c->pool_new, sizeof(double) * npool, cudaMemcpyDeviceToDevice, c->stream);
  if (e == cudaSuccess) e = mark(c, 3);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->red_host, c->red, 4 * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  return e;
}

// Steps (b)+(c) of an unsharded sweep.
cudaError_t enqueue_solve_merge(qflow_ctx* c, int64_t* launches) {
  cudaError_t e = enqueue_solve_phase(c, launches);
  if (e == cudaSuccess) e = enqueue_merge_phase(c, true, launches);
  return e;
}

// Autotuner: time candidate schedules on the first spaces of every class (the dressed integrals
// of the current sweep are in place) and keep the fastest.  Results are cached per problem
// shape for the process.
struct TuneKey {
  int n, nocc;
  int64_t c1, c2, c3;
  bool operator<(const TuneKey& o) const {
    if (n != o.n) return n < o.n;
    if (nocc != o.nocc) return nocc < o.nocc;
    if (c1 != o.c1) return c1 < o.c1;
    if (c2 != o.c2) return c2 < o.c2;
    return c3 < o.c3;
  }
};
std::map<TuneKey, std::array<int, 4>> g_tune_cache;  // persistent, chunk, warps, ladder width
std::mutex g_tune_mu;

// Model layout: parameters, then mu_x[708], s_x[708], mu_y[54], sd_y[54].
float* mlp_stats(qflow_ctx* c, int which) {
  float* p = c->mlp_model + c->mlp_nparam;
  const int64_t off[4] = {0, QFLOW_MLP_NIN, 2 * QFLOW_MLP_NIN, 2 * QFLOW_MLP_NIN + QFLOW_MLP_NOUT};
  return p + off[which];
}

// Dressing of the zero pool (bare Fock matrix and integrals) into F, W; pool_new is scratch.
cudaError_t dress_bare(qflow_ctx* c) {
  cudaError_t e = cudaMemsetAsync(c->pool_new, 0, sizeof(double) * (size_t)(c->n_t1 + c->n_t2), c->stream);
  if (e == cudaSuccess)
    e = dress_pool(c, c->pool_new, c->pool_new + c->n_t1);
  c->fw_of_last_sweep = false;
  return e;
}

// Warm start: the network's start vectors for every 6e6o space, written where the solver reads
// its guesses (the 6e6o root buffer), in chunks of rows.
cudaError_t enqueue_mlp_guess(qflow_ctx* c, int64_t* launches) {
  const int64_t n3 = c->cls_count[3];
  const int64_t CH = 131072;
  const int64_t rows = n3 < CH ? n3 : CH;
  const int H = c->mlp_hidden;
  const size_t fx = (size_t)rows * QFLOW_MLP_NIN * sizeof(float), fy = (size_t)rows * QFLOW_MLP_NOUT * sizeof(float);
  const size_t bytes = fx + fy + qf::mlp_workspace_bytes(QFLOW_MLP_NIN, H, QFLOW_MLP_NOUT, rows) + 512;
  void* buf = nullptr;
  cudaError_t e = cudaMallocAsync(&buf, bytes, c->stream);
  if (e != cudaSuccess) return e;
  float* X = static_cast<float*>(buf);
  float* Y = reinterpret_cast<float*>(static_cast<char*>(buf) + ((fx + 255) / 256) * 256);
  void* work = static_cast<char*>(buf) + ((fx + 255) / 256) * 256 + ((fy + 255) / 256) * 256;
  const bool fp64 = c->opt.precision != QFLOW_PREC_MIXED;
  const size_t esz = fp64 ? sizeof(double) : sizeof(float);
  for (int64_t off = 0; off < n3 && e == cudaSuccess; off += CH) {
    const int64_t r = (n3 - off < CH) ? n3 - off : CH;
    e = qf::mlp_features(c->n, c->F, c->W, c->spaces + c->cls_off[3] + off, r, 1, mlp_stats(c, 0), mlp_stats(c, 1), X,
                         c->stream);
    if (e == cudaSuccess)
      e = qf::mlp_forward(QFLOW_MLP_NIN, H, QFLOW_MLP_NOUT, c->mlp_model, X, r, Y, work, c->stream);
    if (e == cudaSuccess)
      e = qf::mlp_guess(Y, r, mlp_stats(c, 2), mlp_stats(c, 3), static_cast<char*>(c->guess[3]) + (size_t)off * 400 * esz,
                        fp64, c->stream);
    *launches += 5;
  }
  cudaError_t e2 = cudaFreeAsync(buf, c->stream);
  return e != cudaSuccess ? e : e2;
}

cudaError_t autotune(qflow_ctx* c) {
  const TuneKey key{c->n, c->nocc, c->cls_count[1], c->cls_count[2], c->cls_count[3]};
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      c->sched_persistent = it->second[0];
      c->sched_chunk = it->second[1];
      c->sched_warps = it->second[2];
      if (c->opt.ladder_bn == 0 && c->opt.form == QFLOW_FORM_SESCC) c->ladder_bn = it->second[3];
      c->tuned = true;
      return cudaSuccess;
    }
  }
  // candidates: (persistent, items per fetch, warps per CTA).  Only the persistent queue: the
  // per-class grid-stride launch, which can tie on a calibration prefix, loses its L2 locality
  // over a whole list (n82: 90 ms against 76 ms).  Fewer warps per CTA leave more of the SM's
  // 256 KB to the L1 cache (the coupling tables and the gathered blocks) at the cost of latency
  // hiding.  A fixed warps option (qflow_options.warps) keeps only its own candidates.
  constexpr int kCand = 8;
  const int cand[kCand][3] = {{1, 1, 15}, {1, 2, 15}, {1, 4, 15}, {1, 8, 15},
                              {1, 1, 12}, {1, 2, 12}, {1, 4, 12}, {1, 8, 12}};
  static_assert(kCand <= QFLOW_TUNE_MAX, "candidate times");
  // calibration prefix of every class: large enough that the warps' drift through the list
  // (which decides L2 reuse of the W blocks) shows, small next to a full solve
  const int64_t count = 262144;
  cudaEvent_t t0, t1;
  cudaError_t e = cudaEventCreate(&t0);
  if (e == cudaSuccess) e = cudaEventCreate(&t1);
  float best = 1e30f;
  int bi = 0;
  int64_t dummy = 0;
  for (int ci = 0; ci < kCand && e == cudaSuccess; ++ci) {
    float ms = 0.f;
    c->tune_ms[ci] = 0.f;
    if (c->opt.warps > 0 && cand[ci][2] != c->opt.warps) continue;
    if (c->opt.chunk > 0 && cand[ci][1] != c->opt.chunk) continue;
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {  // the first run warms up
      e = cudaEventRecord(t0, c->stream);
      if (e == cudaSuccess) e = enqueue_solve(c, cand[ci][0], cand[ci][1], cand[ci][2], count, &dummy);
      if (e == cudaSuccess) e = cudaEventRecord(t1, c->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(t1);
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
    }
    c->tune_ms[ci] = ms;
    if (ms > 0.f && ms < best) {
      best = ms;
      bi = ci;
    }
  }
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  if (e != cudaSuccess) return e;
  // the dressing's ladder + oooo tile width, on the workspace of this sweep's dressing (which
  // has run: the tuner only overwrites its scratch)
  if (c->opt.ladder_bn == 0 && c->opt.form == QFLOW_FORM_SESCC && c->W32) {
    int bn = 0;
    e = qf::tune_ladder(c->n, c->nocc, c->W32, c->dwork, c->dwork_bytes, c->stream, &bn, c->ladder_ms);
    if (e != cudaSuccess) return e;
    c->ladder_bn = bn;
    c->ladder_count = QFLOW_LADDER_TUNE_MAX;
  }
  c->tune_count = kCand;
  c->sched_persistent = cand[bi][0];
  c->sched_chunk = (c->opt.chunk > 0) ? c->opt.chunk : cand[bi][1];
  c->sched_warps = (c->opt.warps > 0) ? c->opt.warps : cand[bi][2];
  c->tuned = true;
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune_cache[key] = {c->sched_persistent, c->sched_chunk, c->sched_warps, c->ladder_bn};
  return cudaSuccess;
}

// A warm-start sweep: the network's guesses for the 6e6o spaces (outside any captured graph).
bool warm_sweep(const qflow_ctx* c) {
  return c->opt.guess == QFLOW_GUESS_NETWORK && c->mlp_pending && c->cls_count[3] > 0;
}

// Dressing, network guesses of a warm-start sweep, and the schedule calibration: the mixed
// schedule is calibrated at the second sweep, whose work mix (most spaces near their root) is
// that of the rest of a flow; the first sweep runs the default.
cudaError_t enqueue_front(qflow_ctx* c, bool warm, int64_t* launches) {
  cudaError_t e = enqueue_dress(c, launches);
  if (e == cudaSuccess && warm) {
    e = enqueue_mlp_guess(c, launches);
    c->mlp_guess_now = true;
  }
  const bool mixed = c->opt.precision == QFLOW_PREC_MIXED;
  if (e == cudaSuccess && !c->tuned && mixed && c->sweeps >= 1) e = autotune(c);
  if (!mixed) c->tuned = true;  // FP64 runs per-class launches and needs no tuning
  return e;
}

// Host side of a finished sweep (stream synchronised): energy change, scalars, status.
int finish_sweep(qflow_ctx* c, bool warm, int64_t launches, double* d_e, double* max_dt, int32_t* nfailed) {
  if (warm) c->mlp_pending = false;
  c->fw_of_last_sweep = true;
  ++c->sweeps;
  c->last_launches = launches;
  const double em = c->red_host[0];
  const double de = c->have_energy ? em - c->e_mean : std::numeric_limits<double>::infinity();
  c->e_mean = em;
  c->have_energy = true;
  if (d_e) *d_e = de;
  if (max_dt) *max_dt = c->red_host[1];
  const int32_t nf = (int32_t)c->red_host[2];
  if (nfailed) *nfailed = nf;
  if (!isfinite(em) || !isfinite(c->red_host[1])) return QFLOW_ERR_NONFINITE;
  if (nf > 0) {
    const int worst = (int)c->red_host[3];
    if (worst == qf::kSpaceNonFinite) return QFLOW_ERR_NONFINITE;
    if (worst == qf::kSpaceRoot) return QFLOW_ERR_ROOT;
    return QFLOW_ERR_NOCONV;
  }
  return QFLOW_OK;
}

}  // namespace

extern "C" {

int qflow_sweep(qflow_handle c, double* d_e, double* max_dt, int32_t* nfailed) {
  if (!c) return QFLOW_ERR_ARG;
  if (c->shard_n > 1 || c->shard_open) return QFLOW_ERR_STATE;  // sharded: begin / exchange / end
  int64_t launches = 0;
  cudaError_t e = cudaSuccess;
  // a warm-start sweep (network guesses for the 6e6o spaces) runs outside the captured graph
  const bool warm = warm_sweep(c);
  if (c->opt.graph && !c->graph_exec && c->tuned && !warm) {
    // From the second sweep on: capture the sweep's device work once, then replay it.
    int64_t l2 = 0;
    e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t e1 = enqueue_dress(c, &l2);
      if (e1 == cudaSuccess) e1 = enqueue_solve_merge(c, &l2);
      e = cudaStreamEndCapture(c->stream, &c->graph);
      if (e == cudaSuccess) e = e1;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&c->graph_exec, c->graph, 0);
    if (e == cudaSuccess) {
      c->graph_launches = l2;
    } else {  // fall back to plain launches
      if (c->graph) cudaGraphDestroy(c->graph);
      c->graph = nullptr;
      c->graph_exec = nullptr;
      c->opt.graph = 0;
      cudaGetLastError();
      e = cudaSuccess;
    }
  }
  if (c->graph_exec && !warm) {  // replay of the captured sweep
    e = cudaGraphLaunch(c->graph_exec, c->stream);
    launches = c->graph_launches;
  } else {
    e = enqueue_front(c, warm, &launches);
    if (e == cudaSuccess) e = enqueue_solve_merge(c, &launches);
    c->mlp_guess_now = false;
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_status(e);
  return finish_sweep(c, warm, launches, d_e, max_dt, nfailed);
}

int qflow_set_shard(qflow_handle c, int32_t rank, int32_t nranks) {
  if (!c || nranks < 1 || rank < 0 || rank >= nranks) return QFLOW_ERR_ARG;
  if (c->shard_open) return QFLOW_ERR_STATE;
  if (c->space_mask) cudaFree(c->space_mask);
  if (c->pool_mask) cudaFree(c->pool_mask);
  c->space_mask = c->pool_mask = nullptr;
  c->shard_rank = rank;
  c->shard_n = nranks;
  shard_ranges(c->cls_count, rank, nranks, c->shard_lo, c->shard_hi);
  // a captured sweep covers the whole list; sharded sweeps run plain launches
  if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
  if (c->graph) cudaGraphDestroy(c->graph);
  c->graph_exec = nullptr;
  c->graph = nullptr;
  const int64_t ns = c->nspaces, npool = c->n_t1 + c->n_t2;
  std::vector<int64_t> gidx((size_t)ns);
  std::vector<int32_t> own((size_t)npool);
  std::vector<uint8_t> smask((size_t)ns), pmask((size_t)npool);
  cudaError_t e = cudaSuccess;
  if (ns > 0)
    e = cudaMemcpyAsync(gidx.data(), c->sorted_index, sizeof(int64_t) * (size_t)ns, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(own.data(), c->own1, sizeof(int32_t) * (size_t)c->n_t1, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(own.data() + c->n_t1, c->own2, sizeof(int32_t) * (size_t)c->n_t2, cudaMemcpyDeviceToHost,
                        c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_status(e);
  shard_masks(gidx, c->cls_count, c->cls_off, own.data(), c->n_t1, own.data() + c->n_t1, c->n_t2, rank, nranks,
              smask.data(), pmask.data());
  e = dalloc(&c->space_mask, (size_t)std::max<int64_t>(ns, 1));
  if (e == cudaSuccess) e = dalloc(&c->pool_mask, (size_t)npool);
  if (e == cudaSuccess && ns > 0)
    e = cudaMemcpyAsync(c->space_mask, smask.data(), (size_t)ns, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->pool_mask, pmask.data(), (size_t)npool, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  return cuda_status(e);
}

int qflow_sweep_waves(qflow_handle c, int64_t wave, double* d_e, double* max_dt, int32_t* nfailed) {
  if (!c || wave < 1) return QFLOW_ERR_ARG;
  if (c->shard_n > 1 || c->shard_open) return QFLOW_ERR_STATE;
  // the DUCC form reads every internal amplitude of a space, which other spaces of the same wave
  // update in place: waves run in the SES-CC form only
  if (c->opt.form == QFLOW_FORM_DUCC) return QFLOW_ERR_STATE;
  if (wave >= c->nspaces) return qflow_sweep(c, d_e, max_dt, nfailed);  // one wave: Jacobi
  const int64_t ns = c->nspaces;
  const size_t npool = (size_t)(c->n_t1 + c->n_t2);
  cudaError_t e = cudaSuccess;
  if (!c->wave_items) {  // per class, positions in Delta-eps order
    std::vector<int64_t> gidx((size_t)ns), items((size_t)ns);
    e = cudaMemcpyAsync(gidx.data(), c->sorted_index, sizeof(int64_t) * (size_t)ns, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_status(e);
    for (int k = 1; k <= 3; ++k) {
      const int64_t b = c->cls_off[k], n = c->cls_count[k];
      std::vector<int64_t> ord((size_t)n);
      std::iota(ord.begin(), ord.end(), (int64_t)0);
      std::sort(ord.begin(), ord.end(), [&](int64_t x, int64_t y) { return gidx[(size_t)(b + x)] < gidx[(size_t)(b + y)]; });
      c->wave_sidx[k].resize((size_t)n);
      for (int64_t t = 0; t < n; ++t) {
        items[(size_t)(b + t)] = ord[(size_t)t];
        c->wave_sidx[k][(size_t)t] = gidx[(size_t)(b + ord[(size_t)t])];
      }
    }
    e = dalloc(&c->wave_items, (size_t)std::max<int64_t>(ns, 1));
    if (e == cudaSuccess) e = dalloc(&c->pool_start, npool);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(c->wave_items, items.data(), sizeof(int64_t) * (size_t)ns, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_status(e);
  }
  int64_t launches = 0;
  e = cudaMemcpyAsync(c->pool_start, c->pool, sizeof(double) * npool, cudaMemcpyDeviceToDevice, c->stream);
  if (e == cudaSuccess) e = mark(c, 0);
  for (int64_t lo = 0; lo < ns && e == cudaSuccess; lo += wave) {
    const int64_t hi = std::min<int64_t>(ns, lo + wave);
    // dressing of the pool the earlier waves left
    e = dress_pool(c, c->pool, c->pool + c->n_t1);
    launches += dress_pool_launches(c);
    if (e == cudaSuccess && c->W32) {
      const size_t n4 = (size_t)c->n * c->n * c->n * c->n;
      e = qf::launch_to_f32(c->W, c->W32, n4, c->stream);
      if (e == cudaSuccess) e = qf::launch_to_f32(c->F, c->W32 + n4, (size_t)c->n * c->n, c->stream);
      launches += 2;
    }
    if (e == cudaSuccess && lo == 0) e = mark(c, 1);
    // this wave's spaces of every class; owned amplitudes are updated in place (each has one
    // owner, whose warp reads the old value and writes the new one)
    SolveArgs cls[4];
    for (int k = 1; k <= 3; ++k) {
      cls[k] = solve_args(c, k);
      const std::vector<int64_t>& v = c->wave_sidx[k];
      const int64_t a0 = std::lower_bound(v.begin(), v.end(), lo) - v.begin();
      const int64_t a1 = std::lower_bound(v.begin(), v.end(), hi) - v.begin();
      cls[k].items = c->wave_items + c->cls_off[k] + a0;
      cls[k].nspaces = a1 - a0;
      cls[k].t1_new = c->pool;
      cls[k].t2_new = c->pool + c->n_t1;
    }
    if (e == cudaSuccess)
      e = enqueue_solve_cls(c, cls, c->sched_persistent, c->sched_chunk, c->sched_warps, &launches, false);
  }
  if (e == cudaSuccess) e = mark(c, 2);
  if (e == cudaSuccess && c->diis) {
    e = qf::launch_diis(c->diis, c->opt.diis, c->pool_start, c->pool, (int64_t)npool, c->stream);
    launches += 4;
  }
  if (e == cudaSuccess)
    e = qf::launch_reduce(c->energy, c->status, ns, c->pool_start, c->pool, (int64_t)npool, c->red, c->rwork,
                          c->stream);
  launches += 2;
  if (e == cudaSuccess) e = mark(c, 3);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->red_host, c->red, 4 * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_status(e);
  if (c->opt.precision != QFLOW_PREC_MIXED) c->tuned = true;
  return finish_sweep(c, false, launches, d_e, max_dt, nfailed);
}

int64_t qflow_exchange_size(qflow_handle c) {
  return c ? c->n_t1 + c->n_t2 + 2 * c->nspaces : 0;
}

int qflow_sweep_shard_begin(qflow_handle c, double* exchange) {
  if (!c || !exchange) return QFLOW_ERR_ARG;
  if (c->shard_open || !c->space_mask) return QFLOW_ERR_STATE;
  int64_t launches = 0;
  const bool warm = warm_sweep(c);
  cudaError_t e = enqueue_front(c, warm, &launches);
  if (e == cudaSuccess) e = enqueue_solve_phase(c, &launches);
  c->mlp_guess_now = false;
  if (e == cudaSuccess) e = mark(c, 2);
  if (e == cudaSuccess)
    e = qf::launch_exchange_pack(c->pool_new, c->pool_mask, c->n_t1 + c->n_t2, c->energy, c->status, c->iters,
                                 c->space_mask, c->nspaces, exchange, c->stream);
  ++launches;
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_status(e);
  c->shard_open = true;
  c->shard_warm = warm;
  c->last_launches = launches;
  return QFLOW_OK;
}

int qflow_sweep_shard_end(qflow_handle c, const double* exchange, double* d_e, double* max_dt, int32_t* nfailed) {
  if (!c || !exchange) return QFLOW_ERR_ARG;
  if (!c->shard_open) return QFLOW_ERR_STATE;
  c->shard_open = false;
  int64_t launches = c->last_launches;
  cudaError_t e = qf::launch_exchange_unpack(exchange, c->own1, c->n_t1, c->own2, c->n_t2, c->pool_new, c->energy,
                                             c->status, c->iters, c->nspaces, c->stream);
  ++launches;
  if (e == cudaSuccess) e = enqueue_merge_phase(c, false, &launches);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_status(e);
  return finish_sweep(c, c->shard_warm, launches, d_e, max_dt, nfailed);
}

int qflow_energy(qflow_handle c, double* e_mean, double* e_per_space) {
  if (!c) return QFLOW_ERR_ARG;
  if (!c->have_energy) return QFLOW_ERR_STATE;
  if (e_mean) *e_mean = c->e_mean;
  if (e_per_space && c->nspaces > 0) {
    cudaError_t e = cudaMemcpyAsync(e_per_space, c->energy, sizeof(double) * (size_t)c->nspaces,
                                    cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    return cuda_status(e);
  }
  return QFLOW_OK;
}

int qflow_amplitudes(qflow_handle c, double* t1, double* t2) {
  if (!c) return QFLOW_ERR_ARG;
  cudaError_t e = cudaSuccess;
  if (t1) e = cudaMemcpyAsync(t1, c->pool, sizeof(double) * (size_t)c->n_t1, cudaMemcpyDeviceToHost, c->stream);
  if (t2 && e == cudaSuccess)
    e = cudaMemcpyAsync(t2, c->pool + c->n_t1, sizeof(double) * (size_t)c->n_t2, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  return cuda_status(e);
}

int qflow_set_amplitudes(qflow_handle c, const double* t1, const double* t2) {
  if (!c || !t1 || !t2) return QFLOW_ERR_ARG;
  if (c->shard_open) return QFLOW_ERR_STATE;
  cudaError_t e = cudaMemcpyAsync(c->pool, t1, sizeof(double) * (size_t)c->n_t1, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->pool + c->n_t1, t2, sizeof(double) * (size_t)c->n_t2, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess && c->diis) e = qf::diis_reset(c->diis, c->opt.diis, c->n_t1 + c->n_t2, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  return cuda_status(e);
}

int qflow_space_order(qflow_handle c, int64_t* perm) {
  if (!c || !perm) return QFLOW_ERR_ARG;
  memcpy(perm, c->perm.data(), sizeof(int64_t) * c->perm.size());
  return QFLOW_OK;
}

int qflow_space_stats(qflow_handle c, int32_t* iterations, int32_t* status) {
  if (!c) return QFLOW_ERR_ARG;
  if (!c->have_energy) return QFLOW_ERR_STATE;
  cudaError_t e = cudaSuccess;
  if (iterations && c->nspaces > 0)
    e = cudaMemcpyAsync(iterations, c->iters, sizeof(int32_t) * (size_t)c->nspaces, cudaMemcpyDeviceToHost, c->stream);
  if (status && c->nspaces > 0 && e == cudaSuccess)
    e = cudaMemcpyAsync(status, c->status, sizeof(int32_t) * (size_t)c->nspaces, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  return cuda_status(e);
}

int qflow_dressed(qflow_handle c, double* e0, double* F, double* W) {
  if (!c) return QFLOW_ERR_ARG;
  if (c->shard_open) return QFLOW_ERR_STATE;
  const size_t n1 = c->n, n4 = n1 * n1 * n1 * n1;
  cudaError_t e = dress_pool(c, c->pool, c->pool + c->n_t1);
  c->fw_of_last_sweep = false;
  if (e0 && e == cudaSuccess) e = cudaMemcpyAsync(e0, c->e0, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  if (F && e == cudaSuccess) e = cudaMemcpyAsync(F, c->F, sizeof(double) * n1 * n1, cudaMemcpyDeviceToHost, c->stream);
  if (W && e == cudaSuccess) e = cudaMemcpyAsync(W, c->W, sizeof(double) * n4, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  return cuda_status(e);
}

void* qflow_stream(qflow_handle c) { return c ? (void*)c->stream : nullptr; }

int qflow_schedule(qflow_handle c, int32_t* persistent, int32_t* chunk, int32_t* warps_per_cta, int32_t* graph,
                   float* candidate_ms, int32_t* n_candidates) {
  if (!c) return QFLOW_ERR_ARG;
  if (persistent) *persistent = c->sched_persistent;
  if (chunk) *chunk = c->sched_chunk;
  if (warps_per_cta) *warps_per_cta = c->sched_warps;
  if (graph) *graph = c->graph_exec ? 1 : 0;
  if (candidate_ms)
    for (int i = 0; i < c->tune_count; ++i) candidate_ms[i] = c->tune_ms[i];
  if (n_candidates) *n_candidates = c->tune_count;
  return QFLOW_OK;
}

int qflow_dress_schedule(qflow_handle c, int32_t* ladder_bn, float* candidate_ms, int32_t* n_candidates) {
  if (!c) return QFLOW_ERR_ARG;
  if (ladder_bn) *ladder_bn = c->ladder_bn > 0 ? c->ladder_bn : 64;
  if (candidate_ms)
    for (int i = 0; i < c->ladder_count; ++i) candidate_ms[i] = c->ladder_ms[i];
  if (n_candidates) *n_candidates = c->ladder_count;
  return QFLOW_OK;
}

int qflow_last_sweep_info(qflow_handle c, double* phase_ms, int64_t* kernel_launches) {
  if (!c) return QFLOW_ERR_ARG;
  if (!c->have_energy) return QFLOW_ERR_STATE;
  if (phase_ms) {
    for (int k = 0; k < 3; ++k) {
      float ms = 0.f;
      cudaError_t e = cudaEventElapsedTime(&ms, c->ev[k], c->ev[k + 1]);
      if (e != cudaSuccess) return cuda_status(e);
      phase_ms[k] = ms;
    }
  }
  if (kernel_launches) *kernel_launches = c->last_launches;
  return QFLOW_OK;
}

void qflow_destroy(qflow_handle c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  free_ctx(c);
}

const char* qflow_strerror(int code) {
  switch (code) {
    case QFLOW_OK: return "ok";
    case QFLOW_ERR_ARG: return "invalid argument";
    case QFLOW_ERR_CUDA: return "CUDA runtime error";
    case QFLOW_ERR_OOM: return "out of device memory";
    case QFLOW_ERR_NOCONV: return "Davidson solver did not converge for some space";
    case QFLOW_ERR_ROOT: return "no real Phi-dominant root for some space";
    case QFLOW_ERR_NONFINITE: return "non-finite energy or amplitude";
    case QFLOW_ERR_STATE: return "call out of order";
    case QFLOW_WARN_UNCOVERED: return "some amplitudes have no owner space";
    case QFLOW_ERR_TOO_LARGE: return "problem exceeds the static scratch of the allocation-free entry point";
    default: return "unknown qflow status";
  }
}

size_t qflow_dress_workspace(int32_t n, int32_t nocc) {
  if (n < 2 || n > 128 || nocc < 1 || nocc >= n) return 0;
  return qf::dress_workspace_bytes(n, nocc);
}

int qflow_dress_device(const double* h, const double* eri, const double* t1, const double* t2, int32_t n,
                       int32_t nocc, double* e0, double* F, double* W, void* work, size_t work_bytes, void* stream) {
  if (!h || !eri || !t1 || !t2 || !e0 || !F || !W || !work || n < 2 || n > 128 || nocc < 1 || nocc >= n)
    return QFLOW_ERR_ARG;
  if (work_bytes < qf::dress_workspace_bytes(n, nocc)) return QFLOW_ERR_ARG;
  return cuda_status(qf::launch_dress(h, eri, t1, t2, n, nocc, e0, F, W, work, work_bytes, (cudaStream_t)stream));
}

int qflow_solve_device(int32_t n, int32_t nocc, const double* e0, const double* F, const double* W,
                       int32_t size_class, const qflow_space* spaces, int64_t nspaces, int64_t space_base, const int32_t* owner1,
                       const int32_t* owner2, const double* t1_old, const double* t2_old, double* t1_new,
                       double* t2_new, double* energy, int32_t* status, int32_t* iters, void* guess,
                       int32_t save_root, int32_t precision, int32_t max_iter, double tol, void* stream) {
  if (n < 2 || n > 128 || nocc < 1 || nocc >= n || nspaces < 0 || !e0 || !F || !W || !energy || !status)
    return QFLOW_ERR_ARG;
  if (nspaces > 0 && !spaces) return QFLOW_ERR_ARG;
  if ((owner1 || owner2) && (!t1_old || !t2_old || !t1_new || !t2_new)) return QFLOW_ERR_ARG;
  if (precision != QFLOW_PREC_FP64 && precision != QFLOW_PREC_MIXED) return QFLOW_ERR_ARG;
  if (max_iter <= 0 || !(tol > 0.0)) return QFLOW_ERR_ARG;
  if (size_class < 1 || size_class > 3 || size_class > nocc || size_class > n - nocc) return QFLOW_ERR_ARG;
  if (nspaces == 0) return QFLOW_OK;
  SolveArgs a{};
  a.n = n;
  a.nocc = nocc;
  a.nvir = n - nocc;
  a.e0 = e0;
  a.F = F;
  a.W = W;
  a.spaces = spaces;
  a.nspaces = nspaces;
  a.space_base = space_base;
  a.sorted_index = nullptr;
  a.owner1 = owner1;
  a.owner2 = owner2;
  a.t1_old = t1_old;
  a.t2_old = t2_old;
  a.t1_new = t1_new;
  a.t2_new = t2_new;
  a.energy = energy;
  a.status = status;
  a.iters = iters;
  a.guess = guess;
  a.root_out = save_root ? guess : nullptr;
  a.max_iter = max_iter;
  a.tol = tol;
  const cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = qf::launch_solve(size_class, precision, a, st);
  if (e != cudaSuccess || precision != QFLOW_PREC_MIXED || max_iter <= qf::kWarpIterCap) return cuda_status(e);
  // spaces the warp pass left unconverged: the FP64 solver, on stream-ordered scratch
  int64_t* items = nullptr;
  e = cudaMallocAsync(reinterpret_cast<void**>(&items), (size_t)nspaces * sizeof(int64_t) + 16, st);
  if (e != cudaSuccess) return cuda_status(e);
  e = qf::launch_solve_rescue(size_class, a, items, reinterpret_cast<unsigned long long*>(items + nspaces), st);
  const cudaError_t f = cudaFreeAsync(items, st);
  return cuda_status(e != cudaSuccess ? e : f);
}

}  // extern "C"

// ---- warm-start network ---------------------------------------------------------------------

namespace {

bool mlp_sizes_ok(int32_t I, int32_t H, int32_t O) {
  return I >= 1 && I <= 65536 && H >= 1 && H <= 4096 && O >= 1 && O <= 65536;
}

}  // namespace

extern "C" {

int64_t qflow_mlp_param_count(int32_t n_in, int32_t hidden, int32_t n_out) {
  if (!mlp_sizes_ok(n_in, hidden, n_out)) return 0;
  return qf::mlp_param_count(n_in, hidden, n_out);
}

int64_t qflow_mlp_model_size(int32_t hidden) {
  if (hidden < 1 || hidden > 1024) return 0;
  return qf::mlp_param_count(QFLOW_MLP_NIN, hidden, QFLOW_MLP_NOUT) + 2 * QFLOW_MLP_NIN + 2 * QFLOW_MLP_NOUT;
}

int qflow_mlp_set_model(qflow_handle c, int32_t hidden, const float* model, int32_t has_stats) {
  if (!c || !model || hidden < 1 || hidden > 1024) return QFLOW_ERR_ARG;
  const int64_t np = qf::mlp_param_count(QFLOW_MLP_NIN, hidden, QFLOW_MLP_NOUT);
  const int64_t total = qflow_mlp_model_size(hidden);
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_status(e);
  float* ptrs[4] = {c->mlp_model, c->mlp_grad, c->mlp_m, c->mlp_v};
  for (float* p : ptrs)
    if (p) cudaFree(p);
  c->mlp_model = c->mlp_grad = c->mlp_m = c->mlp_v = nullptr;
  c->mlp_hidden = 0;
  e = dalloc(&c->mlp_model, (size_t)total);
  if (e == cudaSuccess) e = dalloc(&c->mlp_grad, (size_t)np);
  if (e == cudaSuccess) e = dalloc(&c->mlp_m, (size_t)np);
  if (e == cudaSuccess) e = dalloc(&c->mlp_v, (size_t)np);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->mlp_model, model, sizeof(float) * total, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->mlp_m, 0, sizeof(float) * np, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->mlp_v, 0, sizeof(float) * np, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_status(e);
  c->mlp_hidden = hidden;
  c->mlp_nparam = np;
  c->mlp_step = 0;
  c->mlp_has_stats = has_stats != 0;
  c->mlp_pending = c->mlp_has_stats;
  return QFLOW_OK;
}

int qflow_mlp_get_model(qflow_handle c, float* model) {
  if (!c || !model) return QFLOW_ERR_ARG;
  if (!c->mlp_model) return QFLOW_ERR_STATE;
  const int64_t total = qflow_mlp_model_size(c->mlp_hidden);
  cudaError_t e = cudaMemcpyAsync(model, c->mlp_model, sizeof(float) * total, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  return cuda_status(e);
}

int qflow_mlp_collect(qflow_handle c, int32_t target, int64_t stride, int64_t max_pairs, int64_t* n_pairs) {
  if (!c || stride < 1 || max_pairs < 1) return QFLOW_ERR_ARG;
  if (target != QFLOW_MLP_TARGET_INCREMENT && target != QFLOW_MLP_TARGET_POOL) return QFLOW_ERR_ARG;
  if (c->shard_open) return QFLOW_ERR_STATE;
  // increment pairs read the roots of every 6e6o space: a shard holds only its own
  if (target == QFLOW_MLP_TARGET_INCREMENT && (c->opt.guess != QFLOW_GUESS_NETWORK || !c->have_energy ||
                                               !c->fw_of_last_sweep || !c->guess[3] || c->shard_n > 1))
    return QFLOW_ERR_STATE;
  if (c->mlp_cap > 0 && c->mlp_target != target) return QFLOW_ERR_STATE;  // one kind of pair per set
  cudaError_t e = cudaSuccess;
  if (c->mlp_cap == 0) {
    e = dalloc(&c->mlp_X, (size_t)max_pairs * QFLOW_MLP_NIN);
    if (e == cudaSuccess) e = dalloc(&c->mlp_T, (size_t)max_pairs * QFLOW_MLP_NOUT);
    if (e == cudaSuccess) e = dalloc(&c->mlp_mask, (size_t)max_pairs);
    if (e != cudaSuccess) return cuda_status(e);
    c->mlp_cap = max_pairs;
    c->mlp_target = target;
  }
  const int64_t n3 = c->cls_count[3];
  int64_t rows = (n3 + stride - 1) / stride;
  if (rows > c->mlp_cap - c->mlp_n) rows = c->mlp_cap - c->mlp_n;
  if (rows > 0) {
    const bool fp64 = c->opt.precision != QFLOW_PREC_MIXED;
    float* X = c->mlp_X + (size_t)c->mlp_n * QFLOW_MLP_NIN;
    float* T = c->mlp_T + (size_t)c->mlp_n * QFLOW_MLP_NOUT;
    if (target == QFLOW_MLP_TARGET_POOL) {  // bare features, the pool's internal amplitudes
      e = dress_bare(c);
      if (e == cudaSuccess)
        e = qf::mlp_features(c->n, c->F, c->W, c->spaces + c->cls_off[3], rows, stride, nullptr, nullptr, X, c->stream);
      if (e == cudaSuccess)
        e = qf::mlp_pool_targets(c->pool, c->spaces + c->cls_off[3], rows, stride, c->nocc, c->nvir, T,
                                 c->mlp_mask + c->mlp_n, c->stream);
    } else {  // the last sweep's features, its roots' increments
      e = qf::mlp_features(c->n, c->F, c->W, c->spaces + c->cls_off[3], rows, stride, nullptr, nullptr, X, c->stream);
      if (e == cudaSuccess)
        e = qf::mlp_targets(c->guess[3], fp64, rows, stride, c->sorted_index + c->cls_off[3], c->status, T,
                            c->mlp_mask + c->mlp_n, c->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_status(e);
    c->mlp_n += rows;
  }
  if (n_pairs) *n_pairs = c->mlp_n;
  return QFLOW_OK;
}

int qflow_mlp_train(qflow_handle c, int32_t epochs, int32_t batch, float lr, const int64_t* order, float* loss) {
  if (!c || epochs < 0 || batch < 1 || !(lr > 0.f)) return QFLOW_ERR_ARG;
  if (!c->mlp_model || c->mlp_n == 0) return QFLOW_ERR_STATE;
  const int64_t n = c->mlp_n;
  if (order)
    for (int64_t i = 0; i < n; ++i)
      if (order[i] < 0 || order[i] >= n) return QFLOW_ERR_ARG;
  std::vector<uint8_t> mask((size_t)n);
  cudaError_t e = cudaMemcpyAsync(mask.data(), c->mlp_mask, (size_t)n, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_status(e);
  int64_t count = 0;
  for (uint8_t m : mask) count += m ? 1 : 0;
  if (count == 0) return QFLOW_ERR_STATE;
  const int I = QFLOW_MLP_NIN, O = QFLOW_MLP_NOUT, H = c->mlp_hidden;
  const int64_t B = batch < n ? batch : n;
  const int64_t nb = (n + B - 1) / B;
  // scratch: batch rows, masks, order, per-batch losses, inverse target scales, workspaces
  const size_t sz[7] = {(size_t)B * I * sizeof(float), (size_t)B * O * sizeof(float), (size_t)B,
                        (size_t)n * sizeof(int64_t), (size_t)(epochs > 0 ? epochs : 1) * nb * sizeof(float),
                        (size_t)O * sizeof(float),
                        std::max(qf::mlp_workspace_bytes(I, H, O, B), qf::mlp_stats_workspace_bytes(n, I))};
  size_t off[8] = {0};
  for (int i = 0; i < 7; ++i) off[i + 1] = off[i] + ((sz[i] + 255) / 256) * 256;
  char* buf = nullptr;
  e = cudaMalloc(reinterpret_cast<void**>(&buf), off[7]);
  if (e != cudaSuccess) return cuda_status(e);
  float* Xb = reinterpret_cast<float*>(buf + off[0]);
  float* Tb = reinterpret_cast<float*>(buf + off[1]);
  uint8_t* Mb = reinterpret_cast<uint8_t*>(buf + off[2]);
  int64_t* ord = reinterpret_cast<int64_t*>(buf + off[3]);
  float* lossd = reinterpret_cast<float*>(buf + off[4]);
  float* inv_sd = reinterpret_cast<float*>(buf + off[5]);
  void* work = buf + off[6];
  std::vector<int64_t> ident;
  if (!order) {
    ident.resize((size_t)n);
    for (int64_t i = 0; i < n; ++i) ident[(size_t)i] = i;
  }
  e = cudaMemcpyAsync(ord, order ? order : ident.data(), sizeof(int64_t) * (size_t)n, cudaMemcpyHostToDevice,
                      c->stream);
  if (e == cudaSuccess && !c->mlp_has_stats) {
    e = qf::mlp_col_stats(c->mlp_X, n, I, c->mlp_mask, count, 1, mlp_stats(c, 0), mlp_stats(c, 1), work, c->stream);
    if (e == cudaSuccess)
      e = qf::mlp_col_stats(c->mlp_T, n, O, c->mlp_mask, count, 0, mlp_stats(c, 2), mlp_stats(c, 3), work, c->stream);
  }
  if (e == cudaSuccess) e = qf::mlp_invert(mlp_stats(c, 3), O, inv_sd, c->stream);
  for (int ep = 0; ep < epochs && e == cudaSuccess; ++ep) {
    for (int64_t b = 0; b < nb && e == cudaSuccess; ++b) {
      const int64_t r = (n - b * B < B) ? n - b * B : B;
      e = qf::mlp_rows(c->mlp_X, r, I, ord + b * B, mlp_stats(c, 0), mlp_stats(c, 1), Xb, c->mlp_mask, Mb, c->stream);
      if (e == cudaSuccess)
        e = qf::mlp_rows(c->mlp_T, r, O, ord + b * B, mlp_stats(c, 2), inv_sd, Tb, nullptr, nullptr, c->stream);
      if (e == cudaSuccess)
        e = qf::mlp_loss_grad(I, H, O, c->mlp_model, Xb, Tb, Mb, r, c->mlp_grad, lossd + (size_t)ep * nb + b, work,
                              c->stream);
      if (e == cudaSuccess)
        e = qf::mlp_adam(c->mlp_nparam, c->mlp_model, c->mlp_grad, c->mlp_m, c->mlp_v, ++c->mlp_step, lr, 0.9f,
                         0.999f, 1e-8f, c->stream);
    }
  }
  std::vector<float> lh((size_t)(epochs > 0 ? epochs : 0) * nb);
  if (e == cudaSuccess && !lh.empty())
    e = cudaMemcpyAsync(lh.data(), lossd, sizeof(float) * lh.size(), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  cudaFree(buf);
  if (e != cudaSuccess) return cuda_status(e);
  c->mlp_has_stats = true;
  c->mlp_pending = c->mlp_target == QFLOW_MLP_TARGET_INCREMENT;  // a guess model: next sweep uses it
  if (loss)
    for (int ep = 0; ep < epochs; ++ep) {
      double s = 0.0;
      for (int64_t b = 0; b < nb; ++b) s += lh[(size_t)ep * nb + b];
      loss[ep] = (float)(s / (double)nb);
    }
  return QFLOW_OK;
}

int qflow_mlp_warm_pool(qflow_handle c) {
  if (!c) return QFLOW_ERR_ARG;
  if (!c->mlp_model || !c->mlp_has_stats || c->shard_open) return QFLOW_ERR_STATE;
  const int64_t n3 = c->cls_count[3];
  const int64_t CH = 131072;
  const int H = c->mlp_hidden;
  cudaError_t e = dress_bare(c);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(c->pool, 0, sizeof(double) * (size_t)(c->n_t1 + c->n_t2), c->stream);
  // only the 6e6o spaces that own an amplitude reach the pool: infer on those alone
  char* own = nullptr;
  const size_t o_flag = 0, o_sp = (((size_t)c->nspaces + 255) / 256) * 256,
               o_idx = o_sp + (((size_t)n3 * sizeof(qflow_space) + 255) / 256) * 256,
               o_cnt = o_idx + (((size_t)n3 * sizeof(int64_t) + 255) / 256) * 256;
  if (e == cudaSuccess && n3 > 0) e = cudaMalloc(reinterpret_cast<void**>(&own), o_cnt + 256);
  int64_t nown = 0;
  if (e == cudaSuccess && n3 > 0) {
    unsigned long long cnt = 0;
    e = qf::mlp_owner_spaces(c->own1, c->n_t1, c->own2, c->n_t2, c->nspaces, c->spaces + c->cls_off[3],
                             c->sorted_index + c->cls_off[3], n3, reinterpret_cast<uint8_t*>(own + o_flag),
                             reinterpret_cast<qflow_space*>(own + o_sp), reinterpret_cast<int64_t*>(own + o_idx),
                             reinterpret_cast<unsigned long long*>(own + o_cnt), c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&cnt, own + o_cnt, sizeof(cnt), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    nown = (int64_t)cnt;
  }
  const qflow_space* osp = reinterpret_cast<const qflow_space*>(own + o_sp);
  const int64_t* oidx = reinterpret_cast<const int64_t*>(own + o_idx);
  const int64_t rows = nown < CH ? nown : CH;
  char* buf = nullptr;
  const size_t fx = ((size_t)rows * QFLOW_MLP_NIN * sizeof(float) + 255) / 256 * 256;
  const size_t fy = ((size_t)rows * QFLOW_MLP_NOUT * sizeof(float) + 255) / 256 * 256;
  if (e == cudaSuccess && rows > 0)
    e = cudaMalloc(reinterpret_cast<void**>(&buf), fx + fy + qf::mlp_workspace_bytes(QFLOW_MLP_NIN, H, QFLOW_MLP_NOUT, rows));
  for (int64_t off = 0; off < nown && e == cudaSuccess; off += CH) {
    const int64_t r = (nown - off < CH) ? nown - off : CH;
    float* X = reinterpret_cast<float*>(buf);
    float* Y = reinterpret_cast<float*>(buf + fx);
    e = qf::mlp_features(c->n, c->F, c->W, osp + off, r, 1, mlp_stats(c, 0), mlp_stats(c, 1), X, c->stream);
    if (e == cudaSuccess)
      e = qf::mlp_forward(QFLOW_MLP_NIN, H, QFLOW_MLP_NOUT, c->mlp_model, X, r, Y, buf + fx + fy, c->stream);
    if (e == cudaSuccess)
      e = qf::mlp_pool_from_pred(Y, mlp_stats(c, 2), mlp_stats(c, 3), osp + off, oidx + off, r, c->nocc, c->nvir,
                                 c->own1, c->own2, c->pool, c->stream);
  }
  if (e == cudaSuccess && c->diis) e = qf::diis_reset(c->diis, c->opt.diis, c->n_t1 + c->n_t2, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (buf) cudaFree(buf);
  if (own) cudaFree(own);
  return cuda_status(e);
}

size_t qflow_mlp_workspace(int32_t n_in, int32_t hidden, int32_t n_out, int64_t rows) {
  if (!mlp_sizes_ok(n_in, hidden, n_out) || rows < 0) return 0;
  return qf::mlp_workspace_bytes(n_in, hidden, n_out, rows);
}

int qflow_mlp_forward_device(int32_t n_in, int32_t hidden, int32_t n_out, const float* params, const float* x,
                             int64_t rows, float* y, void* work, void* stream) {
  if (!mlp_sizes_ok(n_in, hidden, n_out) || rows < 0 || rows > (1 << 30)) return QFLOW_ERR_ARG;
  if (rows == 0) return QFLOW_OK;
  if (!params || !x || !y || !work) return QFLOW_ERR_ARG;
  return cuda_status(qf::mlp_forward(n_in, hidden, n_out, params, x, rows, y, work, (cudaStream_t)stream));
}

int qflow_mlp_grad_device(int32_t n_in, int32_t hidden, int32_t n_out, const float* params, const float* x,
                          const float* target, const uint8_t* mask, int64_t rows, float* grad, float* loss,
                          void* work, void* stream) {
  if (!mlp_sizes_ok(n_in, hidden, n_out) || rows < 1 || rows > (1 << 30)) return QFLOW_ERR_ARG;
  if (!params || !x || !target || !grad || !loss || !work) return QFLOW_ERR_ARG;
  return cuda_status(qf::mlp_loss_grad(n_in, hidden, n_out, params, x, target, mask, rows, grad, loss, work,
                                       (cudaStream_t)stream));
}

int qflow_mlp_adam_device(int64_t n, float* params, const float* grad, float* m, float* v, int32_t step, float lr,
                          float beta1, float beta2, float eps, void* stream) {
  if (n < 0 || step < 1 || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f)) return QFLOW_ERR_ARG;
  if (n == 0) return QFLOW_OK;
  if (!params || !grad || !m || !v) return QFLOW_ERR_ARG;
  return cuda_status(qf::mlp_adam(n, params, grad, m, v, step, lr, beta1, beta2, eps, (cudaStream_t)stream));
}

int qflow_mlp_features_device(int32_t n, const double* F, const double* W, const qflow_space* spaces,
                              int64_t nspaces, float* features, void* stream) {
  if (n < 6 || n > 128 || nspaces < 0) return QFLOW_ERR_ARG;
  if (nspaces == 0) return QFLOW_OK;
  if (!F || !W || !spaces || !features) return QFLOW_ERR_ARG;
  return cuda_status(
      qf::mlp_features(n, F, W, spaces, nspaces, 1, nullptr, nullptr, features, (cudaStream_t)stream));
}

int qflow_mlp_targets_device(const float* roots, int64_t rows, float* targets, void* stream) {
  if (rows < 0) return QFLOW_ERR_ARG;
  if (rows == 0) return QFLOW_OK;
  if (!roots || !targets) return QFLOW_ERR_ARG;
  return cuda_status(qf::mlp_targets(roots, false, rows, 1, nullptr, nullptr, targets, nullptr, (cudaStream_t)stream));
}

int qflow_mlp_guess_device(const float* y, int64_t rows, float* guess, void* stream) {
  if (rows < 0) return QFLOW_ERR_ARG;
  if (rows == 0) return QFLOW_OK;
  if (!y || !guess) return QFLOW_ERR_ARG;
  return cuda_status(qf::mlp_guess(y, rows, nullptr, nullptr, guess, false, (cudaStream_t)stream));
}

}  // extern "C"
