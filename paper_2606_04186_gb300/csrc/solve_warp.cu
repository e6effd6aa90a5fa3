// Mixed-precision batched solver for 6e6o spaces (3 occupied + 3 virtual orbitals, 400
// Sz = 0 determinants): one warp per space, sigma-vectors in FP32 from register tiles.
//
// What it computes is the same as solve.cu (gather + fold, Phi-dominant right eigenpair of the
// space's determinant operator by Davidson, CI -> CC increment, owner-filtered merge), see that
// file for the paper passages.  Differences are in the mapping onto the GB300:
//   * one warp owns one space (no block-wide barriers; all reductions are warp shuffles);
//   * sigma: lane L < 20 owns alpha string I_alpha = L and the 20 determinants of that row.
//     For each of the 12 single replacements (pq, J_alpha, s) into I_alpha it holds the W row
//     W[pq][*] (36 values) and the CI row C[J_alpha][*] (20 values) in registers and applies the
//     whole beta-side replacement table, which is a compile-time constant (same for every
//     space), as 240 register-only FMAs; the same-spin parts are two 20 x 20 x 20 products
//     from vectorised shared-memory rows;
//   * the operator diagonal is built in FP64 relative to E_Phi = <Phi|H|Phi> and removed from
//     the sigma operands, so FP32 sums only off-diagonal couplings;
//   * FP64 is kept for the fold, the diagonal, the projected k x k eigenproblem, the energy and
//     the amplitude update; FP32 for the 400-length vectors and sigma.
// Every loop is bounded; a warp never waits on another warp.
#include <cuda_runtime.h>
#include <math.h>
#include <stddef.h>
#include <stdint.h>

#include <utility>

#include "qflow_internal.h"

namespace qf {
namespace {

constexpr int NS = 20, NSG = 12, NDET = 400, NORB = 6, NF = 36, NW = 1296;
constexpr int KM = 4;        // Davidson subspace limit (restart on the Ritz vector)
constexpr int WARPS = 4;     // spaces (warps) per CTA
constexpr int NPAIR = NF * (NF + 1) / 2;  // unique (pq, rs) pairs of the pair-symmetric W block

struct Tab {
  int mask[NS];
  int idx[64];
  int J[NS][NSG];    // single replacements into string I: <I| a+_p a_q |J> = sg
  int pq[NS][NSG];
  int sg[NS][NSG];
};

__host__ __device__ constexpr int popc6(int m) {
  int c = 0;
  for (int b = 0; b < 6; ++b) c += (m >> b) & 1;
  return c;
}

__host__ __device__ constexpr Tab make_tab() {
  Tab t{};
  int c = 0;
  for (int m = 0; m < 64; ++m) {
    t.idx[m] = -1;
    if (popc6(m) == 3) {
      t.idx[m] = c;
      t.mask[c] = m;
      ++c;
    }
  }
  for (int I = 0; I < NS; ++I) {
    const int mi = t.mask[I];
    int u = 0;
    for (int p = 0; p < NORB; ++p) {
      if (!((mi >> p) & 1)) continue;
      for (int q = 0; q < NORB; ++q) {
        if (q != p && ((mi >> q) & 1)) continue;
        const int mj = (mi & ~(1 << p)) | (1 << q);
        int s = 1;
        if (p != q) {
          int par = popc6(mj & ((1 << q) - 1)) & 1;
          const int m1 = mj & ~(1 << q);
          par ^= popc6(m1 & ((1 << p) - 1)) & 1;
          s = par ? -1 : 1;
        }
        t.J[I][u] = t.idx[mj];
        t.pq[I][u] = p * NORB + q;
        t.sg[I][u] = s;
        ++u;
      }
    }
  }
  return t;
}

// Compile-time copy of the tables: used only in constant expressions (template arguments), so
// the beta-side replacement pattern becomes immediate register operands in sigma.
struct TabHolder {
  static constexpr Tab value = make_tab();
};

template <int B, int V>
__device__ __forceinline__ void ab_term(float (&acc)[NS], const float (&wr)[NF], const float (&cr)[NS]) {
  constexpr int pq = TabHolder::value.pq[B][V];
  constexpr int J = TabHolder::value.J[B][V];
  constexpr int sg = TabHolder::value.sg[B][V];
  if constexpr (sg > 0) acc[B] = fmaf(wr[pq], cr[J], acc[B]);
  else acc[B] = fmaf(-wr[pq], cr[J], acc[B]);
}

template <int... I>
__device__ __forceinline__ void ab_terms(std::integer_sequence<int, I...>, float (&acc)[NS], const float (&wr)[NF],
                                         const float (&cr)[NS]) {
  (ab_term<I / NSG, I % NSG>(acc, wr, cr), ...);
}

struct alignas(16) WarpSmem {  // 16-byte rows: sigma reads them as float4
  float V[KM * NDET];
  float S[KM * NDET];
  float Wt[NW];        // FP32 W block without its [pp][rr] (diagonal-only) entries
  float Hs[NS * NS];   // same-spin string operator, zero diagonal
  float diag[NDET];    // operator diagonal minus E_Phi
  float hp[NF];        // h' = h - 1/2 sum_r W_prrq (off-diagonal part used in FP32)
  double F[NF], J[NF], K[NF];  // F block; J_pr = W_pprr, K_pr = W_prrp (FP64)
  double hd[6];        // folded one-body diagonal h_pp (FP64)
  double hsd[NS];      // same-spin string diagonal (FP64)
  float dh[NS];        // hsd[I] - hsd[0] (FP64 difference, rounded); Hs[I][0] on the Phi path
  float jb[6 * NS];    // jb[p][Ib] = sum_{r in Ib} J_pr
  float G[KM * KM];    // projected matrix, G[i*KM+j] = V_i . S_j
  float yf[KM];        // Ritz coefficients
  float theta;         // Ritz value relative to eshift
  double ecore, eshift;
  int orb[6];
  int ctrl[4];  // [0] subspace size, [1] valid, [2] status, [3] iterations
};

struct alignas(16) CtaSmem {
  int J[NS * NSG];
  int pq[NS * NSG];
  int sg[NS * NSG];
  int mask[NS];
  unsigned short pair[NF * (NF + 1) / 2];  // (P, R) with P <= R, packed P | R << 8
  int c0n[NS];          // number of replacements (pq) with <I| E_pq |Phi string> != 0
  int c0pq[NS][3];      // their pq ...
  int c0sg[NS][3];      // ... and signs
  int xJ[9];            // a+_A a_i |Phi string> = xs * |xJ>, index i*3 + (A-3)
  int xs[9];
  WarpSmem w[WARPS];
};

static_assert(sizeof(WarpSmem) % 16 == 0, "per-warp state must keep 16-byte alignment");
static_assert(offsetof(WarpSmem, V) % 16 == 0 && offsetof(WarpSmem, S) % 16 == 0 && offsetof(WarpSmem, Wt) % 16 == 0 &&
                  offsetof(WarpSmem, Hs) % 16 == 0 && offsetof(WarpSmem, diag) % 16 == 0,
              "float4 rows");
static_assert(offsetof(CtaSmem, w) % 16 == 0, "warp state alignment");

__device__ __forceinline__ float wsum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// sigma = H c restricted to off-diagonal couplings plus the shifted diagonal.
__device__ __noinline__ void sigma_warp(const CtaSmem& cs, const WarpSmem& ws, const float* __restrict__ c,
                                        float* __restrict__ out, int lane) {
  if (lane < NS) {
    const int Ia = lane;
    float acc[NS];
    // diagonal and alpha-alpha: acc[b] = diag * c + sum_J Hs[Ia][J] c[J][b]
    {
      const float4* drow = reinterpret_cast<const float4*>(ws.diag + Ia * NS);
      const float4* crow = reinterpret_cast<const float4*>(c + Ia * NS);
#pragma unroll
      for (int q = 0; q < NS / 4; ++q) {
        const float4 dv = drow[q], cv = crow[q];
        acc[4 * q + 0] = dv.x * cv.x;
        acc[4 * q + 1] = dv.y * cv.y;
        acc[4 * q + 2] = dv.z * cv.z;
        acc[4 * q + 3] = dv.w * cv.w;
      }
    }
#pragma unroll 2
    for (int J = 0; J < NS; ++J) {
      const float hj = ws.Hs[Ia * NS + J];
      const float4* crow = reinterpret_cast<const float4*>(c + J * NS);
#pragma unroll
      for (int q = 0; q < NS / 4; ++q) {
        const float4 cv = crow[q];
        acc[4 * q + 0] = fmaf(hj, cv.x, acc[4 * q + 0]);
        acc[4 * q + 1] = fmaf(hj, cv.y, acc[4 * q + 1]);
        acc[4 * q + 2] = fmaf(hj, cv.z, acc[4 * q + 2]);
        acc[4 * q + 3] = fmaf(hj, cv.w, acc[4 * q + 3]);
      }
    }
    // beta-beta: acc[b] += sum_J Hs[b][J] c[Ia][J]
    {
      float ca[NS];
      const float4* crow = reinterpret_cast<const float4*>(c + Ia * NS);
#pragma unroll
      for (int q = 0; q < NS / 4; ++q) {
        const float4 cv = crow[q];
        ca[4 * q] = cv.x;
        ca[4 * q + 1] = cv.y;
        ca[4 * q + 2] = cv.z;
        ca[4 * q + 3] = cv.w;
      }
#pragma unroll 4
      for (int b = 0; b < NS; ++b) {
        const float4* hrow = reinterpret_cast<const float4*>(ws.Hs + b * NS);
        float s = 0.f;
#pragma unroll
        for (int q = 0; q < NS / 4; ++q) {
          const float4 hv = hrow[q];
          s = fmaf(hv.x, ca[4 * q], s);
          s = fmaf(hv.y, ca[4 * q + 1], s);
          s = fmaf(hv.z, ca[4 * q + 2], s);
          s = fmaf(hv.w, ca[4 * q + 3], s);
        }
        acc[b] += s;
      }
    }
    // alpha-beta: sum over the 12 replacements into Ia, register tiles of W and C rows
#pragma unroll 1
    for (int u = 0; u < NSG; ++u) {
      const int e = Ia * NSG + u;
      const int pq = cs.pq[e], Ja = cs.J[e];
      const float su = (float)cs.sg[e];
      float wr[NF], cr[NS];
      const float4* wrow = reinterpret_cast<const float4*>(ws.Wt + pq * NF);
#pragma unroll
      for (int q = 0; q < NF / 4; ++q) {
        const float4 v = wrow[q];
        wr[4 * q] = v.x;
        wr[4 * q + 1] = v.y;
        wr[4 * q + 2] = v.z;
        wr[4 * q + 3] = v.w;
      }
      const float4* crow = reinterpret_cast<const float4*>(c + Ja * NS);
#pragma unroll
      for (int q = 0; q < NS / 4; ++q) {
        const float4 v = crow[q];
        cr[4 * q] = su * v.x;
        cr[4 * q + 1] = su * v.y;
        cr[4 * q + 2] = su * v.z;
        cr[4 * q + 3] = su * v.w;
      }
      ab_terms(std::make_integer_sequence<int, NS * NSG>{}, acc, wr, cr);
    }
    float4* orow = reinterpret_cast<float4*>(out + Ia * NS);
#pragma unroll
    for (int q = 0; q < NS / 4; ++q) orow[q] = make_float4(acc[4 * q], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3]);
  }
  __syncwarp();
}

// Phi-tracking eigenpair of the k x k projected matrix (lane 0): shifted inverse iteration
// from the previous Ritz value, then Rayleigh-quotient refinement.  The projected matrix is
// built from FP32 vectors, so it is solved in FP32 too.
__device__ __noinline__ void small_eig(const float* G, int k, float shift, float* y, float* theta) {
  float a[KM * KM], z[KM];
  for (int phase = 0; phase < 5; ++phase) {
    const float sg = (phase < 2) ? shift : *theta;
    for (int i = 0; i < k; ++i)
      for (int j = 0; j < k; ++j) a[i * KM + j] = G[i * KM + j] - ((i == j) ? sg : 0.f);
    for (int i = 0; i < k; ++i) z[i] = y[i];
    for (int col = 0; col < k; ++col) {
      int piv = col;
      float best = fabsf(a[col * KM + col]);
      for (int r = col + 1; r < k; ++r)
        if (fabsf(a[r * KM + col]) > best) {
          best = fabsf(a[r * KM + col]);
          piv = r;
        }
      if (piv != col) {
        for (int j = 0; j < k; ++j) {
          const float t = a[col * KM + j];
          a[col * KM + j] = a[piv * KM + j];
          a[piv * KM + j] = t;
        }
        const float t = z[col];
        z[col] = z[piv];
        z[piv] = t;
      }
      float p = a[col * KM + col];
      if (fabsf(p) < 1e-30f) p = (p < 0.f) ? -1e-30f : 1e-30f;
      a[col * KM + col] = p;
      const float ip = 1.f / p;
      for (int r = col + 1; r < k; ++r) {
        const float f = a[r * KM + col] * ip;
        for (int j = col + 1; j < k; ++j) a[r * KM + j] -= f * a[col * KM + j];
        z[r] -= f * z[col];
      }
    }
    for (int r = k - 1; r >= 0; --r) {
      float s = z[r];
      for (int j = r + 1; j < k; ++j) s -= a[r * KM + j] * z[j];
      z[r] = s / a[r * KM + r];
    }
    float nrm = 0.f;
    for (int i = 0; i < k; ++i) nrm += z[i] * z[i];
    nrm = sqrtf(nrm);
    if (!(nrm > 0.f) || !isfinite(nrm)) break;
    const float sc = ((z[0] < 0.f) ? -1.f : 1.f) / nrm;
    for (int i = 0; i < k; ++i) y[i] = sc * z[i];
    float num = 0.f;
    for (int i = 0; i < k; ++i) {
      float gy = 0.f;
      for (int j = 0; j < k; ++j) gy += G[i * KM + j] * y[j];
      num += y[i] * gy;
    }
    *theta = num;
  }
}

__global__ void __launch_bounds__(32 * WARPS) solve_warp_kernel(SolveArgs a, const float* __restrict__ W32,
                                                                 const float* __restrict__ guess_in,
                                                                 float* __restrict__ guess_out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  CtaSmem& cs = *reinterpret_cast<CtaSmem*>(smem_raw);
  if (threadIdx.x == 0) {  // string tables (same construction as make_tab, at run time)
    int c = 0;
    for (int m = 0; m < 64; ++m)
      if (__popc(m) == 3) cs.mask[c++] = m;
    for (int I = 0; I < NS; ++I) {
      const int mi = cs.mask[I];
      int u = 0;
      for (int p = 0; p < NORB; ++p) {
        if (!((mi >> p) & 1)) continue;
        for (int q = 0; q < NORB; ++q) {
          if (q != p && ((mi >> q) & 1)) continue;
          const int mj = (mi & ~(1 << p)) | (1 << q);
          int sgn = 1;
          if (p != q) {
            int par = __popc(mj & ((1 << q) - 1)) & 1;
            const int m1 = mj & ~(1 << q);
            par ^= __popc(m1 & ((1 << p) - 1)) & 1;
            sgn = par ? -1 : 1;
          }
          int J = 0;
          for (int t = 0; t < NS; ++t)
            if (cs.mask[t] == mj) J = t;
          cs.J[I * NSG + u] = J;
          cs.pq[I * NSG + u] = p * NORB + q;
          cs.sg[I * NSG + u] = sgn;
          ++u;
        }
      }
    }
    int t = 0;
    for (int P = 0; P < NF; ++P)
      for (int R = P; R < NF; ++R) cs.pair[t++] = (unsigned short)(P | (R << 8));
    for (int I = 0; I < NS; ++I) {  // connections of each string to the Phi string
      int c = 0;
      for (int u = 0; u < NSG; ++u)
        if (cs.J[I * NSG + u] == 0 && c < 3) {
          cs.c0pq[I][c] = cs.pq[I * NSG + u];
          cs.c0sg[I][c] = cs.sg[I * NSG + u];
          ++c;
        }
      cs.c0n[I] = c;
    }
    for (int x = 0; x < 9; ++x) {  // single replacements i -> A of the Phi string
      const int i = x / 3, A = 3 + x % 3, m0 = cs.mask[0];
      int par = __popc(m0 & ((1 << i) - 1)) & 1;
      const int m1 = m0 & ~(1 << i);
      par ^= __popc(m1 & ((1 << A) - 1)) & 1;
      int J = 0;
      for (int q = 0; q < NS; ++q)
        if (cs.mask[q] == (m1 | (1 << A))) J = q;
      cs.xJ[x] = J;
      cs.xs[x] = par ? -1 : 1;
    }
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  WarpSmem& ws = cs.w[warp];
  const int n = a.n;
  const size_t n1 = (size_t)n, n2 = n1 * n1, n3 = n2 * n1;
  const float tol = (float)a.tol;

#pragma unroll 1
  for (int64_t s = (int64_t)blockIdx.x * WARPS + warp; s < a.nspaces; s += (int64_t)gridDim.x * WARPS) {
    // ---- validate -------------------------------------------------------------------------
    if (lane == 0) {
      const qflow_space& q = a.spaces[s];
      int ok = (q.no == 3 && q.nv == 3);
      for (int t = 0; t < 6; ++t) {
        const int o = q.orb[t];
        ws.orb[t] = o;
        if (t < 3) ok &= (o >= 0 && o < a.nocc);
        else ok &= (o >= a.nocc && o < a.n);
      }
      ws.ctrl[1] = ok;
    }
    __syncwarp();
    const int64_t sidx = a.sorted_index ? a.sorted_index[s] : a.space_base + s;
    const int64_t oidx = a.sorted_index ? sidx : s;
    if (!ws.ctrl[1]) {
      if (lane == 0) {
        a.energy[oidx] = 0.0;
        a.status[oidx] = kSpaceInvalid;
        if (a.iters) a.iters[oidx] = 0;
      }
      __syncwarp();
      continue;
    }
    // ---- gather ------------------------------------------------------------------------------
    // FP32 couplings: the 666 unique elements of the pair-symmetric W block (all loads in
    // flight); FP64: J_pr = W_pprr, K_pr = W_prrp and the F block (energy-carrying parts).
    {
      size_t ro[6];
#pragma unroll
      for (int t = 0; t < 6; ++t) ro[t] = (size_t)ws.orb[t];
      constexpr int PER = (NPAIR + 31) / 32;  // 21
      float wv[PER];
#pragma unroll
      for (int k = 0; k < PER; ++k) {
        const int t = lane + 32 * k;
        wv[k] = 0.f;
        if (t < NPAIR) {
          const int pr = cs.pair[t], P = pr & 255, R = pr >> 8;
          const size_t g = ro[P / 6] * n3 + ro[P % 6] * n2 + ro[R / 6] * n1 + ro[R % 6];
          wv[k] = W32 ? W32[g] : (float)a.W[g];
        }
      }
      double jv[2], kv[2], fv[2];
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const int t = lane + 32 * k;
        jv[k] = kv[k] = fv[k] = 0.0;
        if (t < NF) {
          const size_t p = ro[t / 6], r = ro[t % 6];
          jv[k] = a.W[p * n3 + p * n2 + r * n1 + r];
          kv[k] = a.W[p * n3 + r * n2 + r * n1 + p];
          fv[k] = a.F[p * n1 + r];
        }
      }
#pragma unroll
      for (int k = 0; k < PER; ++k) {
        const int t = lane + 32 * k;
        if (t < NPAIR) {
          const int pr = cs.pair[t], P = pr & 255, R = pr >> 8;
          const bool jj = (P / 6 == P % 6) && (R / 6 == R % 6);  // W_pprr: reaches only the diagonal
          const float wf = jj ? 0.f : wv[k];
          ws.Wt[P * NF + R] = wf;
          ws.Wt[R * NF + P] = wf;
        }
      }
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const int t = lane + 32 * k;
        if (t < NF) {
          ws.J[t] = jv[k];
          ws.K[t] = kv[k];
          ws.F[t] = fv[k];
        }
      }
    }
    __syncwarp();
    // ---- fold (vacuum order over the active orbitals) -------------------------------------
    // h_pp = F_pp - sum_k (2 J_pk - K_pk) in FP64; off-diagonal h' = h - 1/2 sum_r W_prrq in FP32
    if (lane < 6) {
      double v = ws.F[lane * 7];
      for (int k = 0; k < 3; ++k) v -= 2.0 * ws.J[lane * 6 + k] - ws.K[lane * 6 + k];
      ws.hd[lane] = v;
    }
#pragma unroll 1
    for (int idx = lane; idx < NF; idx += 32) {
      const int p = idx / 6, q = idx % 6;
      float v = (float)ws.F[idx];
      for (int k = 0; k < 3; ++k) v -= 2.f * ws.Wt[idx * NF + k * 7] - ws.Wt[(p * 6 + k) * NF + k * 6 + q];
      for (int r = 0; r < 6; ++r) v -= 0.5f * ws.Wt[(p * 6 + r) * NF + r * 6 + q];
      ws.hp[idx] = (p == q) ? 0.f : v;
    }
    __syncwarp();
    if (lane < NS) {  // same-spin string diagonal: sum_{p in I} h_pp + 1/2 sum_{p,r in I} (J_pr - K_pr)
      const int m = cs.mask[lane];
      double v = 0.0;
      for (int p = 0; p < 6; ++p) {
        if (!((m >> p) & 1)) continue;
        v += ws.hd[p];
        for (int r = 0; r < 6; ++r)
          if ((m >> r) & 1) v += 0.5 * (ws.J[p * 6 + r] - ws.K[p * 6 + r]);
      }
      ws.hsd[lane] = v;
    }
    __syncwarp();
    if (lane == 0) {
      double ec = *a.e0;
      for (int k = 0; k < 3; ++k) ec -= ws.hd[k] + ws.F[k * 7];
      ws.ecore = ec;
      double v = ec + 2.0 * ws.hsd[0];
      for (int p = 0; p < 3; ++p)
        for (int r = 0; r < 3; ++r) v += ws.J[p * 6 + r];
      ws.eshift = v;  // <Phi|H|Phi>
      ws.ctrl[0] = 1;
      ws.ctrl[2] = kSpaceNoConv;
      ws.ctrl[3] = 0;
      ws.theta = 0.f;
      ws.G[0] = 0.f;
      ws.yf[0] = 1.f;
    }
    __syncwarp();
    // ---- Phi fast path: sigma(Phi) = column 0 of H (0 at Phi after the shift) --------------
    // Only determinants connected to Phi by single or double replacements are nonzero.  If the
    // residual of Phi is already below the tolerance the root is Phi, the increment is zero and
    // the space is done without building the full string operator or the diagonal.
    const bool phi_start = (guess_in == nullptr);
    if (phi_start) {
      if (lane < NS) {  // dh[I] <- Hs[I][0]: same-spin coupling of string I to the Phi string
        const int I = lane;
        float hc = 0.f;
        if (I != 0) {
#pragma unroll 1
          for (int u = 0; u < NSG; ++u) {
            const int e = I * NSG + u;
            const int pq = cs.pq[e], Kk = cs.J[e];
            const float s1 = (float)cs.sg[e];
            if (Kk == 0) hc = fmaf(s1, ws.hp[pq], hc);
            for (int v = 0; v < cs.c0n[Kk]; ++v)
              hc = fmaf(0.5f * s1 * (float)cs.c0sg[Kk][v], ws.Wt[pq * NF + cs.c0pq[Kk][v]], hc);
          }
        }
        ws.dh[I] = hc;
      }
      for (int d = lane; d < NDET; d += 32) {
        ws.S[d] = 0.f;
        ws.V[d] = (d == 0) ? 1.f : 0.f;
      }
      __syncwarp();
      // alpha-beta couplings: both strings are Phi or single replacements of it (10 x 10 pairs);
      // same-spin couplings sit in row 0 and column 0 of the CI matrix
#pragma unroll 1
      for (int t = lane; t < 100; t += 32) {
        const int x = t / 10, y = t % 10;
        const int Ia = (x == 0) ? 0 : cs.xJ[x - 1], Ib = (y == 0) ? 0 : cs.xJ[y - 1];
        float acc = 0.f;
        for (int u = 0; u < cs.c0n[Ia]; ++u)
          for (int v = 0; v < cs.c0n[Ib]; ++v)
            acc = fmaf((float)(cs.c0sg[Ia][u] * cs.c0sg[Ib][v]), ws.Wt[cs.c0pq[Ia][u] * NF + cs.c0pq[Ib][v]], acc);
        if (t != 0) ws.S[Ia * NS + Ib] = acc;
      }
      __syncwarp();
      if (lane > 0 && lane < NS) {
        ws.S[lane * NS] += ws.dh[lane];
        ws.S[lane] += ws.dh[lane];
      }
      __syncwarp();
      float rr = 0.f;
      for (int d = lane; d < NDET; d += 32) rr = fmaf(ws.S[d], ws.S[d], rr);
      const float rphi = sqrtf(wsum(rr));
      if (rphi < tol) {  // converged at Phi: E = <Phi|H|Phi>, X = 0
        if (lane == 0) {
          a.energy[oidx] = ws.eshift;
          a.status[oidx] = kSpaceOk;
          if (a.iters) a.iters[oidx] = 0;
        }
        if (guess_out)
          for (int d = lane; d < NDET; d += 32) guess_out[(size_t)s * NDET + d] = (d == 0) ? 1.f : 0.f;
        __syncwarp();
        continue;
      }
    }
    // ---- same-spin string operator, off-diagonal (row I owned by lane I) ---------------------
    if (lane < NS) {
      const int I = lane;
#pragma unroll 1
      for (int j = 0; j < NS; ++j) ws.Hs[I * NS + j] = 0.f;
#pragma unroll 1
      for (int u = 0; u < NSG; ++u) {
        const int e = I * NSG + u;
        const int pq = cs.pq[e], Kk = cs.J[e];
        const float s1 = (float)cs.sg[e];
        if (Kk != I) ws.Hs[I * NS + Kk] += s1 * ws.hp[pq];
#pragma unroll 1
        for (int v = 0; v < NSG; ++v) {
          const int e2 = Kk * NSG + v;
          const int J2 = cs.J[e2];
          if (J2 == I) continue;  // the diagonal is kept in FP64
          ws.Hs[I * NS + J2] += 0.5f * s1 * (float)cs.sg[e2] * ws.Wt[pq * NF + cs.pq[e2]];
        }
      }
    }
    // the diagonal relative to <Phi|H|Phi>: string parts as FP64 differences, the alpha-beta
    // Coulomb sum J(Ia, Ib) in FP32 through row sums jb[p][Ib] = sum_{r in Ib} J_pr
    if (lane < NS) ws.dh[lane] = (float)(ws.hsd[lane] - ws.hsd[0]);
#pragma unroll 1
    for (int t = lane; t < 6 * NS; t += 32) {
      const int p = t / NS, b = t % NS, mb = cs.mask[b];
      float v = 0.f;
      for (int r = 0; r < 6; ++r)
        if ((mb >> r) & 1) v += (float)ws.J[p * 6 + r];
      ws.jb[t] = v;
    }
    __syncwarp();
#pragma unroll 1
    for (int d = lane; d < NDET; d += 32) {
      const int ia = d / NS, ib = d % NS;
      const int ma = cs.mask[ia];
      float jj = 0.f, j0 = 0.f;
      for (int p = 0; p < 6; ++p) {
        if ((ma >> p) & 1) jj += ws.jb[p * NS + ib];
        if (p < 3) j0 += ws.jb[p * NS + 0];
      }
      ws.diag[d] = (d == 0) ? 0.f : ws.dh[ia] + ws.dh[ib] + (jj - j0);
      if (!phi_start) ws.V[d] = guess_in[(size_t)s * NDET + d];
    }
    __syncwarp();
    if (!phi_start) {
      float p = 0.f;
      for (int d = lane; d < NDET; d += 32) p = fmaf(ws.V[d], ws.V[d], p);
      const float nr = sqrtf(wsum(p));
      const float inv = (nr > 0.f) ? 1.f / nr : 0.f;
      for (int d = lane; d < NDET; d += 32) ws.V[d] = (nr > 0.f) ? ws.V[d] * inv : ((d == 0) ? 1.f : 0.f);
      __syncwarp();
      sigma_warp(cs, ws, ws.V, ws.S, lane);
      float g = 0.f;
      for (int d = lane; d < NDET; d += 32) g = fmaf(ws.V[d], ws.S[d], g);
      g = wsum(g);
      if (lane == 0) {
        ws.G[0] = g;
        ws.theta = g;
      }
      __syncwarp();
    }
    // ---- Davidson ----------------------------------------------------------------------------
#pragma unroll 1
    for (int it = 0; it < a.max_iter; ++it) {
      int k = ws.ctrl[0];
      if (k == KM) {  // restart on the Ritz vector
        float pv = 0.f, ps = 0.f;
        for (int d = lane; d < NDET; d += 32) {
          float xv = 0.f, sv = 0.f;
          for (int j = 0; j < k; ++j) {
            xv = fmaf(ws.yf[j], ws.V[j * NDET + d], xv);
            sv = fmaf(ws.yf[j], ws.S[j * NDET + d], sv);
          }
          ws.V[d] = xv;
          ws.S[d] = sv;
          pv = fmaf(xv, xv, pv);
          ps = fmaf(xv, sv, ps);
        }
        pv = wsum(pv);
        ps = wsum(ps);
        const float inv = 1.f / sqrtf(pv);
        for (int d = lane; d < NDET; d += 32) {
          ws.V[d] *= inv;
          ws.S[d] *= inv;
        }
        __syncwarp();
        if (lane == 0) {
          ws.G[0] = ps / pv;
          ws.theta = ws.G[0];
          ws.yf[0] = 1.f;
          ws.ctrl[0] = 1;
        }
        __syncwarp();
        k = 1;
      }
      const float th = ws.theta;
      float rr = 0.f;
      float* vk = ws.V + k * NDET;
      for (int d = lane; d < NDET; d += 32) {
        float xv = 0.f, sv = 0.f;
        for (int j = 0; j < k; ++j) {
          xv = fmaf(ws.yf[j], ws.V[j * NDET + d], xv);
          sv = fmaf(ws.yf[j], ws.S[j * NDET + d], sv);
        }
        const float r = sv - th * xv;
        rr = fmaf(r, r, rr);
        float den = th - ws.diag[d];
        if (fabsf(den) < 1e-4f) den = (den < 0.f) ? -1e-4f : 1e-4f;
        vk[d] = r / den;
      }
      const float rnorm = sqrtf(wsum(rr));
      if (!isfinite(rnorm) || !isfinite(th)) {
        if (lane == 0) ws.ctrl[2] = kSpaceNonFinite;
        __syncwarp();
        break;
      }
      if (rnorm < tol) {
        if (lane == 0) {
          ws.ctrl[2] = kSpaceOk;
          ws.ctrl[3] = it;
        }
        __syncwarp();
        break;
      }
      __syncwarp();
      for (int pass = 0; pass < 2; ++pass) {
        float cf[KM];
#pragma unroll
        for (int j = 0; j < KM; ++j) cf[j] = 0.f;
        for (int d = lane; d < NDET; d += 32) {
          const float v = vk[d];
#pragma unroll
          for (int j = 0; j < KM; ++j)
            if (j < k) cf[j] = fmaf(ws.V[j * NDET + d], v, cf[j]);
        }
#pragma unroll
        for (int j = 0; j < KM; ++j)
          if (j < k) cf[j] = wsum(cf[j]);
        for (int d = lane; d < NDET; d += 32) {
          float v = vk[d];
#pragma unroll
          for (int j = 0; j < KM; ++j)
            if (j < k) v = fmaf(-cf[j], ws.V[j * NDET + d], v);
          vk[d] = v;
        }
        __syncwarp();
      }
      float nn = 0.f;
      for (int d = lane; d < NDET; d += 32) nn = fmaf(vk[d], vk[d], nn);
      const float vn = sqrtf(wsum(nn));
      if (!(vn > 1e-6f)) {
        if (lane == 0) {
          ws.ctrl[2] = (rnorm < 100.f * tol) ? kSpaceOk : kSpaceNoConv;
          ws.ctrl[3] = it;
        }
        __syncwarp();
        break;
      }
      const float inv = 1.f / vn;
      for (int d = lane; d < NDET; d += 32) vk[d] *= inv;
      __syncwarp();
      float* sk = ws.S + k * NDET;
      sigma_warp(cs, ws, vk, sk, lane);
      float gc[KM], gr[KM];
#pragma unroll
      for (int j = 0; j < KM; ++j) gc[j] = gr[j] = 0.f;
      float gkk = 0.f;
      for (int d = lane; d < NDET; d += 32) {
        const float vkd = vk[d], skd = sk[d];
        gkk = fmaf(vkd, skd, gkk);
#pragma unroll
        for (int j = 0; j < KM; ++j)
          if (j < k) {
            gc[j] = fmaf(ws.V[j * NDET + d], skd, gc[j]);
            gr[j] = fmaf(vkd, ws.S[j * NDET + d], gr[j]);
          }
      }
      gkk = wsum(gkk);
#pragma unroll
      for (int j = 0; j < KM; ++j)
        if (j < k) {
          gc[j] = wsum(gc[j]);
          gr[j] = wsum(gr[j]);
        }
      if (lane == 0) {
        for (int j = 0; j < k; ++j) {
          ws.G[j * KM + k] = gc[j];
          ws.G[k * KM + j] = gr[j];
        }
        ws.G[k * KM + k] = gkk;
        const int kk = k + 1;
        float yn[KM];
        for (int j = 0; j < kk; ++j) yn[j] = (j < k) ? ws.yf[j] : 0.f;
        float thn = ws.theta;
        small_eig(ws.G, kk, ws.theta - 1e-2f, yn, &thn);
        for (int j = 0; j < kk; ++j) ws.yf[j] = yn[j];
        ws.theta = thn;
        ws.ctrl[0] = kk;
        ws.ctrl[3] = it + 1;
      }
      __syncwarp();
    }
    // ---- root, increment, merge ------------------------------------------------------------
    const int k = ws.ctrl[0];
    float xx = 0.f;
    for (int d = lane; d < NDET; d += 32) {
      float xv = 0.f;
      for (int j = 0; j < k; ++j) xv = fmaf(ws.yf[j], ws.V[j * NDET + d], xv);
      ws.S[d] = xv;
      xx = fmaf(xv, xv, xx);
    }
    xx = wsum(xx);
    __syncwarp();
    const float xn = sqrtf(xx);
    const float c0 = ws.S[0];
    int st = ws.ctrl[2];
    if (st == kSpaceOk && !(fabsf(c0) >= 1e-3f * xn)) st = kSpaceRoot;
    if (!isfinite(c0) || !isfinite(ws.theta)) st = kSpaceNonFinite;
    const float inv0 = (st == kSpaceOk || st == kSpaceNoConv) ? 1.f / c0 : 0.f;
    if (guess_out && st == kSpaceOk)
      for (int d = lane; d < NDET; d += 32) guess_out[(size_t)s * NDET + d] = ws.S[d] * inv0;
    float* x1 = ws.V;  // V is free now: 9 + 81 floats of scratch
    float* x2 = x1 + 9;
    if (lane < 9) {
      const int J = cs.xJ[lane];
      const float f = (cs.xs[lane] < 0) ? -inv0 : inv0;
      x1[lane] = 0.5f * f * (ws.S[J * NS] + ws.S[J]);
    }
    __syncwarp();
#pragma unroll 1
    for (int idx = lane; idx < 81; idx += 32) {
      const int i = idx / 27, j = (idx / 9) % 3, aa = (idx / 3) % 3, b = idx % 3;
      const int xa = i * 3 + aa, xb = j * 3 + b;
      const float f = (cs.xs[xa] != cs.xs[xb]) ? -inv0 : inv0;
      x2[idx] = f * ws.S[cs.xJ[xa] * NS + cs.xJ[xb]] - x1[xa] * x1[xb];
    }
    __syncwarp();
    if (st == kSpaceOk && a.owner1 && lane < 9) {
      const int i = lane / 3, aa = lane % 3;
      const size_t g = (size_t)ws.orb[i] * a.nvir + (ws.orb[3 + aa] - a.nocc);
      if (a.owner1[g] == sidx) a.t1_new[g] = a.t1_old[g] + (double)x1[lane];
    }
    if (st == kSpaceOk && a.owner2) {
#pragma unroll 1
      for (int idx = lane; idx < 81; idx += 32) {
        const int i = idx / 27, j = (idx / 9) % 3, aa = (idx / 3) % 3, b = idx % 3;
        const size_t g = (((size_t)ws.orb[i] * a.nocc + ws.orb[j]) * a.nvir + (ws.orb[3 + aa] - a.nocc)) * a.nvir +
                         (ws.orb[3 + b] - a.nocc);
        if (a.owner2[g] == sidx)
          a.t2_new[g] = a.t2_old[g] + (double)(0.5f * (x2[idx] + x2[((j * 3 + i) * 3 + b) * 3 + aa]));
      }
    }
    if (lane == 0) {
      a.energy[oidx] = ws.eshift + (double)ws.theta;
      a.status[oidx] = st;
      if (a.iters) a.iters[oidx] = ws.ctrl[3];
    }
    __syncwarp();
  }
}

}  // namespace

cudaError_t launch_solve_warp33(const SolveArgs& a, const float* W32, const float* guess_in, float* guess_out,
                                cudaStream_t st) {
  if (a.nspaces <= 0) return cudaSuccess;
  const size_t smem = sizeof(CtaSmem);
  cudaError_t e = cudaFuncSetAttribute(solve_warp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, solve_warp_kernel, 32 * WARPS, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  int64_t grid = (int64_t)sms * per_sm;
  const int64_t need = (a.nspaces + WARPS - 1) / WARPS;
  if (grid > need) grid = need;
  solve_warp_kernel<<<(unsigned)grid, 32 * WARPS, smem, st>>>(a, W32, guess_in, guess_out);
  return cudaGetLastError();
}

size_t solve_warp33_smem() { return sizeof(CtaSmem); }

}  // namespace qf
