// Mixed-precision batched solver, one warp per active space, for the three size classes
// (k occupied + k virtual orbitals, k = 1, 2, 3: 4, 36 and 400 Sz = 0 determinants).
//
// What it computes is the same as solve.cu (gather + fold, Phi-dominant right eigenpair of the
// space's determinant operator by Davidson, CI -> CC increment, owner-filtered merge), see that
// file for the paper passages.  Mapping onto the GB300:
//   * one warp owns one space (no block-wide barriers; all reductions are warp shuffles);
//   * 6e6o sigma: lane L < 20 owns alpha string I_alpha = L and the 20 determinants of that
//     row.  For each of the 12 single replacements (pq, J_alpha, s) into I_alpha it holds the W
//     row W[pq][*] (36 values) and the CI row C[J_alpha][*] (20 values) in registers and applies
//     the whole beta-side replacement table, a compile-time constant (the same for every space),
//     as 240 register-only FMAs; the alpha-alpha part is a 20 x 20 x 20 product from vectorised
//     shared-memory rows and the beta-beta part its transpose (every vector is symmetric under
//     the spin flip).  The small classes use a determinant-per-lane sigma;
//   * the operator diagonal is built relative to E_Phi = <Phi|H|Phi> (which is E0 of the
//     dressing) and kept out of the sigma operands, so the sums carry only off-diagonal
//     couplings;
//   * before anything else a space checks the residual of Phi from Phi's sparse column; spaces
//     already at their root (most of a mid-flow sweep) stop there;
//   * precision: FP32 for the gathered couplings, the fold and set-up (the folded one-body
//     diagonal and the string diagonal, both differences of O(1) terms), the determinant
//     vectors and sigma; FP64 accuracy for the Rayleigh-Ritz step (projected matrix, its root,
//     the Gram-Schmidt coefficients) in double-float arithmetic; FP64 for the energy
//     E0 + theta and the amplitude update;
//   * the root of the projected problem is the real Ritz pair with the largest Phi weight (the
//     space's root is the eigenvector with the largest |c_Phi|); a complex pair with more Phi
//     weight flags the space;
//   * the warp pass runs at most kWarpIterCap Davidson steps: the few spaces it leaves
//     unconverged are solved again by solve.cu's FP64 solver (a larger subspace) in the same
//     sweep.
// Kernels: one per size class (grid-stride over that class), and a persistent kernel whose
// warps take work items from one queue holding every class (largest spaces first).
// Every loop is bounded; a warp never waits on another warp (the queue is a single atomic
// counter).
#include <cuda_runtime.h>
#include <math.h>
#include <stddef.h>
#include <stdint.h>

#include <utility>

#include "qflow_internal.h"

namespace qf {
namespace {

// Loop unrolling of the same-spin table loop (measured: 11 steps per iteration; 6, 22 and 66 were
// not faster)
constexpr int kHsUnroll = 11;
constexpr int KM = 3;     // Davidson subspace limit (restart on the Ritz vector)
// Spaces (warps) per CTA: a launch parameter up to kMaxWarps (the autotuner picks it); one CTA
// fills the shared memory of an SM.  The register file is split over the SM's four
// sub-partitions (16,384 registers each); 15 warps put four warps on some of them, so a thread
// may hold at most 16,384 / (4 x 32) = 128 registers, which every smaller count allows too.
constexpr int kMaxWarps = 15;
constexpr int kMaxRegs = 128;

template <int K>
struct Dim {
  static constexpr int NORB = 2 * K;
  static constexpr int NS = (K == 1) ? 2 : (K == 2) ? 6 : 20;  // C(2k, k) strings per spin
  static constexpr int NSG = K * (K + 1);                       // single replacements into a string
  static constexpr int NDET = NS * NS;
  static constexpr int NF = NORB * NORB;
  static constexpr int NW = NF * NF;
  static constexpr int NPAIR = NF * (NF + 1) / 2;  // unique (pq, rs) pairs of the pair-symmetric block
};

// ---- compile-time string tables (6e6o sigma) ------------------------------------------------

struct Tab3 {
  int mask[20];
  int idx[64];
  int J[20][12];  // single replacements into string I: <I| a+_p a_q |J> = sg
  int pq[20][12];
  int sg[20][12];
};

__host__ __device__ constexpr int popc6(int m) {
  int c = 0;
  for (int b = 0; b < 6; ++b) c += (m >> b) & 1;
  return c;
}

__host__ __device__ constexpr Tab3 make_tab3() {
  Tab3 t{};
  int c = 0;
  for (int m = 0; m < 64; ++m) {
    t.idx[m] = -1;
    if (popc6(m) == 3) {
      t.idx[m] = c;
      t.mask[c] = m;
      ++c;
    }
  }
  for (int I = 0; I < 20; ++I) {
    const int mi = t.mask[I];
    int u = 0;
    for (int p = 0; p < 6; ++p) {
      if (!((mi >> p) & 1)) continue;
      for (int q = 0; q < 6; ++q) {
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
        t.pq[I][u] = p * 6 + q;
        t.sg[I][u] = s;
        ++u;
      }
    }
  }
  return t;
}

// Used only in constant expressions (template arguments), so the beta-side replacement pattern
// becomes immediate register operands in sigma.
struct TabHolder {
  static constexpr Tab3 value = make_tab3();
};

// ---- compile-time coupling tables of the 6e6o class, balanced over the 32 lanes of a warp -------
//
// A table is a list of terms per target element; a term adds c * X[src] to its target, where X is
// the warp state's W block (pq * 36 + rs) followed by h' (1296 + pq), and c is +-1/2, +-1 or +-2
// (merged under the pair symmetry W[pq][rs] = W[rs][pq]).  Whole targets are dealt to lanes in
// order so that every lane gets at most L terms; entry k of lane l is e[k * 32 + l]:
//   bits 0-10 src, 11-19 target, 20 last term of its target, 21 also store at the transposed
//   target, 23-31 sign and exponent of the float c (mantissa 0), so c = as_float(e & 0xff800000);
//   padding entries have c = 0 and src 0 (a W element that is always 0).
// Same-spin string operator: Hs[I][J] = sum_u [J_u = J] s_u h'[pq_u]
//                                     + 1/2 sum_{u,v} [J(J_u, v) = J] s_u s_v W[pq_u][pq_v],  J != I,
// u over the single replacements into string I, v over those into J_u.
// Phi column: sigma(Phi)[d] for d != 0 relative to <Phi|H|Phi>: at (I, 0) and (0, I), Hs[I][0]
// plus the alpha-beta couplings of string I and the Phi string; at (a, b) for single
// replacements a, b of the Phi string, their alpha-beta coupling (the column is symmetric in the
// two spins, so each unique element is computed once and stored at both places).
constexpr int kTermMax = 2400;
struct TermList {
  int ntgt = 0, nterm = 0;
  int tgt[400] = {};
  int mirror[400] = {};
  int first[401] = {};
  int src[kTermMax] = {};
  int c2[kTermMax] = {};  // coefficient in units of 1/2
};

// Adds the merged terms of one target (keys/coefficients gathered by the caller) to the list;
// a coefficient of 3/2 becomes two terms (1 and 1/2) so that every c is a power of two.
__host__ __device__ constexpr void push_target(TermList& L, int target, int mirror, const int* key, const int* c2,
                                               int n) {
  int cnt = 0;
  for (int x = 0; x < n; ++x) cnt += (c2[x] != 0);
  if (cnt == 0) return;
  L.tgt[L.ntgt] = target;
  L.mirror[L.ntgt] = mirror;
  L.first[L.ntgt] = L.nterm;
  for (int x = 0; x < n; ++x) {
    int c = c2[x];
    if (c == 0) continue;
    const int sg = c < 0 ? -1 : 1;
    int m = c * sg;
    while (m > 0) {
      const int part = (m == 3) ? 2 : m;  // 3 -> 2 + 1; 1, 2 and 4 are powers of two
      L.src[L.nterm] = key[x];
      L.c2[L.nterm] = sg * part;
      ++L.nterm;
      m -= part;
    }
  }
  ++L.ntgt;
  L.first[L.ntgt] = L.nterm;
}

__host__ __device__ constexpr int add_key(int* key, int* c2, int n, int k, int c) {
  for (int x = 0; x < n; ++x)
    if (key[x] == k) {
      c2[x] += c;
      return n;
    }
  key[n] = k;
  c2[n] = c;
  return n + 1;
}

__host__ __device__ constexpr int wkey(int a, int b) { return a < b ? a * 36 + b : b * 36 + a; }

// Merged same-spin couplings of string I into target J (J != I); returns the number of keys.
__host__ __device__ constexpr int hs_terms(const Tab3& t, int I, int J, int* key, int* c2) {
  int n = 0;
  for (int u = 0; u < 12; ++u) {
    const int Ku = t.J[I][u];
    if (Ku != I && Ku == J) n = add_key(key, c2, n, 1296 + t.pq[I][u], 2 * t.sg[I][u]);
    for (int v = 0; v < 12; ++v)
      if (t.J[Ku][v] == J) n = add_key(key, c2, n, wkey(t.pq[I][u], t.pq[Ku][v]), t.sg[I][u] * t.sg[Ku][v]);
  }
  return n;
}

__host__ __device__ constexpr TermList make_hs_terms() {
  TermList L{};
  const Tab3 t = make_tab3();
  for (int I = 0; I < 20; ++I)
    for (int J = 0; J < 20; ++J) {
      if (J == I) continue;
      int key[64] = {}, c2[64] = {};
      const int n = hs_terms(t, I, J, key, c2);
      push_target(L, I * 20 + J, 0, key, c2, n);
    }
  return L;
}

__host__ __device__ constexpr TermList make_phi_terms() {
  TermList L{};
  const Tab3 t = make_tab3();
  int c0[20][3] = {}, n0[20] = {};  // replacements u with J[I][u] = 0 (the Phi string)
  for (int I = 0; I < 20; ++I)
    for (int u = 0; u < 12; ++u)
      if (t.J[I][u] == 0 && n0[I] < 3) c0[I][n0[I]++] = u;
  for (int I = 1; I < 20; ++I) {  // (I, 0), mirrored to (0, I)
    int key[64] = {}, c2[64] = {};
    int n = hs_terms(t, I, 0, key, c2);
    for (int x = 0; x < n0[I]; ++x)
      for (int y = 0; y < n0[0]; ++y) {
        const int u = c0[I][x], v = c0[0][y];
        n = add_key(key, c2, n, wkey(t.pq[I][u], t.pq[0][v]), 2 * t.sg[I][u] * t.sg[0][v]);
      }
    push_target(L, I * 20, 1, key, c2, n);
  }
  for (int a = 1; a < 20; ++a)  // (a, b), a <= b single replacements of the Phi string
    for (int b = a; b < 20; ++b) {
      if (n0[a] == 0 || n0[b] == 0) continue;
      int key[16] = {}, c2[16] = {};
      int n = 0;
      for (int x = 0; x < n0[a]; ++x)
        for (int y = 0; y < n0[b]; ++y) {
          const int u = c0[a][x], v = c0[b][y];
          n = add_key(key, c2, n, wkey(t.pq[a][u], t.pq[b][v]), 2 * t.sg[a][u] * t.sg[b][v]);
        }
      push_target(L, a * 20 + b, a != b ? 1 : 0, key, c2, n);
    }
  return L;
}

// Smallest per-lane length that deals the targets, in order, to at most 32 lanes.
__host__ __device__ constexpr int lane_length(const TermList& L) {
  int len = (L.nterm + 31) / 32;
  for (;; ++len) {
    int lanes = 1, cur = 0;
    for (int g = 0; g < L.ntgt; ++g) {
      const int c = L.first[g + 1] - L.first[g];
      if (c > len) {
        lanes = 99;
        break;
      }
      if (cur + c > len) {
        ++lanes;
        cur = 0;
      }
      cur += c;
    }
    if (lanes <= 32) return len;
  }
}

__host__ __device__ constexpr unsigned coef_bits(int c2) {  // float c2 / 2, top 9 bits only
  const unsigned sign = c2 < 0 ? 0x80000000u : 0u;
  const int m = c2 < 0 ? -c2 : c2;
  const unsigned expo = (m == 1) ? 126u : (m == 2) ? 127u : 128u;  // 1/2, 1, 2
  return sign | (expo << 23);
}

template <int LEN>
struct LaneTable {
  unsigned e[LEN * 32];
};

template <int LEN>
__host__ __device__ constexpr LaneTable<LEN> deal(const TermList& L) {
  LaneTable<LEN> T{};
  int lane = 0, cur = 0;
  for (int g = 0; g < L.ntgt; ++g) {
    const int c = L.first[g + 1] - L.first[g];
    if (cur + c > LEN) {
      ++lane;
      cur = 0;
    }
    for (int x = 0; x < c; ++x) {
      const int k = L.first[g] + x;
      unsigned e = (unsigned)L.src[k] | ((unsigned)L.tgt[g] << 11) | coef_bits(L.c2[k]);
      if (x == c - 1) e |= 1u << 20;
      if (L.mirror[g]) e |= 1u << 21;
      T.e[(cur + x) * 32 + lane] = e;
    }
    cur += c;
  }
  return T;
}

__host__ __device__ constexpr bool terms_valid(const TermList& L) {
  if (L.nterm > kTermMax) return false;
  for (int k = 0; k < L.nterm; ++k) {
    const int m = L.c2[k] < 0 ? -L.c2[k] : L.c2[k];
    if (!(m == 1 || m == 2 || m == 4) || L.src[k] < 0 || L.src[k] >= 1296 + 36) return false;
  }
  for (int g = 0; g < L.ntgt; ++g)
    if (L.tgt[g] < 0 || L.tgt[g] >= 400) return false;
  return true;
}

struct TermHolder {
  static constexpr TermList hs = make_hs_terms();
  static constexpr TermList phi = make_phi_terms();
};
static_assert(terms_valid(TermHolder::hs) && terms_valid(TermHolder::phi), "coupling tables");
constexpr int kHsLen = lane_length(TermHolder::hs);
constexpr int kPhiLen = lane_length(TermHolder::phi);
static_assert(kHsLen <= 72 && kPhiLen <= 12, "balanced coupling tables");
__device__ const LaneTable<kHsLen> g_hs_table = deal<kHsLen>(TermHolder::hs);
__device__ const LaneTable<kPhiLen> g_phi_table = deal<kPhiLen>(TermHolder::phi);

template <int B, int V>
__device__ __forceinline__ void ab_term(float (&acc)[20], const float (&wr)[36], const float (&cr)[20]) {
  constexpr int pq = TabHolder::value.pq[B][V];
  constexpr int J = TabHolder::value.J[B][V];
  constexpr int sg = TabHolder::value.sg[B][V];
  if constexpr (sg > 0) acc[B] = fmaf(wr[pq], cr[J], acc[B]);
  else acc[B] = fmaf(-wr[pq], cr[J], acc[B]);
}

template <int... I>
__device__ __forceinline__ void ab_terms(std::integer_sequence<int, I...>, float (&acc)[20], const float (&wr)[36],
                                         const float (&cr)[20]) {
  (ab_term<I / 12, I % 12>(acc, wr, cr), ...);
}

// ---- sigma of the first expansion vector (6e6o) --------------------------------------------
// The first vector is the first-order correction r / (0 - D) on the Phi column's support: the
// determinants (Ia, Ib) whose strings together carry one or two excitations (117 of 400; the
// type of a string is its number of virtual orbitals, 0 for the Phi string).  In the alpha-beta
// part a source row Ja of type 0 then meets columns of types 1, 2 only, type 1 columns of types
// 0, 1, type 2 the Phi string's column, type 3 nothing: 16,848 products instead of 57,600.  The
// (row, replacement) pairs are scheduled at compile time in type-uniform steps (1 step of type 0,
// 4 of type 1, 4 of type 2), so every lane runs the same compile-time product list in a step:
// lane Ia < 20 takes pairs of its own row; lanes 20..31 take a row's remaining pairs of a phase
// and leave their partial row in a scratch slot, which the row's lane adds at the end.
__host__ __device__ constexpr int str_type(int J) { return popc6(TabHolder::value.mask[J] & 0x38); }
__host__ __device__ constexpr bool first_support(int ta, int tb) { return ta + tb >= 1 && ta + tb <= 2; }

constexpr int kFirstSteps = 9;            // step 0: type 0, steps 1-4: type 1, steps 5-8: type 2
constexpr int kFirstSlots = 24;           // helper partial rows (V_2: 20 rows, S_2: 4 rows)
struct FirstSched {
  int e[kFirstSteps][32];    // (Ia << 4) | u of the pair a lane takes in a step, or -1
  int hslot[3][12];          // slot helper h fills at the end of phase t, or -1
  int rslot[20][6];          // slots added to row Ia, in order
  int rcount[20];
  bool ok;
};
__host__ __device__ constexpr FirstSched make_first_sched() {
  FirstSched f{};
  const Tab3 t = TabHolder::value;
  for (int k = 0; k < kFirstSteps; ++k)
    for (int l = 0; l < 32; ++l) f.e[k][l] = -1;
  for (int ph = 0; ph < 3; ++ph)
    for (int h = 0; h < 12; ++h) f.hslot[ph][h] = -1;
  for (int r = 0; r < 20; ++r) f.rcount[r] = 0;
  f.ok = true;
  const int first[3] = {0, 1, 5}, steps[3] = {1, 4, 4};
  int slot = 0;
  for (int ph = 0; ph < 3; ++ph) {
    int helper = 0;
    for (int Ia = 0; Ia < 20; ++Ia) {
      int list[12] = {}, n = 0;
      for (int u = 0; u < 12; ++u)
        if (str_type(t.J[Ia][u]) == ph) list[n++] = u;
      int taken = 0;
      for (; taken < n && taken < steps[ph]; ++taken) f.e[first[ph] + taken][Ia] = (Ia << 4) | list[taken];
      while (taken < n) {  // a helper lane takes up to steps[ph] of this row's remaining pairs
        if (helper >= 12 || slot >= kFirstSlots || f.rcount[Ia] >= 6) {
          f.ok = false;
          return f;
        }
        for (int k = 0; k < steps[ph] && taken < n; ++k, ++taken)
          f.e[first[ph] + k][20 + helper] = (Ia << 4) | list[taken];
        f.hslot[ph][helper] = slot;
        f.rslot[Ia][f.rcount[Ia]++] = slot;
        ++slot;
        ++helper;
      }
    }
  }
  return f;
}
struct FirstHolder {
  static constexpr FirstSched value = make_first_sched();
};
__host__ __device__ constexpr int max_row_slots(const FirstSched& f) {
  int m = 0;
  for (int r = 0; r < 20; ++r) m = f.rcount[r] > m ? f.rcount[r] : m;
  return m;
}
static_assert(FirstHolder::value.ok && max_row_slots(FirstHolder::value) <= 4, "first-vector sigma schedule");
__device__ const FirstSched g_first = make_first_sched();

// Compile-time product lists: the alpha-beta terms (B, V) of a source row of type T (target
// strings J(B, V) of the types first_support allows), and the same-spin terms (J, b) of the
// first vector's support.
template <int T>
struct AbFirst {
  int B[216], V[216], n;
};
template <int T>
__host__ __device__ constexpr AbFirst<T> make_ab_first() {
  AbFirst<T> a{};
  a.n = 0;
  for (int B = 0; B < 20; ++B)
    for (int V = 0; V < 12; ++V)
      if (first_support(T, str_type(TabHolder::value.J[B][V]))) {
        a.B[a.n] = B;
        a.V[a.n] = V;
        ++a.n;
      }
  return a;
}
template <int T>
struct AbFirstHolder {
  static constexpr AbFirst<T> value = make_ab_first<T>();
};
template <int T, int... I>
__device__ __forceinline__ void ab_first_terms(std::integer_sequence<int, I...>, float (&acc)[20], const float (&wr)[36],
                                               const float (&cr)[20]) {
  (ab_term<AbFirstHolder<T>::value.B[I], AbFirstHolder<T>::value.V[I]>(acc, wr, cr), ...);
}
struct AaFirst {
  int J[117], b[117], n;
};
__host__ __device__ constexpr AaFirst make_aa_first() {
  AaFirst a{};
  a.n = 0;
  for (int b = 0; b < 20; ++b)
    for (int J = 0; J < 20; ++J)
      if (first_support(str_type(J), str_type(b))) {
        a.J[a.n] = J;
        a.b[a.n] = b;
        ++a.n;
      }
  return a;
}
struct AaFirstHolder {
  static constexpr AaFirst value = make_aa_first();
};
static_assert(AbFirstHolder<0>::value.n == 216 && AbFirstHolder<1>::value.n == 120 && AbFirstHolder<2>::value.n == 12 &&
                  AaFirstHolder::value.n == 117,
              "first-vector product lists");
template <int... I>
__device__ __forceinline__ void aa_first_terms(std::integer_sequence<int, I...>, float (&acc)[20], const float (&h)[20],
                                               const float* __restrict__ c) {
  ((acc[AaFirstHolder::value.b[I]] =
        fmaf(h[AaFirstHolder::value.J[I]], c[AaFirstHolder::value.J[I] * 20 + AaFirstHolder::value.b[I]],
             acc[AaFirstHolder::value.b[I]])),
   ...);
}

// ---- shared memory -------------------------------------------------------------------------

template <int K>
struct Tabs {  // run-time string tables of one size class (bytes: they share the SM with warps)
  using D = Dim<K>;
  signed char J[D::NS * D::NSG];
  signed char pq[D::NS * D::NSG];
  signed char sg[D::NS * D::NSG];
  signed char mask[D::NS];
  signed char occ[D::NS][K];   // orbitals of each string, ascending
  signed char c0n[D::NS];      // replacements (pq) with <I| E_pq |Phi string> != 0 (<= K of them)
  signed char c0pq[D::NS][K];
  signed char c0sg[D::NS][K];
  signed char xJ[K * K];       // a+_A a_i |Phi string> = xs * |xJ>, index i*K + (A-K)
  signed char xs[K * K];
};

// Set-up data of one space (gather, fold); dead once the Davidson loop has more than two
// vectors, so the 6e6o state keeps it in its third vector slot.
template <int K>
struct SetupF32 {
  using D = Dim<K>;
  float F[D::NF];     // F block
  float hd[D::NORB];  // folded one-body diagonal h_pp
};

__device__ __forceinline__ float wsum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---- precision of the Rayleigh-Ritz step -----------------------------------------------------
// The projected matrix, the Gram-Schmidt coefficients and the Ritz value are kept to FP64
// accuracy as double-float pairs (hi + lo, two FP32 numbers, a 48-bit significand): on this GPU a
// native FP64 instruction occupies the SM's FP64 pipe for about 19 cycles whether one lane or all
// 32 use it, so FP64 arithmetic inside the per-space loop would cost more than the sigma-vectors.
// Inner products of the FP32 vectors are formed as error-free FP32 products summed with
// compensated additions (each lane, then across the warp), and the projected root is refined by
// a Newton step in double-float arithmetic; the energy is E0 + hi + lo in FP64.
struct DF {
  float hi, lo;
};

__device__ __forceinline__ DF df_norm(float a, float b) {  // |a| >= |b| or a = 0: exact renormalisation
  const float s = __fadd_rn(a, b);
  return DF{s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ DF two_sum(float a, float b) {  // a + b = hi + lo exactly
  const float s = __fadd_rn(a, b);
  const float z = __fsub_rn(s, a);
  return DF{s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z))};
}
__device__ __forceinline__ DF df_add(DF x, DF y) {
  const DF s = two_sum(x.hi, y.hi);
  return df_norm(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}
__device__ __forceinline__ DF df_neg(DF x) { return DF{-x.hi, -x.lo}; }
__device__ __forceinline__ DF df_mul(DF x, DF y) {
  const float p = __fmul_rn(x.hi, y.hi);
  const float e = __fmaf_rn(x.hi, y.hi, -p);  // x.hi y.hi = p + e exactly
  return df_norm(p, __fadd_rn(e, __fadd_rn(__fmul_rn(x.hi, y.lo), __fmul_rn(x.lo, y.hi))));
}
__device__ __forceinline__ DF df_mulf(DF x, float y) { return df_mul(x, DF{y, 0.f}); }
__device__ __forceinline__ float df_f(DF x) { return __fadd_rn(x.hi, x.lo); }

// Per-lane sum of products a b, exact products and compensated sums; total() adds the lanes'
// pairs the same way (every lane gets the same pair: each step's exact error term does not
// depend on the order of its two operands).
struct RRAcc {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float a, float b) {
    const float p = __fmul_rn(a, b);
    const float e = __fmaf_rn(a, b, -p);  // a b = p + e exactly
    const DF s = two_sum(hi, p);
    hi = s.hi;
    lo = __fadd_rn(lo, __fadd_rn(s.lo, e));
  }
  __device__ __forceinline__ DF total() const {
    float h = hi, l = lo;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float h2 = __shfl_xor_sync(0xffffffffu, h, o), l2 = __shfl_xor_sync(0xffffffffu, l, o);
      const DF s = two_sum(h, h2);
      h = s.hi;
      l = __fadd_rn(__fadd_rn(l, l2), s.lo);
    }
    return df_norm(h, l);
  }
};

template <int K>
struct alignas(16) WarpState {  // 16-byte rows: the 6e6o sigma reads them as float4
  using D = Dim<K>;
  float V[(KM - 1) * D::NDET];  // V_1 .. V_{KM-1}; V_0 = Phi is implicit (Phi stays in the subspace)
  float S[KM * D::NDET];        // S_j = sigma(V_j)
  // FP32 W block without its [pp][rr] (diagonal-only) entries, then h' = h - 1/2 sum_r W_prrq
  // (off-diagonal part): the coupling tables index both as one array
  float Wt[D::NW + D::NF];
  float Hs[D::NS * D::NS];  // same-spin string operator, zero diagonal
  float dh[(D::NS + 3) / 4 * 4];  // same-spin string diagonal relative to the Phi string
  float Jc[D::NF];          // J_pr = W_pprr: the alpha-beta Coulomb part of the diagonal
  float yf[KM];             // Ritz coefficients (FP32 for the vector updates)
  float j0;                 // sum_{p, r in Phi string} J_pr (FP32, diagonal reference)
  double eshift;             // <Phi|H|Phi> = E0 of the dressing (the fold leaves it unchanged)
  DF theta;                 // Ritz value relative to eshift
  DF G[KM * KM];            // projected matrix, G[i*KM+j] = V_i . S_j
  int orb[D::NORB];
  int ctrl[4];              // [0] subspace size, [1] valid, [2] status, [3] iterations
  // the small classes keep set-up data and gather offsets here (the 6e6o state keeps them in
  // the string operator's slot and the second S slot, which are free until they are filled)
  alignas(16) unsigned char extra[K == 3 ? 16 : sizeof(SetupF32<K>) + 2 * D::NF * sizeof(long long)];
  __device__ __forceinline__ float* hp() { return Wt + D::NW; }
  __device__ __forceinline__ const float* hp() const { return Wt + D::NW; }
};

template <int K>
__device__ __forceinline__ SetupF32<K>& setup(WarpState<K>& ws) {
  if constexpr (K == 3) return *reinterpret_cast<SetupF32<K>*>(ws.Hs);
  else return *reinterpret_cast<SetupF32<K>*>(ws.extra);
}
// gather offsets: element (P, R) of the W block sits at off[P] + off[NF + R]
template <int K>
__device__ __forceinline__ long long* gather_off(WarpState<K>& ws) {
  if constexpr (K == 3) return reinterpret_cast<long long*>(ws.S + Dim<K>::NDET);
  else return reinterpret_cast<long long*>(ws.extra + sizeof(SetupF32<K>));
}
static_assert(KM == 3 && sizeof(SetupF32<3>) <= sizeof(WarpState<3>::Hs) &&
                  2 * Dim<3>::NF * sizeof(long long) <= Dim<3>::NDET * sizeof(float),
              "set-up data must fit the reused 6e6o slots");

union alignas(16) AnyWarpState {
  WarpState<3> w3;
  WarpState<2> w2;
  WarpState<1> w1;
};

// Shared memory of a CTA: the string tables, then one AnyWarpState per warp.
struct alignas(16) CtaTabs {
  Tabs<3> t3;
  Tabs<2> t2;
  Tabs<1> t1;
  unsigned short pair3[Dim<3>::NPAIR];  // (P, R) with P <= R, packed P | R << 8
};
constexpr size_t kTabsBytes = (sizeof(CtaTabs) + 15) / 16 * 16;
__host__ __device__ constexpr size_t cta_smem_bytes(int warps) { return kTabsBytes + (size_t)warps * sizeof(AnyWarpState); }

static_assert(sizeof(WarpState<3>) % 16 == 0 && offsetof(WarpState<3>, S) % 16 == 0 &&
                  offsetof(WarpState<3>, Wt) % 16 == 0 && offsetof(WarpState<3>, Hs) % 16 == 0 &&
                  offsetof(WarpState<3>, dh) % 16 == 0 && offsetof(WarpState<3>, Jc) % 16 == 0 &&
                  (2 * Dim<3>::NDET * sizeof(float)) % 16 == 0,
              "float4 rows of the 6e6o state");
static_assert(kTabsBytes % 16 == 0 && sizeof(AnyWarpState) % 16 == 0, "warp state alignment");
static_assert(cta_smem_bytes(kMaxWarps) <= 232448, "one CTA within the 227 KB of shared memory a block may use");

// Entries of the 6e6o coupling tables (read-only global data, cached on the SM).  A per-CTA
// shared-memory copy was measured slower: it costs one of the 15 warps an SM holds.
__device__ __forceinline__ unsigned phi_entry(const CtaTabs&, int i) { return __ldg(&g_phi_table.e[i]); }
__device__ __forceinline__ unsigned hs_entry(const CtaTabs&, int i) { return __ldg(&g_hs_table.e[i]); }

template <int K>
__device__ Tabs<K>& tabs(CtaTabs& cs);
template <>
__device__ __forceinline__ Tabs<3>& tabs<3>(CtaTabs& cs) { return cs.t3; }
template <>
__device__ __forceinline__ Tabs<2>& tabs<2>(CtaTabs& cs) { return cs.t2; }
template <>
__device__ __forceinline__ Tabs<1>& tabs<1>(CtaTabs& cs) { return cs.t1; }

template <int K>
__device__ WarpState<K>& state(AnyWarpState& a);
template <>
__device__ __forceinline__ WarpState<3>& state<3>(AnyWarpState& a) { return a.w3; }
template <>
__device__ __forceinline__ WarpState<2>& state<2>(AnyWarpState& a) { return a.w2; }
template <>
__device__ __forceinline__ WarpState<1>& state<1>(AnyWarpState& a) { return a.w1; }

// Operator diagonal at determinant (ia, ib) relative to <Phi|H|Phi> (exactly 0 at Phi).
template <int K>
__device__ __forceinline__ float diag_at(const Tabs<K>& tb, const WarpState<K>& ws, int ia, int ib) {
  constexpr int NS = Dim<K>::NS;
  constexpr int NORB = Dim<K>::NORB;
  float jj = 0.f;
#pragma unroll
  for (int l = 0; l < K; ++l) {
    const float* row = ws.Jc + tb.occ[ia][l] * NORB;
#pragma unroll
    for (int m = 0; m < K; ++m) jj += row[tb.occ[ib][m]];
  }
  (void)NS;
  return ws.dh[ia] + ws.dh[ib] + (jj - ws.j0);
}

// String tables of one class (single thread): strings by increasing bit mask (string 0 holds
// the occupied orbitals), single replacements into each string, connections to the Phi string
// and the single replacements i -> A of the Phi string.
template <int K>
__device__ void build_tabs(Tabs<K>& t) {
  using D = Dim<K>;
  int c = 0;
  for (int m = 0; m < (1 << D::NORB); ++m)
    if (__popc(m) == K) t.mask[c++] = m;
  for (int I = 0; I < D::NS; ++I) {
    int j = 0;
    for (int p = 0; p < D::NORB; ++p)
      if ((t.mask[I] >> p) & 1) t.occ[I][j++] = (signed char)p;
  }
  for (int I = 0; I < D::NS; ++I) {
    const int mi = t.mask[I];
    int u = 0;
    for (int p = 0; p < D::NORB; ++p) {
      if (!((mi >> p) & 1)) continue;
      for (int q = 0; q < D::NORB; ++q) {
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
        for (int x = 0; x < D::NS; ++x)
          if (t.mask[x] == mj) J = x;
        t.J[I * D::NSG + u] = J;
        t.pq[I * D::NSG + u] = p * D::NORB + q;
        t.sg[I * D::NSG + u] = sgn;
        ++u;
      }
    }
  }
  for (int I = 0; I < D::NS; ++I) {
    int n0 = 0;
    for (int u = 0; u < D::NSG; ++u)
      if (t.J[I * D::NSG + u] == 0 && n0 < K) {
        t.c0pq[I][n0] = t.pq[I * D::NSG + u];
        t.c0sg[I][n0] = t.sg[I * D::NSG + u];
        ++n0;
      }
    t.c0n[I] = n0;
  }
  for (int x = 0; x < K * K; ++x) {
    const int i = x / K, A = K + x % K, m0 = t.mask[0];
    int par = __popc(m0 & ((1 << i) - 1)) & 1;
    const int m1 = m0 & ~(1 << i);
    par ^= __popc(m1 & ((1 << A) - 1)) & 1;
    int J = 0;
    for (int q = 0; q < D::NS; ++q)
      if (t.mask[q] == (m1 | (1 << A))) J = q;
    t.xJ[x] = J;
    t.xs[x] = par ? -1 : 1;
  }
}

__device__ void build_all_tabs(CtaTabs& cs) {
  if (threadIdx.x == 0) build_tabs<3>(cs.t3);
  if (threadIdx.x == 32) build_tabs<2>(cs.t2);
  if (threadIdx.x == 64) build_tabs<1>(cs.t1);
  if (threadIdx.x == 96) {
    int t = 0;
    for (int P = 0; P < Dim<3>::NF; ++P)
      for (int R = P; R < Dim<3>::NF; ++R) cs.pair3[t++] = (unsigned short)(P | (R << 8));
  }
  __syncthreads();
}

// ---- sigma ------------------------------------------------------------------------------------

// jab[B] = sum_{r in string B} jp[r] (string B's orbitals from the compile-time tables).
template <int B>
__device__ __forceinline__ float coulomb_row(const float (&jp)[6]) {
  constexpr int m = TabHolder::value.mask[B];
  float v = 0.f;
  if constexpr (m & 1) v += jp[0];
  if constexpr (m & 2) v += jp[1];
  if constexpr (m & 4) v += jp[2];
  if constexpr (m & 8) v += jp[3];
  if constexpr (m & 16) v += jp[4];
  if constexpr (m & 32) v += jp[5];
  return v;
}
template <int... B>
__device__ __forceinline__ void coulomb_rows(std::integer_sequence<int, B...>, float (&jab)[20], const float (&jp)[6]) {
  ((jab[B] = coulomb_row<B>(jp)), ...);
}

// 6e6o: sigma = H c restricted to off-diagonal couplings plus the shifted diagonal.
__device__ __noinline__ void sigma33(const Tabs<3>& tb, const WarpState<3>& ws, const float* __restrict__ c,
                                     float* __restrict__ out, int lane) {
  constexpr int NS = 20, NSG = 12, NF = 36;
  constexpr int kSplit = 8;  // alpha-beta: lanes < 20 take replacements [0, 8) of their string
  float acc[NS];
#pragma unroll
  for (int b = 0; b < NS; ++b) acc[b] = 0.f;
  if (lane < NS) {
    const int Ia = lane;
    constexpr unsigned kRows = (1u << NS) - 1u;  // lanes 0..19
    // alpha-alpha: A[Ia][b] = sum_J Hs[Ia][J] c[J][b].  The vectors are symmetric under the spin
    // flip (c[a][b] = c[b][a]: Phi is, and the spin-free operator commutes with the flip), so the
    // beta-beta part is A^T: row Ia of A goes through `out` and comes back as column Ia.
#pragma unroll 4
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
    {
      float4* orow = reinterpret_cast<float4*>(out + Ia * NS);
#pragma unroll
      for (int q = 0; q < NS / 4; ++q) orow[q] = make_float4(acc[4 * q], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3]);
    }
    __syncwarp(kRows);
    {  // + A^T and the diagonal: diag(Ia, b) = dh[Ia] + dh[b] + (sum_{p in Ia, r in b} J_pr - j0),
       // as diag_at, with jp[r] = sum_{p in Ia} J_pr in registers and b's orbitals at compile time
      float jp[6];
#pragma unroll
      for (int r = 0; r < 6; ++r)
        jp[r] = ws.Jc[tb.occ[Ia][0] * 6 + r] + ws.Jc[tb.occ[Ia][1] * 6 + r] + ws.Jc[tb.occ[Ia][2] * 6 + r];
      float jab[NS];
      coulomb_rows(std::make_integer_sequence<int, NS>{}, jab, jp);
      const float4* dhr = reinterpret_cast<const float4*>(ws.dh);
      const float4* crow = reinterpret_cast<const float4*>(c + Ia * NS);
      const float dha = ws.dh[Ia], jz = ws.j0;
#pragma unroll
      for (int q = 0; q < NS / 4; ++q) {
        const float4 dv = dhr[q], cv = crow[q];
        acc[4 * q + 0] += out[(4 * q + 0) * NS + Ia] + (dha + dv.x + (jab[4 * q + 0] - jz)) * cv.x;
        acc[4 * q + 1] += out[(4 * q + 1) * NS + Ia] + (dha + dv.y + (jab[4 * q + 1] - jz)) * cv.y;
        acc[4 * q + 2] += out[(4 * q + 2) * NS + Ia] + (dha + dv.z + (jab[4 * q + 2] - jz)) * cv.z;
        acc[4 * q + 3] += out[(4 * q + 3) * NS + Ia] + (dha + dv.w + (jab[4 * q + 3] - jz)) * cv.w;
      }
    }
  }
  __syncwarp();  // every column of out read before lanes write rows of it again
  // alpha-beta: the 12 replacements into each string Ia, register tiles of W and C rows, on all
  // 32 lanes: lane Ia < 20 takes replacements [0, 8) of string Ia into its row; lane 20 + j takes
  // replacements [8, 12) of string j (first) and of string 12 + j (then, for j < 8), and passes
  // each partial row to its owner through `out` (row Ia is written by exactly one such lane).
  const int j = lane - NS;
  auto flush = [&](int row) {
    float4* orow = reinterpret_cast<float4*>(out + row * NS);
#pragma unroll
    for (int q = 0; q < NS / 4; ++q) orow[q] = make_float4(acc[4 * q], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3]);
#pragma unroll
    for (int b = 0; b < NS; ++b) acc[b] = 0.f;
  };
#pragma unroll 1
  for (int it = 0; it < kSplit; ++it) {
    int Ia = lane, u = it;
    if (lane >= NS) {
      if (it == NSG - kSplit) flush(j);  // the first string's partial row is complete
      Ia = (it < NSG - kSplit) ? j : ((j < NS - NSG) ? NSG + j : 0);  // lanes 28..31: unused second pass
      u = kSplit + (it % (NSG - kSplit));
    }
    const int e = Ia * NSG + u;
    const int pq = tb.pq[e], Ja = tb.J[e];
    const float su = (float)tb.sg[e];
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
  if (lane >= NS && j < NS - NSG) flush(NSG + j);  // second string's partial row (lanes 20..27)
  __syncwarp();
  if (lane < NS) {  // own row + the partial row of replacements [8, 12)
    float4* orow = reinterpret_cast<float4*>(out + lane * NS);
#pragma unroll
    for (int q = 0; q < NS / 4; ++q) {
      const float4 v = orow[q];
      orow[q] = make_float4(acc[4 * q] + v.x, acc[4 * q + 1] + v.y, acc[4 * q + 2] + v.z, acc[4 * q + 3] + v.w);
    }
  }
  __syncwarp();
}

// sigma of the first expansion vector (c on the Phi column's support, spin-flip symmetric): the
// same terms as sigma33 with the products against c's zeros left out (see AbFirst / FirstSched).
// scratch: 480 floats the call may overwrite (the second vector slot and the third sigma slot,
// unused until sigma of the second vector).
__device__ __noinline__ void sigma33_first(const Tabs<3>& tb, const WarpState<3>& ws, const float* __restrict__ c,
                                           float* __restrict__ out, float* __restrict__ scr_a,
                                           float* __restrict__ scr_b, int lane) {
  constexpr int NS = 20, NF = 36;
  // this lane's schedule, loaded up front (its latency runs under the alpha-alpha part)
  int ent[kFirstSteps];
#pragma unroll
  for (int k = 0; k < kFirstSteps; ++k) ent[k] = (int)__ldg(&g_first.e[k][lane]);
  int hsl[3] = {-1, -1, -1}, rsl[4] = {0, 0, 0, 0}, rcnt = 0;
  if (lane >= NS) {
#pragma unroll
    for (int ph = 0; ph < 3; ++ph) hsl[ph] = (int)__ldg(&g_first.hslot[ph][lane - NS]);
  } else {
    rcnt = (int)__ldg(&g_first.rcount[lane]);
#pragma unroll
    for (int i = 0; i < 4; ++i) rsl[i] = (int)__ldg(&g_first.rslot[lane][i]);
  }
  float acc[NS];
#pragma unroll
  for (int b = 0; b < NS; ++b) acc[b] = 0.f;
  if (lane < NS) {
    const int Ia = lane;
    constexpr unsigned kRows = (1u << NS) - 1u;
    // alpha-alpha: A[Ia][b] = sum_J Hs[Ia][J] c[J][b] over c's support (J ascending per b, as the
    // dense product adds them), then A^T and the diagonal as in sigma33
    float h[NS];
    {
      const float4* hr = reinterpret_cast<const float4*>(ws.Hs + Ia * NS);
#pragma unroll
      for (int q = 0; q < NS / 4; ++q) {
        const float4 v = hr[q];
        h[4 * q] = v.x;
        h[4 * q + 1] = v.y;
        h[4 * q + 2] = v.z;
        h[4 * q + 3] = v.w;
      }
    }
    aa_first_terms(std::make_integer_sequence<int, 117>{}, acc, h, c);
    {
      float4* orow = reinterpret_cast<float4*>(out + Ia * NS);
#pragma unroll
      for (int q = 0; q < NS / 4; ++q) orow[q] = make_float4(acc[4 * q], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3]);
    }
    __syncwarp(kRows);
    {
      float jp[6];
#pragma unroll
      for (int r = 0; r < 6; ++r)
        jp[r] = ws.Jc[tb.occ[Ia][0] * 6 + r] + ws.Jc[tb.occ[Ia][1] * 6 + r] + ws.Jc[tb.occ[Ia][2] * 6 + r];
      float jab[NS];
      coulomb_rows(std::make_integer_sequence<int, NS>{}, jab, jp);
      const float4* dhr = reinterpret_cast<const float4*>(ws.dh);
      const float4* crow = reinterpret_cast<const float4*>(c + Ia * NS);
      const float dha = ws.dh[Ia], jz = ws.j0;
#pragma unroll
      for (int q = 0; q < NS / 4; ++q) {
        const float4 dv = dhr[q], cv = crow[q];
        acc[4 * q + 0] += out[(4 * q + 0) * NS + Ia] + (dha + dv.x + (jab[4 * q + 0] - jz)) * cv.x;
        acc[4 * q + 1] += out[(4 * q + 1) * NS + Ia] + (dha + dv.y + (jab[4 * q + 1] - jz)) * cv.y;
        acc[4 * q + 2] += out[(4 * q + 2) * NS + Ia] + (dha + dv.z + (jab[4 * q + 2] - jz)) * cv.z;
        acc[4 * q + 3] += out[(4 * q + 3) * NS + Ia] + (dha + dv.w + (jab[4 * q + 3] - jz)) * cv.w;
      }
    }
  }
  __syncwarp();  // every column of out read before rows are written again
  // alpha-beta over the compile-time schedule: one step adds the products of one (row, source)
  // pair; a helper lane (20..31) hands its partial row to a scratch slot at the end of a phase
  auto slot_ptr = [&](int sl) { return sl < 20 ? scr_a + sl * NS : scr_b + (sl - 20) * NS; };
  auto step = [&](auto type_tag, int e) {
    constexpr int T = decltype(type_tag)::value;
    if (e < 0) return;
    const int x = (e >> 4) * 12 + (e & 15);
    const int pq = tb.pq[x], Ja = tb.J[x];
    const float su = (float)tb.sg[x];
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
    ab_first_terms<T>(std::make_integer_sequence<int, AbFirstHolder<T>::value.n>{}, acc, wr, cr);
  };
  auto flush = [&](int sl) {  // helpers: the phase's partial row to its slot
    if (lane < NS || sl < 0) return;
    float4* orow = reinterpret_cast<float4*>(slot_ptr(sl));
#pragma unroll
    for (int q = 0; q < NS / 4; ++q) orow[q] = make_float4(acc[4 * q], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3]);
#pragma unroll
    for (int b = 0; b < NS; ++b) acc[b] = 0.f;
  };
  // one body per step type (a rolled loop: the kernel's hot code stays small), the lane's entry
  // for step k selected from its registers
  auto entry = [&](int k) {
    int e = ent[0];
#pragma unroll
    for (int j = 1; j < kFirstSteps; ++j) e = (k == j) ? ent[j] : e;
    return e;
  };
  step(std::integral_constant<int, 0>{}, ent[0]);
  flush(hsl[0]);
#pragma unroll 1
  for (int k = 1; k < 5; ++k) step(std::integral_constant<int, 1>{}, entry(k));
  flush(hsl[1]);
#pragma unroll 1
  for (int k = 5; k < 9; ++k) step(std::integral_constant<int, 2>{}, entry(k));
  flush(hsl[2]);
  __syncwarp();
  if (lane < NS) {  // own row + the helpers' partial rows, in slot order
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if (i >= rcnt) break;
      const float4* prow = reinterpret_cast<const float4*>(slot_ptr(rsl[i]));
#pragma unroll
      for (int q = 0; q < NS / 4; ++q) {
        const float4 v = prow[q];
        acc[4 * q] += v.x;
        acc[4 * q + 1] += v.y;
        acc[4 * q + 2] += v.z;
        acc[4 * q + 3] += v.w;
      }
    }
    float4* orow = reinterpret_cast<float4*>(out + lane * NS);
#pragma unroll
    for (int q = 0; q < NS / 4; ++q) orow[q] = make_float4(acc[4 * q], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3]);
  }
  __syncwarp();
}

// 2e2o / 4e4o: one determinant per lane (at most 36 determinants).
template <int K>
__device__ __noinline__ void sigma_small(const Tabs<K>& tb, const WarpState<K>& ws, const float* __restrict__ c,
                                         float* __restrict__ out, int lane) {
  using D = Dim<K>;
  for (int d = lane; d < D::NDET; d += 32) {
    const int ia = d / D::NS, ib = d % D::NS;
    float acc = diag_at<K>(tb, ws, ia, ib) * c[d];
    for (int j = 0; j < D::NS; ++j) {
      acc = fmaf(ws.Hs[ia * D::NS + j], c[j * D::NS + ib], acc);
      acc = fmaf(ws.Hs[ib * D::NS + j], c[ia * D::NS + j], acc);
    }
    for (int u = 0; u < D::NSG; ++u) {
      const int e = ia * D::NSG + u;
      const float* wrow = ws.Wt + tb.pq[e] * D::NF;
      const float* crow = c + tb.J[e] * D::NS;
      float part = 0.f;
      for (int v = 0; v < D::NSG; ++v) {
        const int e2 = ib * D::NSG + v;
        part = fmaf((float)tb.sg[e2] * wrow[tb.pq[e2]], crow[tb.J[e2]], part);
      }
      acc = fmaf((float)tb.sg[e], part, acc);
    }
    out[d] = acc;
  }
  __syncwarp();
}

template <int K>
__device__ __forceinline__ void sigma(const Tabs<K>& tb, const WarpState<K>& ws, const float* c, float* out, int lane) {
  if constexpr (K == 3) sigma33(tb, ws, c, out, lane);
  else sigma_small<K>(tb, ws, c, out, lane);
}

// Imaginary part above which a projected root counts as complex (FP32 closed forms resolve the
// real part of a near-degenerate real pair to about 1e-7 of the matrix scale).
constexpr float kImagMin = 1e-5f;

// Phi-dominant eigenpair of the k x k projected matrix (lane 0).  The subspace basis is Phi
// (component 0 of every other basis vector is exactly zero), so the Phi weight of a Ritz vector
// with coefficients y is |y_0| / |y|: of the real roots, the one with the largest Phi weight is
// taken (the space's root is the eigenvector with the largest |c_Phi|); shifted inverse
// iteration from `shift` is the fallback when the closed forms fail.  Returns 1 when a complex
// pair carries more Phi weight than every real root (the real candidate is still returned),
// else 0.  The closed forms run in FP32 on the rounded double-float matrix; `theta` is the
// previous root (the fallback's second shift).  G and y are the warp state's (shared memory),
// the root comes back by value, so lane 0 makes no local-memory round trips here.
struct EigOut {
  float theta;
  int cx;
};
__device__ __noinline__ EigOut small_eig(const DF* Gd, int k, float shift, float theta, float* y) {
  int cx = 0;
  auto G = [Gd](int i) { return df_f(Gd[i]); };
  // The closed forms below lose absolute accuracy to cancellation (the root sought is small next
  // to the other diagonal entries).  The chosen root is therefore polished with the Phi row of
  // G y = lambda y, lambda = (G y)_0 / y_0 (exact for an eigenpair; G_00 = Phi . sigma(Phi)),
  // alternating with the eigenvector twice: the error shrinks by about |G_0j| / gap per pass.
  if (k == 2) {
    const float g00 = G(0), g01 = G(1), g10 = G(KM), g11 = G(KM + 1);
    const float tr = 0.5f * (g00 + g11), df = 0.5f * (g00 - g11);
    const float disc = df * df + g01 * g10;
    // eigenvector of G for root lam: the better conditioned of the two rows of (G - lam) y = 0
    auto vec2 = [&](float lam, float* y0, float* y1) {
      if (fabsf(g01) + fabsf(lam - g00) >= fabsf(g10) + fabsf(lam - g11)) {
        *y0 = g01;
        *y1 = lam - g00;
      } else {
        *y0 = lam - g11;
        *y1 = g10;
      }
    };
    if (disc < 0.f && sqrtf(-disc) > kImagMin * fmaxf(1.f, fabsf(tr))) cx = 1;  // no real root
    if (disc >= 0.f && isfinite(disc)) {
      const float sq = sqrtf(disc);
      float lam = tr + sq;
      {  // the root with the larger Phi weight
        float a0, a1, b0, b1;
        vec2(tr + sq, &a0, &a1);
        vec2(tr - sq, &b0, &b1);
        const float wa = a0 * a0 / fmaxf(a0 * a0 + a1 * a1, 1e-30f), wb = b0 * b0 / fmaxf(b0 * b0 + b1 * b1, 1e-30f);
        if (wb > wa) lam = tr - sq;
      }
      float y0 = 0.f, y1 = 0.f;
      for (int pass = 0; pass < 3; ++pass) {
        vec2(lam, &y0, &y1);
        if (pass == 2 || !(fabsf(y0) >= 0.3f * sqrtf(y0 * y0 + y1 * y1))) break;
        lam = (g00 * y0 + g01 * y1) / y0;
      }
      const float nrm = sqrtf(y0 * y0 + y1 * y1);
      if (nrm > 0.f && isfinite(nrm) && isfinite(lam)) {
        const float sc = ((y0 < 0.f) ? -1.f : 1.f) / nrm;
        y[0] = sc * y0;
        y[1] = sc * y1;
        return EigOut{lam, cx};
      }
    }
  }
  if (k == 3) {  // roots of the characteristic cubic; eigenvectors from cross products
    const float g00 = G(0), g01 = G(1), g02 = G(2), g10 = G(KM), g11 = G(KM + 1), g12 = G(KM + 2);
    const float g20 = G(2 * KM), g21 = G(2 * KM + 1), g22 = G(2 * KM + 2);
    auto cross = [](const float* u, const float* w, float* o) {
      o[0] = u[1] * w[2] - u[2] * w[1];
      o[1] = u[2] * w[0] - u[0] * w[2];
      o[2] = u[0] * w[1] - u[1] * w[0];
    };
    // null vector of G - lam I (the largest cross product of two of its rows) and its norm^2
    auto vec3 = [&](float lam, float* vb) {
      const float r0[3] = {g00 - lam, g01, g02}, r1[3] = {g10, g11 - lam, g12}, r2[3] = {g20, g21, g22 - lam};
      float c01[3], c02[3], c12[3];
      cross(r0, r1, c01);
      cross(r0, r2, c02);
      cross(r1, r2, c12);
      const float n01 = c01[0] * c01[0] + c01[1] * c01[1] + c01[2] * c01[2];
      const float n02 = c02[0] * c02[0] + c02[1] * c02[1] + c02[2] * c02[2];
      const float n12 = c12[0] * c12[0] + c12[1] * c12[1] + c12[2] * c12[2];
      const float* best = c01;
      float nb = n01;
      if (n02 > nb) { best = c02; nb = n02; }
      if (n12 > nb) { best = c12; nb = n12; }
      vb[0] = best[0];
      vb[1] = best[1];
      vb[2] = best[2];
      return nb;
    };
    // det(lambda I - G) = lambda^3 + a2 lambda^2 + a1 lambda + a0
    const float a2 = -(g00 + g11 + g22);
    const float a1 = g00 * g11 - g01 * g10 + g00 * g22 - g02 * g20 + g11 * g22 - g12 * g21;
    const float a0 = -(g00 * (g11 * g22 - g12 * g21) - g01 * (g10 * g22 - g12 * g20) + g02 * (g10 * g21 - g11 * g20));
    // lambda = mu - a2 / 3:  mu^3 + p mu + q = 0
    const float p = a1 - a2 * a2 / 3.f, q = 2.f * a2 * a2 * a2 / 27.f - a2 * a1 / 3.f + a0;
    float root[3];
    int nr = 0;
    float cre = 0.f, cim = 0.f;  // complex pair re +- i im (one-real-root case)
    const float disc = q * q / 4.f + p * p * p / 27.f;
    if (disc < 0.f && p < 0.f) {  // three real roots (trigonometric form)
      const float m = 2.f * sqrtf(-p / 3.f);
      float c = 3.f * q / (p * m);
      c = fminf(1.f, fmaxf(-1.f, c));
      const float phi = acosf(c) / 3.f;
      for (int j = 0; j < 3; ++j) root[nr++] = m * cosf(phi - 2.0943951f * (float)j) - a2 / 3.f;
    } else {  // one real root
      const float sq = sqrtf(fmaxf(disc, 0.f));
      const float u = cbrtf(-q / 2.f + sq), v = cbrtf(-q / 2.f - sq);
      root[nr++] = u + v - a2 / 3.f;
      // the other two roots: -(u + v) / 2 - a2 / 3 +- i sqrt(3) / 2 (u - v)
      cre = -0.5f * (u + v) - a2 / 3.f;
      cim = 0.8660254f * fabsf(u - v);
    }
    float lam = root[0], wbest = -1.f;
    for (int j = 0; j < nr; ++j) {  // the real root with the largest Phi weight
      float vb[3];
      const float nb = vec3(root[j], vb);
      const float w = vb[0] * vb[0] / fmaxf(nb, 1e-30f);
      if (w > wbest) {
        wbest = w;
        lam = root[j];
      }
    }
    if (nr == 1 && cim > kImagMin * fmaxf(1.f, fabsf(cre))) {
      // Phi weight of the complex pair's eigenvector: cross product of rows 0 and 1 of G - z I,
      // z = cre + i cim (the pair's weights are equal), in real and imaginary parts
      const float ar = g00 - cre, br = g11 - cre, ci = -cim;  // diagonal entries: (ar + i ci), (br + i ci)
      // v0 = g01 g12 - g02 (g11 - z); v1 = g02 g10 - (g00 - z) g12; v2 = (g00 - z)(g11 - z) - g01 g10
      const float v0r = g01 * g12 - g02 * br, v0i = -g02 * ci;
      const float v1r = g02 * g10 - ar * g12, v1i = -ci * g12;
      const float v2r = ar * br - ci * ci - g01 * g10, v2i = ar * ci + ci * br;
      const float n2 = v0r * v0r + v0i * v0i + v1r * v1r + v1i * v1i + v2r * v2r + v2i * v2i;
      if (n2 > 0.f && (v0r * v0r + v0i * v0i) / n2 > wbest) cx = 1;
    }
    float vb[3] = {0.f, 0.f, 0.f}, nb = 0.f;
    for (int pass = 0; pass < 3; ++pass) {
      nb = vec3(lam, vb);
      if (pass == 2 || !(fabsf(vb[0]) >= 0.3f * sqrtf(nb))) break;
      lam = (g00 * vb[0] + g01 * vb[1] + g02 * vb[2]) / vb[0];
    }
    if (nb > 0.f && isfinite(nb) && isfinite(lam)) {
      const float sc = ((vb[0] < 0.f) ? -1.f : 1.f) / sqrtf(nb);
      y[0] = sc * vb[0];
      y[1] = sc * vb[1];
      y[2] = sc * vb[2];
      return EigOut{lam, cx};
    }
  }
  float a[KM * KM], z[KM];
  for (int phase = 0; phase < 5; ++phase) {
    const float sg = (phase < 2) ? shift : theta;
    for (int i = 0; i < k; ++i)
      for (int j = 0; j < k; ++j) a[i * KM + j] = G(i * KM + j) - ((i == j) ? sg : 0.f);
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
      for (int j = 0; j < k; ++j) gy += G(i * KM + j) * y[j];
      num += y[i] * gy;
    }
    theta = num;
  }
  return EigOut{theta, cx};
}

// The Phi-dominant eigenpair of the projected matrix to FP64 accuracy: the FP32 closed forms
// choose the root (and flag a complex one) and give its eigenvector (the coefficients scale FP32
// vectors); one Newton step on the characteristic polynomial of the double-float matrix, with the
// polynomial in double-float arithmetic and the FP32 derivative (the step is a small correction),
// refines the root.  A step that is not finite or moves the root by more than 1e-3 is dropped.
// G, y and theta are the warp state's (shared memory).
__device__ __noinline__ int small_eig_rr(const DF* G, int k, DF shift, float* y, DF* theta) {
  const EigOut r = small_eig(G, k, df_f(shift), df_f(*theta), y);
  const int cx = r.cx;
  const float th = r.theta;
  auto Gf = [G](int i) { return df_f(G[i]); };
  float delta = 0.f;
  const DF lam{th, 0.f};
  if (k == 2) {  // det(lam - G) = (lam - g00)(lam - g11) - g01 g10
    const DF a = df_add(lam, df_neg(G[0])), b = df_add(lam, df_neg(G[KM + 1]));
    const DF f = df_add(df_mul(a, b), df_neg(df_mul(G[1], G[KM])));
    const float fp = 2.f * th - Gf(0) - Gf(KM + 1);
    delta = -df_f(f) / fp;
  } else if (k == 3) {  // det(lam - G) by the rule of Sarrus on the double-float entries of lam - G
    DF m[9];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) m[i * 3 + j] = (i == j) ? df_add(lam, df_neg(G[i * KM + j])) : df_neg(G[i * KM + j]);
    auto t3 = [&](int a, int b, int c) { return df_mul(df_mul(m[a], m[b]), m[c]); };
    DF f = df_add(df_add(t3(0, 4, 8), t3(1, 5, 6)), t3(2, 3, 7));
    f = df_add(f, df_neg(df_add(df_add(t3(2, 4, 6), t3(0, 5, 7)), t3(1, 3, 8))));
    // d/dlam det(lam - G) = sum of the principal 2 x 2 minors of (lam - G), in FP32
    const float d00 = th - Gf(0), d11 = th - Gf(KM + 1), d22 = th - Gf(2 * KM + 2);
    const float fp = (d11 * d22 - Gf(KM + 2) * Gf(2 * KM + 1)) + (d00 * d22 - Gf(2) * Gf(2 * KM)) +
                     (d00 * d11 - Gf(1) * Gf(KM));
    delta = -df_f(f) / fp;
  }
  if (isfinite(delta) && fabsf(delta) <= 1e-3f * (1.f + fabsf(th)))
    *theta = two_sum(th, delta);
  else
    *theta = DF{th, 0.f};
  return cx;
}

// ---- one space -----------------------------------------------------------------------------------

// Solve space s of the class list in `a` (s: index in that list) with the warp's state `ws`.
template <int K>
__device__ void solve_one(const Tabs<K>& tb, const CtaTabs& cs, WarpState<K>& ws,
                          const SolveArgs& a, const float* __restrict__ W32, const float* __restrict__ guess_in,
                          float* __restrict__ guess_out, int64_t s, int lane) {
  using D = Dim<K>;
  constexpr int NS = D::NS, NSG = D::NSG, NDET = D::NDET, NORB = D::NORB, NF = D::NF;
  const unsigned short* __restrict__ pair3 = cs.pair3;
  const int n = a.n;
  const size_t n1 = (size_t)n, n2 = n1 * n1, n3 = n2 * n1;
  const float tol = (float)a.tol;
  // ---- validate -------------------------------------------------------------------------
  // (the sorted index and the owner flag are loaded beside the record: neither waits on it)
  const int64_t sidx = a.sorted_index ? a.sorted_index[s] : a.space_base + s;
  const int64_t oidx = a.sorted_index ? sidx : s;
  // only a space that owns an amplitude forms its increment (loaded here, used at the merge)
  const bool owner = !a.owns || a.owns[s] != 0;
  if (lane == 0) {
    const qflow_space& q = a.spaces[s];
    int ok = (q.no == K && q.nv == K), same = (K == 3);
    for (int t = 0; t < NORB; ++t) {
      const int o = q.orb[t];
      if (t < NORB - 1) same &= (o == ws.orb[t]);
      ws.orb[t] = o;
      if (t < K) ok &= (o >= 0 && o < a.nocc);
      else ok &= (o >= a.nocc && o < a.n);
    }
    if (!ok) ws.orb[0] = -1;  // the W block below is not this record's: nothing to reuse next
    ws.ctrl[1] = ok;
    ws.ctrl[0] = same && ok;
  }
  __syncwarp();
  if (!ws.ctrl[1]) {
    if (lane == 0) {
      a.energy[oidx] = 0.0;
      a.status[oidx] = kSpaceInvalid;
      if (a.iters) a.iters[oidx] = 0;
    }
    __syncwarp();
    return;
  }
  // ---- gather ------------------------------------------------------------------------------
  // FP32 couplings (all loads in flight; the diagonal-only entries W_pprr are J_pr) and the F
  // block.  Element (P, R) of the W block is at off[P] + off[NF + R] (pair offsets built first).
  SetupF32<K>& su = setup(ws);
  {
    long long* off = gather_off(ws);
    for (int t = lane; t < 2 * NF; t += 32) {
      const int P = t % NF;
      const long long o0 = ws.orb[P / NORB], o1 = ws.orb[P % NORB];
      off[t] = (t < NF) ? o0 * (long long)n3 + o1 * (long long)n2 : o0 * (long long)n1 + o1;
    }
    __syncwarp();
    static_assert(NF <= 64, "two rounds of F");
    float f0 = 0.f, f1 = 0.f;
    if (lane < NF) {
      const size_t g = (size_t)ws.orb[lane / NORB] * n1 + ws.orb[lane % NORB];
      f0 = a.F32 ? a.F32[g] : (float)a.F[g];
    }
    if (lane + 32 < NF) {
      const size_t g = (size_t)ws.orb[(lane + 32) / NORB] * n1 + ws.orb[(lane + 32) % NORB];
      f1 = a.F32 ? a.F32[g] : (float)a.F[g];
    }
    if constexpr (K == 3) {  // the 666 unique elements of the pair-symmetric block
      // A space whose first five orbitals are those of this warp's previous space (consecutive
      // spaces of the sorted list differ in the last virtual) keeps the 325 elements without
      // orbital 5 from it: W_t and J_c still hold them.
      const bool reuse = ws.ctrl[0] != 0;
      constexpr int PER = (D::NPAIR + 31) / 32;
      float wv[PER];
#pragma unroll
      for (int k = 0; k < PER; ++k) {
        const int t = lane + 32 * k;
        wv[k] = 0.f;
        if (t < D::NPAIR) {
          const int pr = pair3[t], P = pr & 255, R = pr >> 8;
          if (!reuse || P % NORB == NORB - 1 || P >= NF - NORB || R % NORB == NORB - 1 || R >= NF - NORB) {
            const size_t g = (size_t)(off[P] + off[NF + R]);
            wv[k] = W32 ? W32[g] : (float)a.W[g];
          }
        }
      }
#pragma unroll
      for (int k = 0; k < PER; ++k) {
        const int t = lane + 32 * k;
        if (t < D::NPAIR) {
          const int pr = pair3[t], P = pr & 255, R = pr >> 8;
          if (!reuse || P % NORB == NORB - 1 || P >= NF - NORB || R % NORB == NORB - 1 || R >= NF - NORB) {
            const int p = P / NORB, r = R / NORB;
            const bool jj = (P == p * (NORB + 1)) && (R == r * (NORB + 1));  // W_pprr: diagonal only
            if (jj) {
              ws.Jc[p * NORB + r] = wv[k];
              ws.Jc[r * NORB + p] = wv[k];
            }
            const float wf = jj ? 0.f : wv[k];
            ws.Wt[P * NF + R] = wf;
            ws.Wt[R * NF + P] = wf;
          }
        }
      }
    } else {
      for (int t = lane; t < D::NW; t += 32) {
        const int P = t / NF, R = t % NF;
        const size_t g = (size_t)(off[P] + off[NF + R]);
        const int p = P / NORB, r = R / NORB;
        const bool jj = (P == p * (NORB + 1)) && (R == r * (NORB + 1));
        const float w = W32 ? W32[g] : (float)a.W[g];
        if (jj) ws.Jc[p * NORB + r] = w;
        ws.Wt[t] = jj ? 0.f : w;
      }
    }
    if (lane < NF) su.F[lane] = f0;
    if (lane + 32 < NF) su.F[lane + 32] = f1;
  }
  __syncwarp();
  // ---- fold (vacuum order over the active orbitals) -------------------------------------
  // h_pp = F_pp - sum_k (2 J_pk - K_pk) with K_pk = W_pkkp (J_pp for k = p); off-diagonal
  // h' = h - 1/2 sum_r W_prrq
  if (lane < NORB) {
    const int p = lane;
    float v = su.F[p * (NORB + 1)];
    for (int k = 0; k < K; ++k) {
      const float kx = (k == p) ? ws.Jc[p * NORB + p] : ws.Wt[(p * NORB + k) * NF + k * NORB + p];
      v -= 2.f * ws.Jc[p * NORB + k] - kx;
    }
    su.hd[p] = v;
  }
  for (int idx = lane; idx < NF; idx += 32) {
    const int p = idx / NORB, q = idx % NORB;
    float v = su.F[idx];
    for (int k = 0; k < K; ++k)
      v -= 2.f * ws.Wt[idx * NF + k * (NORB + 1)] - ws.Wt[(p * NORB + k) * NF + k * NORB + q];
    for (int r = 0; r < NORB; ++r) v -= 0.5f * ws.Wt[(p * NORB + r) * NF + r * NORB + q];
    ws.hp()[idx] = (p == q) ? 0.f : v;
  }
  __syncwarp();
  {  // same-spin string diagonal sum_{p in I} h_pp + sum_{p<r in I} (J_pr - K_pr), relative to Phi's
    float hs = 0.f;
    if (lane < NS) {
#pragma unroll
      for (int j = 0; j < K; ++j) {
        const int p = tb.occ[lane][j];
        hs += su.hd[p];
#pragma unroll
        for (int l = j + 1; l < K; ++l) {
          const int r = tb.occ[lane][l];
          hs += ws.Jc[p * NORB + r] - ws.Wt[(p * NORB + r) * NF + r * NORB + p];
        }
      }
    }
    const float hs0 = __shfl_sync(0xffffffffu, hs, 0);
    if (lane < NS) ws.dh[lane] = hs - hs0;
  }
  if (lane == 0) {
    ws.eshift = *a.e0;  // <Phi|H|Phi>: the fold moves the inactive part into E_core exactly
    ws.ctrl[0] = 1;
    ws.ctrl[1] = 0;  // from here on: consecutive steps whose projected root was complex
    ws.ctrl[2] = kSpaceNoConv;
    ws.ctrl[3] = 0;
    ws.theta = DF{0.f, 0.f};
    ws.G[0] = DF{0.f, 0.f};
    ws.yf[0] = 1.f;
  }
  __syncwarp();
  // ---- Phi fast path: sigma(Phi) = column 0 of H (0 at Phi after the shift) ----------------
  // Only determinants connected to Phi by single or double replacements are nonzero.  If the
  // residual of Phi is below the tolerance, the root is Phi, the increment is zero and the
  // space is done without building the full string operator.  Otherwise (and without a caller's
  // guess) the first-order correction r / (0 - diag) goes to V1: if its norm is below what FP32
  // vectors resolve (1e-6) the space stays at Phi (energy error below |r| * 1e-6), else it is
  // the first expansion vector of the Davidson loop.  A guess enters as a second subspace vector.
  float vn_phi = 0.f;
  {
    float rphi;
    unsigned pe[kPhiLen];  // this lane's Phi-table entries, kept for the first-order vector
    if constexpr (K == 3) {  // the column from its coupling table, each unique element once
#pragma unroll
      for (int k = 0; k < kPhiLen; ++k) pe[k] = phi_entry(cs, k * 32 + lane);
      const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
      for (int q = lane; q < NDET / 4; q += 32) {
        reinterpret_cast<float4*>(ws.S)[q] = z4;  // S0 = sigma(Phi)
        reinterpret_cast<float4*>(ws.V)[q] = z4;  // V1
      }
      __syncwarp();
      float acc = 0.f, rr = 0.f;
#pragma unroll
      for (int k = 0; k < kPhiLen; ++k) {
        const unsigned e = pe[k];
        acc = fmaf(__uint_as_float(e & 0xff800000u), ws.Wt[e & 2047u], acc);
        if (e & (1u << 20)) {
          const int d = (int)((e >> 11) & 511u);
          ws.S[d] = acc;
          float w2 = acc * acc;
          if (e & (1u << 21)) {
            ws.S[(d % NS) * NS + d / NS] = acc;
            w2 += w2;
          }
          rr += w2;
          acc = 0.f;
        }
      }
      rphi = sqrtf(wsum(rr));
      __syncwarp();
    } else {
      float hc = 0.f;  // Hs[I][0]: same-spin coupling of string I to the Phi string
      if (lane < NS && lane != 0) {
        const int I = lane;
#pragma unroll 1
        for (int u = 0; u < NSG; ++u) {
          const int e = I * NSG + u;
          const int pq = tb.pq[e], Kk = tb.J[e];
          const float s1 = (float)tb.sg[e];
          if (Kk == 0) hc = fmaf(s1, ws.hp()[pq], hc);
          for (int v = 0; v < tb.c0n[Kk]; ++v)
            hc = fmaf(0.5f * s1 * (float)tb.c0sg[Kk][v], ws.Wt[pq * NF + tb.c0pq[Kk][v]], hc);
        }
      }
      #pragma unroll 1
      for (int d = lane; d < NDET; d += 32) ws.S[d] = 0.f;
      __syncwarp();
      // alpha-beta couplings: both strings are Phi or single replacements of it; same-spin
      // couplings sit in row 0 and column 0 of the CI matrix
      constexpr int NC = 1 + K * K;
#pragma unroll 1
      for (int t = lane; t < NC * NC; t += 32) {
        const int x = t / NC, y = t % NC;
        const int Ia = (x == 0) ? 0 : tb.xJ[x - 1], Ib = (y == 0) ? 0 : tb.xJ[y - 1];
        float acc = 0.f;
        for (int u = 0; u < tb.c0n[Ia]; ++u)
          for (int v = 0; v < tb.c0n[Ib]; ++v)
            acc = fmaf((float)(tb.c0sg[Ia][u] * tb.c0sg[Ib][v]), ws.Wt[tb.c0pq[Ia][u] * NF + tb.c0pq[Ib][v]], acc);
        if (t != 0) ws.S[Ia * NS + Ib] = acc;
      }
      __syncwarp();
      if (lane > 0 && lane < NS) {
        ws.S[lane * NS] += hc;
        ws.S[lane] += hc;
      }
      __syncwarp();
      float rr = 0.f;
      #pragma unroll 1
      for (int d = lane; d < NDET; d += 32) rr = fmaf(ws.S[d], ws.S[d], rr);
      rphi = sqrtf(wsum(rr));
    }
    if (rphi < tol) {  // converged at Phi: E = <Phi|H|Phi>, X = 0
      if (lane == 0) {
        a.energy[oidx] = ws.eshift;
        a.status[oidx] = kSpaceOk;
        if (a.iters) a.iters[oidx] = 0;
      }
      if (guess_out)
        #pragma unroll 1
        for (int d = lane; d < NDET; d += 32) guess_out[(size_t)s * NDET + d] = (d == 0) ? 1.f : 0.f;
      __syncwarp();
      return;
    }
    // the diagonal relative to <Phi|H|Phi> (diag_at) takes its alpha-beta Coulomb sum
    // J(Ia, Ib) = sum_{p in Ia, r in Ib} J_pr from J_c; j0 is that sum at Phi
    if (lane == 0) {
      float j0 = 0.f;
      for (int l = 0; l < K; ++l)
        for (int m = 0; m < K; ++m) j0 += ws.Jc[tb.occ[0][l] * NORB + tb.occ[0][m]];
      ws.j0 = j0;
    }
    __syncwarp();
    if (!guess_in) {
      float nn = 0.f;
      float* v1 = ws.V;
      if constexpr (K == 3) {  // nonzero only where the column is (the diagonal is symmetric too)
        // the diagonal from per-string Coulomb rows jrow[I][r] = sum_{p in I} J_pr, summed as the
        // 6e6o sigma sums them (scratch in the S_1 slot, free until sigma(V_1))
        float* jrow = ws.S + NDET;
        for (int t = lane; t < NS * NORB; t += 32) {
          const int I = t / NORB, r = t % NORB;
          jrow[t] = ws.Jc[tb.occ[I][0] * NORB + r] + ws.Jc[tb.occ[I][1] * NORB + r] + ws.Jc[tb.occ[I][2] * NORB + r];
        }
        __syncwarp();
        const float j0 = ws.j0;
#pragma unroll
        for (int k = 0; k < kPhiLen; ++k) {
          const unsigned e = pe[k];
          if (e & (1u << 20)) {
            const int d = (int)((e >> 11) & 511u);
            const int ia = d / NS, ib = d % NS;
            const float* jr = jrow + ia * NORB;
            const float jab = (jr[tb.occ[ib][0]] + jr[tb.occ[ib][1]]) + jr[tb.occ[ib][2]];
            float den = -(ws.dh[ia] + ws.dh[ib] + (jab - j0));
            if (fabsf(den) < 1e-4f) den = (den < 0.f) ? -1e-4f : 1e-4f;
            const float v = ws.S[d] / den;
            v1[d] = v;
            float w2 = v * v;
            if (e & (1u << 21)) {
              v1[(d % NS) * NS + d / NS] = v;
              w2 += w2;
            }
            nn += w2;
          }
        }
      } else {
        #pragma unroll 1
        for (int d = lane; d < NDET; d += 32) {
          float den = -diag_at<K>(tb, ws, d / NS, d % NS);
          if (fabsf(den) < 1e-4f) den = (den < 0.f) ? -1e-4f : 1e-4f;
          const float v = (d == 0) ? 0.f : ws.S[d] / den;
          v1[d] = v;
          nn = fmaf(v, v, nn);
        }
      }
      vn_phi = sqrtf(wsum(nn));
      if (!(vn_phi > 1e-6f)) {
        const int st = (rphi < 100.f * tol) ? kSpaceOk : kSpaceNoConv;
        if (lane == 0) {
          a.energy[oidx] = ws.eshift;
          a.status[oidx] = st;
          if (a.iters) a.iters[oidx] = 0;
        }
        if (guess_out && st == kSpaceOk)
          #pragma unroll 1
          for (int d = lane; d < NDET; d += 32) guess_out[(size_t)s * NDET + d] = (d == 0) ? 1.f : 0.f;
        __syncwarp();
        return;
      }
    }
  }
  // ---- same-spin string operator, off-diagonal ---------------------------------------------
  if constexpr (K == 3) {  // from its coupling table, targets dealt evenly to the 32 lanes
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int q = lane; q < NS * NS / 4; q += 32) reinterpret_cast<float4*>(ws.Hs)[q] = z4;
    __syncwarp();
    float acc = 0.f;
#pragma unroll kHsUnroll
    for (int k = 0; k < kHsLen; ++k) {
      const unsigned e = hs_entry(cs, k * 32 + lane);
      acc = fmaf(__uint_as_float(e & 0xff800000u), ws.Wt[e & 2047u], acc);
      if (e & (1u << 20)) {
        ws.Hs[(e >> 11) & 511u] = acc;
        acc = 0.f;
      }
    }
  } else if (lane < NS) {
    const int I = lane;
#pragma unroll 1
    for (int j = 0; j < NS; ++j) ws.Hs[I * NS + j] = 0.f;
#pragma unroll 1
    for (int u = 0; u < NSG; ++u) {
      const int e = I * NSG + u;
      const int pq = tb.pq[e], Kk = tb.J[e];
      const float s1 = (float)tb.sg[e];
      if (Kk != I) ws.Hs[I * NS + Kk] += s1 * ws.hp()[pq];
#pragma unroll 1
      for (int v = 0; v < NSG; ++v) {
        const int e2 = Kk * NSG + v;
        const int J2 = tb.J[e2];
        if (J2 == I) continue;  // the diagonal is kept apart (dh, Jc)
        ws.Hs[I * NS + J2] += 0.5f * s1 * (float)tb.sg[e2] * ws.Wt[pq * NF + tb.pq[e2]];
      }
    }
  }
  __syncwarp();
  // ---- caller's guess: subspace {Phi, g - g_Phi Phi}; its sigma counts as one iteration -------
  int it0 = 0;
  if (guess_in && KM >= 2) {
    float* v1 = ws.V;
    float p = 0.f;
    #pragma unroll 1
    for (int d = lane; d < NDET; d += 32) {  // spin-flip symmetric part (where the Phi root lies)
      const int dt = (d % NS) * NS + d / NS;
      const float gv = (d == 0) ? 0.f : 0.5f * (guess_in[(size_t)s * NDET + d] + guess_in[(size_t)s * NDET + dt]);
      v1[d] = gv;
      p = fmaf(gv, gv, p);
    }
    const float nr = sqrtf(wsum(p));
    if (nr > 1e-6f) {  // an all-Phi (or zero) guess adds nothing
      const float inv = 1.f / nr;
      #pragma unroll 1
      for (int d = lane; d < NDET; d += 32) v1[d] *= inv;
      __syncwarp();
      float* s1 = ws.S + NDET;
      sigma<K>(tb, ws, v1, s1, lane);
      RRAcc a10, a11;
      #pragma unroll 1
      for (int d = lane; d < NDET; d += 32) {
        a10.add(v1[d], ws.S[d]);
        a11.add(v1[d], s1[d]);
      }
      const DF g10 = a10.total(), g11 = a11.total();
      const DF g01{s1[0], 0.f};  // Phi . sigma(v1)
      if (lane == 0) {
        ws.G[0] = DF{0.f, 0.f};  // Phi . sigma(Phi) relative to <Phi|H|Phi>
        ws.G[1] = g01;
        ws.G[KM] = g10;
        ws.G[KM + 1] = g11;
        for (int j = 0; j < KM; ++j) ws.yf[j] = (j == 0) ? 1.f : 0.f;
        ws.theta = DF{0.f, 0.f};
        ws.ctrl[1] = small_eig_rr(ws.G, 2, DF{-1e-2f, 0.f}, ws.yf, &ws.theta);
        ws.ctrl[0] = 2;
      }
      it0 = 1;
      __syncwarp();
    }
  }
  // ---- Davidson ----------------------------------------------------------------------------
  // Subspace {Phi = V_0, V_1, ..}: V_0 is implicit (unit vector e_0) and every stored V_j is
  // orthogonal to it (its component 0 is zero), so products with V_0 are single elements.
  constexpr int KMX = (NDET < KM) ? NDET : KM;  // the 2e2o space has only 4 determinants
#pragma unroll 1
  for (int it = 0; it < a.max_iter; ++it) {
    int k = ws.ctrl[0];
    if (k == KMX) {  // restart on {Phi, Ritz vector}: x = y_0 Phi + x', x' = sum_{j>=1} y_j V_j is
                     // already orthogonal to Phi, and sigma(x') = sum_{j>=1} y_j S_j
      RRAcc apv, ap0, ap1;
      #pragma unroll 1
      for (int d = lane; d < NDET; d += 32) {
        float xv = 0.f, sv = 0.f;
        for (int j = 1; j < k; ++j) {
          xv = fmaf(ws.yf[j], ws.V[(j - 1) * NDET + d], xv);
          sv = fmaf(ws.yf[j], ws.S[j * NDET + d], sv);
        }
        ws.V[d] = xv;
        ws.S[NDET + d] = sv;
        apv.add(xv, xv);
        ap0.add(xv, ws.S[d]);
        ap1.add(xv, sv);
      }
      const DF pv = apv.total(), p0 = ap0.total(), p1 = ap1.total();
      const float nx = sqrtf(df_f(pv)), inv = 1.f / nx;
      #pragma unroll 1
      for (int d = lane; d < NDET; d += 32) {
        ws.V[d] *= inv;
        ws.S[NDET + d] *= inv;
      }
      __syncwarp();
      if (lane == 0) {  // projected matrix of {Phi, V_1}; G[0] (Phi . S_0 = 0) is unchanged
        ws.G[1] = DF{ws.S[NDET], 0.f};
        ws.G[KM] = df_mulf(p0, inv);
        ws.G[KM + 1] = df_mulf(df_mulf(p1, inv), inv);
        ws.yf[1] = nx;
        ws.ctrl[0] = 2;
      }
      __syncwarp();
      k = 2;
    }
    const float th = df_f(ws.theta);
    float* vk = ws.V + (k - 1) * NDET;
    float vn = vn_phi;  // first step from Phi: V1 already holds the preconditioned residual
    if (!(it == 0 && !guess_in)) {
      float rr = 0.f;
      #pragma unroll 1
      for (int d = lane; d < NDET; d += 32) {
        float xv = (d == 0) ? ws.yf[0] : 0.f, sv = ws.yf[0] * ws.S[d];
        for (int j = 1; j < k; ++j) {
          xv = fmaf(ws.yf[j], ws.V[(j - 1) * NDET + d], xv);
          sv = fmaf(ws.yf[j], ws.S[j * NDET + d], sv);
        }
        const float r = sv - th * xv;
        rr = fmaf(r, r, rr);
        vk[d] = r;  // the residual; preconditioned below once the space is known not to be done
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
          ws.ctrl[3] = it + it0;
        }
        __syncwarp();
        break;
      }
      #pragma unroll 1
      for (int d = lane; d < NDET; d += 32) {  // diagonal preconditioner r / (theta - D)
        float den = th - diag_at<K>(tb, ws, d / NS, d % NS);
        if (fabsf(den) < 1e-4f) den = (den < 0.f) ? -1e-4f : 1e-4f;
        vk[d] = __fdividef(vk[d], den);
      }
      __syncwarp();
      // expansion vector: the preconditioned residual, orthogonalised against the subspace.  When
      // that leaves (almost) nothing while the residual is still above 100 x tol, the residual
      // itself (orthogonal to the subspace at a Ritz pair) is used instead, so the loop does not
      // stall on a correction that lies in the subspace
#pragma unroll 1
      for (int attempt = 0; attempt < 2; ++attempt) {
        if (attempt == 1) {
          #pragma unroll 1
          for (int d = lane; d < NDET; d += 32) {
            float xv = (d == 0) ? ws.yf[0] : 0.f, sv = ws.yf[0] * ws.S[d];
            for (int j = 1; j < k; ++j) {
              xv = fmaf(ws.yf[j], ws.V[(j - 1) * NDET + d], xv);
              sv = fmaf(ws.yf[j], ws.S[j * NDET + d], sv);
            }
            vk[d] = sv - th * xv;
          }
          __syncwarp();
        }
        for (int pass = 0; pass < 2; ++pass) {  // against Phi: drop component 0
          RRAcc acf[KM];
          float cf[KM];
          #pragma unroll 1
          for (int d = lane; d < NDET; d += 32) {
            const float v = vk[d];
#pragma unroll
            for (int j = 1; j < KM; ++j)
              if (j < k) acf[j].add(ws.V[(j - 1) * NDET + d], v);
          }
#pragma unroll
          for (int j = 0; j < KM; ++j) cf[j] = (j >= 1 && j < k) ? df_f(acf[j].total()) : 0.f;
          #pragma unroll 1
          for (int d = lane; d < NDET; d += 32) {
            float v = vk[d];
#pragma unroll
            for (int j = 1; j < KM; ++j)
              if (j < k) v = fmaf(-cf[j], ws.V[(j - 1) * NDET + d], v);
            vk[d] = (d == 0) ? 0.f : v;
          }
          __syncwarp();
        }
        float nn = 0.f;
        #pragma unroll 1
        for (int d = lane; d < NDET; d += 32) nn = fmaf(vk[d], vk[d], nn);
        vn = sqrtf(wsum(nn));
        if (vn > 1e-6f || rnorm < 100.f * tol) break;
      }
      if (!(vn > 1e-6f)) {  // the subspace cannot grow (complete or stagnated)
        if (lane == 0) {
          ws.ctrl[2] = (rnorm < 100.f * tol) ? kSpaceOk : kSpaceNoConv;
          ws.ctrl[3] = it + it0;
        }
        __syncwarp();
        break;
      }
    }
    const float inv = 1.f / vn;
    #pragma unroll 1
    for (int d = lane; d < NDET; d += 32) vk[d] *= inv;
    __syncwarp();
    float* sk = ws.S + k * NDET;
    if constexpr (K == 3) {
      if (it == 0 && !guess_in)  // the first-order vector: nonzero only on the Phi column's support
        sigma33_first(tb, ws, vk, sk, ws.V + NDET, ws.S + 2 * NDET, lane);
      else
        sigma33(tb, ws, vk, sk, lane);
    } else {
      sigma<K>(tb, ws, vk, sk, lane);
    }
    RRAcc agc[KM], agr[KM], akk;
    #pragma unroll 1
    for (int d = lane; d < NDET; d += 32) {
      const float vkd = vk[d], skd = sk[d];
      akk.add(vkd, skd);
      agr[0].add(vkd, ws.S[d]);
#pragma unroll
      for (int j = 1; j < KM; ++j)
        if (j < k) {
          agc[j].add(ws.V[(j - 1) * NDET + d], skd);
          agr[j].add(vkd, ws.S[j * NDET + d]);
        }
    }
    DF gc[KM], gr[KM];
    const DF gkk = akk.total();
    gr[0] = agr[0].total();
    gc[0] = DF{sk[0], 0.f};  // Phi . sigma(V_k)
#pragma unroll
    for (int j = 1; j < KM; ++j) {
      gc[j] = (j < k) ? agc[j].total() : DF{0.f, 0.f};
      gr[j] = (j < k) ? agr[j].total() : DF{0.f, 0.f};
    }
    if (lane == 0) {
      for (int j = 0; j < k; ++j) {
        ws.G[j * KM + k] = gc[j];
        ws.G[k * KM + j] = gr[j];
      }
      ws.G[k * KM + k] = gkk;
      const int kk = k + 1;
      ws.yf[k] = 0.f;
      const int cx = small_eig_rr(ws.G, kk, df_add(ws.theta, DF{-1e-2f, 0.f}), ws.yf, &ws.theta);
      ws.ctrl[0] = kk;
      ws.ctrl[3] = it + 1 + it0;
      ws.ctrl[1] = cx ? ws.ctrl[1] + 1 : 0;
      if (ws.ctrl[1] >= 2) ws.ctrl[2] = kSpaceRoot;  // a complex root twice in a row: no real root
    }
    __syncwarp();
    if (ws.ctrl[1] >= 2) break;
  }
  // ---- root, increment, merge ------------------------------------------------------------
  // owners and old amplitudes of the space's internal amplitudes are loaded first, so their
  // latency overlaps the Ritz vector and the extraction (only an owner writes an amplitude, so
  // the values read here are the ones the merge below updates)
  constexpr int K4 = K * K * K * K, R2 = (K4 + 31) / 32;
  int32_t own1 = -1, own2[R2];
  double old1 = 0.0, old2[R2];
  size_t g1 = 0, g2[R2];
  if (owner && a.owner1 && lane < K * K) {
    g1 = (size_t)ws.orb[lane / K] * a.nvir + (ws.orb[K + lane % K] - a.nocc);
    own1 = a.owner1[g1];
    old1 = a.t1_old[g1];
  }
#pragma unroll
  for (int r = 0; r < R2; ++r) {
    const int idx = lane + 32 * r;
    own2[r] = -1;
    old2[r] = 0.0;
    g2[r] = 0;
    if (owner && a.owner2 && idx < K4) {
      const int i = idx / (K * K * K), j = (idx / (K * K)) % K, aa = (idx / K) % K, b = idx % K;
      g2[r] = (((size_t)ws.orb[i] * a.nocc + ws.orb[j]) * a.nvir + (ws.orb[K + aa] - a.nocc)) * a.nvir +
              (ws.orb[K + b] - a.nocc);
      own2[r] = a.owner2[g2[r]];
      old2[r] = a.t2_old[g2[r]];
    }
  }
  const int k = ws.ctrl[0];
  float xx = 0.f;
  if (owner || guess_out) {  // the Ritz vector itself: the increment and the saved root read it
#pragma unroll 1
    for (int d = lane; d < NDET; d += 32) {
      float xv = (d == 0) ? ws.yf[0] : 0.f;
      for (int j = 1; j < k; ++j) xv = fmaf(ws.yf[j], ws.V[(j - 1) * NDET + d], xv);
      ws.S[d] = xv;
      xx = fmaf(xv, xv, xx);
    }
    xx = wsum(xx);
    __syncwarp();
  } else {  // only its norm (root test): the stored vectors are orthonormal and orthogonal to Phi
    for (int j = 0; j < k; ++j) xx = fmaf(ws.yf[j], ws.yf[j], xx);
  }
  const float xn = sqrtf(xx);
  const float c0 = ws.yf[0];  // component 0 of the Ritz vector (every stored vector has a zero there)
  int st = ws.ctrl[2];
  if (st == kSpaceNoConv && ws.ctrl[1] > 0) st = kSpaceRoot;  // stopped on a complex projected root
  if (st == kSpaceOk && !(fabsf(c0) >= 1e-3f * xn)) st = kSpaceRoot;
  if (!isfinite(c0) || !isfinite(df_f(ws.theta))) st = kSpaceNonFinite;
  const float inv0 = (st == kSpaceOk || st == kSpaceNoConv) ? 1.f / c0 : 0.f;
  if (guess_out && st == kSpaceOk)
    #pragma unroll 1
    for (int d = lane; d < NDET; d += 32) guess_out[(size_t)s * NDET + d] = ws.S[d] * inv0;
  if (owner) {  // the increment, written where this space owns the amplitude
    float* x1 = ws.V;  // V is free now: K^2 + K^4 floats of scratch
    float* x2 = x1 + K * K;
    if (lane < K * K) {
      const int J = tb.xJ[lane];
      const float f = (tb.xs[lane] < 0) ? -inv0 : inv0;
      x1[lane] = 0.5f * f * (ws.S[J * NS] + ws.S[J]);
    }
    __syncwarp();
#pragma unroll 1
    for (int idx = lane; idx < K4; idx += 32) {
      const int i = idx / (K * K * K), j = (idx / (K * K)) % K, aa = (idx / K) % K, b = idx % K;
      const int xa = i * K + aa, xb = j * K + b;
      const float f = (tb.xs[xa] != tb.xs[xb]) ? -inv0 : inv0;
      x2[idx] = f * ws.S[tb.xJ[xa] * NS + tb.xJ[xb]] - x1[xa] * x1[xb];
    }
    __syncwarp();
    if (st == kSpaceOk && a.owner1 && lane < K * K && own1 == sidx) a.t1_new[g1] = old1 + (double)x1[lane];
    if (st == kSpaceOk && a.owner2) {
#pragma unroll
      for (int r = 0; r < R2; ++r) {
        const int idx = lane + 32 * r;
        if (idx < K4 && own2[r] == sidx) {
          const int i = idx / (K * K * K), j = (idx / (K * K)) % K, aa = (idx / K) % K, b = idx % K;
          a.t2_new[g2[r]] = old2[r] + (double)(0.5f * (x2[idx] + x2[((j * K + i) * K + b) * K + aa]));
        }
      }
    }
  }
  if (lane == 0) {
    a.energy[oidx] = ws.eshift + ((double)ws.theta.hi + (double)ws.theta.lo);
    a.status[oidx] = st;
    if (a.iters) a.iters[oidx] = ws.ctrl[3];
  }
  __syncwarp();
}

// ---- kernels --------------------------------------------------------------------------------------

template <int K>
__global__ void __maxnreg__(kMaxRegs) solve_class_kernel(SolveArgs a, const float* __restrict__ W32,
                                                                  const float* __restrict__ guess_in,
                                                                  float* __restrict__ guess_out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  CtaTabs& cs = *reinterpret_cast<CtaTabs*>(smem_raw);
  AnyWarpState* wst = reinterpret_cast<AnyWarpState*>(smem_raw + kTabsBytes);
  build_all_tabs(cs);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  WarpState<K>& ws = state<K>(wst[warp]);
  if (lane == 0) ws.orb[0] = -1;  // no previous space: nothing to reuse
#pragma unroll 1
  for (int64_t s = (int64_t)blockIdx.x * nw + warp; s < a.nspaces; s += (int64_t)gridDim.x * nw)
    solve_one<K>(tabs<K>(cs), cs, ws, a, W32, guess_in, guess_out, a.items ? a.items[s] : s, lane);
}

struct PersistentArgs {
  SolveArgs cls[4];           // [k] for k = 1..3 (cls[0] unused)
  const float* W32;
  unsigned long long* queue;  // work counter, zero at launch
  int chunk;                  // work items taken per atomic
};

// One queue over every size class: items [0, n3) are 6e6o spaces, then 4e4o, then 2e2o.
__global__ void __maxnreg__(kMaxRegs) solve_persistent_kernel(PersistentArgs p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  CtaTabs& cs = *reinterpret_cast<CtaTabs*>(smem_raw);
  AnyWarpState* wst = reinterpret_cast<AnyWarpState*>(smem_raw + kTabsBytes);
  build_all_tabs(cs);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // no previous 6e6o space: nothing to reuse (a warp's items only increase, so after its first
  // smaller space it never meets a 6e6o space again)
  if (lane == 0) state<3>(wst[warp]).orb[0] = -1;
  const int64_t n3 = p.cls[3].nspaces, n2 = p.cls[2].nspaces, n1 = p.cls[1].nspaces;
  const unsigned long long total = (unsigned long long)(n3 + n2 + n1);
  // each pass takes `chunk` new items, so the loop ends after at most total / chunk + 1 passes
#pragma unroll 1
  for (unsigned long long pass = 0; pass <= total; ++pass) {
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(p.queue, (unsigned long long)p.chunk);
    base = __shfl_sync(0xffffffffu, base, 0);
    if (base >= total) break;
#pragma unroll 1
    for (int c = 0; c < p.chunk; ++c) {
      const unsigned long long item = base + (unsigned long long)c;
      if (item >= total) break;
      const int64_t it = (int64_t)item;
      if (it < n3) {
        const SolveArgs& a = p.cls[3];
        solve_one<3>(cs.t3, cs, state<3>(wst[warp]), a, p.W32, static_cast<const float*>(a.guess),
                     static_cast<float*>(a.root_out), a.items ? a.items[it] : it, lane);
      } else if (it < n3 + n2) {
        const SolveArgs& a = p.cls[2];
        const int64_t l = it - n3;
        solve_one<2>(cs.t2, cs, state<2>(wst[warp]), a, p.W32, static_cast<const float*>(a.guess),
                     static_cast<float*>(a.root_out), a.items ? a.items[l] : l, lane);
      } else {
        const SolveArgs& a = p.cls[1];
        const int64_t l = it - n3 - n2;
        solve_one<1>(cs.t1, cs, state<1>(wst[warp]), a, p.W32, static_cast<const float*>(a.guess),
                     static_cast<float*>(a.root_out), a.items ? a.items[l] : l, lane);
      }
    }
  }
}

template <typename Kern>
cudaError_t grid_for(Kern kern, int warps, int* grid) {
  const size_t smem = cta_smem_bytes(warps);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cta_smem_bytes(kMaxWarps));
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * warps, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  *grid = sms * per_sm;
  return cudaSuccess;
}

}  // namespace

cudaError_t launch_solve_warp(int k, const SolveArgs& a, const float* W32, const float* guess_in, float* guess_out,
                              int warps, cudaStream_t st) {
  if (a.nspaces <= 0) return cudaSuccess;
  if (warps < 1 || warps > kMaxWarps) warps = kMaxWarps;
  int grid = 0;
  cudaError_t e;
  const int64_t need = (a.nspaces + warps - 1) / warps;
  switch (k) {
    case 1: e = grid_for(solve_class_kernel<1>, warps, &grid); break;
    case 2: e = grid_for(solve_class_kernel<2>, warps, &grid); break;
    case 3: e = grid_for(solve_class_kernel<3>, warps, &grid); break;
    default: return cudaErrorInvalidValue;
  }
  if (e != cudaSuccess) return e;
  if (grid > need) grid = (int)need;
  const size_t smem = cta_smem_bytes(warps);
  switch (k) {
    case 1: solve_class_kernel<1><<<grid, 32 * warps, smem, st>>>(a, W32, guess_in, guess_out); break;
    case 2: solve_class_kernel<2><<<grid, 32 * warps, smem, st>>>(a, W32, guess_in, guess_out); break;
    default: solve_class_kernel<3><<<grid, 32 * warps, smem, st>>>(a, W32, guess_in, guess_out); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_solve_persistent(const SolveArgs* cls, const float* W32, unsigned long long* queue, int chunk,
                                    int warps, cudaStream_t st) {
  PersistentArgs p{};
  int64_t total = 0;
  for (int k = 1; k <= 3; ++k) {
    p.cls[k] = cls[k];
    total += cls[k].nspaces;
  }
  if (total <= 0) return cudaSuccess;
  if (warps < 1 || warps > kMaxWarps) warps = kMaxWarps;
  p.W32 = W32;
  p.queue = queue;
  p.chunk = chunk < 1 ? 1 : chunk;
  int grid = 0;
  cudaError_t e = grid_for(solve_persistent_kernel, warps, &grid);
  if (e != cudaSuccess) return e;
  const int64_t need = (total + warps - 1) / warps;
  if (grid > need) grid = (int)need;
  e = cudaMemsetAsync(queue, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  solve_persistent_kernel<<<grid, 32 * warps, cta_smem_bytes(warps), st>>>(p);
  return cudaGetLastError();
}

}  // namespace qf
