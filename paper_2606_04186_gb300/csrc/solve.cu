// Steps (b) and (c) of a flow sweep for one size class of active spaces: gather + fold,
// batched Davidson on the determinant operator, CI -> CC increment, owner-filtered merge.
//
// Paper: Eqs. (5)-(6) with N = 1 define each space's downfolded Hamiltonian; with the SES-CC
// dressing it is the projection of H-bar_<=2 onto the space's Sz = 0 determinants.  The space
// solver (VQE-UCCSD in the paper) is replaced by the exact Phi-dominant root; the singles and
// doubles cluster amplitudes of that root (C1 = t1, C2 = t2 + t1^2/2) are the increment of the
// space's internal amplitudes; each amplitude is written only by its owner space
// (Numerical Implementation: first space in ascending Delta-eps order that reaches it).
//
// Layout of one space with k occupied + k virtual orbitals (k = 1, 2, 3):
//   local orbitals 0..k-1 occupied, k..2k-1 virtual (ascending absolute index);
//   alpha / beta strings = k-electron subsets of the 2k orbitals, numbered by increasing
//   bit mask (string 0 = the occupied orbitals); determinant index = Ialpha * NS + Ibeta;
//   ket phase = alpha creators (ascending) left of beta creators.
// Operator: H = Ecore + Hs (x) 1 + 1 (x) Hs + sum_pqrs W_pqrs E^a_pq E^b_rs, where Hs is the
// same-spin string operator of the one-body part and the same-spin two-body part.
//
// One CTA owns one space at a time (grid-stride loop over the sorted list); everything the
// solver touches lives in shared memory.  All loops are bounded (Davidson iteration limit,
// fixed inner iteration counts); there are no waits on other CTAs.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <type_traits>

#include "qflow_internal.h"

namespace qf {
namespace {

template <int K>
struct Cas {
  static constexpr int NORB = 2 * K;
  static constexpr int NS = (K == 1) ? 2 : (K == 2) ? 6 : 20;  // C(2k, k)
  static constexpr int NSG = K * (K + 1);                       // single replacements per string
  static constexpr int NDET = NS * NS;
  static constexpr int NW = NORB * NORB * NORB * NORB;
  static constexpr int NF = NORB * NORB;
  static constexpr int KMAX = (NDET < 8) ? NDET : 8;           // Davidson subspace limit
  static constexpr int NT = (K == 3) ? 128 : 32;                // threads per CTA
  static constexpr int NWARP = NT / 32;
  static constexpr int NRED = 2 * KMAX + 2;                     // values per block reduction
  static constexpr int PER = (NDET + NT - 1) / NT;              // determinants per thread
};

template <int K, typename T>
struct Smem {
  using C = Cas<K>;
  double W[C::NW];                                   // gathered W block (FP64)
  T Wt[std::is_same<T, double>::value ? 1 : C::NW];  // W in the sigma precision (FP32 path)
  double F[C::NF];                                   // gathered F block
  double h[C::NF];                                   // folded one-body (vacuum order)
  double hp[C::NF];                                  // h - 1/2 sum_r W_prrq
  T Hs[C::NS * C::NS];                               // same-spin string operator (off-diagonal)
  double hsd[C::NS];                                 // its diagonal
  T diag[C::NDET];                                   // operator diagonal
  T V[C::KMAX * C::NDET];                            // subspace basis (orthonormal)
  T S[C::KMAX * C::NDET];                            // H applied to the basis
  double G[C::KMAX * C::KMAX];                       // projected matrix, G[i*KMAX+j] = V_i . S_j
  double y[C::KMAX];                                 // Ritz coefficients
  double ynew[C::KMAX];
  double red[C::NWARP * C::NRED];                    // cross-warp reduction scratch
  double out[C::NRED];                               // reduction results
  double x1[K * K];                                  // singles increment
  double x2raw[K * K * K * K];                       // doubles before symmetrisation
  double ecore, e0, theta, eshift;  // theta is relative to eshift = <Phi|H|Phi>
  int sing[C::NS * C::NSG];                          // packed single replacements into a string
  int smask[C::NS];                                  // string bit masks
  int mask2idx[1 << C::NORB];
  int orb[2 * K];
  int ctrl[4];                                       // [0] k, [1] stop flag, [2] status, [3] iterations
};

__device__ __forceinline__ int popc(unsigned x) { return __popc(x); }

// sign of a+_p a_q acting on string mask m (q in m; p not in m\{q}); returns the new mask.
__device__ __forceinline__ int apply_pq(int m, int p, int q, int* sign) {
  if (p == q) {
    *sign = 1;
    return m;
  }
  int s = popc(m & ((1 << q) - 1)) & 1;
  int m1 = m & ~(1 << q);
  s ^= popc(m1 & ((1 << p) - 1)) & 1;
  *sign = s ? -1 : 1;
  return m1 | (1 << p);
}

// Build string tables in shared memory: strings by increasing mask, and for each target
// string I the K(K+1) entries (pq, J, sign) with <I| a+_p a_q |J> = sign.
template <int K, typename T>
__device__ void build_tables(Smem<K, T>& sm) {
  using C = Cas<K>;
  if (threadIdx.x == 0) {
    int c = 0;
    for (int m = 0; m < (1 << C::NORB); ++m) {
      sm.mask2idx[m] = -1;
      if (popc(m) == K) {
        sm.mask2idx[m] = c;
        sm.smask[c++] = m;
      }
    }
  }
  __syncthreads();
  for (int I = threadIdx.x; I < C::NS; I += C::NT) {
    const int mi = sm.smask[I];
    int u = 0;
    for (int p = 0; p < C::NORB; ++p) {
      if (!((mi >> p) & 1)) continue;
      for (int q = 0; q < C::NORB; ++q) {
        if (q != p && ((mi >> q) & 1)) continue;
        const int mj = (mi & ~(1 << p)) | (1 << q);  // J = I - p + q
        int sg;
        const int back = apply_pq(mj, p, q, &sg);   // a+_p a_q J = sg * I
        (void)back;
        const int J = sm.mask2idx[mj];
        sm.sing[I * C::NSG + u] = (p * C::NORB + q) | (J << 6) | ((sg < 0) ? (1 << 11) : 0);
        ++u;
      }
    }
  }
  __syncthreads();
}

// Reduce m (<= NRED) per-thread partial sums across the block; results in sm.out[0..m).
template <int K, typename T>
__device__ __forceinline__ void block_sums(Smem<K, T>& sm, const T* part, int m) {
  using C = Cas<K>;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < C::NRED; ++j) {
    if (j < m) {
      T v = part[j];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) sm.red[warp * C::NRED + j] = (double)v;
    }
  }
  __syncthreads();
  if (threadIdx.x < m) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < C::NWARP; ++w) s += sm.red[w * C::NRED + threadIdx.x];
    sm.out[threadIdx.x] = s;
  }
  __syncthreads();
}

// sigma = H c for one space (c, out in shared memory, precision T).
template <int K, typename T>
__device__ void sigma(Smem<K, T>& sm, const T* __restrict__ c, T* __restrict__ out) {
  using C = Cas<K>;
  const T* Wv;
  if constexpr (std::is_same<T, double>::value) Wv = sm.W; else Wv = sm.Wt;
  for (int d = threadIdx.x; d < C::NDET; d += C::NT) {
    const int ia = d / C::NS, ib = d - ia * C::NS;
    T acc = sm.diag[d] * c[d];  // diagonal (FP64-built, shifted); Hs and W carry no diagonal part
#pragma unroll 4
    for (int j = 0; j < C::NS; ++j) {
      acc = fma(sm.Hs[ia * C::NS + j], c[j * C::NS + ib], acc);
      acc = fma(sm.Hs[ib * C::NS + j], c[ia * C::NS + j], acc);
    }
    int rsb[C::NSG], jb[C::NSG];
    T sb[C::NSG];
#pragma unroll
    for (int v = 0; v < C::NSG; ++v) {
      const int e = sm.sing[ib * C::NSG + v];
      rsb[v] = e & 63;
      jb[v] = (e >> 6) & 31;
      sb[v] = (e >> 11) ? (T)-1 : (T)1;
    }
#pragma unroll 2
    for (int u = 0; u < C::NSG; ++u) {
      const int e = sm.sing[ia * C::NSG + u];
      const T* wrow = Wv + (e & 63) * C::NF;
      const T* crow = c + ((e >> 6) & 31) * C::NS;
      T part = (T)0;
#pragma unroll
      for (int v = 0; v < C::NSG; ++v) part = fma(sb[v] * wrow[rsb[v]], crow[jb[v]], part);
      acc = (e >> 11) ? acc - part : acc + part;
    }
    out[d] = acc;
  }
}

// Phi-tracking eigenpair of the k x k projected matrix (FP64, one thread): shifted inverse
// iteration from the previous Ritz value, then Rayleigh-quotient refinement.  Returns 1 when
// the result is not an eigenpair of G (|G y - theta y| above 1e-8 of G's scale): real inverse
// iteration cannot settle on a root that is one of a complex pair; else 0.
template <int KM>
__device__ int small_eig(const double* G, int k, double shift, double* y, double* theta) {
  double a[KM * KM], z[KM];
  for (int phase = 0; phase < 8; ++phase) {
    const double sg = (phase < 4) ? shift : *theta;
    for (int i = 0; i < k; ++i)
      for (int j = 0; j < k; ++j) a[i * KM + j] = G[i * KM + j] - ((i == j) ? sg : 0.0);
    for (int i = 0; i < k; ++i) z[i] = y[i];
    // Gaussian elimination with partial pivoting on a copy, solving a z = y.
    for (int col = 0; col < k; ++col) {
      int piv = col;
      double best = fabs(a[col * KM + col]);
      for (int r = col + 1; r < k; ++r)
        if (fabs(a[r * KM + col]) > best) {
          best = fabs(a[r * KM + col]);
          piv = r;
        }
      if (piv != col) {
        for (int j = 0; j < k; ++j) {
          double t = a[col * KM + j];
          a[col * KM + j] = a[piv * KM + j];
          a[piv * KM + j] = t;
        }
        double t = z[col];
        z[col] = z[piv];
        z[piv] = t;
      }
      double p = a[col * KM + col];
      if (fabs(p) < 1e-300) p = (p < 0.0) ? -1e-300 : 1e-300;
      a[col * KM + col] = p;
      for (int r = col + 1; r < k; ++r) {
        const double f = a[r * KM + col] / p;
        for (int j = col; j < k; ++j) a[r * KM + j] -= f * a[col * KM + j];
        z[r] -= f * z[col];
      }
    }
    for (int r = k - 1; r >= 0; --r) {
      double s = z[r];
      for (int j = r + 1; j < k; ++j) s -= a[r * KM + j] * z[j];
      z[r] = s / a[r * KM + r];
    }
    double nrm = 0.0;
    for (int i = 0; i < k; ++i) nrm += z[i] * z[i];
    nrm = sqrt(nrm);
    if (!(nrm > 0.0) || !isfinite(nrm)) break;
    // fix the overall sign so that the Phi-carrying first coefficient stays positive
    const double sgn = (z[0] < 0.0) ? -1.0 : 1.0;
    for (int i = 0; i < k; ++i) y[i] = sgn * z[i] / nrm;
    double num = 0.0;
    for (int i = 0; i < k; ++i) {
      double gy = 0.0;
      for (int j = 0; j < k; ++j) gy += G[i * KM + j] * y[j];
      num += y[i] * gy;
    }
    *theta = num;  // y has unit norm
  }
  double scale = 0.0, res = 0.0;
  for (int i = 0; i < k; ++i) {
    double gy = -(*theta) * y[i];
    for (int j = 0; j < k; ++j) {
      gy += G[i * KM + j] * y[j];
      scale = fmax(scale, fabs(G[i * KM + j]));
    }
    res += gy * gy;
  }
  return (sqrt(res) > 1e-8 * fmax(1.0, scale)) ? 1 : 0;
}

// Symmetric projected problem (DUCC form, Hermitian operator; one thread): G is symmetrised and
// diagonalised by cyclic Jacobi rotations; of its eigenpairs the one whose Ritz vector has the
// largest Phi component (sum_j y_j V_j[Phi]) is taken, as the space's root is the eigenvector
// with the largest |c_Phi|.  y receives the unit eigenvector, theta its eigenvalue.
template <int KM>
__device__ void small_eig_sym(const double* G, int k, const double* v0, double* y, double* theta) {
  double a[KM * KM], z[KM * KM];
  double scale = 0.0;
  for (int i = 0; i < k; ++i)
    for (int j = 0; j < k; ++j) {
      a[i * KM + j] = 0.5 * (G[i * KM + j] + G[j * KM + i]);
      z[i * KM + j] = (i == j) ? 1.0 : 0.0;
      scale = fmax(scale, fabs(a[i * KM + j]));
    }
  for (int sweep = 0; sweep < 16; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < k; ++p)
      for (int q = p + 1; q < k; ++q) off = fmax(off, fabs(a[p * KM + q]));
    if (!(off > 1e-15 * fmax(scale, 1e-300))) break;
    for (int p = 0; p < k; ++p)
      for (int q = p + 1; q < k; ++q) {
        const double apq = a[p * KM + q];
        if (apq == 0.0) continue;
        const double tau = (a[q * KM + q] - a[p * KM + p]) / (2.0 * apq);
        const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
        const double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
        for (int r = 0; r < k; ++r) {  // columns p, q
          const double arp = a[r * KM + p], arq = a[r * KM + q];
          a[r * KM + p] = c * arp - s * arq;
          a[r * KM + q] = s * arp + c * arq;
        }
        for (int r = 0; r < k; ++r) {  // rows p, q
          const double apr = a[p * KM + r], aqr = a[q * KM + r];
          a[p * KM + r] = c * apr - s * aqr;
          a[q * KM + r] = s * apr + c * aqr;
        }
        for (int r = 0; r < k; ++r) {
          const double zrp = z[r * KM + p], zrq = z[r * KM + q];
          z[r * KM + p] = c * zrp - s * zrq;
          z[r * KM + q] = s * zrp + c * zrq;
        }
      }
  }
  int best = 0;
  double wbest = -1.0;
  for (int m = 0; m < k; ++m) {
    double c0 = 0.0;
    for (int j = 0; j < k; ++j) c0 += z[j * KM + m] * v0[j];
    if (fabs(c0) > wbest) {
      wbest = fabs(c0);
      best = m;
    }
  }
  double c0 = 0.0;
  for (int j = 0; j < k; ++j) c0 += z[j * KM + best] * v0[j];
  const double sg = (c0 < 0.0) ? -1.0 : 1.0;
  for (int j = 0; j < k; ++j) y[j] = sg * z[j * KM + best];
  *theta = a[best * KM + best];
}

// ---- DUCC form: the space's internal part L_A ------------------------------------------------------
//
// In the DUCC form (ducc.cu) a space's operator is G|_A - L_A, where
//   L_A = X_A + X_A^+ + 1/2 (Y_A + Y_A^+),  X_A = [H_A, T_A]_(<=2),  Y_A = [B_A, T_A]_(<=2),
// H_A the Hamiltonian and B_A = D.T_A + (D.T_A)^+ restricted to the space's 2K orbitals, T_A the
// space's internal amplitudes.  [O, T]_(<=2) is the T-linear part of the SES-CC dressing
// e^{-T} O e^{T} (its one- and two-body parts normal ordered with respect to Phi): the
// linearisation of the T1 orbital transformation (creators by -K, annihilators by +K, K_ai = t_i^a)
// plus the connected T2-linear terms, each below.  Local orbitals: 0..K-1 occupied, K..2K-1 virtual.
template <int K>
struct DuccSmem {
  static constexpr int NO = 2 * K, NW = NO * NO * NO * NO, NF = NO * NO;
  double g[NW];    // two-body elements of the operator (first H_A, then B_A)
  double Wx[NW];   // [O, T]: two-body part
  double f0[NF];   // bare Fock block of the space
  double h[NF];    // operator's one-body part, vacuum order
  double f[NF];    // operator's one-body part, normal order
  double Fx[NF];   // [O, T]: one-body part
  double t1[K * K];
  double t2[K * K * K * K];
  double ex;       // [O, T]: zero-body part
};

template <int K>
struct LinDress {
  static constexpr int NO = 2 * K;
  const DuccSmem<K>& d;
  __device__ double g(int p, int q, int r, int s) const { return d.g[((p * NO + q) * NO + r) * NO + s]; }
  __device__ double t(int i, int j, int a, int b) const { return d.t2[((i * K + j) * K + a) * K + b]; }
  __device__ double u(int i, int j, int a, int b) const { return 2.0 * t(i, j, a, b) - t(i, j, b, a); }
  __device__ double t1(int i, int a) const { return d.t1[i * K + a]; }
  __device__ double f(int p, int q) const { return d.f[p * NO + q]; }
  __device__ double h(int p, int q) const { return d.h[p * NO + q]; }
  // T1 linearisation: creators (p, r) by -K, annihilators (q, s) by +K
  __device__ double dg(int p, int q, int r, int s) const {
    double v = 0.0;
    for (int x = 0; x < K; ++x) {
      if (p >= K) v -= t1(x, p - K) * g(x, q, r, s);
      if (q < K) v += g(p, K + x, r, s) * t1(q, x);
      if (r >= K) v -= t1(x, r - K) * g(p, q, x, s);
      if (s < K) v += g(p, q, r, K + x) * t1(s, x);
    }
    return v;
  }
  __device__ double dh(int p, int q) const {
    double v = 0.0;
    for (int x = 0; x < K; ++x) {
      if (q < K) v += h(p, K + x) * t1(q, x);
      if (p >= K) v -= t1(x, p - K) * h(x, q);
    }
    return v;
  }
  // T2-linear two-body terms of element (p, q, r, s) (creators p, r; annihilators q, s)
  __device__ double w2(int p, int q, int r, int s) const {
    const int blk = ((p >= K) << 3) | ((q >= K) << 2) | ((r >= K) << 1) | (s >= K);
    double v = 0.0;
    switch (blk) {
      case 0x0:  // oooo (k i l j): sum_ef g_kelf t_ijef
        for (int e = 0; e < K; ++e)
          for (int ff = 0; ff < K; ++ff) v += g(p, K + e, r, K + ff) * t(q, s, e, ff);
        break;
      case 0xF:  // vvvv (a e b f): sum_mn g_menf t_mnab
        for (int m = 0; m < K; ++m)
          for (int nn = 0; nn < K; ++nn) v += g(m, q, nn, s) * t(m, nn, p - K, r - K);
        break;
      case 0x6:  // ovvo (m e b j)
      case 0x9: {  // voov (b j m e) = ovvo (m e b j)
        const int m = (blk == 0x6) ? p : r, e = (blk == 0x6) ? q : s, b = (blk == 0x6) ? r : p, j = (blk == 0x6) ? s : q;
        for (int nn = 0; nn < K; ++nn)
          for (int ff = 0; ff < K; ++ff)
            v += g(m, e, nn, K + ff) * u(j, nn, b - K, ff) - g(m, K + ff, nn, e) * t(j, nn, b - K, ff);
        break;
      }
      case 0x3:  // oovv (i j a b)
      case 0xC: {  // vvoo (a b i j) = oovv (i j a b)
        const int i = (blk == 0x3) ? p : r, j = (blk == 0x3) ? q : s, a = (blk == 0x3) ? r : p, b = (blk == 0x3) ? s : q;
        for (int ff = 0; ff < K; ++ff)
          for (int nn = 0; nn < K; ++nn) v -= g(i, K + ff, nn, b) * t(j, nn, ff, a - K);
        break;
      }
      case 0x2:  // oovo (m i b j)
      case 0x8: {  // vooo (b j m i) = oovo (m i b j)
        const int m = (blk == 0x2) ? p : r, i = (blk == 0x2) ? q : s, b = (blk == 0x2) ? r : p, j = (blk == 0x2) ? s : q;
        for (int e = 0; e < K; ++e) {
          v += f(m, K + e) * t(i, j, e, b - K);
          for (int ff = 0; ff < K; ++ff) v += g(m, K + e, b, K + ff) * t(i, j, e, ff);
          for (int nn = 0; nn < K; ++nn)
            v += g(m, i, nn, K + e) * u(j, nn, b - K, e) - g(m, K + e, nn, i) * t(j, nn, b - K, e) -
                 g(m, K + e, nn, j) * t(i, nn, e, b - K);
        }
        break;
      }
      case 0xE:  // vvvo (a e b i)
      case 0xB: {  // vovv (b i a e) = vvvo (a e b i)
        const int a = (blk == 0xE) ? p : r, e = (blk == 0xE) ? q : s, b = (blk == 0xE) ? r : p, i = (blk == 0xE) ? s : q;
        for (int m = 0; m < K; ++m) {
          v -= f(m, e) * t(m, i, a - K, b - K);
          for (int nn = 0; nn < K; ++nn) v += g(m, e, nn, i) * t(m, nn, a - K, b - K);
          for (int ff = 0; ff < K; ++ff)
            v += g(m, K + ff, a, e) * u(m, i, ff, b - K) - g(m, e, b, K + ff) * t(m, i, a - K, ff) -
                 g(m, e, a, K + ff) * t(m, i, ff, b - K);
        }
        break;
      }
      case 0xA: {  // vovo (a i b j): the doubles block
        const int a = p - K, i = q, b = r - K, j = s;
        for (int e = 0; e < K; ++e) v += f(K + b, K + e) * t(i, j, a, e) + f(K + a, K + e) * t(i, j, e, b);
        for (int m = 0; m < K; ++m) v -= f(m, j) * t(i, m, a, b) + f(m, i) * t(m, j, a, b);
        for (int m = 0; m < K; ++m)
          for (int nn = 0; nn < K; ++nn) v += g(m, i, nn, j) * t(m, nn, a, b);
        for (int e = 0; e < K; ++e)
          for (int ff = 0; ff < K; ++ff) v += g(K + a, K + e, K + b, K + ff) * t(i, j, e, ff);
        for (int m = 0; m < K; ++m)
          for (int e = 0; e < K; ++e)
            v += g(m, K + e, K + b, j) * u(i, m, a, e) - g(m, j, K + b, K + e) * t(i, m, a, e) -
                 g(m, i, K + b, K + e) * t(j, m, e, a) - g(m, j, K + a, K + e) * t(i, m, e, b) +
                 g(m, K + e, K + a, i) * u(j, m, b, e) - g(m, i, K + a, K + e) * t(j, m, b, e);
        break;
      }
      default:
        break;  // ooov, ovoo, ovov, ovvv, vvov: no T2-linear term
    }
    return v;
  }
  // T2-linear one-body terms
  __device__ double f2(int p, int q) const {
    double v = 0.0;
    if (p < K && q < K) {  // oo (m i): sum_nef g_menf u_inef
      for (int nn = 0; nn < K; ++nn)
        for (int e = 0; e < K; ++e)
          for (int ff = 0; ff < K; ++ff) v += g(p, K + e, nn, K + ff) * u(q, nn, e, ff);
    } else if (p >= K && q >= K) {  // vv (a e): -sum_mnf g_menf u_mnaf
      for (int m = 0; m < K; ++m)
        for (int nn = 0; nn < K; ++nn)
          for (int ff = 0; ff < K; ++ff) v -= g(m, q, nn, K + ff) * u(m, nn, p - K, ff);
    } else if (p >= K && q < K) {  // vo (a i)
      const int a = p - K, i = q;
      for (int m = 0; m < K; ++m)
        for (int e = 0; e < K; ++e) {
          v += f(m, K + e) * u(i, m, a, e);
          for (int ff = 0; ff < K; ++ff) v += g(p, K + e, m, K + ff) * u(i, m, e, ff);
          for (int nn = 0; nn < K; ++nn) v -= g(m, i, nn, K + e) * u(m, nn, a, e);
        }
    }
    return v;
  }
};

// Wx, Fx, ex = [O, T]_(<=2) for the operator in d.h (vacuum order), d.f (normal order), d.g.
template <int K, int NT>
__device__ void lin_dress(DuccSmem<K>& d) {
  constexpr int NO = 2 * K, NW = NO * NO * NO * NO, NF = NO * NO;
  const LinDress<K> L{d};
  for (int x = threadIdx.x; x < NW; x += NT) {
    const int p = x / (NO * NO * NO), q = (x / (NO * NO)) % NO, r = (x / NO) % NO, s = x % NO;
    d.Wx[x] = L.dg(p, q, r, s) + L.w2(p, q, r, s);
  }
  for (int x = threadIdx.x; x < NF; x += NT) {
    const int p = x / NO, q = x % NO;
    double v = L.dh(p, q) + L.f2(p, q);
    for (int k = 0; k < K; ++k) v += 2.0 * L.dg(p, q, k, k) - L.dg(p, k, k, q);
    d.Fx[x] = v;
  }
  if (threadIdx.x == NT - 1) {
    double e = 0.0;
    for (int k = 0; k < K; ++k) e += 2.0 * L.dh(k, k);
    for (int k = 0; k < K; ++k)
      for (int l = 0; l < K; ++l) e += 2.0 * L.dg(k, k, l, l) - L.dg(k, l, l, k);
    for (int i = 0; i < K; ++i)
      for (int aa = 0; aa < K; ++aa)
        for (int j = 0; j < K; ++j)
          for (int b = 0; b < K; ++b) e += L.g(i, K + aa, j, K + b) * L.u(i, j, aa, b);
    d.ex = e;
  }
  __syncthreads();
}

// W -= c (Wx + Wx^+), F -= c (Fx + Fx^+), e0 -= 2 c ex.
template <int K, int NT>
__device__ void sub_hermitian(const DuccSmem<K>& d, double c, double* W, double* F, double* e0) {
  constexpr int NO = 2 * K, NW = NO * NO * NO * NO, NF = NO * NO;
  for (int x = threadIdx.x; x < NW; x += NT) {
    const int p = x / (NO * NO * NO), q = (x / (NO * NO)) % NO, r = (x / NO) % NO, s = x % NO;
    W[x] -= c * (d.Wx[x] + d.Wx[((q * NO + p) * NO + s) * NO + r]);
  }
  for (int x = threadIdx.x; x < NF; x += NT) F[x] -= c * (d.Fx[x] + d.Fx[(x % NO) * NO + x / NO]);
  if (threadIdx.x == 0) *e0 -= 2.0 * c * d.ex;
  __syncthreads();
}

// The operator's one-body part in normal order: f = h + sum_k (2 g_pqkk - g_pkkq).
template <int K, int NT>
__device__ void fold_up(DuccSmem<K>& d) {
  constexpr int NO = 2 * K, NF = NO * NO;
  for (int x = threadIdx.x; x < NF; x += NT) {
    const int p = x / NO, q = x % NO;
    double v = d.h[x];
    for (int k = 0; k < K; ++k) v += 2.0 * d.g[((p * NO + q) * NO + k) * NO + k] - d.g[((p * NO + k) * NO + k) * NO + q];
    d.f[x] = v;
  }
  __syncthreads();
}

// G|_A (gathered into W, F, e0) minus the space's internal part L_A.
template <int K, int NT>
__device__ void ducc_local(DuccSmem<K>& d, const SolveArgs& a, const int* orb, double* W, double* F, double* e0) {
  constexpr int NO = 2 * K, NW = NO * NO * NO * NO, NF = NO * NO;
  const size_t n1 = a.n, n2 = n1 * n1, n3 = n2 * n1;
  for (int x = threadIdx.x; x < NW; x += NT) {
    const int p = x / (NO * NO * NO), q = (x / (NO * NO)) % NO, r = (x / NO) % NO, s = x % NO;
    d.g[x] = a.ducc_eri[(size_t)orb[p] * n3 + (size_t)orb[q] * n2 + (size_t)orb[r] * n1 + orb[s]];
  }
  for (int x = threadIdx.x; x < NF; x += NT) d.f0[x] = a.ducc_F0[(size_t)orb[x / NO] * n1 + orb[x % NO]];
  for (int x = threadIdx.x; x < K * K; x += NT)
    d.t1[x] = a.t1_old[(size_t)orb[x / K] * a.nvir + (orb[K + x % K] - a.nocc)];
  for (int x = threadIdx.x; x < K * K * K * K; x += NT) {
    const int i = x / (K * K * K), j = (x / (K * K)) % K, aa = (x / K) % K, b = x % K;
    d.t2[x] = a.t2_old[(((size_t)orb[i] * a.nocc + orb[j]) * a.nvir + (orb[K + aa] - a.nocc)) * a.nvir +
                       (orb[K + b] - a.nocc)];
  }
  __syncthreads();
  // X_A: H_A in vacuum order on the space (its normal order gives back the Fock block f0)
  for (int x = threadIdx.x; x < NF; x += NT) {
    const int p = x / NO, q = x % NO;
    double v = d.f0[x];
    for (int k = 0; k < K; ++k) v -= 2.0 * d.g[((p * NO + q) * NO + k) * NO + k] - d.g[((p * NO + k) * NO + k) * NO + q];
    d.h[x] = v;
    d.f[x] = d.f0[x];
  }
  __syncthreads();
  lin_dress<K, NT>(d);
  sub_hermitian<K, NT>(d, 1.0, W, F, e0);
  // Y_A: B_A = D.T_A + (D.T_A)^+, D from the Fock diagonal
  auto eps = [&](int p) { return d.f0[p * NO + p]; };
  for (int x = threadIdx.x; x < NW; x += NT) {
    const int p = x / (NO * NO * NO), q = (x / (NO * NO)) % NO, r = (x / NO) % NO, s = x % NO;
    double v = 0.0;
    if (p >= K && q < K && r >= K && s < K)
      v = (eps(p) + eps(r) - eps(q) - eps(s)) * d.t2[((q * K + s) * K + (p - K)) * K + (r - K)];
    else if (p < K && q >= K && r < K && s >= K)
      v = (eps(q) + eps(s) - eps(p) - eps(r)) * d.t2[((p * K + r) * K + (q - K)) * K + (s - K)];
    d.g[x] = v;
  }
  for (int x = threadIdx.x; x < NF; x += NT) {
    const int p = x / NO, q = x % NO;
    double v = 0.0;
    if (p >= K && q < K) v = (eps(p) - eps(q)) * d.t1[q * K + (p - K)];
    if (p < K && q >= K) v = (eps(q) - eps(p)) * d.t1[p * K + (q - K)];
    d.h[x] = v;
  }
  __syncthreads();
  fold_up<K, NT>(d);
  lin_dress<K, NT>(d);
  sub_hermitian<K, NT>(d, 0.5, W, F, e0);
}

template <int K, typename T, bool DUCC>
__global__ void __launch_bounds__(Cas<K>::NT) solve_kernel(SolveArgs a) {
  using C = Cas<K>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem<K, T>& sm = *reinterpret_cast<Smem<K, T>*>(smem_raw);
  constexpr size_t kDuccOff = (sizeof(Smem<K, T>) + 15) / 16 * 16;
  const int tid = threadIdx.x;
  build_tables<K, T>(sm);
  const int n = a.n;
  const size_t n1 = (size_t)n, n2 = n1 * n1, n3 = n2 * n1;
  const T tol = (T)a.tol;

  const int64_t nitems = a.count_dev ? (int64_t)*a.count_dev : a.nspaces;
  for (int64_t item = blockIdx.x; item < nitems; item += gridDim.x) {
    const int64_t s = a.items ? a.items[item] : item;
    // ---- gather + fold ---------------------------------------------------------------
    if (tid == 0) {
      const qflow_space& q = a.spaces[s];
      int ok = (q.no == K && q.nv == K);
      for (int t = 0; t < 2 * K; ++t) {
        const int o = q.orb[t];
        sm.orb[t] = o;
        if (t < K) ok &= (o >= 0 && o < a.nocc);
        else ok &= (o >= a.nocc && o < a.n);
      }
      sm.ctrl[1] = ok;
      sm.e0 = *a.e0;
    }
    __syncthreads();
    if (!sm.ctrl[1]) {  // malformed space: report and skip (no memory access with its indices)
      if (tid == 0) {
        const int64_t o = a.sorted_index ? a.sorted_index[s] : s;
        a.energy[o] = 0.0;
        a.status[o] = kSpaceInvalid;
        if (a.iters) a.iters[o] = 0;
      }
      __syncthreads();
      continue;
    }
    for (int idx = tid; idx < C::NW; idx += C::NT) {
      const int p = idx / (C::NORB * C::NORB * C::NORB), q = (idx / (C::NORB * C::NORB)) % C::NORB;
      const int r = (idx / C::NORB) % C::NORB, u = idx % C::NORB;
      const double w = a.W[(size_t)sm.orb[p] * n3 + (size_t)sm.orb[q] * n2 + (size_t)sm.orb[r] * n1 + sm.orb[u]];
      sm.W[idx] = w;
      if constexpr (!std::is_same<T, double>::value) sm.Wt[idx] = (T)w;
    }
    for (int idx = tid; idx < C::NF; idx += C::NT)
      sm.F[idx] = a.F[(size_t)sm.orb[idx / C::NORB] * n1 + sm.orb[idx % C::NORB]];
    __syncthreads();
    if constexpr (DUCC) {  // G|_A minus the space's internal part
      DuccSmem<K>& dz = *reinterpret_cast<DuccSmem<K>*>(smem_raw + kDuccOff);
      ducc_local<K, C::NT>(dz, a, sm.orb, sm.W, sm.F, &sm.e0);
      if constexpr (!std::is_same<T, double>::value)
        for (int idx = tid; idx < C::NW; idx += C::NT) sm.Wt[idx] = (T)sm.W[idx];
      __syncthreads();
    }
    for (int idx = tid; idx < C::NF; idx += C::NT) {
      const int p = idx / C::NORB, q = idx % C::NORB;
      double v = sm.F[idx];
      for (int k = 0; k < K; ++k)
        v -= 2.0 * sm.W[((p * C::NORB + q) * C::NORB + k) * C::NORB + k] -
             sm.W[((p * C::NORB + k) * C::NORB + k) * C::NORB + q];
      sm.h[idx] = v;
    }
    __syncthreads();
    if (tid == 0) {
      double ec = sm.e0;
      for (int k = 0; k < K; ++k) ec -= sm.h[k * C::NORB + k] + sm.F[k * C::NORB + k];
      sm.ecore = ec;
    }
    for (int idx = tid; idx < C::NF; idx += C::NT) {
      const int p = idx / C::NORB, q = idx % C::NORB;
      double v = sm.h[idx];
      for (int r = 0; r < C::NORB; ++r) v -= 0.5 * sm.W[((p * C::NORB + r) * C::NORB + r) * C::NORB + q];
      sm.hp[idx] = v;
    }
    __syncthreads();
    // same-spin string operator (row I owned by one thread) and the diagonal
    for (int I = tid; I < C::NS; I += C::NT) {
      double row[C::NS];
      for (int j = 0; j < C::NS; ++j) row[j] = 0.0;
      for (int u = 0; u < C::NSG; ++u) {
        const int e = sm.sing[I * C::NSG + u];
        const int pq = e & 63, Kk = (e >> 6) & 31;
        const double s1 = (e >> 11) ? -1.0 : 1.0;
        row[Kk] += s1 * sm.hp[pq];
        for (int v = 0; v < C::NSG; ++v) {
          const int e2 = sm.sing[Kk * C::NSG + v];
          const double s2 = (e2 >> 11) ? -1.0 : 1.0;
          row[(e2 >> 6) & 31] += 0.5 * s1 * s2 * sm.W[pq * C::NF + (e2 & 63)];
        }
      }
      for (int j = 0; j < C::NS; ++j) sm.Hs[I * C::NS + j] = (T)row[j];
      sm.hsd[I] = row[I];  // diagonal kept in FP64
    }
    __syncthreads();
    auto diag_of = [&](int ia, int ib) {
      const int ma = sm.smask[ia], mb = sm.smask[ib];
      double v = sm.ecore + sm.hsd[ia] + sm.hsd[ib];
      for (int p = 0; p < C::NORB; ++p) {
        if (!((ma >> p) & 1)) continue;
        for (int r = 0; r < C::NORB; ++r)
          if ((mb >> r) & 1) v += sm.W[(p * C::NORB + p) * C::NF + r * C::NORB + r];
      }
      return v;
    };
    if (tid == 0) sm.eshift = diag_of(0, 0);
    __syncthreads();
    for (int d = tid; d < C::NDET; d += C::NT) {
      const int ia = d / C::NS, ib = d % C::NS;
      sm.diag[d] = (T)(diag_of(ia, ib) - sm.eshift);
      // start vector: Phi or the caller's guess
      T g0 = (d == 0) ? (T)1 : (T)0;
      if (a.guess) g0 = static_cast<const T*>(a.guess)[(size_t)s * C::NDET + d];
      sm.V[d] = g0;
    }
    if (tid == 0) {
      sm.ctrl[0] = 1;
      sm.ctrl[1] = 0;
      sm.ctrl[2] = kSpaceNoConv;
      sm.ctrl[3] = 0;
    }
    __syncthreads();
    // The diagonal now lives in diag[]; strip it from the operands of sigma so that sigma
    // sums only off-diagonal couplings (no cancellation between large diagonal terms).
    for (int I = tid; I < C::NS; I += C::NT) sm.Hs[I * C::NS + I] = (T)0;
    for (int pr = tid; pr < C::NF; pr += C::NT) {
      const int p = pr / C::NORB, r = pr % C::NORB;
      const int w = (p * C::NORB + p) * C::NF + r * C::NORB + r;
      if constexpr (std::is_same<T, double>::value) sm.W[w] = 0.0; else sm.Wt[w] = 0.0f;
    }
    __syncthreads();
    {  // normalise the start vector
      T part[C::NRED];
      part[0] = (T)0;
      for (int d = tid; d < C::NDET; d += C::NT) part[0] = fma(sm.V[d], sm.V[d], part[0]);
      block_sums<K, T>(sm, part, 1);
      const double nr = sqrt(sm.out[0]);
      const T inv = (T)((nr > 0.0) ? 1.0 / nr : 0.0);
      for (int d = tid; d < C::NDET; d += C::NT) sm.V[d] = (nr > 0.0) ? sm.V[d] * inv : (T)((d == 0) ? 1 : 0);
      __syncthreads();
    }
    sigma<K, T>(sm, sm.V, sm.S);
    __syncthreads();
    {
      T part[C::NRED];
      part[0] = (T)0;
      for (int d = tid; d < C::NDET; d += C::NT) part[0] = fma(sm.V[d], sm.S[d], part[0]);
      block_sums<K, T>(sm, part, 1);
      if (tid == 0) {
        sm.G[0] = sm.out[0];
        sm.theta = sm.out[0];
        sm.y[0] = 1.0;
      }
      __syncthreads();
    }

    // ---- Davidson ---------------------------------------------------------------------
    for (int it = 0; it < a.max_iter; ++it) {
      int k = sm.ctrl[0];
      if (k == C::KMAX) {  // restart on the current Ritz vector
        for (int d = tid; d < C::NDET; d += C::NT) {
          T xv = (T)0, sv = (T)0;
          for (int j = 0; j < k; ++j) {
            xv = fma((T)sm.y[j], sm.V[j * C::NDET + d], xv);
            sv = fma((T)sm.y[j], sm.S[j * C::NDET + d], sv);
          }
          sm.V[d] = xv;
          sm.S[d] = sv;
        }
        __syncthreads();
        T part[C::NRED];
        part[0] = part[1] = (T)0;
        for (int d = tid; d < C::NDET; d += C::NT) {
          part[0] = fma(sm.V[d], sm.V[d], part[0]);
          part[1] = fma(sm.V[d], sm.S[d], part[1]);
        }
        block_sums<K, T>(sm, part, 2);
        const double nr = sqrt(sm.out[0]);
        const T inv = (T)(1.0 / nr);
        for (int d = tid; d < C::NDET; d += C::NT) {
          sm.V[d] *= inv;
          sm.S[d] *= inv;
        }
        if (tid == 0) {
          sm.G[0] = sm.out[1] / sm.out[0];
          sm.theta = sm.G[0];
          sm.y[0] = 1.0;
          sm.ctrl[0] = 1;
        }
        __syncthreads();
        k = 1;
      }
      // residual r = S y - theta V y; correction = r / (theta - D) into V[k]
      const double th = sm.theta;
      T part[C::NRED];
      part[0] = (T)0;
      for (int d = tid; d < C::NDET; d += C::NT) {
        T xv = (T)0, sv = (T)0;
        for (int j = 0; j < k; ++j) {
          xv = fma((T)sm.y[j], sm.V[j * C::NDET + d], xv);
          sv = fma((T)sm.y[j], sm.S[j * C::NDET + d], sv);
        }
        const T r = sv - (T)th * xv;
        part[0] = fma(r, r, part[0]);
        T den = (T)th - sm.diag[d];
        if (fabs((double)den) < 1e-4) den = (den < (T)0) ? (T)-1e-4 : (T)1e-4;
        sm.V[k * C::NDET + d] = r / den;
      }
      block_sums<K, T>(sm, part, 1);
      const double rnorm = sqrt(sm.out[0]);
      if (!isfinite(rnorm) || !isfinite(th)) {
        if (tid == 0) sm.ctrl[2] = kSpaceNonFinite;
        __syncthreads();
        break;
      }
      if (rnorm < (double)tol) {
        if (tid == 0) {
          sm.ctrl[2] = kSpaceOk;
          sm.ctrl[3] = it;
        }
        __syncthreads();
        break;
      }
      // two passes of classical Gram-Schmidt against V[0..k)
      T* vk = sm.V + k * C::NDET;
      for (int pass = 0; pass < 2; ++pass) {
        for (int j = 0; j < C::NRED; ++j) part[j] = (T)0;
        for (int d = tid; d < C::NDET; d += C::NT)
          for (int j = 0; j < k; ++j) part[j] = fma(sm.V[j * C::NDET + d], vk[d], part[j]);
        block_sums<K, T>(sm, part, k);
        for (int d = tid; d < C::NDET; d += C::NT) {
          T v = vk[d];
          for (int j = 0; j < k; ++j) v -= (T)sm.out[j] * sm.V[j * C::NDET + d];
          vk[d] = v;
        }
        __syncthreads();
      }
      part[0] = (T)0;
      for (int d = tid; d < C::NDET; d += C::NT) part[0] = fma(vk[d], vk[d], part[0]);
      block_sums<K, T>(sm, part, 1);
      const double vn = sqrt(sm.out[0]);
      const double floor_n = std::is_same<T, double>::value ? 1e-13 : 1e-6;
      if (!(vn > floor_n)) {  // subspace cannot grow (complete or stagnated)
        if (tid == 0) {
          sm.ctrl[2] = (rnorm < 100.0 * (double)tol) ? kSpaceOk : kSpaceNoConv;
          sm.ctrl[3] = it;
        }
        __syncthreads();
        break;
      }
      const T inv = (T)(1.0 / vn);
      for (int d = tid; d < C::NDET; d += C::NT) vk[d] *= inv;
      __syncthreads();
      sigma<K, T>(sm, vk, sm.S + k * C::NDET);
      __syncthreads();
      // new row and column of the projected matrix
      for (int j = 0; j < C::NRED; ++j) part[j] = (T)0;
      const T* sk = sm.S + k * C::NDET;
      for (int d = tid; d < C::NDET; d += C::NT) {
        const T vkd = vk[d], skd = sk[d];
        for (int j = 0; j <= k; ++j) part[j] = fma(sm.V[j * C::NDET + d], skd, part[j]);  // G[j][k]
        for (int j = 0; j < k; ++j) part[k + 1 + j] = fma(vkd, sm.S[j * C::NDET + d], part[k + 1 + j]);  // G[k][j]
      }
      block_sums<K, T>(sm, part, 2 * k + 1);
      if (tid == 0) {
        for (int j = 0; j <= k; ++j) sm.G[j * C::KMAX + k] = sm.out[j];
        for (int j = 0; j < k; ++j) sm.G[k * C::KMAX + j] = sm.out[k + 1 + j];
        const int kk = k + 1;
        for (int j = 0; j < kk; ++j) sm.ynew[j] = (j < k) ? sm.y[j] : 0.0;
        double thn = sm.theta;
        int cx = 0;
        if constexpr (DUCC) {  // Hermitian operator: symmetric projected problem, Phi-weight root
          double v0[C::KMAX];
          for (int j = 0; j < kk; ++j) v0[j] = (double)sm.V[j * C::NDET];
          small_eig_sym<C::KMAX>(sm.G, kk, v0, sm.ynew, &thn);
        } else {
          cx = small_eig<C::KMAX>(sm.G, kk, sm.theta - 1e-2, sm.ynew, &thn);
        }
        for (int j = 0; j < kk; ++j) sm.y[j] = sm.ynew[j];
        sm.theta = thn;
        sm.ctrl[0] = kk;
        sm.ctrl[3] = it + 1;
        sm.ctrl[1] = cx ? sm.ctrl[1] + 1 : 0;  // consecutive steps with a complex projected root
        if (sm.ctrl[1] >= 2) sm.ctrl[2] = kSpaceRoot;
      }
      __syncthreads();
      if (sm.ctrl[1] >= 2) break;  // the selected root is complex: no real root to converge to
    }

    // ---- root, increment, merge --------------------------------------------------------
    const int k = sm.ctrl[0];
    for (int d = tid; d < C::NDET; d += C::NT) {
      T xv = (T)0;
      for (int j = 0; j < k; ++j) xv = fma((T)sm.y[j], sm.V[j * C::NDET + d], xv);
      sm.S[d] = xv;  // Ritz vector (S[0] is free now)
    }
    __syncthreads();
    T part[C::NRED];
    part[0] = (T)0;
    for (int d = tid; d < C::NDET; d += C::NT) part[0] = fma(sm.S[d], sm.S[d], part[0]);
    block_sums<K, T>(sm, part, 1);
    const double xn = sqrt(sm.out[0]);
    const double c0 = (double)sm.S[0];
    int st = sm.ctrl[2];
    if (st == kSpaceNoConv && sm.ctrl[1] > 0) st = kSpaceRoot;  // stopped on a complex projected root
    if (st == kSpaceOk && !(fabs(c0) >= 1e-3 * xn)) st = kSpaceRoot;
    if (!isfinite(c0) || !isfinite(sm.theta)) st = kSpaceNonFinite;
    const double inv0 = (st == kSpaceOk || st == kSpaceNoConv) ? 1.0 / c0 : 0.0;
    if (a.root_out && st == kSpaceOk)
      for (int d = tid; d < C::NDET; d += C::NT)
        static_cast<T*>(a.root_out)[(size_t)s * C::NDET + d] = (T)((double)sm.S[d] * inv0);
    if (tid < K * K) {
      const int i = tid / K, aa = tid % K;
      int sg;
      const int m0 = sm.smask[0];
      const int mj = apply_pq(m0, K + aa, i, &sg);
      const int J = sm.mask2idx[mj];
      const double ca = sg * (double)sm.S[J * C::NS] * inv0;
      const double cb = sg * (double)sm.S[J] * inv0;
      sm.x1[tid] = 0.5 * (ca + cb);
    }
    __syncthreads();
    for (int idx = tid; idx < K * K * K * K; idx += C::NT) {
      const int i = idx / (K * K * K), j = (idx / (K * K)) % K, aa = (idx / K) % K, b = idx % K;
      int sa, sb;
      const int m0 = sm.smask[0];
      const int ja = sm.mask2idx[apply_pq(m0, K + aa, i, &sa)];
      const int jbb = sm.mask2idx[apply_pq(m0, K + b, j, &sb)];
      const double cab = (double)(sa * sb) * (double)sm.S[ja * C::NS + jbb] * inv0;
      sm.x2raw[idx] = cab - sm.x1[i * K + aa] * sm.x1[j * K + b];
    }
    __syncthreads();
    const int64_t sidx = a.sorted_index ? a.sorted_index[s] : a.space_base + s;
    const bool write = (st == kSpaceOk);
    if (write && a.owner1) {
      for (int idx = tid; idx < K * K; idx += C::NT) {
        const int i = idx / K, aa = idx % K;
        const size_t g = (size_t)sm.orb[i] * a.nvir + (sm.orb[K + aa] - a.nocc);
        if (a.owner1[g] == sidx) a.t1_new[g] = (DUCC ? 0.0 : a.t1_old[g]) + sm.x1[idx];  // DUCC: replaced
      }
    }
    if (write && a.owner2) {
      for (int idx = tid; idx < K * K * K * K; idx += C::NT) {
        const int i = idx / (K * K * K), j = (idx / (K * K)) % K, aa = (idx / K) % K, b = idx % K;
        const size_t g = (((size_t)sm.orb[i] * a.nocc + sm.orb[j]) * a.nvir + (sm.orb[K + aa] - a.nocc)) * a.nvir +
                         (sm.orb[K + b] - a.nocc);
        if (a.owner2[g] == sidx) {
          const double x = 0.5 * (sm.x2raw[idx] + sm.x2raw[((j * K + i) * K + b) * K + aa]);
          a.t2_new[g] = (DUCC ? 0.0 : a.t2_old[g]) + x;
        }
      }
    }
    if (tid == 0) {
      const int64_t o = a.sorted_index ? sidx : s;  // outputs in sorted order when indexed
      a.energy[o] = sm.eshift + sm.theta;
      a.status[o] = st;
      if (a.iters) a.iters[o] = sm.ctrl[3];
    }
    __syncthreads();
  }
}

template <int K, typename T, bool DUCC>
cudaError_t launch_k(const SolveArgs& a, cudaStream_t st) {
  using C = Cas<K>;
  if (a.nspaces <= 0) return cudaSuccess;
  const size_t smem = (sizeof(Smem<K, T>) + 15) / 16 * 16 + (DUCC ? sizeof(DuccSmem<K>) : 0);
  cudaError_t e =
      cudaFuncSetAttribute(solve_kernel<K, T, DUCC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, solve_kernel<K, T, DUCC>, C::NT, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  int64_t grid = (int64_t)sms * per_sm;
  if (grid > a.nspaces) grid = a.nspaces;
  solve_kernel<K, T, DUCC><<<(unsigned)grid, C::NT, smem, st>>>(a);
  return cudaGetLastError();
}

// Positions (in a's item numbering) of the spaces whose status is kSpaceNoConv.
__global__ void k_collect_noconv(SolveArgs a, int64_t* __restrict__ items, unsigned long long* __restrict__ count) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.nspaces; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = a.items ? a.items[i] : i;
    const int64_t o = a.sorted_index ? a.sorted_index[s] : s;
    if (a.status[o] == kSpaceNoConv) items[atomicAdd(count, 1ull)] = s;
  }
}

cudaError_t launch_fp64(int k, const SolveArgs& a, cudaStream_t st) {
  const bool ducc = a.ducc_eri != nullptr && a.ducc_F0 != nullptr;
  switch (k) {
    case 1: return ducc ? launch_k<1, double, true>(a, st) : launch_k<1, double, false>(a, st);
    case 2: return ducc ? launch_k<2, double, true>(a, st) : launch_k<2, double, false>(a, st);
    case 3: return ducc ? launch_k<3, double, true>(a, st) : launch_k<3, double, false>(a, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t launch_solve_rescue(int k, const SolveArgs& a, int64_t* items, unsigned long long* count,
                                cudaStream_t st) {
  if (a.nspaces <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(count, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  const int64_t blocks = (a.nspaces + 255) / 256;
  k_collect_noconv<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, st>>>(a, items, count);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  SolveArgs b = a;
  b.items = items;  // positions are class positions: b.spaces / b.sorted_index index them as before
  b.count_dev = count;
  b.guess = nullptr;
  b.root_out = nullptr;
  return launch_fp64(k, b, st);
}

cudaError_t launch_solve(int k, int precision, const SolveArgs& a, cudaStream_t st) {
  if (precision == QFLOW_PREC_MIXED) {
    SolveArgs w = a;
    if (w.max_iter > kWarpIterCap) w.max_iter = kWarpIterCap;
    return launch_solve_warp(k, w, a.W32, static_cast<const float*>(a.guess), static_cast<float*>(a.root_out), 0,
                             st);
  }
  return launch_fp64(k, a, st);
}

}  // namespace qf
