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

template <int K, typename T>
__global__ void __launch_bounds__(Cas<K>::NT) solve_kernel(SolveArgs a) {
  using C = Cas<K>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem<K, T>& sm = *reinterpret_cast<Smem<K, T>*>(smem_raw);
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
        const int cx = small_eig<C::KMAX>(sm.G, kk, sm.theta - 1e-2, sm.ynew, &thn);
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
        if (a.owner1[g] == sidx) a.t1_new[g] = a.t1_old[g] + sm.x1[idx];
      }
    }
    if (write && a.owner2) {
      for (int idx = tid; idx < K * K * K * K; idx += C::NT) {
        const int i = idx / (K * K * K), j = (idx / (K * K)) % K, aa = (idx / K) % K, b = idx % K;
        const size_t g = (((size_t)sm.orb[i] * a.nocc + sm.orb[j]) * a.nvir + (sm.orb[K + aa] - a.nocc)) * a.nvir +
                         (sm.orb[K + b] - a.nocc);
        if (a.owner2[g] == sidx) {
          const double x = 0.5 * (sm.x2raw[idx] + sm.x2raw[((j * K + i) * K + b) * K + aa]);
          a.t2_new[g] = a.t2_old[g] + x;
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

template <int K, typename T>
cudaError_t launch_k(const SolveArgs& a, cudaStream_t st) {
  using C = Cas<K>;
  if (a.nspaces <= 0) return cudaSuccess;
  const size_t smem = sizeof(Smem<K, T>);
  cudaError_t e = cudaFuncSetAttribute(solve_kernel<K, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, solve_kernel<K, T>, C::NT, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  int64_t grid = (int64_t)sms * per_sm;
  if (grid > a.nspaces) grid = a.nspaces;
  solve_kernel<K, T><<<(unsigned)grid, C::NT, smem, st>>>(a);
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
  switch (k) {
    case 1: return launch_k<1, double>(a, st);
    case 2: return launch_k<2, double>(a, st);
    case 3: return launch_k<3, double>(a, st);
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
