// Step (a) of a flow sweep: the dressed one- and two-body integrals that define every active
// space's downfolded Hamiltonian (Eqs. 5-8, N = 1, SES-CC reading):
//   H-bar = e^{-T} H e^{T},  T = T1 + T2 = the current global amplitude pool,
// normal ordered with respect to the closed-shell reference and truncated to <= two-body:
//   E0, F[p][q], W[p][q][r][s] (creators p, r; annihilators q, s; W[pqrs] = W[rspq]).
//
// Construction (one thread per output element, or one block per element for the few long
// sums; the T2 contractions run in FP64, or for the mixed-precision path on the tensor cores
// (tcgen05 GEMMs with three-term TF32 operands and FP32 accumulation, tc_gemm.cuh) on an FP32
// copy of g~ and t2, their FP64 base values being added in FP64):
//   1. T1 exactly: orbital similarity transform of the integrals; creators by (1 - K),
//      annihilators by (1 + K), K_ai = t_i^a (K^2 = 0) -> h~, g~ (four in-place passes).
//   2. f~ = h~ + sum_k [2 g~_pqkk - g~_pkkq], E~ = <Phi|H~|Phi>.
//   3. T2 through its connected contractions with H~ (one- and two-body parts of [H~, T2];
//      the quadratic term 1/2 [[H~,T2],T2] only reaches the doubly excited (vo|vo) block).
//      The mixed path adds the vvvv block's term only where at most three of the four
//      virtual indices differ: every element a (k, k) space with k <= 3 reads.
// Index names: occupied i j k l m n, virtual a b e f (absolute index nocc + a).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "qflow_internal.h"
#include "tc_gemm.cuh"

namespace qf {
namespace {

struct Dims {
  int n, o, v;
};

__device__ __forceinline__ size_t gi(const Dims& d, int p, int q, int r, int s) {
  return (((size_t)p * d.n + q) * d.n + r) * d.n + s;
}
__device__ __forceinline__ size_t ti(const Dims& d, int i, int j, int a, int b) {
  return (((size_t)i * d.o + j) * d.v + a) * d.v + b;
}

constexpr int TPB = 256;
inline unsigned blocks_for(size_t m) { return (unsigned)((m + TPB - 1) / TPB); }

__global__ void k_copy(const double* __restrict__ src, double* __restrict__ dst, size_t m) {
  for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < m; x += (size_t)gridDim.x * blockDim.x)
    dst[x] = src[x];
}

// IEEE-754 conversions between binary64 and binary32 by field arithmetic on the integer pipe
// (GB300 converts floating types on its slow FP64 pipe).  double -> float truncates the
// significand (error below one float ulp) and flushes values below the normal float range to
// zero; float -> double is exact for normal floats (subnormals flush to zero).  Used only for
// the mixed path's FP32 correction sums, whose operands are normal and far from overflow.
__device__ __forceinline__ float d2f_bits(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned sign = hi & 0x80000000u;
  const int ef = (int)((hi >> 20) & 0x7FFu) - 1023 + 127;
  if (ef <= 0) return __uint_as_float(sign);
  if (ef >= 255) return __uint_as_float(sign | 0x7F800000u);
  return __uint_as_float(sign | ((unsigned)ef << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29));
}
__device__ __forceinline__ double f2d_bits(float f) {
  const unsigned u = __float_as_uint(f), sign = u & 0x80000000u, e = (u >> 23) & 0xFFu;
  if (e == 0) return __hiloint2double((int)sign, 0);
  const unsigned hi = sign | ((e - 127u + 1023u) << 20) | ((u & 0x7FFFFFu) >> 3);
  return __hiloint2double((int)hi, (int)((u & 7u) << 29));
}
template <typename A>
__device__ __forceinline__ A to_acc(double x) {
  if constexpr (sizeof(A) == 4) return d2f_bits(x);
  else return x;
}
template <typename A>
__device__ __forceinline__ double from_acc(A x) {
  if constexpr (sizeof(A) == 4) return f2d_bits(x);
  else return x;
}

// Creator index `pos` (0 or 2): rows p >= nocc get  - sum_i t1[i][p-nocc] * row_i.
// The correction sum runs in precision A (FP64, or FP32 for the mixed path) and is added to
// the FP64 element.
template <typename A>
__global__ void k_t1_creator(double* __restrict__ W, const double* __restrict__ t1, Dims d, int pos) {
  const size_t m = (size_t)d.v * d.n * d.n * d.n;
  for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < m; x += (size_t)gridDim.x * blockDim.x) {
    const int a = (int)(x / ((size_t)d.n * d.n * d.n));
    const size_t rest = x % ((size_t)d.n * d.n * d.n);
    const int u = (int)(rest / ((size_t)d.n * d.n)), w = (int)((rest / d.n) % d.n), z = (int)(rest % d.n);
    A acc = 0;
    if (pos == 0) {
      for (int i = 0; i < d.o; ++i) acc += to_acc<A>(t1[i * d.v + a]) * to_acc<A>(W[gi(d, i, u, w, z)]);
      W[gi(d, d.o + a, u, w, z)] -= from_acc<A>(acc);
    } else {
      for (int i = 0; i < d.o; ++i) acc += to_acc<A>(t1[i * d.v + a]) * to_acc<A>(W[gi(d, u, w, i, z)]);
      W[gi(d, u, w, d.o + a, z)] -= from_acc<A>(acc);
    }
  }
}

// Annihilator index `pos` (1 or 3): rows q < nocc get  + sum_a t1[q][a] * row_(nocc+a).
template <typename A>
__global__ void k_t1_annihilator(double* __restrict__ W, const double* __restrict__ t1, Dims d, int pos) {
  const size_t m = (size_t)d.o * d.n * d.n * d.n;
  for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < m; x += (size_t)gridDim.x * blockDim.x) {
    const int q = (int)(x / ((size_t)d.n * d.n * d.n));
    const size_t rest = x % ((size_t)d.n * d.n * d.n);
    const int u = (int)(rest / ((size_t)d.n * d.n)), w = (int)((rest / d.n) % d.n), z = (int)(rest % d.n);
    A acc = 0;
    if (pos == 1) {
      for (int a = 0; a < d.v; ++a) acc += to_acc<A>(t1[q * d.v + a]) * to_acc<A>(W[gi(d, u, d.o + a, w, z)]);
      W[gi(d, u, q, w, z)] += from_acc<A>(acc);
    } else {
      for (int a = 0; a < d.v; ++a) acc += to_acc<A>(t1[q * d.v + a]) * to_acc<A>(W[gi(d, u, w, z, d.o + a)]);
      W[gi(d, u, w, z, q)] += from_acc<A>(acc);
    }
  }
}

// The same four passes with each element read once per pass: thread per index triple (the
// three positions other than the transformed one), t1 in shared memory, the occupied-index
// values (creator) or the o accumulators (annihilator) in registers.  Used when o <= kT1Omax.
// Shared t1 is stored transposed, t1s[a][i] with rows padded to kT1Omax (zeros), so the o
// coefficients of one virtual index come in 16-byte loads that every lane shares.
constexpr int kT1Omax = 16;
// FP32 sums: resident CTAs per SM the register budget keeps (5 x 256 threads; the creator
// pass, which holds no accumulators, 6)
constexpr int kT1Blocks = 5;

template <typename A>
__device__ __forceinline__ void load_t1_t(const double* __restrict__ t1, A* t1s, const Dims& d) {
  for (int x = threadIdx.x; x < d.v * kT1Omax; x += blockDim.x) {
    const int a = x / kT1Omax, i = x % kT1Omax;
    t1s[x] = (i < d.o) ? to_acc<A>(t1[i * d.v + a]) : (A)0;
  }
  __syncthreads();
}
// the kT1Omax coefficients t1[0..o)[a] (then zeros) of virtual index a
template <typename A>
__device__ __forceinline__ void t1_row(const A* t1s, int a, A (&c)[kT1Omax]) {
  static_assert(kT1Omax * sizeof(A) % 16 == 0, "16-byte rows");
  const uint4* r = reinterpret_cast<const uint4*>(t1s + a * kT1Omax);
#pragma unroll
  for (int q = 0; q < kT1Omax * (int)sizeof(A) / 16; ++q) {
    const uint4 u = r[q];
    memcpy(reinterpret_cast<unsigned char*>(c) + 16 * q, &u, 16);
  }
}

template <typename A, int POS>
__device__ __forceinline__ size_t t1_index(const Dims& d, int p, size_t rest) {
  const size_t n1 = d.n, n2 = n1 * n1;
  const size_t u = rest / n2, w = (rest / n1) % n1, z = rest % n1;
  // the transformed index p sits at position POS; (u, w, z) fill the other three in order
  if constexpr (POS == 0) return ((size_t)p * n1 + u) * n2 + w * n1 + z;
  else if constexpr (POS == 1) return ((u * n1 + p) * n1 + w) * n1 + z;
  else if constexpr (POS == 2) return ((u * n1 + w) * n1 + p) * n1 + z;
  else return ((u * n1 + w) * n1 + z) * n1 + p;
}

template <typename A, int POS>
__global__ void __launch_bounds__(TPB, sizeof(A) == 4 ? kT1Blocks + 1 : 1) k_t1_creator_fast(double* __restrict__ W, const double* __restrict__ t1, Dims d) {
  extern __shared__ __align__(16) double t1raw[];  // [v][kT1Omax], in the accumulation type
  A* t1s = reinterpret_cast<A*>(t1raw);
  load_t1_t<A>(t1, t1s, d);
  const size_t m = (size_t)d.n * d.n * d.n;
  for (size_t rest = blockIdx.x * (size_t)blockDim.x + threadIdx.x; rest < m; rest += (size_t)gridDim.x * blockDim.x) {
    A wi[kT1Omax];
#pragma unroll
    for (int i = 0; i < kT1Omax; ++i) wi[i] = (i < d.o) ? to_acc<A>(W[t1_index<A, POS>(d, i, rest)]) : (A)0;
    for (int a = 0; a < d.v; ++a) {
      A c[kT1Omax];
      t1_row<A>(t1s, a, c);
      A acc = 0;
#pragma unroll
      for (int i = 0; i < kT1Omax; ++i)
        if (i < d.o) acc += c[i] * wi[i];
      W[t1_index<A, POS>(d, d.o + a, rest)] -= from_acc<A>(acc);
    }
  }
}

// The first pass of the fast form also copies: it reads the bare integrals and writes every row
// of W (occupied rows unchanged, virtual rows corrected), so no separate copy pass reads and
// writes W first.  Same arithmetic as k_t1_creator_fast at POS 0.
template <typename A>
__global__ void __launch_bounds__(TPB, sizeof(A) == 4 ? kT1Blocks : 1) k_t1_creator_copy(const double* __restrict__ src, double* __restrict__ W, const double* __restrict__ t1,
                                  Dims d) {
  extern __shared__ __align__(16) double t1raw[];  // [v][kT1Omax], in the accumulation type
  A* t1s = reinterpret_cast<A*>(t1raw);
  load_t1_t<A>(t1, t1s, d);
  const size_t m = (size_t)d.n * d.n * d.n;
  for (size_t rest = blockIdx.x * (size_t)blockDim.x + threadIdx.x; rest < m; rest += (size_t)gridDim.x * blockDim.x) {
    A wi[kT1Omax];
#pragma unroll
    for (int i = 0; i < kT1Omax; ++i) {
      wi[i] = (A)0;
      if (i < d.o) {
        const size_t g = t1_index<A, 0>(d, i, rest);
        const double x = src[g];
        W[g] = x;
        wi[i] = to_acc<A>(x);
      }
    }
    for (int a = 0; a < d.v; ++a) {
      A c[kT1Omax];
      t1_row<A>(t1s, a, c);
      A acc = 0;
#pragma unroll
      for (int i = 0; i < kT1Omax; ++i)
        if (i < d.o) acc += c[i] * wi[i];
      const size_t g = t1_index<A, 0>(d, d.o + a, rest);
      W[g] = src[g] - from_acc<A>(acc);
    }
  }
}

template <typename A, int POS>
__global__ void __launch_bounds__(TPB, sizeof(A) == 4 ? kT1Blocks : 1) k_t1_annihilator_fast(double* __restrict__ W, const double* __restrict__ t1, Dims d) {
  extern __shared__ __align__(16) double t1raw[];  // [v][kT1Omax], in the accumulation type
  A* t1s = reinterpret_cast<A*>(t1raw);
  load_t1_t<A>(t1, t1s, d);
  const size_t m = (size_t)d.n * d.n * d.n;
  for (size_t rest = blockIdx.x * (size_t)blockDim.x + threadIdx.x; rest < m; rest += (size_t)gridDim.x * blockDim.x) {
    A acc[kT1Omax];
#pragma unroll
    for (int q = 0; q < kT1Omax; ++q) acc[q] = 0;
    for (int a = 0; a < d.v; ++a) {
      const A wa = to_acc<A>(W[t1_index<A, POS>(d, d.o + a, rest)]);
      A c[kT1Omax];
      t1_row<A>(t1s, a, c);
#pragma unroll
      for (int q = 0; q < kT1Omax; ++q)
        if (q < d.o) acc[q] += c[q] * wa;
    }
#pragma unroll
    for (int q = 0; q < kT1Omax; ++q)
      if (q < d.o) W[t1_index<A, POS>(d, q, rest)] += from_acc<A>(acc[q]);
  }
}

template <typename A>
void t1_passes(const double* eri, double* W, const double* t1, const Dims& d, cudaStream_t st) {
  const size_t mc = (size_t)d.v * d.n * d.n * d.n, ma = (size_t)d.o * d.n * d.n * d.n;
  const size_t n3 = (size_t)d.n * d.n * d.n;
  if (d.o <= kT1Omax) {
    const size_t sm = sizeof(A) * kT1Omax * d.v;
    const unsigned g = blocks_for(n3) > 152u * 16u ? 152u * 16u : blocks_for(n3);
    k_t1_creator_copy<A><<<g, TPB, sm, st>>>(eri, W, t1, d);
    k_t1_creator_fast<A, 2><<<g, TPB, sm, st>>>(W, t1, d);
    k_t1_annihilator_fast<A, 1><<<g, TPB, sm, st>>>(W, t1, d);
    k_t1_annihilator_fast<A, 3><<<g, TPB, sm, st>>>(W, t1, d);
  } else {
    const size_t n4 = n3 * d.n;
    k_copy<<<blocks_for(n4) > 152u * 64u ? 152u * 64u : blocks_for(n4), TPB, 0, st>>>(eri, W, n4);
    k_t1_creator<A><<<blocks_for(mc), TPB, 0, st>>>(W, t1, d, 0);
    k_t1_creator<A><<<blocks_for(mc), TPB, 0, st>>>(W, t1, d, 2);
    k_t1_annihilator<A><<<blocks_for(ma), TPB, 0, st>>>(W, t1, d, 1);
    k_t1_annihilator<A><<<blocks_for(ma), TPB, 0, st>>>(W, t1, d, 3);
  }
}

// h~ = (1 - K) h (1 + K)
__global__ void k_h_tilde(const double* __restrict__ h, const double* __restrict__ t1, double* __restrict__ ht, Dims d) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= d.n * d.n) return;
  const int r = x / d.n, s = x % d.n;
  // (h (1+K))_{p s} = h_ps + [s occ] sum_a h_{p,nocc+a} t1[s][a]
  auto hk = [&](int p) {
    double v = h[p * d.n + s];
    if (s < d.o)
      for (int a = 0; a < d.v; ++a) v += h[p * d.n + d.o + a] * t1[s * d.v + a];
    return v;
  };
  double v = hk(r);
  if (r >= d.o)
    for (int i = 0; i < d.o; ++i) v -= t1[i * d.v + (r - d.o)] * hk(i);
  ht[x] = v;
}

// f~ = h~ + sum_k [2 g~_pqkk - g~_pkkq]
__global__ void k_fock(const double* __restrict__ ht, const double* __restrict__ W, double* __restrict__ F, Dims d) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= d.n * d.n) return;
  const int p = x / d.n, q = x % d.n;
  double v = ht[x];
  for (int k = 0; k < d.o; ++k) v += 2.0 * W[gi(d, p, q, k, k)] - W[gi(d, p, k, k, q)];
  F[x] = v;
}

// E0 = sum_k 2 h~_kk + sum_kl [2 g~_kkll - g~_kllk] + sum_ijab g~_iajb (2 t_ij^ab - t_ij^ba).
// Fixed-order reduction: EGRID block partials (grid-stride), then one block sums them in order.
constexpr int EGRID = 256;
__global__ void k_energy_part(const double* __restrict__ ht, const double* __restrict__ W,
                              const double* __restrict__ t2, double* __restrict__ part, Dims d) {
  __shared__ double red[TPB];
  double acc = 0.0;
  const size_t m = (size_t)d.o * d.o * d.v * d.v;
  for (size_t x = blockIdx.x * (size_t)TPB + threadIdx.x; x < m; x += (size_t)EGRID * TPB) {
    const int i = (int)(x / ((size_t)d.o * d.v * d.v)), j = (int)((x / ((size_t)d.v * d.v)) % d.o);
    const int a = (int)((x / d.v) % d.v), b = (int)(x % d.v);
    acc += W[gi(d, i, d.o + a, j, d.o + b)] * (2.0 * t2[x] - t2[ti(d, i, j, b, a)]);
  }
  if (blockIdx.x == 0) {
    for (int x = threadIdx.x; x < d.o * d.o; x += TPB) {
      const int k = x / d.o, l = x % d.o;
      acc += 2.0 * W[gi(d, k, k, l, l)] - W[gi(d, k, l, l, k)];
    }
    for (int k = threadIdx.x; k < d.o; k += TPB) acc += 2.0 * ht[k * d.n + k];
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = TPB / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void k_energy_sum(const double* __restrict__ part, double* __restrict__ e0) {
  __shared__ double red[EGRID];
  red[threadIdx.x] = part[threadIdx.x];
  __syncthreads();
  for (int s = EGRID / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) *e0 = red[0];
}

// u = 2 t_ij^ab - t_ij^ba in the contraction precision T
template <typename T>
__device__ __forceinline__ T Ut(const T* t2, const Dims& d, int i, int j, int a, int b) {
  return (T)2 * t2[ti(d, i, j, a, b)] - t2[ti(d, i, j, b, a)];
}

// Fixed-order block sum (TPB threads) of a per-thread partial; result valid in thread 0.
__device__ __forceinline__ double block_sum(double v, double* red) {
  red[threadIdx.x] = v;
  __syncthreads();
  for (int s = TPB / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  const double r = red[0];
  __syncthreads();
  return r;
}

// One block per output element (FP64, these outputs are few and their sums long):
//   Foo[m][i] = f~_mi + sum_nef g~_menf u_in^ef           (blocks 0 .. o^2-1)
//   Fvv[a][e] = f~_ae - sum_mnf g~_menf u_mn^af           (next v^2 blocks)
//   R1[a][i]  = f~_ai + sum_me f~_me u_im^ae + sum_mef g~_aemf u_im^ef - sum_mne g~_mine u_mn^ae
//   Woooo[k][i][l][j] = g~_kilj + sum_ef g~_kelf t_ij^ef
// u[i j a b] = 2 t_ij^ab - t_ij^ba once per dressing (the small blocks read it many times)
__global__ void k_make_u(const double* __restrict__ t2, double* __restrict__ U, Dims d) {
  const size_t m = (size_t)d.o * d.o * d.v * d.v;
  for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < m; x += (size_t)gridDim.x * blockDim.x) {
    const int b = (int)(x % d.v), a = (int)((x / d.v) % d.v);
    const int j = (int)((x / ((size_t)d.v * d.v)) % d.o), i = (int)(x / ((size_t)d.v * d.v * d.o));
    U[x] = Ut(t2, d, i, j, a, b);
  }
}

// Index walk of a grid-stride loop over t = (x0 n1 + x1) n2 + x2 (x2 fastest) in steps of
// `step`: the digits advance by the step's own digits with carries instead of three divisions
// per term (the same t sequence, so the same summation order).
struct Walk3 {
  int x0, x1, x2, s0, s1, s2, n1, n2;
  __device__ Walk3(int t, int step, int n1_, int n2_) : n1(n1_), n2(n2_) {
    x2 = t % n2;
    x1 = (t / n2) % n1;
    x0 = t / (n1 * n2);
    s2 = step % n2;
    s1 = (step / n2) % n1;
    s0 = step / (n1 * n2);
  }
  __device__ __forceinline__ void next() {
    x2 += s2;
    int c = x2 >= n2;
    x2 -= c ? n2 : 0;
    x1 += s1 + c;
    c = x1 >= n1;
    x1 -= c ? n1 : 0;
    x0 += s0 + c;
  }
};

__global__ void k_small_blocks(const double* __restrict__ F, const double* __restrict__ W,
                               const double* __restrict__ U, const double* __restrict__ t2, double* __restrict__ foo, double* __restrict__ fvv,
                               double* __restrict__ r1, double* __restrict__ wo, Dims d) {
  __shared__ double red[TPB];
  const int o = d.o, v = d.v;
  const size_t n1 = d.n, n2 = n1 * n1, n3 = n2 * n1;
  const int x = blockIdx.x;
  double acc = 0.0;
  if (x < o * o) {
    const int m = x / o, i = x % o;
    // t = (nn, e, f): W[m, o+e, nn, o+f] U[i, nn, e, f]
    for (Walk3 w(threadIdx.x, TPB, v, v); w.x0 < o; w.next()) {
      const int nn = w.x0, e = w.x1, f = w.x2;
      acc += W[(size_t)m * n3 + (size_t)(o + e) * n2 + (size_t)nn * n1 + (o + f)] *
             U[((i * o + nn) * v + e) * v + f];
    }
    acc = block_sum(acc, red);
    if (threadIdx.x == 0) foo[x] = F[m * d.n + i] + acc;
  } else if (x < o * o + v * v) {
    const int y = x - o * o, a = y / v, e = y % v;
    // t = (m, nn, f): W[m, o+e, nn, o+f] U[m, nn, a, f]
    for (Walk3 w(threadIdx.x, TPB, o, v); w.x0 < o; w.next()) {
      const int m = w.x0, nn = w.x1, f = w.x2;
      acc -= W[(size_t)m * n3 + (size_t)(o + e) * n2 + (size_t)nn * n1 + (o + f)] *
             U[((m * o + nn) * v + a) * v + f];
    }
    acc = block_sum(acc, red);
    if (threadIdx.x == 0) fvv[y] = F[(o + a) * d.n + o + e] + acc;
  } else if (x < o * o + v * v + v * o) {
    const int y = x - o * o - v * v, a = y / o, i = y % o;
    // t = (m, e, f): W[o+a, o+e, m, o+f] U[i, m, e, f]
    for (Walk3 w(threadIdx.x, TPB, v, v); w.x0 < o; w.next()) {
      const int m = w.x0, e = w.x1, f = w.x2;
      acc += W[(size_t)(o + a) * n3 + (size_t)(o + e) * n2 + (size_t)m * n1 + (o + f)] *
             U[((i * o + m) * v + e) * v + f];
    }
    // t = (m, nn, e): W[m, i, nn, o+e] U[m, nn, a, e]
    for (Walk3 w(threadIdx.x, TPB, o, v); w.x0 < o; w.next()) {
      const int m = w.x0, nn = w.x1, e = w.x2;
      acc -= W[(size_t)m * n3 + (size_t)i * n2 + (size_t)nn * n1 + (o + e)] * U[((m * o + nn) * v + a) * v + e];
    }
    // t = (m, e): F[m, o+e] U[i, m, a, e]
    for (Walk3 w(threadIdx.x, TPB, o, v); w.x0 < 1; w.next()) {
      const int m = w.x1, e = w.x2;
      acc += F[m * d.n + o + e] * U[((i * o + m) * v + a) * v + e];
    }
    acc = block_sum(acc, red);
    if (threadIdx.x == 0) r1[y] = F[(o + a) * d.n + i] + acc;
  } else {
    const int y = x - o * o - v * v - v * o;
    const int k = y / (o * o * o), i = (y / (o * o)) % o, l = (y / o) % o, j = y % o;
    // t = (e, f): W[k, o+e, l, o+f] t2[i, j, e, f]
    for (Walk3 w(threadIdx.x, TPB, v, v); w.x0 < 1; w.next()) {
      const int e = w.x1, f = w.x2;
      acc += W[(size_t)k * n3 + (size_t)(o + e) * n2 + (size_t)l * n1 + (o + f)] * t2[((i * o + j) * v + e) * v + f];
    }
    acc = block_sum(acc, red);
    if (threadIdx.x == 0) wo[y] = W[gi(d, k, i, l, j)] + acc;
  }
}

// Ring intermediates for the quadratic doubles terms, each [i][a][n][f] (o v o v), precision T:
//   A = sum_me u_im^ae g~_menf,  B = sum_me u_im^ae g~_mfne,  Cq = sum_me t_im^ae g~_mfne,
//   D[j][a][n][f] = sum_me t_jm^ea g~_mfne
template <typename T>
__global__ void k_rings(const T* __restrict__ G, const T* __restrict__ t2, T* __restrict__ A, T* __restrict__ B,
                        T* __restrict__ Cq, T* __restrict__ D, Dims d) {
  const size_t m_all = (size_t)d.o * d.v * d.o * d.v;
  const size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (x >= m_all) return;
  const int i = (int)(x / ((size_t)d.v * d.o * d.v)), a = (int)((x / ((size_t)d.o * d.v)) % d.v);
  const int nn = (int)((x / d.v) % d.o), f = (int)(x % d.v);
  T sa = 0, sb = 0, sc = 0, sd = 0;
  for (int m = 0; m < d.o; ++m)
    for (int e = 0; e < d.v; ++e) {
      const T g1 = G[gi(d, m, d.o + e, nn, d.o + f)];
      const T g2 = G[gi(d, m, d.o + f, nn, d.o + e)];
      const T t = t2[ti(d, i, m, a, e)];
      const T tx = t2[ti(d, i, m, e, a)];
      const T u = (T)2 * t - tx;
      sa += u * g1;
      sb += u * g2;
      sc += t * g2;
      sd += tx * g2;
    }
  A[x] = sa;
  B[x] = sb;
  Cq[x] = sc;
  D[x] = sd;
}

// R2[i][j][a][b] = <Phi_{ij}^{ab}|H-bar|Phi> (alpha-beta): bare g~ vo|vo (FP64, from W) plus the
// T2 terms in precision T (G: g~ in precision T; W is only read at untouched bare blocks).
template <typename T>
__global__ void k_r2(const double* __restrict__ W, const T* __restrict__ G, const T* __restrict__ t2,
                     const double* __restrict__ foo, const double* __restrict__ fvv, const double* __restrict__ wo,
                     const T* __restrict__ A, const T* __restrict__ B, const T* __restrict__ Cq,
                     const T* __restrict__ D, double* __restrict__ r2, Dims d) {
  const size_t m_all = (size_t)d.o * d.o * d.v * d.v;
  const size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (x >= m_all) return;
  const int i = (int)(x / ((size_t)d.o * d.v * d.v)), j = (int)((x / ((size_t)d.v * d.v)) % d.o);
  const int a = (int)((x / d.v) % d.v), b = (int)(x % d.v);
  const int A_ = d.o + a, B_ = d.o + b;
  T v = 0;
  for (int e = 0; e < d.v; ++e)
    v += (T)fvv[b * d.v + e] * t2[ti(d, i, j, a, e)] + (T)fvv[a * d.v + e] * t2[ti(d, i, j, e, b)];
  for (int m = 0; m < d.o; ++m)
    v -= (T)foo[m * d.o + j] * t2[ti(d, i, m, a, b)] + (T)foo[m * d.o + i] * t2[ti(d, m, j, a, b)];
  for (int m = 0; m < d.o; ++m)
    for (int nn = 0; nn < d.o; ++nn) v += (T)wo[((m * d.o + i) * d.o + nn) * d.o + j] * t2[ti(d, m, nn, a, b)];
  // particle-particle ladder
  for (int e = 0; e < d.v; ++e)
    for (int f = 0; f < d.v; ++f) v += G[gi(d, A_, d.o + e, B_, d.o + f)] * t2[ti(d, i, j, e, f)];
  // linear rings
  for (int m = 0; m < d.o; ++m)
    for (int e = 0; e < d.v; ++e) {
      const int E_ = d.o + e;
      v += G[gi(d, m, E_, B_, j)] * Ut(t2, d, i, m, a, e);
      v -= G[gi(d, m, j, B_, E_)] * t2[ti(d, i, m, a, e)];
      v -= G[gi(d, m, i, B_, E_)] * t2[ti(d, j, m, e, a)];
      v -= G[gi(d, m, j, A_, E_)] * t2[ti(d, i, m, e, b)];
      v += G[gi(d, m, E_, A_, i)] * Ut(t2, d, j, m, b, e);
      v -= G[gi(d, m, i, A_, E_)] * t2[ti(d, j, m, b, e)];
    }
  // quadratic rings through the intermediates
  const size_t ovov_i = (size_t)d.v * d.o * d.v, ovov_a = (size_t)d.o * d.v;
  for (int nn = 0; nn < d.o; ++nn)
    for (int f = 0; f < d.v; ++f) {
      const size_t ia = i * ovov_i + a * ovov_a + (size_t)nn * d.v + f;
      const size_t ja = j * ovov_i + a * ovov_a + (size_t)nn * d.v + f;
      v += A[ia] * Ut(t2, d, j, nn, b, f) - B[ia] * t2[ti(d, j, nn, b, f)] + Cq[ia] * t2[ti(d, j, nn, f, b)] +
           D[ja] * t2[ti(d, i, nn, f, b)];
    }
  r2[x] = W[gi(d, A_, i, B_, j)] + (double)v;
}

// W[a,e,b,f] += sum_mn g~_menf t_mn^ab  (vvvv block; G reads only the ovov block)
template <typename T>
__global__ void k_vvvv(double* __restrict__ W, const T* __restrict__ G, const T* __restrict__ t2, Dims d) {
  const size_t m_all = (size_t)d.v * d.v * d.v * d.v;
  const size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (x >= m_all) return;
  const int a = (int)(x / ((size_t)d.v * d.v * d.v)), e = (int)((x / ((size_t)d.v * d.v)) % d.v);
  const int b = (int)((x / d.v) % d.v), f = (int)(x % d.v);
  T v = 0;
  for (int m = 0; m < d.o; ++m)
    for (int nn = 0; nn < d.o; ++nn) v += G[gi(d, m, d.o + e, nn, d.o + f)] * t2[ti(d, m, nn, a, b)];
  W[gi(d, d.o + a, d.o + e, d.o + b, d.o + f)] += (double)v;
}

// (ov|vo) and its pair partner (vo|ov):
//   W[m,e,b,j] = g~_mebj + sum_nf g~_menf u_jn^bf - sum_nf g~_mfne t_jn^bf
template <typename T>
__global__ void k_ovvo(double* __restrict__ W, const T* __restrict__ G, const T* __restrict__ t2, Dims d) {
  const size_t m_all = (size_t)d.o * d.v * d.v * d.o;
  const size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (x >= m_all) return;
  const int m = (int)(x / ((size_t)d.v * d.v * d.o)), e = (int)((x / ((size_t)d.v * d.o)) % d.v);
  const int b = (int)((x / d.o) % d.v), j = (int)(x % d.o);
  T v = 0;
  for (int nn = 0; nn < d.o; ++nn)
    for (int f = 0; f < d.v; ++f)
      v += G[gi(d, m, d.o + e, nn, d.o + f)] * Ut(t2, d, j, nn, b, f) -
           G[gi(d, m, d.o + f, nn, d.o + e)] * t2[ti(d, j, nn, b, f)];
  const double w = W[gi(d, m, d.o + e, d.o + b, j)] + (double)v;
  W[gi(d, m, d.o + e, d.o + b, j)] = w;
  W[gi(d, d.o + b, j, m, d.o + e)] = w;
}

// (oo|vv) and (vv|oo):  W[i,j,a,b] = g~_ijab - sum_nf g~_ifnb t_jn^fa
template <typename T>
__global__ void k_oovv(double* __restrict__ W, const T* __restrict__ G, const T* __restrict__ t2, Dims d) {
  const size_t m_all = (size_t)d.o * d.o * d.v * d.v;
  const size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (x >= m_all) return;
  const int i = (int)(x / ((size_t)d.o * d.v * d.v)), j = (int)((x / ((size_t)d.v * d.v)) % d.o);
  const int a = (int)((x / d.v) % d.v), b = (int)(x % d.v);
  T v = 0;
  for (int nn = 0; nn < d.o; ++nn)
    for (int f = 0; f < d.v; ++f) v -= G[gi(d, i, d.o + f, nn, d.o + b)] * t2[ti(d, j, nn, f, a)];
  const double w = W[gi(d, i, j, d.o + a, d.o + b)] + (double)v;
  W[gi(d, i, j, d.o + a, d.o + b)] = w;
  W[gi(d, d.o + a, d.o + b, i, j)] = w;
}

// (oo|vo) and (vo|oo):
//   W[m,i,b,j] = g~_mibj + sum_e f~_me t_ij^eb + sum_ef g~_mebf t_ij^ef
//              + sum_ne [g~_mine u_jn^be - g~_meni t_jn^be - g~_menj t_in^eb]
template <typename T>
__global__ void k_oovo(double* __restrict__ W, const T* __restrict__ G, const double* __restrict__ F,
                       const T* __restrict__ t2, Dims d) {
  const size_t m_all = (size_t)d.o * d.o * d.v * d.o;
  const size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (x >= m_all) return;
  const int m = (int)(x / ((size_t)d.o * d.v * d.o)), i = (int)((x / ((size_t)d.v * d.o)) % d.o);
  const int b = (int)((x / d.o) % d.v), j = (int)(x % d.o);
  const int B_ = d.o + b;
  T v = 0;
  for (int e = 0; e < d.v; ++e) {
    const int E_ = d.o + e;
    v += (T)F[m * d.n + E_] * t2[ti(d, i, j, e, b)];
    for (int f = 0; f < d.v; ++f) v += G[gi(d, m, E_, B_, d.o + f)] * t2[ti(d, i, j, e, f)];
    for (int nn = 0; nn < d.o; ++nn)
      v += G[gi(d, m, i, nn, E_)] * Ut(t2, d, j, nn, b, e) - G[gi(d, m, E_, nn, i)] * t2[ti(d, j, nn, b, e)] -
           G[gi(d, m, E_, nn, j)] * t2[ti(d, i, nn, e, b)];
  }
  const double w = W[gi(d, m, i, B_, j)] + (double)v;
  W[gi(d, m, i, B_, j)] = w;
  W[gi(d, B_, j, m, i)] = w;
}

// (vv|vo) and (vo|vv):
//   W[a,e,b,i] = g~_aebi - sum_m f~_me t_mi^ab + sum_mn g~_meni t_mn^ab
//              + sum_mf [g~_mfae u_mi^fb - g~_mebf t_mi^af - g~_meaf t_mi^fb]
template <typename T>
__global__ void k_vvvo(double* __restrict__ W, const T* __restrict__ G, const double* __restrict__ F,
                       const T* __restrict__ t2, Dims d) {
  const size_t m_all = (size_t)d.v * d.v * d.v * d.o;
  const size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (x >= m_all) return;
  const int a = (int)(x / ((size_t)d.v * d.v * d.o)), e = (int)((x / ((size_t)d.v * d.o)) % d.v);
  const int b = (int)((x / d.o) % d.v), i = (int)(x % d.o);
  const int A_ = d.o + a, E_ = d.o + e, B_ = d.o + b;
  T v = 0;
  for (int m = 0; m < d.o; ++m) {
    v -= (T)F[m * d.n + E_] * t2[ti(d, m, i, a, b)];
    for (int nn = 0; nn < d.o; ++nn) v += G[gi(d, m, E_, nn, i)] * t2[ti(d, m, nn, a, b)];
    for (int f = 0; f < d.v; ++f) {
      const int F_ = d.o + f;
      v += G[gi(d, m, F_, A_, E_)] * Ut(t2, d, m, i, f, b) - G[gi(d, m, E_, B_, F_)] * t2[ti(d, m, i, a, f)] -
           G[gi(d, m, E_, A_, F_)] * t2[ti(d, m, i, f, b)];
    }
  }
  const double w = W[gi(d, A_, E_, B_, i)] + (double)v;
  W[gi(d, A_, E_, B_, i)] = w;
  W[gi(d, B_, i, A_, E_)] = w;
}

// Write the dressed oooo, vo|vo blocks and the oo / vv / vo Fock blocks.
__global__ void k_finalize(double* __restrict__ W, double* __restrict__ F, const double* __restrict__ foo,
                           const double* __restrict__ fvv, const double* __restrict__ r1, const double* __restrict__ wo,
                           const double* __restrict__ r2, Dims d) {
  const size_t n_r2 = (size_t)d.o * d.o * d.v * d.v;
  const size_t n_wo = (size_t)d.o * d.o * d.o * d.o;
  const size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (x < n_r2) {
    const int i = (int)(x / ((size_t)d.o * d.v * d.v)), j = (int)((x / ((size_t)d.v * d.v)) % d.o);
    const int a = (int)((x / d.v) % d.v), b = (int)(x % d.v);
    W[gi(d, d.o + a, i, d.o + b, j)] = r2[x];
  } else if (x < n_r2 + n_wo) {
    const int y = (int)(x - n_r2);
    const int k = y / (d.o * d.o * d.o), i = (y / (d.o * d.o)) % d.o, l = (y / d.o) % d.o, j = y % d.o;
    W[gi(d, k, i, l, j)] = wo[y];
  } else if (x < n_r2 + n_wo + (size_t)d.o * d.o) {
    const int y = (int)(x - n_r2 - n_wo);
    F[(y / d.o) * d.n + (y % d.o)] = foo[y];
  } else if (x < n_r2 + n_wo + (size_t)d.o * d.o + (size_t)d.v * d.v) {
    const int y = (int)(x - n_r2 - n_wo - (size_t)d.o * d.o);
    F[(d.o + y / d.v) * d.n + d.o + (y % d.v)] = fvv[y];
  } else if (x < n_r2 + n_wo + (size_t)d.o * d.o + (size_t)d.v * d.v + (size_t)d.v * d.o) {
    const int y = (int)(x - n_r2 - n_wo - (size_t)d.o * d.o - (size_t)d.v * d.v);
    F[(d.o + y / d.o) * d.n + (y % d.o)] = r1[y];
  }
}

struct Work {
  double *ht, *foo, *fvv, *wo, *r1, *r2, *A, *B, *Cq, *D, *t2f;  // A..D, t2f hold T values
  double* epart;  // energy partials
  float* acc;     // mixed path: FP32 GEMM results (v^3 o floats)
  float* f32;     // mixed path: FP32 copies of f~ (n^2), Foo (o^2), Fvv (v^2) for the FP32 finishing sums
  int* err;       // mixed path: set by a GEMM tile that gave up waiting
  float* arena;   // mixed path: packed GEMM operands and partial products
};

size_t tc_arena_floats(int n, int nocc);

size_t carve(void* base, int n, int o, Work* w, bool mixed = false) {
  const int v = n - o;
  const size_t sizes[] = {(size_t)n * n, (size_t)o * o, (size_t)v * v, (size_t)o * o * o * o, (size_t)v * o,
                          (size_t)o * o * v * v, (size_t)o * v * o * v, (size_t)o * v * o * v, (size_t)o * v * o * v,
                          (size_t)o * v * o * v, (size_t)o * o * v * v, (size_t)EGRID};
  double** ptrs[] = {&w->ht, &w->foo, &w->fvv, &w->wo, &w->r1, &w->r2, &w->A, &w->B, &w->Cq, &w->D, &w->t2f,
                     &w->epart};
  size_t off = 0;
  for (int k = 0; k < 12; ++k) {
    if (base) *ptrs[k] = reinterpret_cast<double*>(static_cast<char*>(base) + off);
    off += ((sizes[k] * sizeof(double) + 255) / 256) * 256;
  }
  w->acc = nullptr;
  w->f32 = nullptr;
  w->err = nullptr;
  w->arena = nullptr;
  if (mixed && v > 0 && o > 0) {
    const size_t na = (size_t)v * v * v * o > (size_t)o * o * v * v ? (size_t)v * v * v * o : (size_t)o * o * v * v;
    if (base) w->acc = reinterpret_cast<float*>(static_cast<char*>(base) + off);
    off += ((na * sizeof(float) + 255) / 256) * 256;
    if (base) w->f32 = reinterpret_cast<float*>(static_cast<char*>(base) + off);
    off += (((size_t)n * n + (size_t)o * o + (size_t)v * v) * sizeof(float) + 255) / 256 * 256;
    if (base) w->err = reinterpret_cast<int*>(static_cast<char*>(base) + off);
    off += 256;
    if (base) w->arena = reinterpret_cast<float*>(static_cast<char*>(base) + off);
    off += ((tc_arena_floats(n, o) * sizeof(float) + 255) / 256) * 256;
  }
  return off;
}

__global__ void k_to_f32(const double* __restrict__ W, float* __restrict__ W32, size_t m) {
  for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < m; x += (size_t)gridDim.x * blockDim.x)
    W32[x] = (float)W[x];
}

}  // namespace

cudaError_t launch_to_f32(const double* W, float* W32, size_t count, cudaStream_t st) {
  const unsigned g = blocks_for(count) > 152u * 64u ? 152u * 64u : blocks_for(count);
  k_to_f32<<<g, TPB, 0, st>>>(W, W32, count);
  return cudaGetLastError();
}

size_t dress_workspace_bytes(int n, int nocc) {
  Work w;
  return carve(nullptr, n, nocc, &w);
}

size_t dress_workspace_bytes_mixed(int n, int nocc) {
  Work w;
  return carve(nullptr, n, nocc, &w, true);
}

int dress_launch_count(int n, int nocc, bool mixed) {
  // 4 T1 passes (the first one copies; for nocc > kT1Omax a separate copy + 4), h~, f~, 2 energy,
  // u, small blocks, finalize; T2 terms: 7 SIMT kernels (FP64) or 2 FP32 copies + 33 operand
  // packs + 9 GEMM launches + the vvvv pack and two product kernels + FP32 Fock copies + 4 finalize
  // kernels + error check (mixed)
  if (!(n - nocc > 0 && nocc > 0)) return 5;
  const int front = (nocc <= kT1Omax ? 4 : 5) + 7;
  return front + (mixed ? 53 : 7);
}

namespace {

template <typename T>
void t2_terms(const Dims& d, double* W, const T* G, const double* F, const T* t2, const Work& w, cudaStream_t st) {
  const size_t o = d.o, v = d.v;
  T* A = reinterpret_cast<T*>(w.A);
  T* B = reinterpret_cast<T*>(w.B);
  T* Cq = reinterpret_cast<T*>(w.Cq);
  T* D = reinterpret_cast<T*>(w.D);
  k_rings<T><<<blocks_for(o * v * o * v), TPB, 0, st>>>(G, t2, A, B, Cq, D, d);
  k_r2<T><<<blocks_for(o * o * v * v), TPB, 0, st>>>(W, G, t2, w.foo, w.fvv, w.wo, A, B, Cq, D, w.r2, d);
  // blocks that read only unmodified bare blocks (through G) may now be overwritten in W
  k_vvvv<T><<<blocks_for(v * v * v * v), TPB, 0, st>>>(W, G, t2, d);
  k_ovvo<T><<<blocks_for(o * v * v * o), TPB, 0, st>>>(W, G, t2, d);
  k_oovv<T><<<blocks_for(o * o * v * v), TPB, 0, st>>>(W, G, t2, d);
  k_oovo<T><<<blocks_for(o * o * v * o), TPB, 0, st>>>(W, G, F, t2, d);
  k_vvvo<T><<<blocks_for(v * v * v * o), TPB, 0, st>>>(W, G, F, t2, d);
}


// ---- mixed precision: the T2 contractions as tensor-core GEMMs ----------------------------
// Every contraction below is a GEMM over index pairs, D[(r1 r2)][(c1 c2)] = sum_k A(r, k) B(c, k),
// with several terms of one output map concatenated along k (segments of o*v or v^2).  Loaders
// read the FP32 copy g of g~ (after the T1 transform, before any T2 term) and the FP32 t2; the
// stores add into FP32 scratch or, for blocks with a single GEMM, directly onto the FP64 base.
struct TcCtx {
  const float* g;   // g~ [n^4]
  const float* t;   // t2 [o o v v]
  const float* ra;  // ring intermediates [i a][n f] (A, B, Cq, D)
  const float* rb;
  const float* rc;
  const float* rd;
  const double* wo;  // dressed oooo block [k i l j] (FP64)
  int n, o, v;
  __device__ __forceinline__ float G(int p, int q, int r, int s) const {
    return g[(((size_t)p * n + q) * n + r) * n + s];
  }
  __device__ __forceinline__ float T(int i, int j, int a, int b) const {
    return t[(((size_t)i * o + j) * v + a) * v + b];
  }
  __device__ __forceinline__ float U(int i, int j, int a, int b) const { return 2.f * T(i, j, a, b) - T(i, j, b, a); }
};

// rings: rows (i, a), cols (n, f), k = (m, e)
struct LRingA {  // sel 0: u[i m a e], 1: t[i m a e], 2: t[i m e a]
  TcCtx c;
  int sel;
  __device__ float operator()(int r, int k) const {
    const int i = r / c.v, a = r % c.v, m = k / c.v, e = k % c.v;
    return sel == 0 ? c.U(i, m, a, e) : (sel == 1 ? c.T(i, m, a, e) : c.T(i, m, e, a));
  }
};
struct LRingB {  // swap 0: g[m E n F], 1: g[m F n E]
  TcCtx c;
  int swap;
  __device__ float operator()(int col, int k) const {
    const int nn = col / c.v, f = col % c.v, m = k / c.v, e = k % c.v;
    return swap ? c.G(m, c.o + f, nn, c.o + e) : c.G(m, c.o + e, nn, c.o + f);
  }
};
// Stores of the GEMM epilogue: run(r, col, vals, cnt) writes vals[j] at (r, col + j), j < cnt
// (<= 32).  The column index is split into its two factors once and then walked, so the
// epilogue does no division per element.
struct StoreRows {
  float* p;
  int ld;
  __device__ void run(int m, int n, const float (&v)[32], int cnt) const {
    float* q = p + (size_t)m * ld + n;
#pragma unroll
    for (int j = 0; j < 32; ++j)
      if (j < cnt) q[j] = v[j];
  }
};

// Woooo (mixed path): rows (k, l), cols (i, j), k = (e, f):  sum_ef g~_kelf t_ij^ef, split K
// into kWoSplit partial maps summed in order onto the FP64 base g~_kilj by k_wo_fin
constexpr int kWoSplit = 8;
struct LWOA {
  TcCtx c;
  __device__ float operator()(int r, int k) const { return c.G(r / c.o, c.o + k / c.v, r % c.o, c.o + k % c.v); }
};
struct LWOB {
  TcCtx c;
  __device__ float operator()(int col, int k) const { return c.T(col / c.o, col % c.o, k / c.v, k % c.v); }
};
__global__ void k_wo_fin(const double* __restrict__ W, const float* __restrict__ part, double* __restrict__ wo,
                         Dims d) {
  const int o = d.o, oo = o * o;
  const int m_all = oo * oo;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;  // wo index [k i l j]
  if (x >= m_all) return;
  const int k = x / (o * oo), i = (x / oo) % o, l = (x / o) % o, j = x % o;
  float v = 0.f;
  for (int z = 0; z < kWoSplit; ++z) v += part[(size_t)z * m_all + (k * o + l) * oo + i * o + j];
  wo[x] = W[gi(d, k, i, l, j)] + (double)v;
}

// r2, ladder + oooo: rows (i, j), cols (a, b), k = (e, f) then (m, n)
struct LR2G1A {
  TcCtx c;
  __device__ float operator()(int r, int k) const {
    const int i = r / c.o, j = r % c.o, vv = c.v * c.v;
    if (k < vv) return c.T(i, j, k / c.v, k % c.v);
    k -= vv;
    const int m = k / c.o, nn = k % c.o;
    return (float)c.wo[(((size_t)m * c.o + i) * c.o + nn) * c.o + j];
  }
};
struct LR2G1B {
  TcCtx c;
  __device__ float operator()(int col, int k) const {
    const int a = col / c.v, b = col % c.v, vv = c.v * c.v;
    if (k < vv) return c.G(c.o + a, c.o + k / c.v, c.o + b, c.o + k % c.v);
    k -= vv;
    return c.T(k / c.o, k % c.o, a, b);
  }
};
// r2 part at (i, j, a, b) from a GEMM whose rows / cols are pairs of (i|j, a|b); every job of
// a launch writes its own buffer (jobs run concurrently)
struct StoreR2 {
  float* acc;
  int o, v, mode;  // 0: (i a)(j b)  1: (j a)(i b)  2: (i b)(j a)  3: (j b)(i a)  4: (i j)(a b)
  __device__ void run(int r, int col, const float (&val)[32], int cnt) const {
    if (mode == 4) {
      float* q = acc + (size_t)r * v * v + col;
#pragma unroll
      for (int t = 0; t < 32; ++t)
        if (t < cnt) q[t] = val[t];
      return;
    }
    const int r1 = r / v, r2 = r % v;
    int c1 = col / v, c2 = col % v;
#pragma unroll
    for (int t = 0; t < 32; ++t) {
      if (t < cnt) {
        int i, j, a, b;
        if (mode == 0) { i = r1; a = r2; j = c1; b = c2; }
        else if (mode == 1) { j = r1; a = r2; i = c1; b = c2; }
        else if (mode == 2) { i = r1; b = r2; j = c1; a = c2; }
        else { j = r1; b = r2; i = c1; a = c2; }
        acc[(((size_t)i * o + j) * v + a) * v + b] = val[t];
      }
      if (++c2 == v) {
        c2 = 0;
        ++c1;
      }
    }
  }
};
// rows (i, a), cols (j, b): linear rings through (m, e) and quadratic rings through (n, f)
struct LR2G3A {
  TcCtx c;
  __device__ float operator()(int r, int k) const {
    const int ov = c.o * c.v, seg = k / ov, kk = k % ov, i = r / c.v, a = r % c.v, m = kk / c.v, e = kk % c.v;
    switch (seg) {
      case 0: return c.U(i, m, a, e);
      case 1: return c.T(i, m, a, e);
      case 2: return c.ra[(size_t)r * ov + kk];
      case 3: return c.rb[(size_t)r * ov + kk];
      default: return c.rc[(size_t)r * ov + kk];
    }
  }
};
struct LR2G3B {
  TcCtx c;
  __device__ float operator()(int col, int k) const {
    const int ov = c.o * c.v, seg = k / ov, kk = k % ov, j = col / c.v, b = col % c.v, m = kk / c.v, e = kk % c.v;
    switch (seg) {
      case 0: return c.G(m, c.o + e, c.o + b, j);
      case 1: return -c.G(m, j, c.o + b, c.o + e);
      case 2: return c.U(j, m, b, e);
      case 3: return -c.T(j, m, b, e);
      default: return c.T(j, m, e, b);
    }
  }
};
// rows (j, a), cols (i, b)
struct LR2G4A {
  TcCtx c;
  __device__ float operator()(int r, int k) const {
    const int ov = c.o * c.v, kk = k % ov, j = r / c.v, a = r % c.v;
    return (k < ov) ? c.T(j, kk / c.v, kk % c.v, a) : c.rd[(size_t)r * ov + kk];
  }
};
struct LR2G4B {
  TcCtx c;
  __device__ float operator()(int col, int k) const {
    const int ov = c.o * c.v, kk = k % ov, i = col / c.v, b = col % c.v, m = kk / c.v, e = kk % c.v;
    return (k < ov) ? -c.G(m, i, c.o + b, c.o + e) : c.T(i, m, e, b);
  }
};
// rows (i, b), cols (j, a)
struct LR2G5A {
  TcCtx c;
  __device__ float operator()(int r, int k) const { return c.T(r / c.v, k / c.v, k % c.v, r % c.v); }
};
struct LR2G5B {
  TcCtx c;
  __device__ float operator()(int col, int k) const {
    return -c.G(k / c.v, col / c.v, c.o + col % c.v, c.o + k % c.v);
  }
};
// rows (j, b), cols (i, a)
struct LR2G6A {
  TcCtx c;
  __device__ float operator()(int r, int k) const {
    const int ov = c.o * c.v, kk = k % ov, j = r / c.v, b = r % c.v, m = kk / c.v, e = kk % c.v;
    return (k < ov) ? c.U(j, m, b, e) : c.T(j, m, b, e);
  }
};
struct LR2G6B {
  TcCtx c;
  __device__ float operator()(int col, int k) const {
    const int ov = c.o * c.v, kk = k % ov, i = col / c.v, a = col % c.v, m = kk / c.v, e = kk % c.v;
    return (k < ov) ? c.G(m, c.o + e, c.o + a, i) : -c.G(m, i, c.o + a, c.o + e);
  }
};

// ovvo: rows (m, e), cols (j, b), k = (n, f) twice; W[m E B j] = W[B j m E] = base + D
struct LOVA {
  TcCtx c;
  __device__ float operator()(int r, int k) const {
    const int ov = c.o * c.v, kk = k % ov, m = r / c.v, e = r % c.v, nn = kk / c.v, f = kk % c.v;
    return (k < ov) ? c.G(m, c.o + e, nn, c.o + f) : -c.G(m, c.o + f, nn, c.o + e);
  }
};
struct LOVB {
  TcCtx c;
  __device__ float operator()(int col, int k) const {
    const int ov = c.o * c.v, kk = k % ov, j = col / c.v, b = col % c.v, nn = kk / c.v, f = kk % c.v;
    return (k < ov) ? c.U(j, nn, b, f) : c.T(j, nn, b, f);
  }
};
struct StoreOV {
  double* W;
  int n, o, v;
  __device__ void run(int r, int col, const float (&val)[32], int cnt) const {
    const int m = r / v, E = o + r % v;
    double old[32];
    {
      int j = col / v, B = o + col % v;
#pragma unroll
      for (int t = 0; t < 32; ++t) {
        old[t] = (t < cnt) ? W[(((size_t)m * n + E) * n + B) * n + j] : 0.0;
        if (++B == o + v) {
          B = o;
          ++j;
        }
      }
    }
    int j = col / v, B = o + col % v;
#pragma unroll
    for (int t = 0; t < 32; ++t) {
      if (t < cnt) {
        const size_t x = (((size_t)m * n + E) * n + B) * n + j, y = (((size_t)B * n + j) * n + m) * n + E;
        const double w = old[t] + (double)val[t];
        W[x] = w;
        W[y] = w;
      }
      if (++B == o + v) {
        B = o;
        ++j;
      }
    }
  }
};

// oovv: rows (i, b), cols (j, a), k = (n, f); W[i j A B] = W[A B i j] = base + D
struct LOOA {
  TcCtx c;
  __device__ float operator()(int r, int k) const {
    return c.G(r / c.v, c.o + k % c.v, k / c.v, c.o + r % c.v);
  }
};
struct LOOB {
  TcCtx c;
  __device__ float operator()(int col, int k) const { return -c.T(col / c.v, k / c.v, k % c.v, col % c.v); }
};
struct StoreOO {
  double* W;
  int n, o, v;
  __device__ void run(int r, int col, const float (&val)[32], int cnt) const {
    const int i = r / v, B = o + r % v;
    double old[32];
    {
      int j = col / v, A = o + col % v;
#pragma unroll
      for (int t = 0; t < 32; ++t) {
        old[t] = (t < cnt) ? W[(((size_t)i * n + j) * n + A) * n + B] : 0.0;
        if (++A == o + v) {
          A = o;
          ++j;
        }
      }
    }
    int j = col / v, A = o + col % v;
#pragma unroll
    for (int t = 0; t < 32; ++t) {
      if (t < cnt) {
        const size_t x = (((size_t)i * n + j) * n + A) * n + B, y = (((size_t)A * n + B) * n + i) * n + j;
        const double w = old[t] + (double)val[t];
        W[x] = w;
        W[y] = w;
      }
      if (++A == o + v) {
        A = o;
        ++j;
      }
    }
  }
};

// oovo, the v^2 term: rows (m, b), cols (i, j), k = (e, f) -> acc[m i b j]
struct LOVOA {
  TcCtx c;
  __device__ float operator()(int r, int k) const {
    return c.G(r / c.v, c.o + k / c.v, c.o + r % c.v, c.o + k % c.v);
  }
};
struct LOVOB {
  TcCtx c;
  __device__ float operator()(int col, int k) const { return c.T(col / c.o, col % c.o, k / c.v, k % c.v); }
};
struct StoreOVO {
  float* acc;
  int o, v;
  __device__ void run(int r, int col, const float (&val)[32], int cnt) const {
    const int m = r / v, b = r % v;
    int i = col / o, j = col % o;
#pragma unroll
    for (int t = 0; t < 32; ++t) {
      if (t < cnt) acc[(((size_t)m * o + i) * v + b) * o + j] = val[t];
      if (++j == o) {
        j = 0;
        ++i;
      }
    }
  }
};

// oovo, the O(o v) terms, k = (n, e):
//   rows (m, i), cols (b, j), k twice:  sum_ne g~_mine u_jn^be  - sum_ne g~_meni t_jn^be
//   rows (m, j), cols (b, i):          -sum_ne g~_menj t_in^eb
// (each into a row-major [rows][o v] buffer, added by k_oovo_fin)
struct LOV2A {
  TcCtx c;
  __device__ float operator()(int r, int k) const {
    const int ov = c.o * c.v, m = r / c.o, i = r % c.o;
    if (k < ov) return c.G(m, i, k / c.v, c.o + k % c.v);
    const int kk = k - ov;
    return -c.G(m, c.o + kk % c.v, kk / c.v, i);
  }
};
struct LOV2B {
  TcCtx c;
  __device__ float operator()(int col, int k) const {
    const int ov = c.o * c.v, b = col / c.o, j = col % c.o;
    const int kk = k < ov ? k : k - ov, nn = kk / c.v, e = kk % c.v;
    return k < ov ? c.U(j, nn, b, e) : c.T(j, nn, b, e);
  }
};
struct LOV3A {
  TcCtx c;
  __device__ float operator()(int r, int k) const { return -c.G(r / c.o, c.o + k % c.v, k / c.v, r % c.o); }
};
struct LOV3B {
  TcCtx c;
  __device__ float operator()(int col, int k) const { return c.T(col % c.o, k / c.v, k % c.v, col / c.o); }
};

// vvvo: acc[a e b i] from three GEMMs
struct LVV1A {  // rows (a, e), k = (m, f) twice: g[m F A E], -g[m E A F]
  TcCtx c;
  __device__ float operator()(int r, int k) const {
    const int ov = c.o * c.v, kk = k % ov, a = r / c.v, e = r % c.v, m = kk / c.v, f = kk % c.v;
    return (k < ov) ? c.G(m, c.o + f, c.o + a, c.o + e) : -c.G(m, c.o + e, c.o + a, c.o + f);
  }
};
struct LVV1B {  // cols (b, i): u[m i f b], t[m i f b]
  TcCtx c;
  __device__ float operator()(int col, int k) const {
    const int ov = c.o * c.v, kk = k % ov, b = col / c.o, i = col % c.o, m = kk / c.v, f = kk % c.v;
    return (k < ov) ? c.U(m, i, f, b) : c.T(m, i, f, b);
  }
};
struct LVV2A {  // rows (a, b), k = (m, n): t[m n a b]
  TcCtx c;
  __device__ float operator()(int r, int k) const { return c.T(k / c.o, k % c.o, r / c.v, r % c.v); }
};
struct LVV2B {  // cols (e, i): g[m E n i]
  TcCtx c;
  __device__ float operator()(int col, int k) const { return c.G(k / c.o, c.o + col / c.o, k % c.o, col % c.o); }
};
struct LVV3A {  // rows (e, b), k = (m, f): -g[m E B F]
  TcCtx c;
  __device__ float operator()(int r, int k) const {
    return -c.G(k / c.v, c.o + r / c.v, c.o + r % c.v, c.o + k % c.v);
  }
};
struct LVV3B {  // cols (a, i): t[m i a f]
  TcCtx c;
  __device__ float operator()(int col, int k) const { return c.T(k / c.v, col % c.o, col / c.o, k % c.v); }
};
struct StoreVV {  // each job its own buffer
  float* acc;
  int o, v, mode;  // 0: (a e)(b i)  1: (a b)(e i)  2: (e b)(a i)
  __device__ void run(int r, int col, const float (&val)[32], int cnt) const {
    const int r1 = r / v, r2 = r % v;
    int c1 = col / o, c2 = col % o;
#pragma unroll
    for (int t = 0; t < 32; ++t) {
      if (t < cnt) {
        int a, e, b;
        if (mode == 0) { a = r1; e = r2; b = c1; }
        else if (mode == 1) { a = r1; b = r2; e = c1; }
        else { e = r1; b = r2; a = c1; }
        acc[(((size_t)a * v + e) * v + b) * o + c2] = val[t];
      }
      if (++c2 == o) {
        c2 = 0;
        ++c1;
      }
    }
  }
};

// r2 = bare vo|vo + GEMM parts (ladder/oooo in acc, four ring maps in part[0..3]) + the O(v)
// Fock terms (FP32), added in FP64
// FP32 copies of f~, Foo and Fvv (the finishing kernels' O(v) sums multiply them with FP32 t2;
// converting once keeps those loops off the FP64 pipe, with the same rounded values).
__global__ void k_fock_f32(const double* __restrict__ F, const double* __restrict__ foo, const double* __restrict__ fvv,
                           float* __restrict__ out, Dims d) {
  const int nf = d.n * d.n, no = d.o * d.o, nv = d.v * d.v;
  for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < nf + no + nv; x += gridDim.x * blockDim.x)
    out[x] = (float)(x < nf ? F[x] : (x < nf + no ? foo[x - nf] : fvv[x - nf - no]));
}

__global__ void k_r2_fin(const double* __restrict__ W, const float* __restrict__ t2, const float* __restrict__ foo,
                         const float* __restrict__ fvv, const float* __restrict__ acc, const float* __restrict__ part,
                         double* __restrict__ r2, Dims d) {
  const size_t m_all = (size_t)d.o * d.o * d.v * d.v;
  const size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (x >= m_all) return;
  const int i = (int)(x / ((size_t)d.o * d.v * d.v)), j = (int)((x / ((size_t)d.v * d.v)) % d.o);
  const int a = (int)((x / d.v) % d.v), b = (int)(x % d.v);
  float v = acc[x] + part[x] + part[m_all + x] + part[2 * m_all + x] + part[3 * m_all + x];
  for (int e = 0; e < d.v; ++e)
    v += fvv[b * d.v + e] * t2[ti(d, i, j, a, e)] + fvv[a * d.v + e] * t2[ti(d, i, j, e, b)];
  for (int m = 0; m < d.o; ++m)
    v -= foo[m * d.o + j] * t2[ti(d, i, m, a, b)] + foo[m * d.o + i] * t2[ti(d, m, j, a, b)];
  r2[x] = W[gi(d, d.o + a, i, d.o + b, j)] + (double)v;
}

// oovo: the GEMM's v^2 term plus the O(v) and O(ov) terms, onto the FP64 base and its mirror
__global__ void k_oovo_fin(double* __restrict__ W, const float* __restrict__ F, const float* __restrict__ t2,
                           const float* __restrict__ part, int nsplit, Dims d) {
  const size_t m_all = (size_t)d.o * d.o * d.v * d.o;
  const size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (x >= m_all) return;
  const int m = (int)(x / ((size_t)d.o * d.v * d.o)), i = (int)((x / ((size_t)d.v * d.o)) % d.o);
  const int b = (int)((x / d.o) % d.v), j = (int)(x % d.o);
  const int B_ = d.o + b;
  float v = 0.f;
  for (int z = 0; z < nsplit; ++z) v += part[(size_t)z * m_all + x];  // split-K partials, in order
  // the O(o v) maps: [m i][b j] (same order as x) and [m j][b i]
  v += part[(size_t)nsplit * m_all + x];
  v += part[(size_t)(nsplit + 1) * m_all + (((size_t)m * d.o + j) * d.v + b) * d.o + i];
  for (int e = 0; e < d.v; ++e) v += F[m * d.n + d.o + e] * t2[ti(d, i, j, e, b)];
  const double w = W[gi(d, m, i, B_, j)] + (double)v;
  W[gi(d, m, i, B_, j)] = w;
  W[gi(d, B_, j, m, i)] = w;
}

// vvvo: GEMM part minus the f~ term, onto the FP64 base and its mirror
__global__ void k_vvvo_fin(double* __restrict__ W, const float* __restrict__ F, const float* __restrict__ t2,
                           const float* __restrict__ acc, const float* __restrict__ p1, const float* __restrict__ p2,
                           Dims d) {
  const size_t m_all = (size_t)d.v * d.v * d.v * d.o;
  const size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (x >= m_all) return;
  const int a = (int)(x / ((size_t)d.v * d.v * d.o)), e = (int)((x / ((size_t)d.v * d.o)) % d.v);
  const int b = (int)((x / d.o) % d.v), i = (int)(x % d.o);
  const int A_ = d.o + a, E_ = d.o + e, B_ = d.o + b;
  float v = acc[x] + p1[x] + p2[x];
  for (int m = 0; m < d.o; ++m) v -= F[m * d.n + E_] * t2[ti(d, m, i, a, b)];
  const double w = W[gi(d, A_, E_, B_, i)] + (double)v;
  W[gi(d, A_, E_, B_, i)] = w;
  W[gi(d, B_, i, A_, E_)] = w;
}

// A tensor-core tile that gave up waiting poisons E0, so the sweep reports a non-finite energy.
__global__ void k_gemm_check(const int* __restrict__ err, double* __restrict__ e0) {
  if (threadIdx.x == 0 && *err) *e0 = nan("");
}

// Scratch for packed operands: a bump allocator over one region, reset between phases; a dry
// run (base == nullptr) only records the peak, which sizes the workspace.
// vvvv block restricted to what (k, k) spaces with k <= 3 read: W[A E B F] with at most three
// distinct virtual indices among a, e, b, f (about 6 v^3 of the v^4 elements), each getting the
// ladder-type term  D = sum_mn g~_menf t_mn^ab  (FP32 products and sums, added in FP64).  Operands
// packed once as rows of o^2:  Gt[(e v + f)][m o + n] = g~[m][o+e][n][o+f],
// Tt[(a v + b)][m o + n] = t2[m][n][a][b].  The restricted set is the disjoint union of six
// families, each a batch of v products C_x = T_x G_x^T (v x v, K = o^2) over rows of Tt and Gt:
//   0  a = b (all e, f):            x = a, C[e][f] = Tt(a,a).Gt(e,f)  -> W[A E A F]
//   1  e = a != b (all f):          x = a, C[b][f] = Tt(a,b).Gt(a,f)  -> W[A A B F]
//   2  e = b != a (all f):          x = b, C[a][f] = Tt(a,b).Gt(b,f)  -> W[A B B F]
//   3  f = a, a != b, e not in {a, b}: x = a, C[b][e] = Tt(a,b).Gt(e,a) -> W[A E B A]
//   4  f = b, a != b, e not in {a, b}: x = b, C[a][e] = Tt(a,b).Gt(e,b) -> W[A E B B]
//   5  e = f, a != b, e not in {a, b}: x = a, C[b][e] = Tt(a,b).Gt(e,e) -> W[A E B E]
__global__ void k_pack_vvvv(const float* __restrict__ g, const float* __restrict__ t2, float* __restrict__ Gt,
                            float* __restrict__ Tt, Dims d) {
  const int o = d.o, v = d.v, oo = o * o;
  const size_t m_all = (size_t)v * v * oo;
  for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < m_all; x += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(x % oo), ef = (int)(x / oo);
    const int m = k / o, nn = k % o, e = ef / v, f = ef % v;
    Gt[x] = g[gi(d, m, o + e, nn, o + f)];
    Tt[x] = t2[ti(d, m, nn, e, f)];
  }
}

constexpr int kV4Tile = 128;  // v <= 128: one CTA holds a family's whole v x v product
constexpr int kV4K = 32;      // K chunk staged in shared memory

__global__ void __launch_bounds__(256) k_vvvv_restricted(double* __restrict__ W, const float* __restrict__ Gt,
                                                         const float* __restrict__ Tt, Dims d) {
  __shared__ float ts[kV4K][kV4Tile + 4], gs[kV4K][kV4Tile + 4];  // [k][row]
  const int o = d.o, v = d.v, oo = o * o;
  const int fam = 1 + blockIdx.x / v, x = blockIdx.x % v;  // families 1..5 (0: k_vvvv_diag)
  const size_t n1 = d.n, n2 = n1 * n1, n3 = n2 * n1;
  // row selectors of the batch: T row i, G row j
  auto trow = [&](int i) -> int { return (fam == 1 || fam == 3 || fam == 5) ? x * v + i : i * v + x; };
  auto grow = [&](int j) -> int {
    switch (fam) {
      case 1: case 2: return x * v + j;
      case 3: case 4: return j * v + x;
      default: return j * (v + 1);  // 5
    }
  };
  const int tid = threadIdx.x, ty = tid / 16, tx = tid % 16;  // 16 x 16 threads, 8 x 8 outputs each
  float acc[8][8];
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[r][c] = 0.f;
  for (int k0 = 0; k0 < oo; k0 += kV4K) {
    __syncthreads();
    for (int t = tid; t < kV4K * kV4Tile; t += 256) {
      const int kk = t / kV4Tile, r = t % kV4Tile, k = k0 + kk;
      float tv = 0.f, gv = 0.f;
      if (r < v && k < oo) {
        tv = Tt[(size_t)trow(r) * oo + k];
        gv = Gt[(size_t)grow(r) * oo + k];
      }
      ts[kk][r] = tv;
      gs[kk][r] = gv;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < kV4K; ++kk) {
      float a[8], b[8];
#pragma unroll
      for (int r = 0; r < 8; ++r) a[r] = ts[kk][ty * 8 + r];
#pragma unroll
      for (int c = 0; c < 8; ++c) b[c] = gs[kk][tx * 8 + c];
#pragma unroll
      for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[r][c] = fmaf(a[r], b[c], acc[r][c]);
    }
  }
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int i = ty * 8 + r;
    if (i >= v) continue;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int j = tx * 8 + c;
      if (j >= v) continue;
      int a, e, b, f;
      bool keep;
      switch (fam) {
        case 1: a = x; b = i; e = x; f = j; keep = (i != x); break;
        case 2: a = i; b = x; e = x; f = j; keep = (i != x); break;
        case 3: a = x; b = i; e = j; f = x; keep = (i != x && j != x && j != i); break;
        case 4: a = i; b = x; e = j; f = x; keep = (i != x && j != x && j != i); break;
        default: a = x; b = i; e = j; f = j; keep = (i != x && j != x && j != i); break;
      }
      if (keep) {
        const size_t w = (size_t)(o + a) * n3 + (size_t)(o + e) * n2 + (size_t)(o + b) * n1 + (size_t)(o + f);
        W[w] += (double)acc[r][c];
      }
    }
  }
}

// Family 0 (a = b, every (e, f)): C[e][f] = Tt(a,a).Gt(e v + f), a warp per output streaming
// Gt's rows (contiguous) with Tt(a,a) in registers; kV4Diag blocks share one a.
constexpr int kV4Diag = 8;
__global__ void __launch_bounds__(256) k_vvvv_diag(double* __restrict__ W, const float* __restrict__ Gt,
                                                   const float* __restrict__ Tt, Dims d) {
  const int o = d.o, v = d.v, oo = o * o, lane = threadIdx.x & 31;
  const int a = blockIdx.x / kV4Diag, part = blockIdx.x % kV4Diag;
  const size_t n1 = d.n, n2 = n1 * n1, n3 = n2 * n1;
  const float* trow = Tt + (size_t)(a * v + a) * oo;
  const int rows = v * v, per = (rows + kV4Diag - 1) / kV4Diag;
  const int r1 = (part + 1) * per < rows ? (part + 1) * per : rows;
  for (int r = part * per + (int)(threadIdx.x >> 5); r < r1; r += (int)(blockDim.x >> 5)) {
    const float* gr = Gt + (size_t)r * oo;
    float acc = 0.f;
    for (int k = lane; k < oo; k += 32) acc = fmaf(trow[k], gr[k], acc);
#pragma unroll
    for (int s2 = 16; s2 > 0; s2 >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, s2);
    if (lane == 0) {
      const int e = r / v, f = r % v;
      const size_t w = (size_t)(o + a) * n3 + (size_t)(o + e) * n2 + (size_t)(o + a) * n1 + (size_t)(o + f);
      W[w] += (double)acc;
    }
  }
}

struct Arena {
  float* base;
  size_t used = 0, peak = 0;
  float* take(size_t n) {
    float* p = base ? base + used : nullptr;
    used += (n + 63) / 64 * 64;
    if (used > peak) peak = used;
    return p;
  }
  void reset() { used = 0; }
};

struct Op {  // a packed operand: hi / lo parts, rows padded to the tile (rows_p), K padded to 32
  float *hi, *lo;
  int rows, rows_p, K, ld;
};

template <class L>
cudaError_t pack_op(L ld, int rows, int K, int tile, Arena& ar, Op* out, cudaStream_t st) {
  const int rows_p = tc::pad_to(rows, tile), Kp = tc::pad_to(K, tc::BK);
  out->rows = rows;
  out->rows_p = rows_p;
  out->K = K;
  out->ld = Kp;
  out->hi = ar.take((size_t)rows_p * Kp);
  out->lo = ar.take((size_t)rows_p * Kp);
  if (!ar.base) return cudaSuccess;
  return tc::pack(ld, rows, K, rows_p, Kp, out->hi, out->lo, st);
}

// operand tiles: A rows pad to 128; B rows pad to the launch's BN
constexpr int kTileM = tc::BM;

template <class Store>
tc::PackedJob<Store> job(const Op& a, const Op& b, Store st, int split = 0, int nsplit = 1) {
  tc::PackedJob<Store> j{};
  j.ahi = a.hi;
  j.alo = a.lo;
  j.bhi = b.hi;
  j.blo = b.lo;
  j.M = a.rows;
  j.N = b.rows;
  j.ma_p = a.rows_p;
  j.nb_p = b.rows_p;
  j.ld = a.ld;
  const int slabs = a.ld / tc::BK, per = (slabs + nsplit - 1) / nsplit;
  j.k_begin = split * per * tc::BK;
  j.k_slabs = (split * per >= slabs) ? 0 : ((split + 1) * per > slabs ? slabs - split * per : per);
  j.st = st;
  return j;
}

template <int BN, class Store>
cudaError_t run_jobs(tc::PackedJobs<Store>& jobs, const Arena& ar, int* err, cudaStream_t st) {
  if (!ar.base) return cudaSuccess;
  return tc::gemm_packed<BN>(jobs, err, st);
}

// The ladder + oooo product's tile width is a run-time choice among kLadderBN (timed by
// tune_ladder); its B operand is padded to the widest candidate so any of them can run on it.
constexpr int kLadderBN[3] = {32, 64, 128};
constexpr int kLadderPad = 128;
constexpr int kLadderDefault = 64;  // one wave of 81 tiles at o = 10 (v^2 = 5184)

cudaError_t run_ladder(tc::PackedJobs<StoreR2>& js, const Arena& ar, int* err, int bn, cudaStream_t st) {
  switch (bn) {
    case 32: return run_jobs<32>(js, ar, err, st);
    case 128: return run_jobs<128>(js, ar, err, st);
    default: return run_jobs<64>(js, ar, err, st);
  }
}

// The packed operands of the ladder + oooo product: rows (i, j), cols (a, b), k = (e, f) then
// (m, n).
cudaError_t pack_ladder(const TcCtx& c, int o, int v, Arena& ar, Op* a1, Op* b1, cudaStream_t st) {
  const int oo = o * o, vv = v * v;
  cudaError_t e = pack_op(LR2G1A{c}, oo, vv + oo, kTileM, ar, a1, st);
  if (e == cudaSuccess) e = pack_op(LR2G1B{c}, vv, vv + oo, kLadderPad, ar, b1, st);
  return e;
}

constexpr int kOvoSplit = 6;  // split K of the oovo v^2 product (720 x 100 x v^2)

// The T2 terms of the mixed path; with ar.base == nullptr only sizes the packed scratch.
cudaError_t t2_terms_tc(const Dims& d, double* W, const float* G, const double* F, const float* t2, const Work& w,
                        double* e0, Arena& ar, cudaStream_t st, int ladder_bn = kLadderDefault) {
  const int o = d.o, v = d.v, ov = o * v, vv = v * v, oo = o * o;
  const bool run = ar.base != nullptr;
  float* A = run ? reinterpret_cast<float*>(w.A) : nullptr;
  float* B = run ? reinterpret_cast<float*>(w.B) : nullptr;
  float* Cq = run ? reinterpret_cast<float*>(w.Cq) : nullptr;
  float* D = run ? reinterpret_cast<float*>(w.D) : nullptr;
  TcCtx c{G, t2, A, B, Cq, D, w.wo, d.n, o, v};
  int* err = w.err;
  float* acc = w.acc;
  cudaError_t e = run ? cudaMemsetAsync(err, 0, sizeof(int), st) : cudaSuccess;
#define QF_TRY(x)                       \
  do {                                  \
    if (e == cudaSuccess) e = (x);      \
  } while (0)
  // Woooo first: the ladder + oooo map reads it
  {
    ar.reset();
    Op a, b;
    QF_TRY(pack_op(LWOA{c}, oo, vv, kTileM, ar, &a, st));
    QF_TRY(pack_op(LWOB{c}, oo, vv, 32, ar, &b, st));
    float* wp = ar.take((size_t)oo * oo * kWoSplit);
    tc::PackedJobs<StoreRows> js{};
    for (int z = 0; z < kWoSplit; ++z) js.j[z] = job(a, b, StoreRows{wp + (run ? (size_t)oo * oo * z : 0), oo}, z, kWoSplit);
    js.count = kWoSplit;
    QF_TRY((run_jobs<32>(js, ar, err, st)));
    if (run && e == cudaSuccess) {
      k_wo_fin<<<blocks_for((size_t)oo * oo), TPB, 0, st>>>(W, wp, w.wo, d);
      e = cudaGetLastError();
    }
  }
  // ring intermediates: one launch of four jobs sharing packed operands
  {
    ar.reset();
    Op au, at, atx, b0, b1;
    QF_TRY(pack_op(LRingA{c, 0}, ov, ov, kTileM, ar, &au, st));
    QF_TRY(pack_op(LRingA{c, 1}, ov, ov, kTileM, ar, &at, st));
    QF_TRY(pack_op(LRingA{c, 2}, ov, ov, kTileM, ar, &atx, st));
    QF_TRY(pack_op(LRingB{c, 0}, ov, ov, 64, ar, &b0, st));
    QF_TRY(pack_op(LRingB{c, 1}, ov, ov, 64, ar, &b1, st));
    tc::PackedJobs<StoreRows> js{};
    js.j[0] = job(au, b0, StoreRows{A, ov});
    js.j[1] = job(au, b1, StoreRows{B, ov});
    js.j[2] = job(at, b1, StoreRows{Cq, ov});
    js.j[3] = job(atx, b1, StoreRows{D, ov});
    js.count = 4;
    QF_TRY((run_jobs<64>(js, ar, err, st)));
  }
  // r2: ladder + oooo term
  {
    ar.reset();
    Op a1, b1;
    QF_TRY(pack_ladder(c, o, v, ar, &a1, &b1, st));
    tc::PackedJobs<StoreR2> js{};
    js.j[0] = job(a1, b1, StoreR2{acc, o, v, 4});
    js.count = 1;
    QF_TRY(run_ladder(js, ar, err, ladder_bn, st));
  }
  // r2: rings (four output maps, one launch)
  {
    ar.reset();
    Op a3, b3, a4, b4, a5, b5, a6, b6;
    QF_TRY(pack_op(LR2G3A{c}, ov, 5 * ov, kTileM, ar, &a3, st));
    QF_TRY(pack_op(LR2G3B{c}, ov, 5 * ov, 64, ar, &b3, st));
    QF_TRY(pack_op(LR2G4A{c}, ov, 2 * ov, kTileM, ar, &a4, st));
    QF_TRY(pack_op(LR2G4B{c}, ov, 2 * ov, 64, ar, &b4, st));
    QF_TRY(pack_op(LR2G5A{c}, ov, ov, kTileM, ar, &a5, st));
    QF_TRY(pack_op(LR2G5B{c}, ov, ov, 64, ar, &b5, st));
    QF_TRY(pack_op(LR2G6A{c}, ov, 2 * ov, kTileM, ar, &a6, st));
    QF_TRY(pack_op(LR2G6B{c}, ov, 2 * ov, 64, ar, &b6, st));
    const size_t n_r2 = (size_t)oo * vv;
    float* part = ar.take(4 * n_r2);
    tc::PackedJobs<StoreR2> js{};
    js.j[0] = job(a3, b3, StoreR2{part, o, v, 0});
    js.j[1] = job(a4, b4, StoreR2{run ? part + n_r2 : nullptr, o, v, 1});
    js.j[2] = job(a5, b5, StoreR2{run ? part + 2 * n_r2 : nullptr, o, v, 2});
    js.j[3] = job(a6, b6, StoreR2{run ? part + 3 * n_r2 : nullptr, o, v, 3});
    js.count = 4;
    QF_TRY((run_jobs<64>(js, ar, err, st)));
    if (run && e == cudaSuccess) {
      const float* f32 = w.f32;
      k_fock_f32<<<blocks_for((size_t)d.n * d.n + oo + vv), TPB, 0, st>>>(F, w.foo, w.fvv, w.f32, d);
      k_r2_fin<<<blocks_for(n_r2), TPB, 0, st>>>(W, t2, f32 + (size_t)d.n * d.n, f32 + (size_t)d.n * d.n + oo, acc, part,
                                                  w.r2, d);
      e = cudaGetLastError();
    }
  }
  // blocks written in place (their bases are read from W by the store of their single job)
  {  // vvvv: only the elements (k, k) spaces read, six batched SIMT products (v <= 128)
    static_assert(kV4Tile >= 128, "n <= 128 orbitals: v fits one tile");
    ar.reset();
    float* Gt = ar.take((size_t)vv * oo);
    float* Tt = ar.take((size_t)vv * oo);
    if (run && e == cudaSuccess) {
      const size_t m_all = (size_t)vv * oo;
      k_pack_vvvv<<<blocks_for(m_all) > 152u * 32u ? 152u * 32u : blocks_for(m_all), TPB, 0, st>>>(G, t2, Gt, Tt, d);
      k_vvvv_diag<<<kV4Diag * v, 256, 0, st>>>(W, Gt, Tt, d);
      k_vvvv_restricted<<<5 * v, 256, 0, st>>>(W, Gt, Tt, d);
      e = cudaGetLastError();
    }
  }
  {
    ar.reset();
    Op a, b;
    QF_TRY(pack_op(LOVA{c}, ov, 2 * ov, kTileM, ar, &a, st));
    QF_TRY(pack_op(LOVB{c}, ov, 2 * ov, 32, ar, &b, st));
    tc::PackedJobs<StoreOV> js{};
    js.j[0] = job(a, b, StoreOV{W, d.n, o, v});
    js.count = 1;
    QF_TRY((run_jobs<32>(js, ar, err, st)));
  }
  {
    ar.reset();
    Op a, b;
    QF_TRY(pack_op(LOOA{c}, ov, ov, kTileM, ar, &a, st));
    QF_TRY(pack_op(LOOB{c}, ov, ov, 32, ar, &b, st));
    tc::PackedJobs<StoreOO> js{};
    js.j[0] = job(a, b, StoreOO{W, d.n, o, v});
    js.count = 1;
    QF_TRY((run_jobs<32>(js, ar, err, st)));
  }
  // oovo v^2 term, split K into partial outputs summed in order by k_oovo_fin
  float* part = nullptr;
  {
    ar.reset();
    Op a, b;
    QF_TRY(pack_op(LOVOA{c}, ov, vv, kTileM, ar, &a, st));
    QF_TRY(pack_op(LOVOB{c}, oo, vv, 32, ar, &b, st));
    const size_t n_ovo = (size_t)oo * v * o;
    part = ar.take(n_ovo * (kOvoSplit + 2));  // + the two O(o v) maps
    tc::PackedJobs<StoreOVO> js{};
    for (int z = 0; z < kOvoSplit; ++z) js.j[z] = job(a, b, StoreOVO{part + (run ? n_ovo * z : 0), o, v}, z, kOvoSplit);
    js.count = kOvoSplit;
    QF_TRY((run_jobs<32>(js, ar, err, st)));
    Op a2, b2, a3, b3;
    QF_TRY(pack_op(LOV2A{c}, oo, 2 * ov, kTileM, ar, &a2, st));
    QF_TRY(pack_op(LOV2B{c}, ov, 2 * ov, 32, ar, &b2, st));
    QF_TRY(pack_op(LOV3A{c}, oo, ov, kTileM, ar, &a3, st));
    QF_TRY(pack_op(LOV3B{c}, ov, ov, 32, ar, &b3, st));
    tc::PackedJobs<StoreRows> jr{};
    jr.j[0] = job(a2, b2, StoreRows{part + (run ? n_ovo * kOvoSplit : 0), ov});
    jr.j[1] = job(a3, b3, StoreRows{part + (run ? n_ovo * (kOvoSplit + 1) : 0), ov});
    jr.count = 2;
    QF_TRY((run_jobs<32>(jr, ar, err, st)));
  }
  if (run && e == cudaSuccess) {
    k_oovo_fin<<<blocks_for((size_t)oo * v * o), TPB, 0, st>>>(W, w.f32, t2, part, kOvoSplit, d);
    e = cudaGetLastError();
  }
  // vvvo: three output maps, one launch; each job its own buffer, summed by k_vvvo_fin
  {
    ar.reset();
    Op a1, b1, a2, b2, a3, b3;
    QF_TRY(pack_op(LVV1A{c}, vv, 2 * ov, kTileM, ar, &a1, st));
    QF_TRY(pack_op(LVV1B{c}, v * o, 2 * ov, 128, ar, &b1, st));
    QF_TRY(pack_op(LVV2A{c}, vv, oo, kTileM, ar, &a2, st));
    QF_TRY(pack_op(LVV2B{c}, v * o, oo, 128, ar, &b2, st));
    QF_TRY(pack_op(LVV3A{c}, vv, ov, kTileM, ar, &a3, st));
    QF_TRY(pack_op(LVV3B{c}, v * o, ov, 128, ar, &b3, st));
    const size_t n_vvvo = (size_t)vv * v * o;
    float* p1 = ar.take(n_vvvo);
    float* p2 = ar.take(n_vvvo);
    tc::PackedJobs<StoreVV> js{};
    js.j[0] = job(a1, b1, StoreVV{acc, o, v, 0});
    js.j[1] = job(a2, b2, StoreVV{p1, o, v, 1});
    js.j[2] = job(a3, b3, StoreVV{p2, o, v, 2});
    js.count = 3;
    // 128-column tiles: half the re-reads of the v^2-row operand from L2
    QF_TRY((run_jobs<128>(js, ar, err, st)));
    if (run && e == cudaSuccess) {
      k_vvvo_fin<<<blocks_for(n_vvvo), TPB, 0, st>>>(W, w.f32, t2, acc, p1, p2, d);
      e = cudaGetLastError();
    }
  }
#undef QF_TRY
  if (run && e == cudaSuccess) {
    k_gemm_check<<<1, 32, 0, st>>>(err, e0);
    e = cudaGetLastError();
  }
  return e;
}

size_t tc_arena_floats(int n, int nocc) {
  Dims d{n, nocc, n - nocc};
  Work w{};
  Arena ar{nullptr};
  t2_terms_tc(d, nullptr, nullptr, nullptr, nullptr, w, nullptr, ar, nullptr);
  return ar.peak;
}
}  // namespace

cudaError_t launch_dress(const double* h, const double* eri, const double* t1, const double* t2, int n, int nocc,
                         double* e0, double* F, double* W, void* work, size_t work_bytes, cudaStream_t st,
                         float* g32, int ladder_bn) {
  Work w;
  const bool mixed = g32 != nullptr;
  if (work_bytes < carve(nullptr, n, nocc, &w, mixed)) return cudaErrorInvalidValue;
  carve(work, n, nocc, &w, mixed);
  Dims d{n, nocc, n - nocc};
  const size_t n4 = (size_t)n * n * n * n;
  const size_t o = nocc, v = n - nocc;
  if (v > 0 && o > 0) {  // W = the bare integrals with T1 applied (the first pass copies them)
    if (mixed) t1_passes<float>(eri, W, t1, d, st);  // FP32 correction sums onto the FP64 elements
    else t1_passes<double>(eri, W, t1, d, st);
  } else {
    k_copy<<<blocks_for(n4) > 152u * 64u ? 152u * 64u : blocks_for(n4), TPB, 0, st>>>(eri, W, n4);
  }
  k_h_tilde<<<blocks_for((size_t)n * n), TPB, 0, st>>>(h, t1, w.ht, d);
  k_fock<<<blocks_for((size_t)n * n), TPB, 0, st>>>(w.ht, W, F, d);
  k_energy_part<<<EGRID, TPB, 0, st>>>(w.ht, W, t2, w.epart, d);
  k_energy_sum<<<1, EGRID, 0, st>>>(w.epart, e0);
  if (v > 0 && o > 0) {
    // U lives in the r2 slot until the doubles residual is written there
    k_make_u<<<blocks_for(o * o * v * v), TPB, 0, st>>>(t2, w.r2, d);
    // the mixed path forms Woooo (a W block) on the tensor cores with its other T2 terms; the
    // Fock-like blocks stay FP64 sums
    const unsigned nsb = (unsigned)(o * o + v * v + v * o + (g32 ? 0 : o * o * o * o));
    k_small_blocks<<<nsb, TPB, 0, st>>>(F, W, w.r2, t2, w.foo, w.fvv, w.r1, w.wo, d);
    if (g32) {  // contractions of the T2 terms in FP32 (mixed precision), bases kept in FP64
      float* t2f = reinterpret_cast<float*>(w.t2f);
      const unsigned gg = blocks_for(n4) > 152u * 64u ? 152u * 64u : blocks_for(n4);
      k_to_f32<<<gg, TPB, 0, st>>>(W, g32, n4);
      k_to_f32<<<blocks_for(o * o * v * v), TPB, 0, st>>>(t2, t2f, o * o * v * v);
      Arena ar{w.arena};
      cudaError_t e = t2_terms_tc(d, W, g32, F, t2f, w, e0, ar, st, ladder_bn > 0 ? ladder_bn : kLadderDefault);
      if (e != cudaSuccess) return e;
    } else {
      t2_terms<double>(d, W, W, F, t2, w, st);
    }
    const size_t nf = o * o * v * v + o * o * o * o + o * o + v * v + v * o;
    k_finalize<<<blocks_for(nf), TPB, 0, st>>>(W, F, w.foo, w.fvv, w.r1, w.wo, w.r2, d);
  }
  return cudaGetLastError();
}

// Times the ladder + oooo product with each tile width of kLadderBN on the workspace of a mixed
// dressing that has run (its packed scratch and FP32 copies are overwritten, its results are
// not read): each candidate runs twice on the stream, the second run timed with CUDA events.
// *best = the fastest width; ms[3] = the candidates' times.  Not capturable (it synchronises).
cudaError_t tune_ladder(int n, int nocc, const float* g32, void* work, size_t work_bytes, cudaStream_t st, int* best,
                        float* ms) {
  *best = kLadderDefault;
  for (int i = 0; i < 3; ++i) ms[i] = 0.f;
  const int o = nocc, v = n - nocc;
  if (!(o > 0 && v > 0) || !g32) return cudaSuccess;
  Work w;
  if (work_bytes < carve(nullptr, n, nocc, &w, true)) return cudaErrorInvalidValue;
  carve(work, n, nocc, &w, true);
  TcCtx c{g32, reinterpret_cast<const float*>(w.t2f), nullptr, nullptr, nullptr, nullptr, w.wo, n, o, v};
  Arena ar{w.arena};
  Op a1, b1;
  cudaError_t e = pack_ladder(c, o, v, ar, &a1, &b1, st);
  tc::PackedJobs<StoreR2> js{};
  js.j[0] = job(a1, b1, StoreR2{w.acc, o, v, 4});
  js.count = 1;
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&t0);
  if (e == cudaSuccess) e = cudaEventCreate(&t1);
  float bt = 0.f;
  for (int i = 0; i < 3 && e == cudaSuccess; ++i) {
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
      e = cudaEventRecord(t0, st);
      if (e == cudaSuccess) e = run_ladder(js, ar, w.err, kLadderBN[i], st);
      if (e == cudaSuccess) e = cudaEventRecord(t1, st);
      if (e == cudaSuccess) e = cudaEventSynchronize(t1);
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms[i], t0, t1);
    }
    if (e == cudaSuccess && ms[i] > 0.f && (bt == 0.f || ms[i] < bt)) {
      bt = ms[i];
      *best = kLadderBN[i];
    }
  }
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  return e;
}

}  // namespace qf
