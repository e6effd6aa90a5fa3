// Tensor-core GEMM for the dressing contractions (sm_103a, tcgen05).
//
// D[M][N] = sum_k A(m, k) B(n, k) in FP32 with operands taken as three-term TF32 splits
// (x = hi + lo, hi = tf32(x), lo = tf32(x - hi); A B ~ Ah Bh + Ah Bl + Al Bh), which keeps the
// product at FP32-level accuracy while the tensor cores do the work.  A(m, k) and B(n, k) come
// from loader functors (any layout, any permutation of a 4-index block), the result goes to a
// store functor, so a contraction needs no transposed copies in HBM.
//
// The general engine (loader functors, used by the device-level GEMM entry point): one CTA of
// 128 threads computes a 128 x BN tile:
//   * all threads load a 128 x 32 slab of A and a BN x 32 slab of B, split them and write them
//     to shared memory in the canonical K-major, no-swizzle layout (core matrices of 8 rows x
//     16 bytes; LBO = 128 B between core matrices along K, SBO = 1 KB between 8-row groups);
//   * one thread issues 4 K-steps x 3 tcgen05.mma (kind::tf32, M = 128, K = 8 per instruction)
//     and commits them to an mbarrier.  Ah Bh accumulates in one tensor-memory accumulator (BN
//     FP32 columns), the two small terms Ah Bl + Al Bh in a second one: the tensor cores' FP32
//     accumulation drops the bits below the accumulator's last place, so the small terms are
//     kept apart from the large running sum and added to it once, in the epilogue;
//   * two slab buffers alternate, so loading slab s+1 overlaps the MMAs of slab s;
//   * the epilogue reads the accumulator with tcgen05.ld (warp w owns rows 32w..32w+31).
// Every mbarrier wait is bounded; on timeout the CTA records an error, stops issuing work,
// waits (bounded) for its committed MMAs, frees its tensor memory and returns.
// The packed engine further down, which the dressing uses, takes operands split ahead of time and
// brings them in with TMA (see its own description).
#pragma once
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace qf {
namespace tc {

constexpr int BM = 128;
constexpr int BK = 32;       // K elements per slab (4 MMAs of K = 8)
constexpr int THREADS = 128;
constexpr unsigned kSpinLimit = 1u << 26;  // bounded waits (far above any real MMA latency)

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for phase `parity` of the barrier to complete; false after kSpinLimit polls.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (unsigned it = 0; it < kSpinLimit; ++it)
    if (mbar_test(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Warp-wide: allocate ncols tensor-memory columns (power of two >= 32); address to *dst.
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// Shared-memory matrix descriptor: K-major, no swizzle (layout type 0), version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor of kind::tf32: D F32, A and B TF32, both K-major, M = 128, N = bn.
__host__ __device__ constexpr uint32_t idesc_tf32(int bn) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(bn >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accum)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// 32 consecutive FP32 columns of this thread's tensor-memory lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ float tf32_round(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Byte offset of element (row, k) of a slab in the canonical K-major no-swizzle layout
// (4-byte elements, BK = 32 per row: 8 core matrices along K, LBO = 128 B, SBO = 1024 B).
__device__ __forceinline__ uint32_t slab_off(int row, int k) {
  return (uint32_t)((row >> 3) * 1024 + (k >> 2) * 128 + (row & 7) * 16 + (k & 3) * 4);
}

template <int BN>
struct Smem {
  float a_hi[2][BM * BK], a_lo[2][BM * BK];
  float b_hi[2][BN * BK], b_lo[2][BN * BK];
  uint64_t bar[2];
  uint32_t tmem;
  int abort;
};

// Split x_ = hi + lo and write both parts of four consecutive k of one row.
__device__ __forceinline__ void put4(float* hi, float* lo, int row, int k4, const float (&x)[4]) {
  float h[4], l[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    h[j] = tf32_round(x[j]);
    l[j] = tf32_round(x[j] - h[j]);
  }
  const uint32_t off = slab_off(row, k4) / 4;
  *reinterpret_cast<float4*>(hi + off) = make_float4(h[0], h[1], h[2], h[3]);
  *reinterpret_cast<float4*>(lo + off) = make_float4(l[0], l[1], l[2], l[3]);
}

// LoadA: float operator()(int m, int k) const, only called in range.  Same for LoadB(n, k).
// Store: void operator()(int m, int n, float v) const, only called in range.
template <int BN, class LoadA, class LoadB, class Store>
__global__ void __launch_bounds__(THREADS) k_gemm_tf32x3(int M, int N, int K, LoadA la, LoadB lb, Store st,
                                                         int* __restrict__ err) {
  static_assert(BN % 32 == 0 && BN >= 32 && BN <= 256, "tile width");
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  Smem<BN>& sm = *reinterpret_cast<Smem<BN>*>(smem_raw);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  if (tid == 0) {
    mbar_init(&sm.bar[0], 1);
    mbar_init(&sm.bar[1], 1);
    sm.abort = 0;
  }
  if (warp == 0) tmem_alloc(&sm.tmem, 2 * BN);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = sm.tmem;
  constexpr uint32_t idesc = idesc_tf32(BN);
  const int nslab = (K + BK - 1) / BK;
  uint32_t phase[2] = {0u, 0u};
  int issued[2] = {0, 0};
  for (int s = 0; s < nslab; ++s) {
    const int buf = s & 1;
    // the MMAs that last read this buffer (slab s - 2) must be done before it is rewritten
    if (issued[buf]) {
      if (!mbar_wait(&sm.bar[buf], phase[buf])) sm.abort = 1;  // benign race: any writer sets 1
      phase[buf] ^= 1u;
      issued[buf] = 0;
    }
    __syncthreads();
    if (sm.abort) break;
    const int k0 = s * BK;
    // A slab: thread t owns row t, all 32 k
    {
      const int m = m0 + tid;
#pragma unroll
      for (int k4 = 0; k4 < BK; k4 += 4) {
        float x[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int k = k0 + k4 + j;
          x[j] = (m < M && k < K) ? la(m, k) : 0.f;
        }
        put4(sm.a_hi[buf], sm.a_lo[buf], tid, k4, x);
      }
    }
    // B slab: BN rows over 128 threads
#pragma unroll 1
    for (int r = tid; r < BN; r += THREADS) {
      const int n = n0 + r;
#pragma unroll
      for (int k4 = 0; k4 < BK; k4 += 4) {
        float x[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int k = k0 + k4 + j;
          x[j] = (n < N && k < K) ? lb(n, k) : 0.f;
        }
        put4(sm.b_hi[buf], sm.b_lo[buf], r, k4, x);
      }
    }
    fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t ah = smem_u32(sm.a_hi[buf]), al = smem_u32(sm.a_lo[buf]);
      const uint32_t bh = smem_u32(sm.b_hi[buf]), bl = smem_u32(sm.b_lo[buf]);
#pragma unroll
      for (int ks = 0; ks < BK / 8; ++ks) {
        const uint32_t koff = (uint32_t)ks * 256;  // two core matrices (8 tf32) per K step
        const uint64_t dah = smem_desc(ah + koff, 128, 1024), dal = smem_desc(al + koff, 128, 1024);
        const uint64_t dbh = smem_desc(bh + koff, 128, 1024), dbl = smem_desc(bl + koff, 128, 1024);
        const uint32_t acc0 = (s > 0 || ks > 0) ? 1u : 0u;
        mma_tf32(tmem, dah, dbh, idesc, acc0);
        mma_tf32(tmem + BN, dah, dbl, idesc, acc0);
        mma_tf32(tmem + BN, dal, dbh, idesc, 1u);
      }
      mma_commit(&sm.bar[buf]);
    }
    issued[buf] = 1;
  }
  // drain: every committed slab, bounded
  for (int b = 0; b < 2; ++b)
    if (issued[b]) {
      if (!mbar_wait(&sm.bar[b], phase[b])) sm.abort = 1;
      phase[b] ^= 1u;
    }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const bool ok = (sm.abort == 0);
  if (ok && nslab > 0) {
    const int m = m0 + warp * 32 + (tid & 31);
#pragma unroll 1
    for (int c = 0; c < BN; c += 32) {
      float v[32], w[32];
      const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
      tmem_ld32(tmem + lane_base + (uint32_t)c, v);
      tmem_ld32(tmem + lane_base + (uint32_t)(BN + c), w);
      if (m < M) {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int n = n0 + c + j;
          if (n < N) st(m, n, v[j] + w[j]);
        }
      }
    }
  }
  if (!ok && tid == 0) atomicExch(err, 1);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tmem_dealloc(tmem, 2 * BN);
    tmem_relinquish();
  }
}

template <int BN, class LoadA, class LoadB, class Store>
cudaError_t gemm_tf32x3(int M, int N, int K, LoadA la, LoadB lb, Store st, int* err, cudaStream_t stream) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  const size_t smem = sizeof(Smem<BN>) + 1024;
  auto kern = k_gemm_tf32x3<BN, LoadA, LoadB, Store>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const dim3 grid((unsigned)((N + BN - 1) / BN), (unsigned)((M + BM - 1) / BM));
  kern<<<grid, THREADS, smem, stream>>>(M, N, K, la, lb, st, err);
  return cudaGetLastError();
}

}  // namespace tc
}  // namespace qf

// ---- packed operands --------------------------------------------------------------------------
// A second engine for operands prepared by k_pack: hi and lo TF32 parts as row-major FP32
// matrices with K padded to a multiple of 32 and rows padded to the tile.  A slab (32 K x tile
// rows, 128-byte rows) is one TMA box per array, written to shared memory with the 128-byte
// swizzle that the MMA descriptors read, while the tensor cores work on the previous slabs.  Up
// to kMaxJobs independent jobs of one store type share a launch (blockIdx.z selects the job);
// jobs may also be K-ranges of one product (split K) writing separate partial outputs.  A CTA has
// two warpgroups: in the epilogue warps w and w + 4 read the same 32 accumulator lanes (a warp
// reaches the lanes 32 (w mod 4) .. 32 (w mod 4) + 31) and take alternate 32-column chunks, so
// twice as many output loads and stores are in flight as with one warpgroup.
namespace qf {
namespace tc {

constexpr int PTHREADS = 256;  // threads of a packed-engine CTA

// out_hi/out_lo[r][k] = split(L(r, k)) for r < rows, k < K; zero in the padding.
// (r, k) of the grid-stride index x = r Kp + k advance by the stride's own digits with a carry,
// so no 64-bit division runs per element.
template <class L>
__global__ void k_pack(L ld, int rows, int K, int rows_p, int Kp, float* __restrict__ hi, float* __restrict__ lo) {
  const size_t total = (size_t)rows_p * Kp;
  const size_t x0 = blockIdx.x * (size_t)blockDim.x + threadIdx.x, step = (size_t)gridDim.x * blockDim.x;
  int r = (int)(x0 / Kp), k = (int)(x0 % Kp);
  const int sr = (int)(step / Kp), sk = (int)(step % Kp);
  for (size_t x = x0; x < total; x += step) {
    const float v = (r < rows && k < K) ? ld(r, k) : 0.f;
    const float h = tf32_round(v);
    hi[x] = h;
    lo[x] = tf32_round(v - h);
    k += sk;
    const int c = k >= Kp;
    k -= c ? Kp : 0;
    r += sr + c;
  }
}

template <class L>
cudaError_t pack(L ld, int rows, int K, int rows_p, int Kp, float* hi, float* lo, cudaStream_t st) {
  const size_t total = (size_t)rows_p * Kp;
  size_t g = (total + 255) / 256;
  if (g > 152 * 64) g = 152 * 64;
  if (g < 1) g = 1;
  k_pack<L><<<(unsigned)g, 256, 0, st>>>(ld, rows, K, rows_p, Kp, hi, lo);
  return cudaGetLastError();
}

__host__ __device__ constexpr int pad_to(int x, int m) { return (x + m - 1) / m * m; }

template <class Store>
struct PackedJob {
  // tensor maps of the four packed arrays (filled by gemm_packed from the pointers below): 2-D
  // views [rows_p][ld] whose boxes are one slab (32 K x tile rows) with the 128-byte swizzle
  CUtensorMap tahi, talo, tbhi, tblo;
  const float *ahi, *alo, *bhi, *blo;  // [ma_p][ld], [nb_p][ld]
  int M, N, ld;                        // ld = padded K of the packed arrays
  int ma_p, nb_p;                      // allocated (padded) rows of the A and B arrays
  int k_begin, k_slabs;                // slabs [k_begin / 32, k_begin / 32 + k_slabs)
  Store st;
};

constexpr int kMaxJobs = 8;
template <class Store>
struct PackedJobs {
  PackedJob<Store> j[kMaxJobs];
  int count;
};

template <int BN, int S>
struct SmemP {  // S-stage buffers of the packed engine (each slab 128-byte rows, swizzled)
  float a_hi[S][BM * BK], a_lo[S][BM * BK];
  float b_hi[S][BN * BK], b_lo[S][BN * BK];
  uint64_t full[S];  // slab landed (TMA transaction count)
  uint64_t bar[S];   // MMAs of the slab done (stage free)
  uint32_t tmem;
  int abort;
};

// Non-blocking probe of a phase; polled a bounded number of times.
__device__ __forceinline__ bool mbar_probe(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_probe(uint64_t* bar, uint32_t parity) {
  for (unsigned it = 0; it < kSpinLimit; ++it)
    if (mbar_probe(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// One box of a 2-D tensor map (x = K element, y = row) into shared memory, counted on `bar`.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// Shared-memory matrix descriptor of a K-major tile with the 128-byte swizzle: rows of 128 bytes
// (32 TF32), 8-row groups 1 KB apart (SBO); the leading offset is unused for this layout.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;  // layout: 128-byte swizzle
  return d;
}

// S-stage pipeline driven by one thread: TMA brings slab s+S-1 while the tensor cores work on
// slab s; a stage is refilled once the MMAs that read it have completed.  The other threads wait
// at the barrier before the epilogue.  Every wait is a bounded poll; on a timeout the CTA records
// an error and waits (bounded) for what it has in flight before it frees its tensor memory.
template <int BN, int S, class Store>
__global__ void __launch_bounds__(PTHREADS, 1) k_gemm_packed(const __grid_constant__ PackedJobs<Store> jobs,
                                                             int* __restrict__ err) {
  static_assert(S >= 2 && S <= 4, "stages");
  if ((int)blockIdx.z >= jobs.count) return;
  const PackedJob<Store>& jb = jobs.j[blockIdx.z];
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  if (m0 >= jb.M || n0 >= jb.N) return;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  SmemP<BN, S>& sm = *reinterpret_cast<SmemP<BN, S>*>(smem_raw);
  const int tid = threadIdx.x, warp = tid >> 5;
  if (tid == 0) {
    for (int i = 0; i < S; ++i) {
      mbar_init(&sm.full[i], 1);
      mbar_init(&sm.bar[i], 1);
    }
    sm.abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    fence_async_smem();
  }
  if (warp == 0) tmem_alloc(&sm.tmem, 2 * BN);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = sm.tmem;
  const int nslab = jb.k_slabs, s0 = jb.k_begin / BK;
  if (tid == 0 && nslab > 0) {
    constexpr uint32_t idesc = idesc_tf32(BN);
    constexpr uint32_t kStageBytes = (uint32_t)(BM + BN) * BK * 4u * 2u;
    uint32_t fph = 0u, mph = 0u;       // parity to wait for, per stage, on full[] and bar[]
    uint32_t loaded = 0u, pend = 0u;   // stages with a load / an MMA commit not yet waited for
    bool bad = false;
    auto load = [&](int slab, int st) {
      const int kx = (s0 + slab) * BK;
      mbar_expect_tx(&sm.full[st], kStageBytes);
      tma_load_2d(smem_u32(sm.a_hi[st]), &jb.tahi, kx, m0, &sm.full[st]);
      tma_load_2d(smem_u32(sm.a_lo[st]), &jb.talo, kx, m0, &sm.full[st]);
      tma_load_2d(smem_u32(sm.b_hi[st]), &jb.tbhi, kx, n0, &sm.full[st]);
      tma_load_2d(smem_u32(sm.b_lo[st]), &jb.tblo, kx, n0, &sm.full[st]);
      loaded |= 1u << st;
    };
    for (int p = 0; p < S && p < nslab; ++p) load(p, p);
    for (int s = 0; s < nslab; ++s) {
      const int st = s % S;
      if (!mbar_wait_probe(&sm.full[st], (fph >> st) & 1u)) {
        bad = true;
        break;
      }
      fph ^= 1u << st;
      loaded &= ~(1u << st);
      tc_fence_after();
      const uint32_t ah = smem_u32(sm.a_hi[st]), al = smem_u32(sm.a_lo[st]);
      const uint32_t bh = smem_u32(sm.b_hi[st]), bl = smem_u32(sm.b_lo[st]);
#pragma unroll
      for (int ks = 0; ks < BK / 8; ++ks) {
        const uint32_t koff = (uint32_t)ks * 32;  // 8 TF32 along the 128-byte row
        const uint64_t dah = smem_desc_sw128(ah + koff), dal = smem_desc_sw128(al + koff);
        const uint64_t dbh = smem_desc_sw128(bh + koff), dbl = smem_desc_sw128(bl + koff);
        const uint32_t acc0 = (s > 0 || ks > 0) ? 1u : 0u;
        mma_tf32(tmem, dah, dbh, idesc, acc0);
        mma_tf32(tmem + BN, dah, dbl, idesc, acc0);
        mma_tf32(tmem + BN, dal, dbh, idesc, 1u);
      }
      mma_commit(&sm.bar[st]);
      pend |= 1u << st;
      // refill the stage of slab s-1 with slab s-1+S once its MMAs are done
      const int nxt = s - 1 + S;
      if (s >= 1 && nxt < nslab) {
        const int ps = (s - 1) % S;
        if (!mbar_wait_probe(&sm.bar[ps], (mph >> ps) & 1u)) {
          bad = true;
          break;
        }
        mph ^= 1u << ps;
        pend &= ~(1u << ps);
        load(nxt, ps);
      }
    }
    for (int b = 0; b < S; ++b) {
      if ((pend >> b) & 1u) {
        if (!mbar_wait_probe(&sm.bar[b], (mph >> b) & 1u)) bad = true;
        mph ^= 1u << b;
      }
      if ((loaded >> b) & 1u) {  // only after a failure: copies still in flight
        if (!mbar_wait_probe(&sm.full[b], (fph >> b) & 1u)) bad = true;
        fph ^= 1u << b;
      }
    }
    if (bad) sm.abort = 1;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const bool ok = (sm.abort == 0);
  // A job whose K range is empty (a split-K part past the last slab) stores zeros: its partial
  // output is summed like the others.
  if (ok) {
    const int quad = warp & 3;  // accumulator lanes 32 quad .. 32 quad + 31
    const int m = m0 + quad * 32 + (tid & 31);
#pragma unroll 1
    for (int c = (warp >> 2) * 32; c < BN; c += 64) {
      float v[32], w[32];
      const uint32_t lane_base = (uint32_t)(quad * 32) << 16;
      if (nslab > 0) {  // uniform over the CTA: every warp takes the collective loads or none
        tmem_ld32(tmem + lane_base + (uint32_t)c, v);
        tmem_ld32(tmem + lane_base + (uint32_t)(BN + c), w);
      } else {
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] = w[j] = 0.f;
      }
      if (m < jb.M && n0 + c < jb.N) {
        // 32 consecutive columns of row m in one call, so the store can walk its output indices
        // instead of splitting every column index
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] += w[j];
        const int cnt = (jb.N - (n0 + c) < 32) ? jb.N - (n0 + c) : 32;
        jb.st.run(m, n0 + c, v, cnt);
      }
    }
  }
  if (!ok && tid == 0) atomicExch(err, 1);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tmem_dealloc(tmem, 2 * BN);
    tmem_relinquish();
  }
}

// cuTensorMapEncodeTiled from the driver (through the runtime, no link against libcuda).
inline PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      f = nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  }();
  return fn;
}

// 2-D view [rows_p][ld] of one packed array; box = one slab (32 K) of `box_rows` rows.
inline bool encode_operand(CUtensorMap* m, const float* p, int rows_p, int ld, int box_rows) {
  const PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc || !p || ((uintptr_t)p & 15u) != 0 || ld % BK != 0 || rows_p % box_rows != 0) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)ld, (cuuint64_t)rows_p};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(p), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int BN, class Store>
cudaError_t gemm_packed(const PackedJobs<Store>& in, int* err, cudaStream_t stream) {
  constexpr int S = (BN <= 32) ? 4 : 3;  // 3 x 64 KB stages at BN = 128
  PackedJobs<Store> jobs = in;
  int gx = 1, gy = 1;
  for (int i = 0; i < jobs.count; ++i) {
    PackedJob<Store>& j = jobs.j[i];
    const int ma = j.ma_p, nb = j.nb_p;
    // every box of the grid must lie inside the allocated rows
    if (ma < pad_to(j.M, BM) || nb < pad_to(j.N, BN)) return cudaErrorInvalidValue;
    if (!encode_operand(&j.tahi, j.ahi, ma, j.ld, BM) || !encode_operand(&j.talo, j.alo, ma, j.ld, BM) ||
        !encode_operand(&j.tbhi, j.bhi, nb, j.ld, BN) || !encode_operand(&j.tblo, j.blo, nb, j.ld, BN))
      return cudaErrorInvalidValue;
    const int x = (j.N + BN - 1) / BN, y = (j.M + BM - 1) / BM;
    gx = x > gx ? x : gx;
    gy = y > gy ? y : gy;
  }
  static_assert(sizeof(SmemP<BN, S>) + 1024 <= 232448, "stages within the shared memory of a block");
  const size_t smem = sizeof(SmemP<BN, S>) + 1024;
  auto kern = k_gemm_packed<BN, S, Store>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<dim3((unsigned)gx, (unsigned)gy, (unsigned)jobs.count), PTHREADS, smem, stream>>>(jobs, err);
  return cudaGetLastError();
}

}  // namespace tc
}  // namespace qf
