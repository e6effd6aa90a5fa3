// Warm-start network for the 6e6o solver (not in the paper; the paper mentions learning only
// for the choice of active spaces).  A small FP32 network maps the folded integrals of a
// (3,3) space to its CI -> CC increment; the increment is expanded into a start vector for the
// Davidson solver, which alone decides every energy and amplitude.
//
//   features (708): vacuum-ordered h[p][q] over the six local orbitals (36, row-major), the
//       pair-symmetric W[p][q][r][s] once per P = 6p+q <= R = 6r+s (666, row-major over (P,R)),
//       the dressed Fock diagonal F_pp of the six orbitals (6);
//   targets (54): X1[i][a] (9) and X2[i][j][a][b] once per P = 3i+a <= R = 3j+b (45);
//   network: H1 = tanh(X W1 + b1), H2 = tanh(H1 W2 + b2), Y = H2 W3 + b3 with W stored
//       [fan_in][fan_out]; loss 1/(2N) sum (Y - T)^2 over rows whose mask is set; Adam;
//   start vector: Phi + X1 Phi + (X2 + X1^2/2) Phi (the rank <= 2 part of e^X Phi), written
//       in the solver's determinant layout (alpha string index * 20 + beta string index,
//       strings of three electrons in six local orbitals by increasing bit mask, local
//       orbitals 0..2 occupied in Phi).
//
// Every reduction runs in a fixed order, so results do not depend on scheduling.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "qflow_internal.h"
#include "tc_gemm.cuh"

namespace qf {
namespace {

// ---- matrix products on the tensor cores, with fused epilogues --------------------------------
// C[M][N] = op(A) op(B) through the repo's tcgen05 engine (three-term TF32 products, FP32
// accumulation in tensor memory: FP32-accurate): op(A) is A[M][K] (lda) or, when TA, A stored
// [K][M]; op(B) is B[K][N] (ldb) or, when TB, B stored [N][K].  Epilogues: kBiasTanh
// C = tanh(acc + bias[n]); kBias C = acc + bias[n]; kTanhGrad C = acc * (1 - aux[m][n]^2) (aux has
// C's layout).  `err` is set by a tile that gave up waiting on its operands (k_mlp_check then
// makes the first output NaN, so a failed product cannot pass silently).
enum Epi { kStore = 0, kBiasTanh = 1, kBias = 2, kTanhGrad = 3 };

template <bool T>
struct LoadOp {  // element (r, k) of op(X): X[r][k] (T = false) or X stored [k][r] (T = true)
  const float* p;
  int ld;
  __device__ float operator()(int r, int k) const { return T ? p[(size_t)k * ld + r] : p[(size_t)r * ld + k]; }
};
template <int EPI>
struct StoreEpi {
  float* C;
  int ldc;
  const float* bias;
  const float* aux;
  __device__ void operator()(int m, int n, float v) const {
    const size_t x = (size_t)m * ldc + n;
    if (EPI == kBiasTanh) v = tanhf(v + bias[n]);
    else if (EPI == kBias) v = v + bias[n];
    else if (EPI == kTanhGrad) v = v * (1.f - aux[x] * aux[x]);
    C[x] = v;
  }
};

__global__ void k_mlp_check(const int* __restrict__ err, float* __restrict__ y) {
  if (threadIdx.x == 0 && *err) y[0] = __int_as_float(0x7fc00000);
}

template <bool TA, bool TB, int EPI>
cudaError_t gemm(int M, int N, int K, const float* A, int lda, const float* B, int ldb, float* C, int ldc,
                 const float* bias, const float* aux, int* err, cudaStream_t st) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  // the engine forms sum_k a(m, k) b(n, k): op(B)^T element (n, k) is B[k][n], or B[n][k] when TB.
  // Tile width: the widest that N fills while the tiles still cover every SM (op(A) streamed
  // fewer times); products with few 128-row tiles (the weight gradients, K = rows) take 64.
  const LoadOp<TA> la{A, lda};
  const LoadOp<!TB> lb{B, ldb};
  const StoreEpi<EPI> sv{C, ldc, bias, aux};
  const int mt = (M + 127) / 128;
  if (N > 128 && mt * ((N + 255) / 256) >= 152) return tc::gemm_tf32x3<256>(M, N, K, la, lb, sv, err, st);
  if (N > 64 && mt * ((N + 127) / 128) >= 152) return tc::gemm_tf32x3<128>(M, N, K, la, lb, sv, err, st);
  return tc::gemm_tf32x3<64>(M, N, K, la, lb, sv, err, st);
}

// out[c] = sum over rows r (ascending) of X[r][c]
__global__ void k_colsum(const float* __restrict__ X, int rows, int cols, float* __restrict__ out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  float s = 0.f;
  for (int r = 0; r < rows; ++r) s += X[(size_t)r * cols + c];
  out[c] = s;
}

constexpr int LB = 256;    // threads of the loss kernel
constexpr int LGRID = 64;  // its fixed grid

// dY = m (Y - T) / rows and per-block partial sums of m (Y - T)^2 (m = mask or 1).
__global__ void k_loss_grad(const float* __restrict__ Y, const float* __restrict__ T,
                            const uint8_t* __restrict__ mask, int rows, int cols, float* __restrict__ dY,
                            float* __restrict__ partial) {
  __shared__ float red[LB];
  float acc = 0.f;
  const int64_t total = (int64_t)rows * cols;
  const float inv = 1.f / (float)rows;
  for (int64_t i = (int64_t)blockIdx.x * LB + threadIdx.x; i < total; i += (int64_t)LGRID * LB) {
    const int r = (int)(i / cols);
    const float w = (mask && !mask[r]) ? 0.f : 1.f;
    const float d = w * (Y[i] - T[i]);
    dY[i] = d * inv;
    acc = fmaf(d, d, acc);
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = LB / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

__global__ void k_loss_final(const float* __restrict__ partial, int rows, float* __restrict__ loss) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s = 0.0;
  for (int b = 0; b < LGRID; ++b) s += (double)partial[b];
  *loss = (float)(0.5 * s / (double)rows);
}

__global__ void k_adam(int64_t n, float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float eps, float bc1, float bc2) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
  }
}

// ---- features of (3,3) spaces ---------------------------------------------------------------
constexpr int FW = 4;  // warps per CTA of the feature kernel

// Warp per row.  out[s][708] = features of spaces[s * stride], standardised as
// (x - mu) * sc when mu is given.
__global__ void __launch_bounds__(32 * FW) k_features(int n, const double* __restrict__ F,
                                                      const double* __restrict__ W,
                                                      const qflow_space* __restrict__ spaces, int64_t nspaces,
                                                      int64_t stride, const float* __restrict__ mu,
                                                      const float* __restrict__ sc, float* __restrict__ out) {
  __shared__ unsigned short pairs[666];
  for (int t = threadIdx.x; t < 666; t += blockDim.x) {  // t -> (P, R), P <= R, row-major
    int P = 0, start = 0;
    while (start + (36 - P) <= t) {
      start += 36 - P;
      ++P;
    }
    const int R = P + (t - start);
    pairs[t] = (unsigned short)(P | (R << 8));
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const size_t n1 = (size_t)n, n2 = n1 * n1, n3 = n2 * n1;
  for (int64_t s = (int64_t)blockIdx.x * FW + warp; s < nspaces; s += (int64_t)gridDim.x * FW) {
    size_t o[6];
#pragma unroll
    for (int t = 0; t < 6; ++t) o[t] = (size_t)spaces[s * stride].orb[t];
    float* row = out + (size_t)s * QFLOW_MLP_NIN;
    for (int c = lane; c < QFLOW_MLP_NIN; c += 32) {
      double x;
      if (c < 36) {  // h_pq = F_pq - sum_{k occupied} (2 W_pqkk - W_pkkq)
        const size_t p = o[c / 6], q = o[c % 6];
        x = F[p * n1 + q];
        for (int k = 0; k < 3; ++k) x -= 2.0 * W[p * n3 + q * n2 + o[k] * n1 + o[k]] - W[p * n3 + o[k] * n2 + o[k] * n1 + q];
      } else if (c < 702) {
        const int pr = pairs[c - 36], P = pr & 255, R = pr >> 8;
        x = W[o[P / 6] * n3 + o[P % 6] * n2 + o[R / 6] * n1 + o[R % 6]];
      } else {
        const size_t p = o[c - 702];
        x = F[p * n1 + p];
      }
      float v = (float)x;
      if (mu) v = (v - mu[c]) * sc[c];
      row[c] = v;
    }
  }
}

// ---- determinant bookkeeping of the (3,3) space ---------------------------------------------
// Strings: three electrons in six local orbitals, indexed by increasing bit mask, which is the
// colexicographic order: index = C(b1,1) + C(b2,2) + C(b3,3) for set bits b1 < b2 < b3.
__device__ __forceinline__ int binom(int m, int k) {
  if (m < k) return 0;
  int r = 1;
  for (int t = 0; t < k; ++t) r = r * (m - t) / (t + 1);
  return r;
}
__device__ __forceinline__ int string_index(int mask) {
  int idx = 0, k = 1;
  for (int b = 0; b < 6; ++b)
    if ((mask >> b) & 1) idx += binom(b, k++);
  return idx;
}
__device__ __forceinline__ int string_mask(int idx) {
  int seen = 0;
  for (int m = 0; m < 64; ++m) {
    if (__popc(m) != 3) continue;
    if (seen == idx) return m;
    ++seen;
  }
  return 0;
}
// Annihilate (create) orbital b on a string: the sign is (-1)^(occupied orbitals below b).
__device__ __forceinline__ int annihilate(int& mask, int b) {
  const int sgn = (__popc(mask & ((1 << b) - 1)) & 1) ? -1 : 1;
  mask &= ~(1 << b);
  return sgn;
}
__device__ __forceinline__ int create(int& mask, int b) {
  const int sgn = (__popc(mask & ((1 << b) - 1)) & 1) ? -1 : 1;
  mask |= 1 << b;
  return sgn;
}
constexpr int kPhiMask = 0b000111;

// Sign and string index of a+_{3+a} a_i acting on the Phi string.
__device__ __forceinline__ int single_on_phi(int i, int a, int* sign) {
  int m = kPhiMask;
  int s = annihilate(m, i);
  s *= create(m, 3 + a);
  *sign = s;
  return string_index(m);
}

// Packed position of X2[i][j][a][b] (symmetric under (i a) <-> (j b)).
__device__ __forceinline__ int x2_slot(int i, int a, int j, int b) {
  int P = 3 * i + a, R = 3 * j + b;
  if (P > R) {
    const int t = P;
    P = R;
    R = t;
  }
  return 9 + P * 9 - P * (P - 1) / 2 + (R - P);
}

// targets[r][54] from the saved root of class position r * stride; mask[r] = 1 when that
// space's solve finished with status 0 (its root was saved), else 0 and the row is zero.
template <typename R>
__global__ void k_targets(const R* __restrict__ roots, int64_t rows, int64_t stride,
                          const int64_t* __restrict__ sorted_index, const int32_t* __restrict__ status,
                          float* __restrict__ targets, uint8_t* __restrict__ mask) {
  const int64_t total = rows * QFLOW_MLP_NOUT;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t / QFLOW_MLP_NOUT;
    const int c = (int)(t % QFLOW_MLP_NOUT);
    const int64_t pos = r * stride;
    const bool ok = status ? status[sorted_index ? sorted_index[pos] : pos] == 0 : true;
    if (c == 0 && mask) mask[r] = ok ? 1 : 0;
    if (!ok) {
      targets[t] = 0.f;
      continue;
    }
    const R* v = roots + (size_t)pos * 400;
    auto x1 = [&](int i, int a) {  // mean of the alpha and beta single coefficients
      int sg = 0;
      const int J = single_on_phi(i, a, &sg);
      return 0.5f * (float)sg * ((float)v[J * 20] + (float)v[J]);
    };
    float y;
    if (c < 9) {
      y = x1(c / 3, c % 3);
    } else {
      int k = c - 9, P = 0;
      while (k >= 9 - P) {
        k -= 9 - P;
        ++P;
      }
      const int R = P + k;
      const int i = P / 3, a = P % 3, j = R / 3, b = R % 3;
      int sa = 0, sb = 0, sa2 = 0, sb2 = 0;
      const int Ja = single_on_phi(i, a, &sa), Jb = single_on_phi(j, b, &sb);
      const int Ja2 = single_on_phi(j, b, &sa2), Jb2 = single_on_phi(i, a, &sb2);
      const float cab = (float)(sa * sb) * (float)v[Ja * 20 + Jb];      // alpha (i->a), beta (j->b)
      const float cba = (float)(sa2 * sb2) * (float)v[Ja2 * 20 + Jb2];  // alpha (j->b), beta (i->a)
      y = 0.5f * (cab + cba) - x1(i, a) * x1(j, b);
    }
    targets[t] = y;
  }
}

// Start vectors guess[r][400] from network outputs pred[r][54]; y = mu + sd * pred when mu is
// given.  Thread per determinant.
template <typename T>
__global__ void k_guess(const float* __restrict__ pred, int64_t rows, const float* __restrict__ mu,
                        const float* __restrict__ sd, T* __restrict__ guess) {
  __shared__ int masks[20];
  if (threadIdx.x < 20) masks[threadIdx.x] = string_mask(threadIdx.x);
  __syncthreads();
  const int64_t total = rows * 400;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t / 400;
    const int d = (int)(t % 400);
    const float* y = pred + (size_t)r * QFLOW_MLP_NOUT;
    auto val = [&](int c) { return mu ? mu[c] + sd[c] * y[c] : y[c]; };
    auto X1 = [&](int i, int a) { return val(3 * i + a); };
    auto X2 = [&](int i, int j, int a, int b) { return val(x2_slot(i, a, j, b)); };
    const int ma = masks[d / 20], mb = masks[d % 20];
    const int ra = __popc(ma & 0b111000), rb = __popc(mb & 0b111000);
    // holes (local occupied orbitals missing) and particles (local virtuals present), ascending
    int ha[3], pa[3], hb[3], pb[3], nha = 0, npa = 0, nhb = 0, npb = 0;
    for (int o = 0; o < 3; ++o) {
      if (!((ma >> o) & 1)) ha[nha++] = o;
      if (!((mb >> o) & 1)) hb[nhb++] = o;
      if ((ma >> (3 + o)) & 1) pa[npa++] = o;
      if ((mb >> (3 + o)) & 1) pb[npb++] = o;
    }
    float c = 0.f;
    if (ra + rb == 0) {
      c = 1.f;
    } else if (ra + rb == 1) {  // a+_a a_i on one string
      const bool alpha = ra == 1;
      const int i = alpha ? ha[0] : hb[0], a = alpha ? pa[0] : pb[0];
      int sg = 0;
      single_on_phi(i, a, &sg);
      c = (float)sg * X1(i, a);
    } else if (ra == 1 && rb == 1) {  // alpha (i->a), beta (j->b)
      int s1 = 0, s2 = 0;
      single_on_phi(ha[0], pa[0], &s1);
      single_on_phi(hb[0], pb[0], &s2);
      c = (float)(s1 * s2) * (X2(ha[0], hb[0], pa[0], pb[0]) + X1(ha[0], pa[0]) * X1(hb[0], pb[0]));
    } else if (ra + rb == 2) {  // same spin: a+_a a+_b a_j a_i, i < j, a < b
      const int* h = (ra == 2) ? ha : hb;
      const int* p = (ra == 2) ? pa : pb;
      const int i = h[0], j = h[1], a = p[0], b = p[1];
      int m = kPhiMask;
      int sg = annihilate(m, i);
      sg *= annihilate(m, j);
      sg *= create(m, 3 + b);
      sg *= create(m, 3 + a);
      const float amp = X2(i, j, a, b) - X2(i, j, b, a) + X1(i, a) * X1(j, b) - X1(i, b) * X1(j, a);
      c = (float)sg * amp;
    }
    guess[(size_t)r * 400 + d] = (T)c;
  }
}

// ---- column statistics (FP64 accumulation, fixed order) --------------------------------------
constexpr int SB = 256;       // threads per block of the statistics kernels
constexpr int SROWS = 2048;   // rows per partial block

// partial[b][c] = sum over rows of block b (ascending) of m_r * f(X[r][c]); f = x or (x - mu)^2
__global__ void k_col_partial(const float* __restrict__ X, int64_t rows, int cols, const uint8_t* __restrict__ mask,
                              const double* __restrict__ mu, double* __restrict__ partial) {
  const int64_t r0 = (int64_t)blockIdx.y * SROWS;
  const int64_t r1 = (r0 + SROWS < rows) ? r0 + SROWS : rows;
  for (int c = blockIdx.x * SB + threadIdx.x; c < cols; c += gridDim.x * SB) {
    double s = 0.0;
    for (int64_t r = r0; r < r1; ++r) {
      if (mask && !mask[r]) continue;
      const double x = (double)X[(size_t)r * cols + c];
      s += mu ? (x - mu[c]) * (x - mu[c]) : x;
    }
    partial[(size_t)blockIdx.y * cols + c] = s;
  }
}

__global__ void k_col_final(const double* __restrict__ partial, int nblk, int cols, double count,
                            double* __restrict__ out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += partial[(size_t)b * cols + c];
  out[c] = s / count;
}

// mu[c] = mean, scale[c] = 1/sd (inverse) or sd; a column with sd <= 1e-12 (1 + |mean|) gets
// scale 0 (inverse) or 1.
__global__ void k_col_store(const double* __restrict__ mean, const double* __restrict__ var, int cols, int inverse,
                            float* __restrict__ mu, float* __restrict__ scale) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  const double sd = sqrt(var[c]);
  const bool flat = !(sd > 1e-12 * (1.0 + fabs(mean[c])));
  mu[c] = (float)mean[c];
  scale[c] = inverse ? (flat ? 0.f : (float)(1.0 / sd)) : (flat ? 1.f : (float)sd);
}

// out[r][c] = (X[src(r)][c] - mu[c]) * sc[c]; src(r) = order[r] when order is given.
// Also copies the row masks when given.
__global__ void k_rows(const float* __restrict__ X, int64_t rows, int cols, const int64_t* __restrict__ order,
                       const float* __restrict__ mu, const float* __restrict__ sc, float* __restrict__ out,
                       const uint8_t* __restrict__ mask_in, uint8_t* __restrict__ mask_out) {
  const int64_t total = rows * cols;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t / cols;
    const int c = (int)(t % cols);
    const int64_t src = order ? order[r] : r;
    float v = X[(size_t)src * cols + c];
    if (mu) v = (v - mu[c]) * sc[c];
    out[t] = v;
    if (mask_out && c == 0) mask_out[r] = mask_in ? mask_in[src] : 1;
  }
}

unsigned grid1(int64_t n, int threads) {
  const int64_t g = (n + threads - 1) / threads;
  return (unsigned)(g < 1 ? 1 : (g > 65536 ? 65536 : g));
}

struct Net {
  int I, H, O;
  const float *W1, *b1, *W2, *b2, *W3, *b3;
  Net(int i, int h, int o, const float* p) : I(i), H(h), O(o) {
    W1 = p;
    b1 = W1 + (size_t)I * H;
    W2 = b1 + H;
    b2 = W2 + (size_t)H * H;
    W3 = b2 + H;
    b3 = W3 + (size_t)H * O;
  }
};

}  // namespace

int64_t mlp_param_count(int I, int H, int O) { return (int64_t)I * H + H + (int64_t)H * H + H + (int64_t)H * O + O; }

size_t mlp_workspace_bytes(int I, int H, int O, int64_t rows) {
  (void)I;
  // H1, H2, dZ (rows x H each), Y, dY (rows x O each), loss partials + loss
  return sizeof(float) * ((size_t)rows * (3 * (size_t)H + 2 * (size_t)O) + LGRID + 4) + 512;
}
// the products' timeout flag: the workspace's last 256 bytes
int* mlp_err(void* work, int I, int H, int O, int64_t rows) {
  return reinterpret_cast<int*>(static_cast<char*>(work) + mlp_workspace_bytes(I, H, O, rows) - 256);
}

cudaError_t mlp_forward(int I, int H, int O, const float* params, const float* x, int64_t rows, float* y, void* work,
                        cudaStream_t st) {
  const Net net(I, H, O, params);
  float* H1 = static_cast<float*>(work);
  float* H2 = H1 + (size_t)rows * H;
  const int R = (int)rows;
  int* err = mlp_err(work, I, H, O, rows);
  cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int), st);
  if (e == cudaSuccess) e = gemm<false, false, kBiasTanh>(R, H, I, x, I, net.W1, H, H1, H, net.b1, nullptr, err, st);
  if (e == cudaSuccess) e = gemm<false, false, kBiasTanh>(R, H, H, H1, H, net.W2, H, H2, H, net.b2, nullptr, err, st);
  if (e == cudaSuccess) e = gemm<false, false, kBias>(R, O, H, H2, H, net.W3, O, y, O, net.b3, nullptr, err, st);
  if (e == cudaSuccess && R > 0) {
    k_mlp_check<<<1, 32, 0, st>>>(err, y);
    e = cudaGetLastError();
  }
  return e;
}

cudaError_t mlp_loss_grad(int I, int H, int O, const float* params, const float* x, const float* t,
                          const uint8_t* mask, int64_t rows, float* grad, float* loss, void* work, cudaStream_t st) {
  const Net net(I, H, O, params);
  const int R = (int)rows;
  float* H1 = static_cast<float*>(work);
  float* H2 = H1 + (size_t)rows * H;
  float* dZ = H2 + (size_t)rows * H;
  float* Y = dZ + (size_t)rows * H;
  float* dY = Y + (size_t)rows * O;
  float* part = dY + (size_t)rows * O;
  float* gW1 = grad;
  float* gb1 = gW1 + (size_t)I * H;
  float* gW2 = gb1 + H;
  float* gb2 = gW2 + (size_t)H * H;
  float* gW3 = gb2 + H;
  float* gb3 = gW3 + (size_t)H * O;
  int* err = mlp_err(work, I, H, O, rows);
  cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int), st);
  if (e == cudaSuccess) e = gemm<false, false, kBiasTanh>(R, H, I, x, I, net.W1, H, H1, H, net.b1, nullptr, err, st);
  if (e == cudaSuccess) e = gemm<false, false, kBiasTanh>(R, H, H, H1, H, net.W2, H, H2, H, net.b2, nullptr, err, st);
  if (e == cudaSuccess) e = gemm<false, false, kBias>(R, O, H, H2, H, net.W3, O, Y, O, net.b3, nullptr, err, st);
  if (e != cudaSuccess) return e;
  k_loss_grad<<<LGRID, LB, 0, st>>>(Y, t, mask, R, O, dY, part);
  k_loss_final<<<1, 32, 0, st>>>(part, R, loss);
  // layer 3: gW3 = H2^T dY, gb3 = colsum dY, dZ2 = (dY W3^T) (1 - H2^2)
  e = gemm<true, false, kStore>(H, O, R, H2, H, dY, O, gW3, O, nullptr, nullptr, err, st);
  if (e != cudaSuccess) return e;
  k_colsum<<<grid1(O, 128), 128, 0, st>>>(dY, R, O, gb3);
  e = gemm<false, true, kTanhGrad>(R, H, O, dY, O, net.W3, O, dZ, H, nullptr, H2, err, st);
  // layer 2: gW2 = H1^T dZ2, gb2 = colsum dZ2, dZ1 = (dZ2 W2^T) (1 - H1^2) (into H2's buffer)
  if (e == cudaSuccess) e = gemm<true, false, kStore>(H, H, R, H1, H, dZ, H, gW2, H, nullptr, nullptr, err, st);
  if (e != cudaSuccess) return e;
  k_colsum<<<grid1(H, 128), 128, 0, st>>>(dZ, R, H, gb2);
  e = gemm<false, true, kTanhGrad>(R, H, H, dZ, H, net.W2, H, H2, H, nullptr, H1, err, st);
  // layer 1: gW1 = X^T dZ1, gb1 = colsum dZ1
  if (e == cudaSuccess) e = gemm<true, false, kStore>(I, H, R, x, I, H2, H, gW1, H, nullptr, nullptr, err, st);
  if (e != cudaSuccess) return e;
  k_colsum<<<grid1(H, 128), 128, 0, st>>>(H2, R, H, gb1);
  k_mlp_check<<<1, 32, 0, st>>>(err, loss);  // a failed product shows as a NaN loss
  return cudaGetLastError();
}

cudaError_t mlp_adam(int64_t n, float* p, const float* g, float* m, float* v, int step, float lr, float b1, float b2,
                     float eps, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const float bc1 = (float)(1.0 - pow((double)b1, (double)step));
  const float bc2 = (float)(1.0 - pow((double)b2, (double)step));
  k_adam<<<grid1(n, 256) > 2048 ? 2048 : grid1(n, 256), 256, 0, st>>>(n, p, g, m, v, lr, b1, b2, eps, bc1, bc2);
  return cudaGetLastError();
}

cudaError_t mlp_features(int n, const double* F, const double* W, const qflow_space* spaces, int64_t nspaces,
                         int64_t stride, const float* mu, const float* sc, float* out, cudaStream_t st) {
  if (nspaces <= 0) return cudaSuccess;
  const int64_t need = (nspaces + FW - 1) / FW;
  const unsigned g = (unsigned)(need > 152 * 16 ? 152 * 16 : need);
  k_features<<<g, 32 * FW, 0, st>>>(n, F, W, spaces, nspaces, stride, mu, sc, out);
  return cudaGetLastError();
}

cudaError_t mlp_targets(const void* roots, bool fp64, int64_t rows, int64_t stride, const int64_t* sorted_index,
                        const int32_t* status, float* targets, uint8_t* mask, cudaStream_t st) {
  if (rows <= 0) return cudaSuccess;
  const unsigned g = grid1(rows * QFLOW_MLP_NOUT, 256) > 4096 ? 4096 : grid1(rows * QFLOW_MLP_NOUT, 256);
  if (fp64)
    k_targets<double><<<g, 256, 0, st>>>(static_cast<const double*>(roots), rows, stride, sorted_index, status,
                                         targets, mask);
  else
    k_targets<float><<<g, 256, 0, st>>>(static_cast<const float*>(roots), rows, stride, sorted_index, status,
                                        targets, mask);
  return cudaGetLastError();
}

// Absolute pool index of packed component c of a (3,3) space with orbitals o[6] (occupied
// first): t1[i][a] for c < 9, else t2[i][j][a][b] of the pair P = 3i+a <= R = 3j+b.
__device__ __forceinline__ int64_t pool_index(const int* o, int c, int nocc, int nvir, int64_t n_t1, int* is_t2,
                                              int64_t* mirror) {
  if (c < 9) {
    *is_t2 = 0;
    *mirror = -1;
    return (int64_t)o[c / 3] * nvir + (o[3 + c % 3] - nocc);
  }
  int k = c - 9, P = 0;
  while (k >= 9 - P) {
    k -= 9 - P;
    ++P;
  }
  const int R = P + k;
  const int i = o[P / 3], a = o[3 + P % 3] - nocc, j = o[R / 3], b = o[3 + R % 3] - nocc;
  *is_t2 = 1;
  *mirror = n_t1 + (((int64_t)j * nocc + i) * nvir + b) * nvir + a;  // t2[j][i][b][a]
  return n_t1 + (((int64_t)i * nocc + j) * nvir + a) * nvir + b;
}

// targets[r][54] = the pool's internal amplitudes of the space at class position r * stride.
__global__ void k_pool_targets(const double* __restrict__ pool, const qflow_space* __restrict__ spaces, int64_t rows,
                               int64_t stride, int nocc, int nvir, float* __restrict__ targets,
                               uint8_t* __restrict__ mask) {
  const int64_t n_t1 = (int64_t)nocc * nvir;
  const int64_t total = rows * QFLOW_MLP_NOUT;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t / QFLOW_MLP_NOUT;
    const int c = (int)(t % QFLOW_MLP_NOUT);
    const qflow_space& q = spaces[r * stride];
    const int o[6] = {q.orb[0], q.orb[1], q.orb[2], q.orb[3], q.orb[4], q.orb[5]};
    int is_t2 = 0;
    int64_t mirror = 0;
    targets[t] = (float)pool[pool_index(o, c, nocc, nvir, n_t1, &is_t2, &mirror)];
    if (c == 0 && mask) mask[r] = 1;
  }
}

// pool[x] = mu + sd * pred[r][c] for every amplitude x whose owner is the space at class
// position r (sorted index sorted_index[r]); t2 entries are written with their mirror.
__global__ void k_pool_from_pred(const float* __restrict__ pred, const float* __restrict__ mu,
                                 const float* __restrict__ sd, const qflow_space* __restrict__ spaces,
                                 const int64_t* __restrict__ sorted_index, int64_t rows, int nocc, int nvir,
                                 const int32_t* __restrict__ owner1, const int32_t* __restrict__ owner2,
                                 double* __restrict__ pool) {
  const int64_t n_t1 = (int64_t)nocc * nvir;
  const int64_t total = rows * QFLOW_MLP_NOUT;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t / QFLOW_MLP_NOUT;
    const int c = (int)(t % QFLOW_MLP_NOUT);
    const qflow_space& q = spaces[r];
    const int o[6] = {q.orb[0], q.orb[1], q.orb[2], q.orb[3], q.orb[4], q.orb[5]};
    int is_t2 = 0;
    int64_t mirror = 0;
    const int64_t x = pool_index(o, c, nocc, nvir, n_t1, &is_t2, &mirror);
    const int32_t own = is_t2 ? owner2[x - n_t1] : owner1[x];
    if (own != (int32_t)sorted_index[r]) continue;
    const double v = (double)(mu ? mu[c] + sd[c] * pred[t] : pred[t]);
    pool[x] = v;
    if (is_t2) pool[mirror] = v;
  }
}

__global__ void k_invert(const float* __restrict__ sd, int n, float* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = sd[i] > 0.f ? 1.f / sd[i] : 0.f;
}

cudaError_t mlp_pool_targets(const double* pool, const qflow_space* spaces, int64_t rows, int64_t stride, int nocc,
                             int nvir, float* targets, uint8_t* mask, cudaStream_t st) {
  if (rows <= 0) return cudaSuccess;
  const unsigned g = grid1(rows * QFLOW_MLP_NOUT, 256) > 4096 ? 4096 : grid1(rows * QFLOW_MLP_NOUT, 256);
  k_pool_targets<<<g, 256, 0, st>>>(pool, spaces, rows, stride, nocc, nvir, targets, mask);
  return cudaGetLastError();
}

cudaError_t mlp_pool_from_pred(const float* pred, const float* mu, const float* sd, const qflow_space* spaces,
                               const int64_t* sorted_index, int64_t rows, int nocc, int nvir, const int32_t* owner1,
                               const int32_t* owner2, double* pool, cudaStream_t st) {
  if (rows <= 0) return cudaSuccess;
  const unsigned g = grid1(rows * QFLOW_MLP_NOUT, 256) > 4096 ? 4096 : grid1(rows * QFLOW_MLP_NOUT, 256);
  k_pool_from_pred<<<g, 256, 0, st>>>(pred, mu, sd, spaces, sorted_index, rows, nocc, nvir, owner1, owner2, pool);
  return cudaGetLastError();
}

// Spaces that own at least one amplitude: flag[sorted index] = 1 from the owner maps; then the
// flagged positions of one class list are gathered (space records and sorted indices) in any
// order, with their count.  Only those spaces' predictions reach the pool in a warm start.
__global__ void k_flag_owners(const int32_t* __restrict__ own, int64_t m, uint8_t* __restrict__ flag) {
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < m; x += (int64_t)gridDim.x * blockDim.x)
    if (own[x] >= 0) flag[own[x]] = 1;
}

__global__ void k_gather_flagged(const qflow_space* __restrict__ spaces, const int64_t* __restrict__ sorted_index,
                                 int64_t rows, const uint8_t* __restrict__ flag, qflow_space* __restrict__ out_sp,
                                 int64_t* __restrict__ out_idx, unsigned long long* __restrict__ count) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rows; r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t si = sorted_index[r];
    if (flag[si]) {
      const unsigned long long k = atomicAdd(count, 1ull);
      out_sp[k] = spaces[r];
      out_idx[k] = si;
    }
  }
}

cudaError_t mlp_owner_spaces(const int32_t* owner1, int64_t n1, const int32_t* owner2, int64_t n2, int64_t nspaces,
                             const qflow_space* spaces, const int64_t* sorted_index, int64_t rows, uint8_t* flag,
                             qflow_space* out_sp, int64_t* out_idx, unsigned long long* count, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(flag, 0, (size_t)nspaces, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(count, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  k_flag_owners<<<grid1(n1, 256) > 4096 ? 4096 : grid1(n1, 256), 256, 0, st>>>(owner1, n1, flag);
  k_flag_owners<<<grid1(n2, 256) > 4096 ? 4096 : grid1(n2, 256), 256, 0, st>>>(owner2, n2, flag);
  if (rows > 0)
    k_gather_flagged<<<grid1(rows, 256) > 4096 ? 4096 : grid1(rows, 256), 256, 0, st>>>(spaces, sorted_index, rows,
                                                                                        flag, out_sp, out_idx, count);
  return cudaGetLastError();
}

cudaError_t mlp_invert(const float* sd, int n, float* out, cudaStream_t st) {
  k_invert<<<grid1(n, 128), 128, 0, st>>>(sd, n, out);
  return cudaGetLastError();
}

cudaError_t mlp_guess(const float* pred, int64_t rows, const float* mu, const float* sd, void* guess, bool fp64,
                      cudaStream_t st) {
  if (rows <= 0) return cudaSuccess;
  const unsigned g = grid1(rows * 400, 256) > 8192 ? 8192 : grid1(rows * 400, 256);
  if (fp64)
    k_guess<double><<<g, 256, 0, st>>>(pred, rows, mu, sd, static_cast<double*>(guess));
  else
    k_guess<float><<<g, 256, 0, st>>>(pred, rows, mu, sd, static_cast<float*>(guess));
  return cudaGetLastError();
}

size_t mlp_stats_workspace_bytes(int64_t rows, int cols) {
  const int64_t nblk = (rows + SROWS - 1) / SROWS;
  return sizeof(double) * ((size_t)(nblk < 1 ? 1 : nblk) * cols + 2 * (size_t)cols) + 256;
}

cudaError_t mlp_col_stats(const float* X, int64_t rows, int cols, const uint8_t* mask, int64_t count, int inverse,
                          float* mu, float* scale, void* work, cudaStream_t st) {
  if (rows <= 0 || count <= 0) return cudaErrorInvalidValue;
  const int nblk = (int)((rows + SROWS - 1) / SROWS);
  double* partial = static_cast<double*>(work);
  double* mean = partial + (size_t)nblk * cols;
  double* var = mean + cols;
  const dim3 g((unsigned)((cols + SB - 1) / SB), (unsigned)nblk);
  k_col_partial<<<g, SB, 0, st>>>(X, rows, cols, mask, nullptr, partial);
  k_col_final<<<grid1(cols, 128), 128, 0, st>>>(partial, nblk, cols, (double)count, mean);
  k_col_partial<<<g, SB, 0, st>>>(X, rows, cols, mask, mean, partial);
  k_col_final<<<grid1(cols, 128), 128, 0, st>>>(partial, nblk, cols, (double)count, var);
  k_col_store<<<grid1(cols, 128), 128, 0, st>>>(mean, var, cols, inverse, mu, scale);
  return cudaGetLastError();
}

cudaError_t mlp_rows(const float* X, int64_t rows, int cols, const int64_t* order, const float* mu, const float* sc,
                     float* out, const uint8_t* mask_in, uint8_t* mask_out, cudaStream_t st) {
  if (rows <= 0) return cudaSuccess;
  k_rows<<<grid1(rows * cols, 256) > 8192 ? 8192 : grid1(rows * cols, 256), 256, 0, st>>>(X, rows, cols, order, mu, sc,
                                                                                          out, mask_in, mask_out);
  return cudaGetLastError();
}

}  // namespace qf
