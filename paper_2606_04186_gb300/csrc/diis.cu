// Optional Pulay DIIS on the amplitude pool (FP64).  Not part of the paper: an acceleration of
// the sweep-to-sweep fixed-point iteration that leaves its fixed point unchanged.
//
// After each sweep: error e = t_new - t_old, vector x = t_new are stored in a ring of m slots;
// B_ij = e_i . e_j is updated for the new slot; the extrapolated pool is sum_i c_i x_i with c from
//   [B  -1][c]   [ 0]
//   [-1  0][l] = [-1]
// solved in FP64 over the stored slots in age order (oldest first).  With fewer than two stored
// vectors, or an exactly singular system, the pool is left as t_new.  Every reduction has a
// fixed shape, so results do not depend on scheduling; the ring state lives on the device, so
// the whole step is stream-ordered (no host round trip).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "qflow_internal.h"

namespace qf {
namespace {

constexpr int DB = 256;     // threads per block
constexpr int DGRID = 256;  // blocks of the dot-product pass (fixed)

__global__ void k_diis_store(const double* __restrict__ t_old, const double* __restrict__ t_new, double* X,
                             double* E, const int* __restrict__ state, int64_t N) {
  const int slot = state[1];
  double* xs = X + (size_t)slot * N;
  double* es = E + (size_t)slot * N;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const double tn = t_new[i];
    xs[i] = tn;
    es[i] = tn - t_old[i];
  }
}

// partial[b * DIIS_MAX + j] = sum over block b's chunk of E[slot] . E[j]
__global__ void k_diis_dots(const double* __restrict__ E, const int* __restrict__ state, int m, int64_t N,
                            double* __restrict__ partial) {
  __shared__ double red[DB];
  const int slot = state[1];
  const int count = state[0] + 1 < m ? state[0] + 1 : m;  // slots holding data after this store
  const double* es = E + (size_t)slot * N;
  for (int j = 0; j < m; ++j) {
    double acc = 0.0;
    if (j < count || j == slot) {
      const double* ej = E + (size_t)j * N;
      for (int64_t i = blockIdx.x * (int64_t)DB + threadIdx.x; i < N; i += (int64_t)DGRID * DB) acc += es[i] * ej[i];
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = DB / 2; s > 0; s >>= 1) {
      if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
      __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x * QFLOW_DIIS_MAX + j] = red[0];
    __syncthreads();
  }
}

// Update B, the ring state and the coefficients (one block; solve on thread 0).
__global__ void k_diis_update(const double* __restrict__ partial, double* B, int* state, double* coeff, int m) {
  __shared__ double dots[QFLOW_DIIS_MAX];
  const int slot = state[1];
  if ((int)threadIdx.x < m) {
    double s = 0.0;
    for (int b = 0; b < DGRID; ++b) s += partial[b * QFLOW_DIIS_MAX + threadIdx.x];
    dots[threadIdx.x] = s;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  int count = state[0] + 1;
  if (count > m) count = m;
  for (int j = 0; j < m; ++j) {
    B[slot * QFLOW_DIIS_MAX + j] = dots[j];
    B[j * QFLOW_DIIS_MAX + slot] = dots[j];
  }
  const int head = (slot + 1) % m;
  state[0] = count;
  state[1] = head;
  state[2] = 0;  // 1 when coeff holds an extrapolation
  if (count < 2) return;
  // slots in age order: oldest = head - count (mod m)
  int order[QFLOW_DIIS_MAX];
  for (int i = 0; i < count; ++i) order[i] = ((head - count + i) % m + m) % m;
  const int dim = count + 1;
  double a[(QFLOW_DIIS_MAX + 1) * (QFLOW_DIIS_MAX + 1)], rhs[QFLOW_DIIS_MAX + 1];
  for (int i = 0; i < count; ++i) {
    for (int j = 0; j < count; ++j) a[i * dim + j] = B[order[i] * QFLOW_DIIS_MAX + order[j]];
    a[i * dim + count] = -1.0;
    a[count * dim + i] = -1.0;
    rhs[i] = 0.0;
  }
  a[count * dim + count] = 0.0;
  rhs[count] = -1.0;
  for (int col = 0; col < dim; ++col) {  // Gaussian elimination with partial pivoting
    int piv = col;
    for (int r = col + 1; r < dim; ++r)
      if (fabs(a[r * dim + col]) > fabs(a[piv * dim + col])) piv = r;
    if (a[piv * dim + col] == 0.0) return;  // exactly singular: keep t_new
    if (piv != col) {
      for (int j = 0; j < dim; ++j) {
        const double t = a[col * dim + j];
        a[col * dim + j] = a[piv * dim + j];
        a[piv * dim + j] = t;
      }
      const double t = rhs[col];
      rhs[col] = rhs[piv];
      rhs[piv] = t;
    }
    for (int r = col + 1; r < dim; ++r) {
      const double f = a[r * dim + col] / a[col * dim + col];
      for (int j = col; j < dim; ++j) a[r * dim + j] -= f * a[col * dim + j];
      rhs[r] -= f * rhs[col];
    }
  }
  double c[QFLOW_DIIS_MAX + 1];
  for (int r = dim - 1; r >= 0; --r) {
    double s = rhs[r];
    for (int j = r + 1; j < dim; ++j) s -= a[r * dim + j] * c[j];
    c[r] = s / a[r * dim + r];
  }
  for (int i = 0; i < count; ++i) {
    if (!isfinite(c[i])) return;
  }
  for (int i = 0; i < QFLOW_DIIS_MAX; ++i) coeff[i] = 0.0;
  for (int i = 0; i < count; ++i) coeff[i] = c[i];  // in age order
  state[2] = 1;
}

// t_new = sum_i coeff_i X[order_i] (age order) when an extrapolation was made.
__global__ void k_diis_combine(const double* __restrict__ X, const int* __restrict__ state,
                               const double* __restrict__ coeff, int m, double* __restrict__ t_new, int64_t N) {
  if (state[2] != 1) return;
  const int count = state[0], head = state[1];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    double v = 0.0;
    for (int k = 0; k < count; ++k) {
      const int slot = ((head - count + k) % m + m) % m;
      v += coeff[k] * X[(size_t)slot * N + i];
    }
    t_new[i] = v;
  }
}

}  // namespace

size_t diis_workspace_bytes(int m, int64_t N) {
  // X, E rings + B + coeff + partials + state
  return (size_t)2 * m * N * sizeof(double) + QFLOW_DIIS_MAX * QFLOW_DIIS_MAX * sizeof(double) +
         QFLOW_DIIS_MAX * sizeof(double) + (size_t)DGRID * QFLOW_DIIS_MAX * sizeof(double) + 4 * sizeof(int) + 256;
}

cudaError_t launch_diis(void* work, int m, const double* t_old, double* t_new, int64_t N, cudaStream_t st) {
  char* p = static_cast<char*>(work);
  double* X = reinterpret_cast<double*>(p);
  double* E = X + (size_t)m * N;
  double* B = E + (size_t)m * N;
  double* coeff = B + QFLOW_DIIS_MAX * QFLOW_DIIS_MAX;
  double* partial = coeff + QFLOW_DIIS_MAX;
  int* state = reinterpret_cast<int*>(partial + (size_t)DGRID * QFLOW_DIIS_MAX);
  const unsigned g = (unsigned)((N + DB - 1) / DB > 4096 ? 4096 : (N + DB - 1) / DB);
  k_diis_store<<<g, DB, 0, st>>>(t_old, t_new, X, E, state, N);
  k_diis_dots<<<DGRID, DB, 0, st>>>(E, state, m, N, partial);
  k_diis_update<<<1, 32, 0, st>>>(partial, B, state, coeff, m);
  k_diis_combine<<<g, DB, 0, st>>>(X, state, coeff, m, t_new, N);
  return cudaGetLastError();
}

cudaError_t diis_reset(void* work, int m, int64_t N, cudaStream_t st) {
  char* p = static_cast<char*>(work);
  double* X = reinterpret_cast<double*>(p);
  double* E = X + (size_t)m * N;
  double* B = E + (size_t)m * N;
  double* coeff = B + QFLOW_DIIS_MAX * QFLOW_DIIS_MAX;
  double* partial = coeff + QFLOW_DIIS_MAX;
  int* state = reinterpret_cast<int*>(partial + (size_t)DGRID * QFLOW_DIIS_MAX);
  cudaError_t e = cudaMemsetAsync(B, 0, QFLOW_DIIS_MAX * QFLOW_DIIS_MAX * sizeof(double), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(state, 0, 4 * sizeof(int), st);
  return e;
}

}  // namespace qf
