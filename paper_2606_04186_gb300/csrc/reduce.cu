// Step (c) reductions of a sweep: E_QFlow = mean_i E(i) (Results: the reported energy is the
// average over all active spaces), max |t_new - t_old| over the pool (convergence test), and
// the count / worst status of failed spaces.  Two fixed-shape passes, so the summation order
// and hence the result are identical run to run.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "qflow_internal.h"

namespace qf {
namespace {

constexpr int RB = 256;     // threads per block
constexpr int RGRID = 512;  // blocks of the first pass (fixed: deterministic order)

struct Partial {
  double esum, dmax, nfail, smax;
};

__global__ void k_partials(const double* __restrict__ energy, const int32_t* __restrict__ status, int64_t ns,
                           const double* __restrict__ t_old, const double* __restrict__ t_new, int64_t nt,
                           Partial* __restrict__ out) {
  __shared__ double se[RB], sd[RB], sf[RB], ss[RB];
  double e = 0.0, dm = 0.0, nf = 0.0, sm = 0.0;
  const int64_t stride = (int64_t)RGRID * RB;
  for (int64_t x = (int64_t)blockIdx.x * RB + threadIdx.x; x < ns; x += stride) {
    e += energy[x];
    if (status[x] != 0) {
      nf += 1.0;
      sm = fmax(sm, (double)status[x]);
    }
  }
  for (int64_t x = (int64_t)blockIdx.x * RB + threadIdx.x; x < nt; x += stride) {
    const double d = fabs(t_new[x] - t_old[x]);
    dm = (d > dm || d != d) ? d : dm;
  }
  se[threadIdx.x] = e;
  sd[threadIdx.x] = dm;
  sf[threadIdx.x] = nf;
  ss[threadIdx.x] = sm;
  __syncthreads();
  for (int s = RB / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) {
      se[threadIdx.x] += se[threadIdx.x + s];
      sd[threadIdx.x] = fmax(sd[threadIdx.x], sd[threadIdx.x + s]);
      sf[threadIdx.x] += sf[threadIdx.x + s];
      ss[threadIdx.x] = fmax(ss[threadIdx.x], ss[threadIdx.x + s]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = Partial{se[0], sd[0], sf[0], ss[0]};
}

__global__ void k_final(const Partial* __restrict__ in, int64_t ns, double* __restrict__ out4) {
  __shared__ double se[RB], sd[RB], sf[RB], ss[RB];
  double e = 0.0, dm = 0.0, nf = 0.0, sm = 0.0;
  for (int b = threadIdx.x; b < RGRID; b += RB) {
    e += in[b].esum;
    dm = fmax(dm, in[b].dmax);
    nf += in[b].nfail;
    sm = fmax(sm, in[b].smax);
  }
  se[threadIdx.x] = e;
  sd[threadIdx.x] = dm;
  sf[threadIdx.x] = nf;
  ss[threadIdx.x] = sm;
  __syncthreads();
  for (int s = RB / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) {
      se[threadIdx.x] += se[threadIdx.x + s];
      sd[threadIdx.x] = fmax(sd[threadIdx.x], sd[threadIdx.x + s]);
      sf[threadIdx.x] += sf[threadIdx.x + s];
      ss[threadIdx.x] = fmax(ss[threadIdx.x], ss[threadIdx.x + s]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out4[0] = (ns > 0) ? se[0] / (double)ns : 0.0;
    out4[1] = sd[0];
    out4[2] = sf[0];
    out4[3] = ss[0];
  }
}

// Exchange vector of a sharded sweep: [pool (np) | energy (ns) | code (ns)], code = status * 2^20
// + Davidson iterations (an exact integer in FP64; both fields are small and non-negative).
// Entries this shard did not produce hold -0.0, the identity of floating-point addition for every
// value (x + (-0.0) = x, also for x = +0.0 and -0.0), so the element-wise sum over the ranks
// reproduces each produced entry exactly, in any summation order.
constexpr int kCodeShift = 20;  // iterations below 2^20
__global__ void k_exchange_pack(const double* __restrict__ pool_new, const uint8_t* __restrict__ pool_mask, int64_t np,
                                const double* __restrict__ energy, const int32_t* __restrict__ status,
                                const int32_t* __restrict__ iters, const uint8_t* __restrict__ space_mask, int64_t ns,
                                double* __restrict__ x) {
  const int64_t total = np + 2 * ns;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    double v = -0.0;
    if (i < np) {
      if (pool_mask[i]) v = pool_new[i];
    } else {
      const int64_t j = (i - np) % ns, seg = (i - np) / ns;
      if (space_mask[j])
        v = (seg == 0) ? energy[j] : (double)(((int64_t)status[j] << kCodeShift) + (int64_t)iters[j]);
    }
    x[i] = v;
  }
}

// After the sum over ranks: owned amplitudes take the summed value (each has exactly one owner
// space, solved by exactly one rank); unowned ones keep t_old (already in pool_new).
__global__ void k_exchange_unpack(const double* __restrict__ x, const int32_t* __restrict__ own1, int64_t n1,
                                  const int32_t* __restrict__ own2, int64_t n2, double* __restrict__ pool_new,
                                  double* __restrict__ energy, int32_t* __restrict__ status,
                                  int32_t* __restrict__ iters, int64_t ns) {
  const int64_t np = n1 + n2, total = np + 2 * ns;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    if (i < np) {
      const int32_t o = (i < n1) ? own1[i] : own2[i - n1];
      if (o >= 0) pool_new[i] = x[i];
    } else {
      const int64_t j = (i - np) % ns, seg = (i - np) / ns;
      if (seg == 0) {
        energy[j] = x[i];
      } else {
        const int64_t c = (int64_t)x[i];
        status[j] = (int32_t)(c >> kCodeShift);
        iters[j] = (int32_t)(c & ((1 << kCodeShift) - 1));
      }
    }
  }
}

}  // namespace

cudaError_t launch_exchange_pack(const double* pool_new, const uint8_t* pool_mask, int64_t np, const double* energy,
                                 const int32_t* status, const int32_t* iters, const uint8_t* space_mask, int64_t ns,
                                 double* x, cudaStream_t st) {
  const int64_t total = np + 2 * ns;
  if (total == 0) return cudaSuccess;
  const int64_t blocks = std::min<int64_t>((total + RB - 1) / RB, 152 * 16);
  k_exchange_pack<<<(unsigned)blocks, RB, 0, st>>>(pool_new, pool_mask, np, energy, status, iters, space_mask, ns, x);
  return cudaGetLastError();
}

cudaError_t launch_exchange_unpack(const double* x, const int32_t* own1, int64_t n1, const int32_t* own2, int64_t n2,
                                   double* pool_new, double* energy, int32_t* status, int32_t* iters, int64_t ns,
                                   cudaStream_t st) {
  const int64_t total = n1 + n2 + 2 * ns;
  if (total == 0) return cudaSuccess;
  const int64_t blocks = std::min<int64_t>((total + RB - 1) / RB, 152 * 16);
  k_exchange_unpack<<<(unsigned)blocks, RB, 0, st>>>(x, own1, n1, own2, n2, pool_new, energy, status, iters, ns);
  return cudaGetLastError();
}

size_t mean_maxdiff_workspace(int64_t, int64_t) { return sizeof(Partial) * RGRID; }

// out4: [mean energy, max |dt|, failed spaces, worst status]; status is read from the int32
// array that follows `energy`'s owner (passed through `work` layout by the caller).
cudaError_t launch_reduce(const double* energy, const int32_t* status, int64_t nspaces, const double* t_old,
                          const double* t_new, int64_t nt, double* out4, void* work, cudaStream_t st) {
  Partial* part = static_cast<Partial*>(work);
  k_partials<<<RGRID, RB, 0, st>>>(energy, status, nspaces, t_old, t_new, nt, part);
  k_final<<<1, RB, 0, st>>>(part, nspaces, out4);
  return cudaGetLastError();
}

}  // namespace qf
