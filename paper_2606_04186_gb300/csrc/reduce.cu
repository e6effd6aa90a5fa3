// Step (c) reductions of a sweep: E_QFlow = mean_i E(i) (Results: the reported energy is the
// average over all active spaces), max |t_new - t_old| over the pool (convergence test), and
// the count / worst status of failed spaces.  Two fixed-shape passes, so the summation order
// and hence the result are identical run to run.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

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

}  // namespace

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
