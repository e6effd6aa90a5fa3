// Step (a) in the Hermitian (DUCC) form: the global part of every space's downfolded
// Hamiltonian (Eqs. 1-8 with N = 1 and an anti-Hermitian sigma = T - T^+; the paper leaves the
// truncation open, this library uses all terms through second order, each commutator normal
// ordered with respect to Phi and kept to <= two-body):
//
//   H_eff(i) = P_i [ H + [H, s] + 1/2 [[F, s], s] ]_(<=2) P_i,   s = sigma_ext(i),
//
// with F the (diagonal) Fock operator of the reference.  By linearity it splits into a part
// common to every space, G = [H + [H, sigma] + 1/2 [[F, sigma], sigma]]_(<=2) over the whole pool,
// restricted to the space's orbitals, minus a part L_A built from the space's internal
// amplitudes alone (solve.cu, per space): a commutator with an operator whose indices all lie in
// the space only sees the other factor's part inside the space, and F does not mix orbitals.
//
// G here, in the spin-free (E0, F, W) layout of the SES-CC dressing:
//   [H, sigma] = X + X^+,  X = [H, T]_(<=2);   1/2 [[F, sigma], sigma] = 1/2 (Y + Y^+),  Y = [B, T]_(<=2),
//   B = [F, sigma] = D.T + (D.T)^+ (D = orbital-energy differences of each excitation).
// X and Y are the T-linear parts of the SES-CC dressing e^{-T} O e^{T} of O = H and O = B: that
// dressing is a polynomial of degree four in T, so its linear part is exactly the five-point
// central difference  [8 (O(T) - O(-T)) - (O(2T) - O(-2T))] / 12  of four FP64 dressings
// (dress.cu; its formulas assume no index symmetry of the operator beyond W_pqrs = W_rspq, which B
// has).  The operator part O itself cancels in the difference.
#include <cuda_runtime.h>
#include <stdint.h>

#include "qflow_internal.h"

namespace qf {
namespace {

constexpr int TPB = 256;
inline unsigned grid_for(size_t m) {
  const size_t b = (m + TPB - 1) / TPB;
  return (unsigned)(b < 65535 * 8 ? b : 65535 * 8);
}

// Bare Fock matrix F0_pq = h_pq + sum_k [2 (pq|kk) - (pk|kq)] and E_HF = sum_k (h_kk + F0_kk).
__global__ void k_fock0(const double* __restrict__ h, const double* __restrict__ eri, int n, int nocc,
                        double* __restrict__ F0) {
  const size_t n1 = n, n2 = n1 * n1, n3 = n2 * n1;
  for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < n * n; x += gridDim.x * blockDim.x) {
    const int p = x / n, q = x % n;
    double v = h[x];
    for (int k = 0; k < nocc; ++k)
      v += 2.0 * eri[p * n3 + q * n2 + k * n1 + k] - eri[p * n3 + k * n2 + k * n1 + q];
    F0[x] = v;
  }
}

__global__ void k_e_hf(const double* __restrict__ h, const double* __restrict__ F0, int n, int nocc,
                       double* __restrict__ e0) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    double e = 0.0;
    for (int k = 0; k < nocc; ++k) e += h[k * n + k] + F0[k * n + k];
    *e0 = e;
  }
}

__global__ void k_scaled(const double* __restrict__ x, double s, double* __restrict__ y, size_t m) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < m; i += (size_t)gridDim.x * blockDim.x)
    y[i] = s * x[i];
}

// B = D.T + (D.T)^+ as a spin-free operator on n orbitals: one-body hB_ai = hB_ia = (e_a - e_i) t_i^a,
// two-body gB_aibj = gB_iajb = (e_a + e_b - e_i - e_j) t_ij^ab, every other element zero (the caller
// zeroes gB).  Its normal ordering adds nothing (no element of the form (pq|kk) or (pk|kq) with k
// occupied), so hB is also its normal-ordered one-body part.
__global__ void k_b_operator(const double* __restrict__ F0, const double* __restrict__ t1,
                             const double* __restrict__ t2, int n, int nocc, double* __restrict__ hB,
                             double* __restrict__ gB) {
  const int v = n - nocc;
  const size_t n1 = n, n2 = n1 * n1, n3 = n2 * n1;
  const size_t m2 = (size_t)nocc * nocc * v * v;
  for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < m2; x += (size_t)gridDim.x * blockDim.x) {
    const int b = (int)(x % v), a = (int)((x / v) % v), j = (int)((x / ((size_t)v * v)) % nocc),
              i = (int)(x / ((size_t)v * v * nocc));
    const int A = nocc + a, Bv = nocc + b;
    const double d = F0[A * n + A] + F0[Bv * n + Bv] - F0[i * n + i] - F0[j * n + j];
    const double val = d * t2[x];
    gB[A * n3 + i * n2 + Bv * n1 + j] = val;
    gB[i * n3 + A * n2 + j * n1 + Bv] = val;
  }
  for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < n2; x += (size_t)gridDim.x * blockDim.x) {
    const int p = (int)(x / n), q = (int)(x % n);
    double val = 0.0;
    if (p >= nocc && q < nocc) val = (F0[p * n + p] - F0[q * n + q]) * t1[(size_t)q * v + (p - nocc)];
    if (p < nocc && q >= nocc) val = (F0[q * n + q] - F0[p * n + p]) * t1[(size_t)p * v + (q - nocc)];
    hB[x] = val;
  }
}

// out += c (X + X^+) for a dressing's (e0, F, W): W^+_pqrs = W_qpsr, F^+_pq = F_qp, e0^+ = e0.
__global__ void k_acc_hermitian(const double* __restrict__ e0, const double* __restrict__ F,
                                const double* __restrict__ W, double c, int n, double* __restrict__ oe,
                                double* __restrict__ oF, double* __restrict__ oW) {
  const size_t n1 = n, n2 = n1 * n1, n3 = n2 * n1, n4 = n3 * n1;
  for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < n4; x += (size_t)gridDim.x * blockDim.x) {
    const size_t p = x / n3, q = (x / n2) % n1, r = (x / n1) % n1, s = x % n1;
    oW[x] += c * (W[x] + W[q * n3 + p * n2 + s * n1 + r]);
  }
  for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < n2; x += (size_t)gridDim.x * blockDim.x) {
    const size_t p = x / n1, q = x % n1;
    oF[x] += c * (F[x] + F[q * n1 + p]);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *oe += c * 2.0 * (*e0);
}

// Workspace layout (bytes, each part 256-aligned).
struct DuccWork {
  size_t dress, t1s, t2s, e, F, W, hB, gB, total;
};
DuccWork ducc_layout(int n, int nocc) {
  auto al = [](size_t b) { return (b + 255) / 256 * 256; };
  const size_t n1 = n, n2 = n1 * n1, n4 = n2 * n2;
  const size_t ov = (size_t)nocc * (n - nocc), oovv = ov * ov;
  DuccWork w{};
  size_t off = 0;
  w.dress = off;
  off += al(dress_workspace_bytes(n, nocc));
  w.t1s = off;
  off += al(ov * sizeof(double));
  w.t2s = off;
  off += al(oovv * sizeof(double));
  w.e = off;
  off += al(sizeof(double));
  w.F = off;
  off += al(n2 * sizeof(double));
  w.W = off;
  off += al(n4 * sizeof(double));
  w.hB = off;
  off += al(n2 * sizeof(double));
  w.gB = off;
  off += al(n4 * sizeof(double));
  w.total = off;
  return w;
}

}  // namespace

size_t ducc_workspace_bytes(int n, int nocc) { return ducc_layout(n, nocc).total; }

int ducc_launch_count(int n, int nocc) { return 6 + 8 * (3 + dress_launch_count(n, nocc, false)); }

cudaError_t launch_dress_ducc(const double* h, const double* eri, const double* t1, const double* t2, int n, int nocc,
                              double* e0, double* F, double* W, double* F0, void* work, size_t work_bytes,
                              cudaStream_t st) {
  const DuccWork L = ducc_layout(n, nocc);
  if (work_bytes < L.total) return cudaErrorInvalidValue;
  unsigned char* base = static_cast<unsigned char*>(work);
  double* t1s = reinterpret_cast<double*>(base + L.t1s);
  double* t2s = reinterpret_cast<double*>(base + L.t2s);
  double* ek = reinterpret_cast<double*>(base + L.e);
  double* Fk = reinterpret_cast<double*>(base + L.F);
  double* Wk = reinterpret_cast<double*>(base + L.W);
  double* hB = reinterpret_cast<double*>(base + L.hB);
  double* gB = reinterpret_cast<double*>(base + L.gB);
  const size_t n1 = n, n2 = n1 * n1, n4 = n2 * n2;
  const size_t ov = (size_t)nocc * (n - nocc), oovv = ov * ov;
  // G starts as H: E_HF, the bare Fock matrix, the integrals
  k_fock0<<<grid_for(n2), TPB, 0, st>>>(h, eri, n, nocc, F0);
  k_e_hf<<<1, 32, 0, st>>>(h, F0, n, nocc, e0);
  cudaError_t e = cudaMemcpyAsync(F, F0, n2 * sizeof(double), cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(W, eri, n4 * sizeof(double), cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(gB, 0, n4 * sizeof(double), st);
  if (e != cudaSuccess) return e;
  k_b_operator<<<grid_for(oovv > n2 ? oovv : n2), TPB, 0, st>>>(F0, t1, t2, n, nocc, hB, gB);
  // the T-linear parts: X of H (weight 1 on X + X^+) and Y of B (weight 1/2 on Y + Y^+)
  const double lam[4] = {1.0, -1.0, 2.0, -2.0};
  const double cof[4] = {8.0 / 12.0, -8.0 / 12.0, -1.0 / 12.0, 1.0 / 12.0};
  for (int op = 0; op < 2 && e == cudaSuccess; ++op) {
    const double* oh = op == 0 ? h : hB;
    const double* og = op == 0 ? eri : gB;
    const double w = op == 0 ? 1.0 : 0.5;
    for (int k = 0; k < 4 && e == cudaSuccess; ++k) {
      k_scaled<<<grid_for(ov), TPB, 0, st>>>(t1, lam[k], t1s, ov);
      k_scaled<<<grid_for(oovv), TPB, 0, st>>>(t2, lam[k], t2s, oovv);
      e = launch_dress(oh, og, t1s, t2s, n, nocc, ek, Fk, Wk, base + L.dress, L.t1s - L.dress, st);
      if (e == cudaSuccess) {
        k_acc_hermitian<<<grid_for(n4), TPB, 0, st>>>(ek, Fk, Wk, w * cof[k], n, e0, F, W);
        e = cudaGetLastError();
      }
    }
  }
  return e;
}

}  // namespace qf
