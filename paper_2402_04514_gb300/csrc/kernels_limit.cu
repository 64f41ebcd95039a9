// Sweeps C and D: symmetrisation of the limiter coefficients, the limited updates of Sec. 5.3,
// eq. (LimitedScheme), and the second limiter pass of Sec. 6.1.  One thread per row.
#include "gdg_internal.cuh"

namespace gdg {

namespace {

constexpr int kThreads = 256;

// Sweep C: l_ij = min(l_ij^(i), l_ji^(j)) (Lemma ConsInvariants needs l_ij = l_ji);
// U^(1)_i = U^L_i + (sum_j l_ij A_ij + sum_k l_i^k A_i^k) / m_i; then the second pass limits the
// remainder (1 - l) A from U^(1) against the same bounds.  With one pass it writes U_out from U^(1).
template <int DIM>
__global__ void __launch_bounds__(kThreads) k_limit2(Dev D, Scratch S, const double* __restrict__ Ubase,
                                                     double alpha, double* __restrict__ Uout, int last) {
  constexpr int M = DIM + 2;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= D.n) return;
  const size_t n = D.n, nnz = D.nnz, nb = D.nb;
  double acc[M];
#pragma unroll
  for (int q = 0; q < M; ++q) acc[q] = 0.0;
  const int r0 = D.row_ptr[i], r1 = D.row_ptr[i + 1];
  for (int e = r0; e < r1; ++e) {
    double l = fmin(S.l1[e], S.l1[D.tr[e]]);
#pragma unroll
    for (int q = 0; q < M; ++q) acc[q] += l * S.A[q * nnz + e];
  }
  for (int b = D.b_ptr[i]; b < D.b_ptr[i + 1]; ++b) {
    double l = S.l1B[b];
#pragma unroll
    for (int q = 0; q < M; ++q) acc[q] += l * S.AB[q * nb + b];
  }
  const double inv_mi = D.inv_mi[i];
  double U1[M];
#pragma unroll
  for (int q = 0; q < M; ++q) U1[q] = S.UL[q * n + i] + acc[q] * inv_mi;
  if (last) {
#pragma unroll
    for (int q = 0; q < M; ++q)
      Uout[q * n + i] = alpha != 0.0 ? alpha * Ubase[q * n + i] + (1.0 - alpha) * U1[q] : U1[q];
    return;
  }
#pragma unroll
  for (int q = 0; q < M; ++q) S.U1[q * n + i] = U1[q];
  LsRow<DIM> ls;
  ls_row<DIM>(D, ls, U1, S.bounds[i], S.bounds[n + i], S.bounds[2 * n + i]);
  const double ikm = D.inv_km[i];
  // an entry with l1 = 1 has no remainder: its l2 multiplies zero and is set to 1 without a search
  for (int e = r0; e < r1; ++e) {
    double rem = 1.0 - fmin(S.l1[e], S.l1[D.tr[e]]);
    if (rem == 0.0) {
      S.l2[e] = 1.0;
      continue;
    }
    double A[M];
#pragma unroll
    for (int q = 0; q < M; ++q) A[q] = S.A[q * nnz + e];
    S.l2[e] = line_search<DIM>(D, ls, A, rem * ikm);
  }
  for (int b = D.b_ptr[i]; b < D.b_ptr[i + 1]; ++b) {
    double rem = 1.0 - S.l1B[b];
    if (rem == 0.0) {
      S.l2B[b] = 1.0;
      continue;
    }
    double A[M];
#pragma unroll
    for (int q = 0; q < M; ++q) A[q] = S.AB[q * nb + b];
    S.l2B[b] = line_search<DIM>(D, ls, A, rem * ikm);
  }
}

// Sweep D: U^(2)_i = U^(1)_i + (sum_j l2_ij (1 - l1_ij) A_ij + sum_k l2_i^k (1 - l1_i^k) A_i^k) / m_i,
// symmetrised as in sweep C, and U_out = alpha U_base + (1 - alpha) U^(2).
template <int DIM>
__global__ void __launch_bounds__(kThreads) k_final(Dev D, Scratch S, const double* __restrict__ Ubase,
                                                    double alpha, double* __restrict__ Uout) {
  constexpr int M = DIM + 2;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= D.n) return;
  const size_t n = D.n, nnz = D.nnz, nb = D.nb;
  double acc[M];
#pragma unroll
  for (int q = 0; q < M; ++q) acc[q] = 0.0;
  for (int e = D.row_ptr[i]; e < D.row_ptr[i + 1]; ++e) {
    int t = D.tr[e];
    double w = fmin(S.l2[e], S.l2[t]) * (1.0 - fmin(S.l1[e], S.l1[t]));
#pragma unroll
    for (int q = 0; q < M; ++q) acc[q] += w * S.A[q * nnz + e];
  }
  for (int b = D.b_ptr[i]; b < D.b_ptr[i + 1]; ++b) {
    double w = S.l2B[b] * (1.0 - S.l1B[b]);
#pragma unroll
    for (int q = 0; q < M; ++q) acc[q] += w * S.AB[q * nb + b];
  }
  const double inv_mi = D.inv_mi[i];
#pragma unroll
  for (int q = 0; q < M; ++q) {
    double u2 = S.U1[q * n + i] + acc[q] * inv_mi;
    Uout[q * n + i] = alpha != 0.0 ? alpha * Ubase[q * n + i] + (1.0 - alpha) * u2 : u2;
  }
}

template <int DIM>
cudaError_t limit2_impl(const Dev& D, const Scratch& S, const double* Ubase, double alpha, double* Uout,
                        cudaStream_t s) {
  if (D.n == 0) return cudaSuccess;
  k_limit2<DIM><<<(D.n + kThreads - 1) / kThreads, kThreads, 0, s>>>(D, S, Ubase, alpha, Uout,
                                                                     D.passes == 1 ? 1 : 0);
  return cudaGetLastError();
}

template <int DIM>
cudaError_t final_impl(const Dev& D, const Scratch& S, const double* Ubase, double alpha, double* Uout,
                       cudaStream_t s) {
  if (D.n == 0) return cudaSuccess;
  k_final<DIM><<<(D.n + kThreads - 1) / kThreads, kThreads, 0, s>>>(D, S, Ubase, alpha, Uout);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_limit2(int dim, const Dev& D, const Scratch& S, const double* Ubase, double alpha, double* Uout,
                          cudaStream_t s) {
  GDG_DISPATCH(dim, limit2_impl, D, S, Ubase, alpha, Uout, s);
}

cudaError_t launch_final(int dim, const Dev& D, const Scratch& S, const double* Ubase, double alpha, double* Uout,
                         cudaStream_t s) {
  GDG_DISPATCH(dim, final_impl, D, S, Ubase, alpha, Uout, s);
}

}  // namespace gdg
