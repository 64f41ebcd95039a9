// Sweeps C and D: symmetrisation of the limiter coefficients, the limited updates of Sec. 5.3,
// eq. (LimitedScheme), and the second limiter pass of Sec. 6.1.  One thread per row.
#include <algorithm>

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
    double l = pmin(S.l1[e], S.l1[D.tr[e]]);  // limiter coefficients are in [0, 1]: integer min
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
    const double l1s = pmin(S.l1[e], S.l1[D.tr[e]]);
    if (is_one_bits(l1s)) {
      S.l2[e] = 1.0;
      continue;
    }
    const double w = (1.0 - l1s) * ikm;
    double A[M];
#pragma unroll
    for (int q = 0; q < M; ++q) A[q] = S.A[q * nnz + e];
    double l, fb;
    if (line_search_head<DIM>(D, ls, A, w, d2f_fast(w), &l, &fb))
      S.l2[e] = l;
    else
      ls_defer(S, 1, e, i);
  }
  for (int b = D.b_ptr[i]; b < D.b_ptr[i + 1]; ++b) {
    if (is_one_bits(S.l1B[b])) {
      S.l2B[b] = 1.0;
      continue;
    }
    const double w = (1.0 - S.l1B[b]) * ikm;
    double A[M];
#pragma unroll
    for (int q = 0; q < M; ++q) A[q] = S.AB[q * nb + b];
    double l, fb;
    if (line_search_head<DIM>(D, ls, A, w, d2f_fast(w), &l, &fb))
      S.l2B[b] = l;
    else
      ls_defer(S, 1, -(b + 1), i);
  }
}

// The deferred line searches of one limiter pass (pass 0: from U^L with P = A / (kappa_i m_i), written to
// l1; pass 1: from U^(1) with P = (1 - l1_ij) A / (kappa_i m_i), written to l2).  One thread per queued
// entry, grid-stride over the queue: every lane runs a bracketed iteration.  The row context, l_rho and
// psi(l_rho) are recomputed from the same stored values by the same code as in the queuing kernel.
template <int DIM>
__global__ void __launch_bounds__(128) k_lsfix(Dev D, Scratch S, int pass) {
  constexpr int M = DIM + 2;
  const unsigned count = S.lsq_n[pass];
  const size_t n = D.n, nnz = D.nnz, nb = D.nb;
  for (unsigned k = blockIdx.x * blockDim.x + threadIdx.x; k < count; k += gridDim.x * blockDim.x) {
    const int2 it = S.lsq[k];
    const int i = it.y;
    const bool bnd = it.x < 0;
    const int e = bnd ? -(it.x + 1) : it.x;
    double U0[M], A[M];
    const double* Usrc = pass == 0 ? S.UL : S.U1;
#pragma unroll
    for (int q = 0; q < M; ++q) {
      U0[q] = Usrc[q * n + i];
      A[q] = bnd ? S.AB[q * nb + e] : S.A[q * nnz + e];
    }
    double w = D.inv_km[i];
    if (pass == 1) w = (1.0 - (bnd ? S.l1B[e] : pmin(S.l1[e], S.l1[D.tr[e]]))) * w;
    LsRow<DIM> ls;
    ls_row<DIM>(D, ls, U0, S.bounds[i], S.bounds[n + i], S.bounds[2 * n + i]);
    double l, fb;
    if (!line_search_head<DIM>(D, ls, A, w, d2f_fast(w), &l, &fb)) l = line_search_tail<DIM>(D, ls, A, w, l, fb);
    double* dst = pass == 0 ? (bnd ? S.l1B : S.l1) : (bnd ? S.l2B : S.l2);
    dst[e] = l;
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
    double w = pmin(S.l2[e], S.l2[t]) * (1.0 - pmin(S.l1[e], S.l1[t]));
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

template <int DIM>
cudaError_t lsfix_impl(const Dev& D, const Scratch& S, int pass, cudaStream_t s) {
  if (D.n == 0) return cudaSuccess;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // the queue length is only known on the device: a grid of 4 blocks per SM strides over it
  const long long cap = ((long long)D.nnz + D.nb + 127) / 128;
  const int blocks = (int)std::max(1LL, std::min<long long>(4LL * std::max(1, sms), cap));
  k_lsfix<DIM><<<blocks, 128, 0, s>>>(D, S, pass);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_lsfix(int dim, const Dev& D, const Scratch& S, int pass, cudaStream_t s) {
  GDG_DISPATCH(dim, lsfix_impl, D, S, pass, s);
}

cudaError_t launch_limit2(int dim, const Dev& D, const Scratch& S, const double* Ubase, double alpha, double* Uout,
                          cudaStream_t s) {
  GDG_DISPATCH(dim, limit2_impl, D, S, Ubase, alpha, Uout, s);
}

cudaError_t launch_final(int dim, const Dev& D, const Scratch& S, const double* Ubase, double alpha, double* Uout,
                         cudaStream_t s) {
  GDG_DISPATCH(dim, final_impl, D, S, Ubase, alpha, Uout, s);
}

}  // namespace gdg
