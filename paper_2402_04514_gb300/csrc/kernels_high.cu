// Sweep B: high-order update with the consistent element mass, relaxed local bounds, antidiffusive
// fluxes and the first convex-limiting pass.  One thread per node; a block holds whole elements so the
// element solve and the m_ij coupling of A_ij stay in shared memory.
#include "gdg_internal.cuh"

namespace gdg {

namespace {

constexpr int kMaxBlock = kHighMaxBlock;

// Per node i of the block:
//  1. d_ij^H = max(d^min, d^ev) (Sec. 5, eq. (HighOrderViscosity); Sec. 5.1, eq. (ViscMin); Sec. 5.2),
//     the boundary d^{d,H} = max(c_k h_i^{p_k}, min(c_ev |N_i|, 1)) d^{d,L} (ghost node read as
//     collocated with x_i), and the high-order right-hand side
//       RHS^H_i = RHS^L_i - sum_j (d^H_ij - d^L_ij)(U_j - U_i) - sum_k (d^{d,H} - d^{d,L})(U^{d,k} - U_i);
//  2. the element solve of Sec. 5, eq. (HighScheme): dU^H_K = -tau M_K^{-1} RHS^H_K;
//  3. the relaxed bounds of Sec. 5.4, eq. (eq:local_bounds), from the one-hop aggregates of i and of
//     its stencil neighbours and node i's own boundary bar states;
//  4. A_ij = tau (d^H_ij - d^L_ij)(U_j - U_i) - m_ij (dU^H_j - dU^H_i) and
//     A_i^{d,k} = tau (d^{d,H} - d^{d,L})(U^{d,k} - U_i) (Sec. 5.3, eq. (HighLowOrderIdentity)), and the
//     pass-1 line search of Sec. 5.4, eq. (ConvexScheme), from U^L with P = A / (kappa_i m_i); the rare
//     searches that need the bracketed iteration are queued for k_lsfix.
// With order HIGH the kernel stops after 2 and writes U_out = alpha U_base + (1 - alpha)(U + dU^H).
template <int DIM, class Src>
__global__ void __launch_bounds__(kMaxBlock, 3) k_high(Src src, int nodes_per_block) {
  constexpr int M = DIM + 2;
  __shared__ double sR[M][kMaxBlock];
  __shared__ double sdU[M][kMaxBlock];
  __shared__ Ctx sctx;
  int lb;
  const Ctx& c = src.get(&sctx, &lb);
  if (finished(c)) return;
  const Dev& D = c.D;
  const Scratch& S = c.S;
  const double* U = c.U;
  const double* bdata = c.bdata;
  const int t = threadIdx.x;
  const int i = lb * nodes_per_block + t;
  const bool valid = t < nodes_per_block && i < D.n;
  const size_t n = D.n;
  const double tau = stage_tau(c);
  double Ui[M], dUi[M];
  double Ni = 0.0;
  if (valid) {
    load_state<DIM>(U, D.n, i, Ui);
    Ni = abs_bits(S.N[i]);
    double rhs[M];
#pragma unroll
    for (int q = 0; q < M; ++q) rhs[q] = S.RHSL[(size_t)q * n + i];
    // min / max of non-negative values and the m_ij-only test on the integer pipe
    for (int e = D.row_ptr[i]; e < D.row_ptr[i + 1]; ++e) {
      if (is_zero_bits(D.cnorm[e])) continue;  // m_ij-only entry: not in I(i)
      const double dl = S.dL[e];
      const int j = D.col[e];
      const double dev = dl * pmin(D.c_ev * pmax(Ni, abs_bits(S.N[j])), 1.0);
      const double dd = pmax(D.mu[e] * dl, dev) - dl;
      const double td = tau * dd;
#pragma unroll
      for (int q = 0; q < M; ++q) {
        const double du = U[(size_t)q * n + j] - Ui[q];
        rhs[q] = fma(-dd, du, rhs[q]);
        S.A[(size_t)q * D.nnz + e] = td * du;  // viscous part of A_ij, completed below
      }
    }
    for (int b = D.b_ptr[i]; b < D.b_ptr[i + 1]; ++b) {
      double nv[DIM], UB[M];
#pragma unroll
      for (int k = 0; k < DIM; ++k) nv[k] = D.bn[(size_t)k * D.nb + b];
      boundary_state<DIM>(D, b, Ui, bdata, nv, UB);
      double dl = S.dB[b];
      double dd = (pmax(D.muB[i], pmin(D.c_ev * Ni, 1.0)) - 1.0) * dl;
#pragma unroll
      for (int q = 0; q < M; ++q) {
        rhs[q] -= dd * (UB[q] - Ui[q]);
        S.AB[(size_t)q * D.nb + b] = tau * dd * (UB[q] - Ui[q]);
      }
    }
#pragma unroll
    for (int q = 0; q < M; ++q) sR[q][t] = rhs[q];
  }
  __syncthreads();
  if (valid) {
    const int nl = D.n_loc;
    const int il = i % nl;
    const int t0 = t - il;  // first node of the element in the block
    const double* Minv = D.MKinv + ((size_t)(i / nl) * nl + il) * nl;
    double acc[M];
#pragma unroll
    for (int q = 0; q < M; ++q) acc[q] = 0.0;
    for (int l = 0; l < nl; ++l) {
      double w = Minv[l];
#pragma unroll
      for (int q = 0; q < M; ++q) acc[q] += w * sR[q][t0 + l];
    }
#pragma unroll
    for (int q = 0; q < M; ++q) {
      dUi[q] = -tau * acc[q];
      sdU[q][t] = dUi[q];
    }
    if (D.order == GDG_ORDER_HIGH) {
#pragma unroll
      for (int q = 0; q < M; ++q) {
        c.Uout[(size_t)q * n + i] = rk_out(c, (size_t)q * n + i, Ui[q] + dUi[q]);
      }
    }
  }
  if (D.order == GDG_ORDER_HIGH) return;
  __syncthreads();
  if (!valid) return;
  // relaxed local bounds
  double lo = S.agg[i], hi = S.agg[n + i], sl = S.agg[2 * n + i];
  for (int b = D.b_ptr[i]; b < D.b_ptr[i + 1]; ++b) {
    lo = pmin(lo, S.bbar[b]);
    hi = pmax(hi, S.bbar[b]);
    sl = pmin(sl, S.bbar[(size_t)D.nb + b]);
  }
  for (int e = D.row_ptr[i]; e < D.row_ptr[i + 1]; ++e) {
    if (is_zero_bits(D.cnorm[e])) continue;
    int j = D.col[e];
    lo = pmin(lo, S.agg[j]);
    hi = pmax(hi, S.agg[n + j]);
    sl = pmin(sl, S.agg[2 * n + j]);
  }
  double rmin, rmax, smin;
  if (D.bounds_mode == 0) {
    rmin = D.rminus[i] * lo;
    rmax = D.rplus[i] * hi;
    smin = D.rminus[i] * sl;
  } else {
    rmin = 0.0;
    rmax = INFINITY;
    smin = 0.0;
  }
  S.bounds[i] = rmin;
  S.bounds[n + i] = rmax;
  S.bounds[2 * n + i] = smin;
  // antidiffusive fluxes and pass-1 line search
  double UL[M];
#pragma unroll
  for (int q = 0; q < M; ++q) UL[q] = S.UL[(size_t)q * n + i];
  LsRow<DIM> ls;
  ls_row<DIM>(D, ls, UL, rmin, rmax, smin);
  const double ikm = D.inv_km[i];
  const float ikmf = d2f_fast(ikm);
  const int nl = D.n_loc;
  const int elem = i / nl;
  const int t0 = t - (i % nl);
  for (int e = D.row_ptr[i]; e < D.row_ptr[i + 1]; ++e) {
    int j = D.col[e];
    double A[M];
    const bool stencil = !is_zero_bits(D.cnorm[e]);
    const bool same = (j / nl) == elem;
    const double mij = same ? D.mij[e] : 0.0;
    const int tj = t0 + (j % nl);
#pragma unroll
    for (int q = 0; q < M; ++q) {
      double a = stencil ? S.A[(size_t)q * D.nnz + e] : 0.0;
      if (same) a = fma(-mij, sdU[q][tj] - dUi[q], a);
      A[q] = a;
      S.A[(size_t)q * D.nnz + e] = a;
    }
    double l, fb;
    if (line_search_head<DIM>(D, ls, A, ikm, ikmf, &l, &fb))
      S.l1[e] = l;
    else
      ls_defer(S, 0, e, i);
  }
  for (int b = D.b_ptr[i]; b < D.b_ptr[i + 1]; ++b) {
    double A[M];
#pragma unroll
    for (int q = 0; q < M; ++q) A[q] = S.AB[(size_t)q * D.nb + b];
    double l, fb;
    if (line_search_head<DIM>(D, ls, A, ikm, ikmf, &l, &fb))
      S.l1B[b] = l;
    else
      ls_defer(S, 0, -(b + 1), i);
  }
}

template <int DIM, class Src>
cudaError_t high_launch(const Src& src, long long blocks, int npb, cudaStream_t s) {
  if (blocks <= 0) return cudaSuccess;
  if (npb < 1 || npb > kMaxBlock) return cudaErrorInvalidValue;
  k_high<DIM, Src><<<(unsigned)blocks, high_threads(npb), 0, s>>>(src, npb);
  return cudaGetLastError();
}

}  // namespace

// npb: nodes per block, whole elements (all instances of a batch share n_loc, hence the block shape).
cudaError_t launch_high_file(int dim, const Ctx& c, long long blocks, int npb, cudaStream_t s) {
  const One src{c};
  switch (dim) {
    case 1: return high_launch<1, One>(src, blocks, npb, s);
    case 2: return high_launch<2, One>(src, blocks, npb, s);
    case 3: return high_launch<3, One>(src, blocks, npb, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_high_file_many(int dim, const Many& m, long long blocks, int npb, cudaStream_t s) {
  switch (dim) {
    case 1: return high_launch<1, Many>(m, blocks, npb, s);
    case 2: return high_launch<2, Many>(m, blocks, npb, s);
    case 3: return high_launch<3, Many>(m, blocks, npb, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace gdg
