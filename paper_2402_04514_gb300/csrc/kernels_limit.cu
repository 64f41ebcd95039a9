// Sweeps C and D: symmetrisation of the limiter coefficients, the limited updates of Sec. 5.3,
// eq. (LimitedScheme), and the second limiter pass of Sec. 6.1.  One thread per row.
#include "gdg_internal.cuh"

namespace gdg {

namespace {

constexpr int kLimThreads = kRowMaxThreads;  // launch bound; the schedule launches 128, 256 or 512

// Sweep C: l_ij = min(l_ij^(i), l_ji^(j)) (Lemma ConsInvariants needs l_ij = l_ji);
// U^(1)_i = U^L_i + (sum_j l_ij A_ij + sum_k l_i^k A_i^k) / m_i; then the second pass limits the
// remainder (1 - l) A from U^(1) against the same bounds.  With one pass it writes U_out from U^(1).
// Capped at 72 registers (seven 128-thread blocks per SM; a few bytes of spills in the search): the row
// sums, which every row runs, need far fewer, and the searches of the rare rows with a remainder would
// otherwise set the kernel's occupancy.
template <int DIM, class Src>
__device__ __forceinline__ void limit2_body(const Src& src, int sliced, int last) {
  constexpr int M = DIM + 2;
  __shared__ Ctx sctx;
  int lb;
  const Ctx& c = src.get(&sctx, &lb);
  if (finished(c)) return;
  const Dev& D = c.D;
  const Scratch& S = c.S;
  const int i = row_node(D, lb * blockDim.x + threadIdx.x, sliced && !(last && c.Uhost));
  if (i < 0) return;
  const size_t n = D.n, nnz = D.nnz, nb = D.nb;
  double acc[M];
#pragma unroll
  for (int q = 0; q < M; ++q) acc[q] = 0.0;
  const int r0 = D.rbeg[i], r1 = D.rend[i];
  bool remainder = false;  // some entry has l1 < 1, so that pass 2 has a remainder to limit
  for (int e = r0; e < r1; e += kEll) {
    double l = pmin(S.l1[e], S.l1[D.tr[e]]);  // limiter coefficients are in [0, 1]: integer min
    remainder |= !is_one_bits(l);
#pragma unroll
    for (int q = 0; q < M; ++q) acc[q] += l * S.A[q * nnz + e];
  }
  for (int b = D.b_ptr[i]; b < D.b_ptr[i + 1]; ++b) {
    double l = S.l1B[b];
    remainder |= !is_one_bits(l);
#pragma unroll
    for (int q = 0; q < M; ++q) acc[q] += l * S.AB[q * nb + b];
  }
  const double inv_mi = D.inv_mi[i];
  double U1[M];
#pragma unroll
  for (int q = 0; q < M; ++q) U1[q] = S.UL[q * n + i] + acc[q] * inv_mi;
  if (last) {
#pragma unroll
    for (int q = 0; q < M; ++q) store_out(c, q * n + i, rk_out(c, q * n + i, U1[q]));
    return;
  }
#pragma unroll
  for (int q = 0; q < M; ++q) S.U1[q * n + i] = U1[q];
  S.rem[i] = remainder;
  // l2 is computed only where it multiplies a nonzero remainder (1 - l1)A: k_final reads no other, and a
  // row without a remainder (the flag above) takes no row context and no search
  if (!remainder) return;
  LsRow<DIM> ls;
  ls_row<DIM>(D, ls, U1, S.bounds[i], S.bounds[n + i], S.bounds[2 * n + i]);
  const double ikm = D.inv_km[i];
  for (int e = r0; e < r1; e += kEll) {
    const double l1s = pmin(S.l1[e], S.l1[D.tr[e]]);
    if (is_one_bits(l1s)) continue;
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
    if (is_one_bits(S.l1B[b])) continue;
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

template <int DIM, class Src>
__global__ void __maxnreg__(72) k_limit2(Src src, int sliced, int last) {
  limit2_body<DIM, Src>(src, sliced, last);
}

// The deferred line searches of one limiter pass (pass 0: from U^L with P = A / (kappa_i m_i), written to
// l1; pass 1: from U^(1) with P = (1 - l1_ij) A / (kappa_i m_i), written to l2).  One thread per queued
// entry, grid-stride over the queue: every lane runs a bracketed iteration.  The row context, l_rho and
// psi(l_rho) are recomputed from the same stored values by the same code as in the queuing kernel.
template <int DIM, class Src>
__device__ __forceinline__ void lsfix_body(const Src& src, int pass) {
  constexpr int M = DIM + 2;
  __shared__ Ctx sctx;
  int lb, blocks_per_inst;
  if ((unsigned)src.queue_length(pass, &lb) <= (unsigned)lb * blockDim.x) return;  // a block with no item
  const Ctx& c = src.get(&sctx, &lb, &blocks_per_inst);
  if (finished(c)) return;
  const Dev& D = c.D;
  const Scratch& S = c.S;
  const unsigned count = S.lsq_n[pass];
  const size_t n = D.n, nnz = D.nnz, nb = D.nb;
  const unsigned stride = (unsigned)blocks_per_inst * blockDim.x;
  for (unsigned k = lb * blockDim.x + threadIdx.x; k < count; k += stride) {
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

template <int DIM, class Src>
__global__ void __launch_bounds__(kLsfixThreads) k_lsfix(Src src, int pass) {
  lsfix_body<DIM, Src>(src, pass);
}

// Sweep D: U^(2)_i = U^(1)_i + (sum_j l2_ij (1 - l1_ij) A_ij + sum_k l2_i^k (1 - l1_i^k) A_i^k) / m_i,
// symmetrised as in sweep C, and U_out = alpha U_base + (1 - alpha) U^(2).  A writer of the step's host
// output (c.Uhost) takes its rows in node order whatever the schedule says, so that each warp's stores
// over the host link are contiguous (sweep C with one pass and the low-order sweep likewise).
template <int DIM, class Src>
__device__ __forceinline__ void final_body(const Src& src, int sliced) {
  constexpr int M = DIM + 2;
  __shared__ Ctx sctx;
  int lb;
  const Ctx& c = src.get(&sctx, &lb);
  if (finished(c)) return;
  const Dev& D = c.D;
  const Scratch& S = c.S;
  const int i = row_node(D, lb * blockDim.x + threadIdx.x, sliced && !c.Uhost);
  if (i < 0) return;
  const size_t n = D.n, nnz = D.nnz, nb = D.nb;
  if (!S.rem[i]) {  // no remainder in the row: U^(2)_i = U^(1)_i
#pragma unroll
    for (int q = 0; q < M; ++q) store_out(c, q * n + i, rk_out(c, q * n + i, S.U1[q * n + i]));
    return;
  }
  double acc[M];
#pragma unroll
  for (int q = 0; q < M; ++q) acc[q] = 0.0;
  // an entry with l1 = 1 has no remainder (its weight is 0): skipped, with the loads of its A
  for (int e = D.rbeg[i], e1 = D.rend[i]; e < e1; e += kEll) {
    int t = D.tr[e];
    const double l1s = pmin(S.l1[e], S.l1[t]);
    if (is_one_bits(l1s)) continue;
    double w = pmin(S.l2[e], S.l2[t]) * (1.0 - l1s);
#pragma unroll
    for (int q = 0; q < M; ++q) acc[q] += w * S.A[q * nnz + e];
  }
  for (int b = D.b_ptr[i]; b < D.b_ptr[i + 1]; ++b) {
    if (is_one_bits(S.l1B[b])) continue;
    double w = S.l2B[b] * (1.0 - S.l1B[b]);
#pragma unroll
    for (int q = 0; q < M; ++q) acc[q] += w * S.AB[q * nb + b];
  }
  const double inv_mi = D.inv_mi[i];
#pragma unroll
  for (int q = 0; q < M; ++q) store_out(c, q * n + i, rk_out(c, q * n + i, S.U1[q * n + i] + acc[q] * inv_mi));
}

template <int DIM, class Src>
__global__ void __launch_bounds__(kLimThreads) k_final(Src src, int sliced) {
  final_body<DIM, Src>(src, sliced);
}

// End of a fused step for one instance's clock: t += dt of the step (the dt every kernel of the step
// used), the step is counted, and the bound is reset for the next step.  Steps taken after t reached
// t_end are no-ops and are not counted.
__device__ __forceinline__ void clock_advance(Clock* k, double dt_factor) {
  if (!(k->t < k->t_end)) {  // finished before this step: the step did nothing and is not counted
    k->tau = 0.0;
    k->tau_bits = kTauNone;
    return;
  }
  bool clipped;
  const double dt = clock_dt(k, dt_factor, &clipped);
  if (k->tau_bits == kTauNone) clipped = k->t_end < INFINITY;  // no viscosity anywhere: nothing evolves
  k->tau = dt;
  k->t = clipped ? k->t_end : k->t + dt;  // a step clipped to t_end lands on it exactly
  k->steps += 1;
  k->tau_bits = kTauNone;
}

__global__ void k_clock_one(Clock* k, double dt_factor) {
  if (threadIdx.x == 0 && blockIdx.x == 0) clock_advance(k, dt_factor);
}

__global__ void k_clock_many(const Ctx* ctx, int ninst) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < ninst) clock_advance(ctx[k].clk, ctx[k].dt_factor);
}

// U_out = alpha U_base + (1 - alpha) U_in at every node and component (alpha = 0: a copy): the linear
// stage combinations of a Runge-Kutta step that involve no forward-Euler evaluation.
template <int DIM, class Src>
__device__ __forceinline__ void axpy_body(const Src& src) {
  constexpr int M = DIM + 2;
  __shared__ Ctx sctx;
  int lb;
  const Ctx& c = src.get(&sctx, &lb);
  if (finished(c)) return;
  const int i = lb * blockDim.x + threadIdx.x;
  if (i >= c.D.n) return;
  const size_t n = c.D.n;
  const double alpha = c.alpha;
#pragma unroll
  for (int q = 0; q < M; ++q) {
    const size_t idx = (size_t)q * n + i;
    c.Uout[idx] = alpha != 0.0 ? fma(1.0 - alpha, c.U[idx], sf::mul(alpha, c.Ubase[idx])) : c.U[idx];
  }
}

template <int DIM, class Src>
__global__ void __launch_bounds__(kLimThreads) k_axpy(Src src) {
  axpy_body<DIM, Src>(src);
}

template <int DIM, class Src>
cudaError_t limit_launch(int kern, const Src& src, long long blocks, int threads, int sliced, int arg,
                         cudaStream_t s) {
  if (blocks <= 0) return cudaSuccess;
  if (threads < 32 || threads > kLimThreads || threads % 32) return cudaErrorInvalidValue;
  const unsigned g = (unsigned)blocks;
  switch (kern) {
    case KN_LIMIT2: k_limit2<DIM, Src><<<g, threads, 0, s>>>(src, sliced, arg); break;
    case KN_FINAL: k_final<DIM, Src><<<g, threads, 0, s>>>(src, sliced); break;
    case KN_AXPY: k_axpy<DIM, Src><<<g, threads, 0, s>>>(src); break;
    case KN_LSFIX: k_lsfix<DIM, Src><<<g, kLsfixThreads, 0, s>>>(src, arg); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace

#ifndef GDG_BODIES_ONLY  // (a file that includes this one for its kernel bodies defines it)
cudaError_t launch_limit_file(int kern, int dim, const Ctx& c, long long blocks, int threads, int sliced, int arg,
                              cudaStream_t s) {
  const One src{c};
  switch (dim) {
    case 1: return limit_launch<1, One>(kern, src, blocks, threads, sliced, arg, s);
    case 2: return limit_launch<2, One>(kern, src, blocks, threads, sliced, arg, s);
    case 3: return limit_launch<3, One>(kern, src, blocks, threads, sliced, arg, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_limit_file_many(int kern, int dim, const Many& m, long long blocks, int threads, int sliced,
                                   int arg, cudaStream_t s) {
  switch (dim) {
    case 1: return limit_launch<1, Many>(kern, m, blocks, threads, sliced, arg, s);
    case 2: return limit_launch<2, Many>(kern, m, blocks, threads, sliced, arg, s);
    case 3: return limit_launch<3, Many>(kern, m, blocks, threads, sliced, arg, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_clock_one(Clock* clk, double dt_factor, cudaStream_t s) {
  k_clock_one<<<1, 32, 0, s>>>(clk, dt_factor);
  return cudaGetLastError();
}

cudaError_t launch_clock_many(const Ctx* ctx, int ninst, cudaStream_t s) {
  if (ninst <= 0) return cudaSuccess;
  k_clock_many<<<(ninst + 127) / 128, 128, 0, s>>>(ctx, ninst);
  return cudaGetLastError();
}

#endif  // GDG_BODIES_ONLY

}  // namespace gdg
