// Sweep B: high-order update with the consistent element mass, relaxed local bounds, antidiffusive
// fluxes and the first convex-limiting pass.  One thread per node; a block holds whole elements so the
// element solve and the m_ij coupling of A_ij stay in shared memory.
#include <type_traits>

#include "gdg_internal.cuh"

namespace gdg {

namespace {

constexpr int kMaxBlock = kHighMaxBlock;
constexpr int kMaxLocal = 32;  // n_loc limit of gdg_setup

// Thread-to-node map of an element block.  A block holds eb elements (a power of two <= kEll) of one
// ELL group of kEll consecutive elements: block lb of an instance takes group g = lb / (kEll / eb) and its
// elements e0 .. e0 + eb - 1 with e0 = (lb % (kEll / eb)) eb.  Thread t takes local index t / eb of
// element e0 + t % eb, so the lanes of a warp hold one local index of consecutive elements: rows of one
// shape (equal trip counts through the row loops) whose entries lie side by side in the ELL slices.
struct ElemSlot {
  int i;      // the node, valid only if ok
  int el, l;  // the element's place in the block and the node's local index
  bool ok;
};
__device__ __forceinline__ ElemSlot element_slot(const Dev& D, int lb, int eb) {
  const int per_group = kEll / eb;
  const int g = lb / per_group;
  const int t = threadIdx.x;
  ElemSlot r;
  r.l = t / eb;
  r.el = t - r.l * eb;
  const int E = g * kEll + (lb - g * per_group) * eb + r.el;
  r.ok = r.l < D.n_loc && E < D.nel;
  r.i = E * D.n_loc + r.l;
  return r;
}

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
// The mixed path (MX) runs steps 1, 2 and the A_ij of step 4 in FP32 (the differences U_j - U_i in FP64
// first); the bounds and the line search stay FP64.
template <int DIM, bool MX, class Src>
__device__ __forceinline__ void high_sweep(const Src& src, int eb) {
  constexpr int M = DIM + 2;
  constexpr int kShared = kMaxBlock + kEll;        // room for one pad slot per element
  using R = std::conditional_t<MX, float, double>;  // arithmetic of steps 1, 2 and the A_ij of step 4
  __shared__ R sR[M][kShared];
  __shared__ R sdU[M][kShared];
  __shared__ Ctx sctx;
  int lb;
  const Ctx& c = src.get(&sctx, &lb);
  if (finished(c)) return;
  const Dev& D = c.D;
  const Scratch& S = c.S;
  const double* U = c.U;
  const double* bdata = c.bdata;
  const ElemSlot es = element_slot(D, lb, eb);
  const int i = es.i;
  const bool valid = es.ok;
  // the shared arrays space elements n_loc + 1 apart for even n_loc: the lanes of a warp read one node of
  // each of consecutive elements, and an even stride would put pairs of them in the same bank
  const int stride_sh = D.n_loc + !(D.n_loc & 1);
  const int t0 = es.el * stride_sh;  // the element's first slot in the shared arrays
  const int sh = t0 + es.l;
  const size_t n = D.n;
  const double tau = stage_tau(c);
  const R tau_r = MX ? R(to_f32(tau)) : R(tau);
  double Ui[M];
  R dUi[M];
  double Ni = 0.0;
  const bool lim = D.order != GDG_ORDER_HIGH;  // the limiter's steps 3 and 4 follow the solve
  double lo = 0.0, hi = 0.0, sl = 0.0;         // two-hop aggregates of node i (step 3)
  if (valid) {
    load_state<DIM>(U, D.n, i, Ui);
    Ni = abs_bits(S.N[i]);
    R rhs[M];
#pragma unroll
    for (int q = 0; q < M; ++q) {
      if constexpr (MX)
        rhs[q] = to_f32(S.RHSL[(size_t)q * n + i]);
      else
        rhs[q] = S.RHSL[(size_t)q * n + i];
    }
    // min / max of non-negative values on the integer pipe; every input of the loop is read-only in this
    // kernel, so its loads take the read-only path and may move ahead of the stores of A.  The same pass
    // over I(i) gathers the two-hop aggregates of the relaxed bounds (step 3).
    const int e1 = D.sten_end[i];
    if (lim) {
      lo = S.agg[i];
      hi = S.agg[n + i];
      sl = S.agg[2 * n + i];
    }
    // not unrolled: with its products on the integer pipe the loop body is large, and unrolled by 2 the
    // kernel stalled on instruction fetch (4.24 against 4.14 ms per launch at Q2 1024^2)
#pragma unroll 1
    for (int e = D.rbeg[i]; e < e1; e += kEll) {  // I(i)
      const int j = __ldg(D.col + e);
      const double dl64 = __ldg(S.dL + e), mu = __ldg(D.mu + e), Nj = abs_bits(__ldg(S.N + j));
      double Uj[M];
#pragma unroll
      for (int q = 0; q < M; ++q) Uj[q] = __ldg(U + (size_t)q * n + j);
      if (lim) {
        lo = pmin(lo, __ldg(S.agg + j));
        hi = pmax(hi, __ldg(S.agg + n + j));
        sl = pmin(sl, __ldg(S.agg + 2 * n + j));
      }
      if constexpr (MX) {
        // d^H - d^L from FP32 operands: every factor is symmetric in (i, j), so the same bits come out
        // of row j, and A_ji = -A_ij holds exactly
        const float dl = to_f32(dl64);
        const float dev = dl * fminf(D.c_ev_f * to_f32(pmax(Ni, Nj)), 1.f);
        const float dd = fmaxf(to_f32(mu) * dl, dev) - dl;
        const float td = tau_r * dd;
#pragma unroll
        for (int q = 0; q < M; ++q) {
          const float du = to_f32(Uj[q] - Ui[q]);
          rhs[q] = fmaf(-dd, du, rhs[q]);
          S.A[(size_t)q * D.nnz + e] = to_f64(td * du);  // viscous part of A_ij, completed below
        }
      } else {
        // products on the integer pipe (sf::mul, the same bits as the FP64 instruction)
        const double dl = dl64;
        const double dev = sf::mul(dl, pmin(sf::mul(D.c_ev, pmax(Ni, Nj)), 1.0));
        const double dd = pmax(sf::mul(mu, dl), dev) - dl;
        const double td = sf::mul(tau, dd);
#pragma unroll
        for (int q = 0; q < M; ++q) {
          const double du = Uj[q] - Ui[q];
          rhs[q] = fma(-dd, du, rhs[q]);
          S.A[(size_t)q * D.nnz + e] = sf::mul(td, du);  // viscous part of A_ij, completed below
        }
      }
    }
    for (int b = D.b_ptr[i]; b < D.b_ptr[i + 1]; ++b) {
      if (lim) {
        lo = pmin(lo, S.bbar[b]);
        hi = pmax(hi, S.bbar[b]);
        sl = pmin(sl, S.bbar[(size_t)D.nb + b]);
      }
      double nv[DIM], UB[M];
#pragma unroll
      for (int k = 0; k < DIM; ++k) nv[k] = D.bn[(size_t)k * D.nb + b];
      boundary_state<DIM>(D, b, Ui, bdata, nv, UB);
      double dl = S.dB[b];
      double dd = (pmax(D.muB[i], pmin(D.c_ev * Ni, 1.0)) - 1.0) * dl;
#pragma unroll
      for (int q = 0; q < M; ++q) {
        if constexpr (MX)
          rhs[q] -= to_f32(dd * (UB[q] - Ui[q]));
        else
          rhs[q] -= dd * (UB[q] - Ui[q]);
        S.AB[(size_t)q * D.nb + b] = tau * dd * (UB[q] - Ui[q]);
      }
    }
#pragma unroll
    for (int q = 0; q < M; ++q) sR[q][sh] = rhs[q];
    if (lim) {  // relaxed local bounds, read back after the solve
      double rmin = 0.0, rmax = INFINITY, smin = 0.0;
      if (D.bounds_mode == 0) {
        rmin = D.rminus[i] * lo;
        rmax = D.rplus[i] * hi;
        smin = D.rminus[i] * sl;
      }
      S.bounds[i] = rmin;
      S.bounds[n + i] = rmax;
      S.bounds[2 * n + i] = smin;
    }
  }
  __syncthreads();
  if (valid) {
    const int nl = D.n_loc;
    const int ei = div_nl(D, i);
    // row il of the element's M_K^{-1}, stored grouped like the entries: (E, a, b) at
    // ((E / kEll * n_loc + a) * n_loc + b) * kEll + E % kEll
    const double* Minv = D.MKinv + ((size_t)(ei / kEll) * nl + es.l) * nl * kEll + (ei % kEll);
    R acc[M];
#pragma unroll
    for (int q = 0; q < M; ++q) acc[q] = R(0);
    for (int l = 0; l < nl; ++l) {
      R w;
      if constexpr (MX)
        w = to_f32(Minv[(size_t)l * kEll]);
      else
        w = Minv[(size_t)l * kEll];
#pragma unroll
      for (int q = 0; q < M; ++q) acc[q] += w * sR[q][t0 + l];
    }
#pragma unroll
    for (int q = 0; q < M; ++q) {
      if constexpr (MX)
        dUi[q] = -tau_r * acc[q];
      else
        dUi[q] = -tau * acc[q];
      sdU[q][sh] = dUi[q];
    }
    if (D.order == GDG_ORDER_HIGH) {
#pragma unroll
      for (int q = 0; q < M; ++q) {
        double du;
        if constexpr (MX)
          du = to_f64(dUi[q]);
        else
          du = dUi[q];
        store_out(c, (size_t)q * n + i, rk_out(c, (size_t)q * n + i, Ui[q] + du));
      }
    }
  }
  if (D.order == GDG_ORDER_HIGH) return;
  __syncthreads();
  if (!valid) return;
  const double rmin = S.bounds[i], rmax = S.bounds[n + i], smin = S.bounds[2 * n + i];
  const int se = D.sten_end[i];
  // antidiffusive fluxes and pass-1 line search
  double UL[M];
#pragma unroll
  for (int q = 0; q < M; ++q) UL[q] = S.UL[(size_t)q * n + i];
  LsRow<DIM> ls;
  ls_row<DIM>(D, ls, UL, rmin, rmax, smin);
  const double ikm = D.inv_km[i];
  const float ikmf = d2f_fast(ikm);
  const int nl = D.n_loc;
  const int elem = div_nl(D, i);
  for (int e = D.rbeg[i], e1 = D.rend[i]; e < e1; e += kEll) {
    int j = D.col[e];
    double A[M];
    const bool stencil = e < se;
    const int ej = div_nl(D, j);
    const bool same = ej == elem;
    const int tj = t0 + (j - ej * nl);
    if constexpr (MX) {
      const float mij = same ? to_f32(D.mij[e]) : 0.f;
#pragma unroll
      for (int q = 0; q < M; ++q) {
        float a = stencil ? to_f32(S.A[(size_t)q * D.nnz + e]) : 0.f;
        if (same) a = fmaf(-mij, sdU[q][tj] - dUi[q], a);
        A[q] = to_f64(a);
        S.A[(size_t)q * D.nnz + e] = A[q];
      }
    } else {
      const double mij = same ? D.mij[e] : 0.0;
#pragma unroll
      for (int q = 0; q < M; ++q) {
        double a = stencil ? S.A[(size_t)q * D.nnz + e] : 0.0;
        if (same) a = fma(-mij, sdU[q][tj] - dUi[q], a);
        A[q] = a;
        S.A[(size_t)q * D.nnz + e] = a;
      }
    }
    // A = 0 (a uniform neighbourhood): the search's outcome is l = 1 exactly when the FP32 tests it
    // starts with pass, which here reduce to a density gap above and psi(0) > 0; then skip them
    unsigned long long abits = 0;
#pragma unroll
    for (int q = 0; q < M; ++q) abits |= (unsigned long long)__double_as_longlong(A[q]) << 1;
    if (abits == 0 && ls.dhi > 0.f && ls.psi0f > 0.f) {
      S.l1[e] = 1.0;
      continue;
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

// The element sweep of each path as its own kernel with its own register budget.  Both run fastest at 72
// registers (three 288-thread blocks per SM, a few spills): with the per-entry streams contiguous, the
// resident warps matter more than the spills (the mixed path took 3.97 ms per launch at 96 registers,
// 3.37 ms at 72, at 1024^2 Q2; with the integer-pipe products the FP64 path 4.36 ms at 64, 4.15 at 72).
template <int DIM, class Src>
__global__ void __maxnreg__(72) k_high(Src src, int eb) {
  high_sweep<DIM, false, Src>(src, eb);
}
template <int DIM, class Src>
__global__ void __maxnreg__(72) k_high_mixed(Src src, int eb) {
  high_sweep<DIM, true, Src>(src, eb);
}

// eb: elements per block, a power of two <= kEll with eb * n_loc <= kMaxBlock (one element may exceed
// no block: n_loc <= kMaxLocal); n_loc is the one of the instance (a batch shares it).
template <int DIM, bool MX, class Src>
cudaError_t high_launch(const Src& src, long long blocks, int n_loc, int eb, cudaStream_t s) {
  if (blocks <= 0) return cudaSuccess;
  if (eb < 1 || eb > kEll || (eb & (eb - 1)) || n_loc < 1 || n_loc > kMaxLocal || eb * n_loc > kMaxBlock)
    return cudaErrorInvalidValue;
  const int threads = high_threads(n_loc, eb);
  if constexpr (MX)
    k_high_mixed<DIM, Src><<<(unsigned)blocks, threads, 0, s>>>(src, eb);
  else
    k_high<DIM, Src><<<(unsigned)blocks, threads, 0, s>>>(src, eb);
  return cudaGetLastError();
}

template <class Src>
cudaError_t high_dispatch(int dim, bool mx, const Src& src, long long blocks, int n_loc, int eb, cudaStream_t s) {
  switch (dim * 2 + (mx ? 1 : 0)) {
    case 2: return high_launch<1, false, Src>(src, blocks, n_loc, eb, s);
    case 3: return high_launch<1, true, Src>(src, blocks, n_loc, eb, s);
    case 4: return high_launch<2, false, Src>(src, blocks, n_loc, eb, s);
    case 5: return high_launch<2, true, Src>(src, blocks, n_loc, eb, s);
    case 6: return high_launch<3, false, Src>(src, blocks, n_loc, eb, s);
    case 7: return high_launch<3, true, Src>(src, blocks, n_loc, eb, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

#ifndef GDG_BODIES_ONLY  // (a file that includes this one for its kernel bodies defines it)
// eb: elements per block (all instances of a batch share n_loc, hence the block shape).
cudaError_t launch_high_file(int dim, const Ctx& c, long long blocks, int eb, cudaStream_t s) {
  return high_dispatch(dim, c.D.mixed != 0, One{c}, blocks, c.D.n_loc, eb, s);
}

cudaError_t launch_high_file_many(int dim, bool mixed, const Many& m, int n_loc, long long blocks, int eb,
                                  cudaStream_t s) {
  return high_dispatch(dim, mixed, m, blocks, n_loc, eb, s);
}

#endif  // GDG_BODIES_ONLY

}  // namespace gdg
