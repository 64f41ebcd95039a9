// Low-order sweep: per-node primitives, the time-step reduction (Sec. 3.3, eq. (MaxCFLdt)) and the
// first stage sweep (low-order update, entropy-viscosity indicator, one-hop bound aggregates).
// Every kernel takes its context from a source (One: a single instance, Many: a batch; gdg_internal.cuh).
#include <type_traits>

#include "gdg_internal.cuh"

namespace gdg {

namespace {

constexpr int kThreads = kRowMaxThreads;  // launch bound; the schedule launches 128, 256 or 512

// Per-node primitives (Sec. 2.2): 1/rho, p, 1/p, a = sqrt(gamma p / rho), p^{-e}, the entropy function
// f(s) = exp(s / (gamma + 1)) of the entropy-viscosity indicator and s~ = rho^{-gamma} eps (Sec. 5.4).
// Flags a state outside the admissible set of eq. (AddSet).  Being the first kernel of every stage, it
// also empties the stage's deferred line-search queues.  The mixed path (MX) keeps 1/rho and p in FP64
// (the fluxes use them) and computes the rest in FP32.  With c.Ucopy set (the first stage of a step whose
// state comes from host memory, read here over the host link) it also stores the state it read there, for
// the later sweeps of the stage; when the instance's clock has finished, the step is a no-op and it also
// writes that state to c.Uhost, the step's host output, where the last stage's writers would have.
template <int DIM, bool MX, class Src>
__device__ __forceinline__ void prim_body(const Src& src) {
  __shared__ Ctx sctx;
  int lb;
  const Ctx& c = src.get(&sctx, &lb);
  const bool done = finished(c);
  if (done && !c.Ucopy) return;
  const Dev& D = c.D;
  const Scratch& S = c.S;
  const int i = lb * blockDim.x + threadIdx.x;
  if (i == 0 && !done) {
    S.lsq_n[0] = 0u;
    S.lsq_n[1] = 0u;
  }
  if (i >= D.n) return;
  double Ui[DIM + 2];
  load_state<DIM>(c.U, D.n, i, Ui);
  if (c.Ucopy) {
#pragma unroll
    for (int q = 0; q < DIM + 2; ++q) c.Ucopy[(size_t)q * D.n + i] = Ui[q];
    if (done) {
      if (c.Uhost)
#pragma unroll
        for (int q = 0; q < DIM + 2; ++q) c.Uhost[(size_t)q * D.n + i] = Ui[q];
      return;
    }
  }
  double irho = rcp64(Ui[0]);
  // products on the integer pipe (sf::mul, the same bits as the FP64 instruction) where no sum follows
  double m2 = sf::mul(Ui[1], Ui[1]);
#pragma unroll
  for (int k = 1; k < DIM; ++k) m2 = fma(Ui[1 + k], Ui[1 + k], m2);
  double eps = fma(-sf::mul_pow2(m2, -1), irho, Ui[DIM + 1]);
  if (!(Ui[0] > 0.0) || !(eps > 0.0)) atomicOr(S.flags, (unsigned)GDG_FLAG_INADMISSIBLE);
  double p = sf::mul(D.gm1, eps);
  double* P = S.prim;
  size_t n = D.n;
  if constexpr (MX) {
    const PrimF f = prim_mx(D, Ui[0], p);
    float st = powf(to_f32(Ui[0]), -D.gamma_f) * to_f32(eps);
    double st64 = to_f64(st);
    if (!finite_f32(st)) {  // rho^{-gamma} beyond the FP32 range
      double ir;
      st64 = rho_neg_gamma(D, Ui[0], &ir) * eps;
      st = to_f32(st64);
    }
    P[PR_IRHO * n + i] = irho;
    P[PR_P * n + i] = p;
    P[PR_IP * n + i] = to_f64(f.ip);
    P[PR_A * n + i] = to_f64(f.a);
    P[PR_PME * n + i] = to_f64(f.pme);
    P[PR_F * n + i] = to_f64(powf(2.f * D.gm1h_f * st, D.inv_gp1_f));
    P[PR_ST * n + i] = st64;
    return;
  }
  double ir;
  double st = sf::mul(rho_neg_gamma<false>(D, Ui[0], &ir), eps);
  P[PR_IRHO * n + i] = irho;
  P[PR_P * n + i] = p;
  P[PR_IP * n + i] = rcp64(p);
  P[PR_A * n + i] = sqrt64(sf::mul(sf::mul(D.gamma, p), irho));
  P[PR_PME * n + i] = D.ie_root > 0 ? rootinv(p, D.root_ie) : pow(p, -D.e_exp);
  // f = (gm1 s~)^{1/(gamma+1)} = x^{q/(p+q)} = x (x^{-1/(p+q)})^p for gamma = p/q
  double x = sf::mul(D.gm1, st);
  P[PR_F * n + i] =
      (D.gq > 0 && D.gp + D.gq <= 16) ? sf::mul(x, ipow(rootinv(x, D.root_gpq), D.gp)) : pow(x, D.inv_gp1);
  P[PR_ST * n + i] = st;
}

template <int DIM, bool MX, class Src>
__global__ void __launch_bounds__(kThreads) k_prim(Src src) {
  prim_body<DIM, MX, Src>(src);
}

// d_i^{d,k} = |c_i^{d,k}| lambda_max^+(U_i, U^{d,k}, n_i^k) of boundary entry b (Sec. 4.2,
// eq. (eq:dij_low_order_modified); interior state on the left), from node i's primitives.
template <int DIM, bool MX>
__device__ __forceinline__ double boundary_viscosity(const Dev& D, int b, const double* Ui, const double* bdata,
                                                     double irho_i, double p_i, double ip_i, double a_i,
                                                     double pme_i) {
  constexpr int M = DIM + 2;
  double nv[DIM], UB[M];
#pragma unroll
  for (int k = 0; k < DIM; ++k) nv[k] = D.bn[(size_t)k * D.nb + b];
  boundary_state<DIM>(D, b, Ui, bdata, nv, UB);
  double irB = 1.0 / UB[0];
  double pB = sf::mul(D.gm1, internal_energy<DIM>(UB));
  const double uL = dot<DIM>(Ui + 1, nv), uR = dot<DIM>(UB + 1, nv);
  double ipB, aB, pmeB;
  prim_of<MX>(D, UB[0], irB, pB, &ipB, &aB, &pmeB);
  return sf::mul(D.bnorm[b], lambda_pair<MX>(D, sf::mul(uL, irho_i), p_i, irho_i, ip_i, a_i, pme_i, sf::mul(uR, irB),
                                             pB, irB, ipB, aB, pmeB));
}

// Block minimum of val, then one 64-bit atomicMin per block on the bit pattern (positive doubles order
// like uint64).  Every thread of the block calls it.
__device__ __forceinline__ void block_min_to(double val, unsigned long long* dst) {
  __shared__ double red[kThreads / 32];
  for (int off = 16; off > 0; off >>= 1) val = fmin(val, __shfl_xor_sync(0xffffffffu, val, off));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = val;
  __syncthreads();
  if (threadIdx.x < 32) {
    val = threadIdx.x < blockDim.x / 32 ? red[threadIdx.x] : INFINITY;
    for (int off = 16; off > 0; off >>= 1) val = fmin(val, __shfl_xor_sync(0xffffffffu, val, off));
    if (threadIdx.x == 0 && val < INFINITY) atomicMin(dst, (unsigned long long)__double_as_longlong(val));
  }
}

// Sum over the row of d_ij^L plus the boundary viscosities, i.e. -d_ii of
// eq. (eq:dij_low_order_supplement), then min over nodes of m_i / (2 |d_ii|), with d_ij^L evaluated here
// (gdg_max_dt, before any stage).
template <int DIM, bool MX, class Src>
__device__ __forceinline__ void maxdt_body(const Src& src, int sliced) {
  constexpr int M = DIM + 2;
  __shared__ Ctx sctx;
  int lb;
  const Ctx& c = src.get(&sctx, &lb);
  if (finished(c)) return;
  const Dev& D = c.D;
  const Scratch& S = c.S;
  const double* U = c.U;
  const int i = row_node(D, lb * blockDim.x + threadIdx.x, sliced);
  double val = INFINITY;
  if (i >= 0) {
    size_t n = D.n;
    double Ui[M];
    load_state<DIM>(U, D.n, i, Ui);
    const double* P = S.prim;
    double irho_i = P[PR_IRHO * n + i], p_i = P[PR_P * n + i], ip_i = P[PR_IP * n + i], a_i = P[PR_A * n + i],
           pme_i = P[PR_PME * n + i];
    double dsum = 0.0;
    const int e1 = D.sten_end[i];
    for (int e = D.rbeg[i]; e < e1; e += kEll) {  // I(i)
      double cnm = D.cnorm[e];
      int j = D.col[e];
      double nv[DIM], mj[DIM];
#pragma unroll
      for (int k = 0; k < DIM; ++k) {
        nv[k] = D.cn[(size_t)k * D.nnz + e];
        mj[k] = U[(size_t)(1 + k) * n + j];
      }
      const double irho_j = P[PR_IRHO * n + j];
      const double uL = sf::mul(dot<DIM>(Ui + 1, nv), irho_i), uR = sf::mul(dot<DIM>(mj, nv), irho_j);
      dsum = fma(cnm, lambda_pair<MX>(D, uL, p_i, irho_i, ip_i, a_i, pme_i, uR, P[PR_P * n + j], irho_j,
                                      P[PR_IP * n + j], P[PR_A * n + j], P[PR_PME * n + j]), dsum);
    }
    for (int b = D.b_ptr[i]; b < D.b_ptr[i + 1]; ++b)
      dsum += boundary_viscosity<DIM, MX>(D, b, Ui, c.bdata, irho_i, p_i, ip_i, a_i, pme_i);
    if (dsum > 0.0) val = sf::mul(sf::mul_pow2(D.mi[i], -1), rcp64(dsum));
  }
  block_min_to(val, S.tau_bits);
}

template <int DIM, bool MX, class Src>
__global__ void __launch_bounds__(kThreads) k_maxdt(Src src, int sliced) {
  maxdt_body<DIM, MX, Src>(src, sliced);
}

// The same bound inside the fused SSP-RK3 step, after the edge sweep of the step's first stage: the row
// sums of the stored d_ij^L plus the boundary viscosities, reduced into the instance's clock.  Capped at
// 48 registers: the row sum, which every row runs, is latency-bound and wants many warps; the boundary
// viscosities of the few boundary rows would otherwise take 117 and spill at the cap.
template <int DIM, bool MX, class Src>
__device__ __forceinline__ void tau_body(const Src& src, int sliced) {
  constexpr int M = DIM + 2;
  __shared__ Ctx sctx;
  int lb;
  const Ctx& c = src.get(&sctx, &lb);
  if (finished(c)) return;
  const Dev& D = c.D;
  const Scratch& S = c.S;
  const int i = row_node(D, lb * blockDim.x + threadIdx.x, sliced);
  double val = INFINITY;
  if (i >= 0) {
    double dsum = 0.0;
    const int e0 = D.rbeg[i], e1 = D.sten_end[i];
#pragma unroll 4
    for (int e = e0; e < e1; e += kEll) dsum += __ldg(S.dL + e);  // loads issued ahead of the in-order sum
    const int b0 = D.b_ptr[i], b1 = D.b_ptr[i + 1];
    if (b0 < b1) {
      const size_t n = D.n;
      const double* P = S.prim;
      double Ui[M];
      load_state<DIM>(c.U, D.n, i, Ui);
      for (int b = b0; b < b1; ++b)
        dsum += boundary_viscosity<DIM, MX>(D, b, Ui, c.bdata, P[PR_IRHO * n + i], P[PR_P * n + i], P[PR_IP * n + i],
                                        P[PR_A * n + i], P[PR_PME * n + i]);
    }
    if (dsum > 0.0) val = sf::mul(sf::mul_pow2(D.mi[i], -1), rcp64(dsum));
  }
  block_min_to(val, &c.clk->tau_bits);
}

template <int DIM, bool MX, class Src>
__global__ void __maxnreg__(48) k_tau(Src src, int sliced) {
  tau_body<DIM, MX, Src>(src, sliced);
}

// Edge sweep, one thread per undirected stencil edge {i, j} (i < j): the quantities of a pair that are
// symmetric in i and j are computed once and written to both entries (i, j) and (j, i):
//  - d_ij^L = d_ji^L = |c_ij| lambda_max^+(U_i, U_j, n_ij) (Sec. 3.1, eq. (eq:dij_low_order); the bound
//    is symmetric under (U_i, U_j, n) -> (U_j, U_i, -n), which is also what makes d^L symmetric);
//  - the bar state Ubar_ij = Ubar_ji (eq. (UsualBarState)), of which only rho and s~ are kept (for the
//    local bounds of eq. (eq:local_bounds));
//  - G_ij = f(U_j) c_ij and G_ji = f(U_i) c_ji = -|c_ij| f(U_i) n_ij for the row sums of sweep A.
// The mixed path (MX) takes lambda from lambda_pair<true> and the entropy power of the bar state in FP32;
// the fluxes, G and the bar state itself stay FP64.
template <int DIM, bool MX, class Src>
__device__ __forceinline__ void edge_body(const Src& src) {
  constexpr int M = DIM + 2;
  __shared__ Ctx sctx;
  int lb;
  const Ctx& c = src.get(&sctx, &lb);
  if (finished(c)) return;
  const Dev& D = c.D;
  const Scratch& S = c.S;
  const int k = lb * blockDim.x + threadIdx.x;
  if (k >= D.ne) return;
  const size_t n = D.n, nnz = D.nnz;
  const int e = D.edge_e[k], i = D.edge_i[k];
  const int j = D.col[e], t = D.tr[e];
  const double* P = S.prim;
  double Ui[M], Uj[M], nv[DIM];
  load_state<DIM>(c.U, D.n, i, Ui);
  load_state<DIM>(c.U, D.n, j, Uj);
  const double cnm = D.cnorm[e];
  // products on the integer pipe (sf::mul, the same bits as the FP64 instruction) where no sum follows
#pragma unroll
  for (int q = 0; q < DIM; ++q) nv[q] = D.cn[(size_t)q * nnz + e];
  double mnL = sf::mul(Ui[1], nv[0]), mnR = sf::mul(Uj[1], nv[0]);
#pragma unroll
  for (int q = 1; q < DIM; ++q) {
    mnL = fma(Ui[1 + q], nv[q], mnL);
    mnR = fma(Uj[1 + q], nv[q], mnR);
  }
  const double p_i = P[PR_P * n + i], p_j = P[PR_P * n + j];
  const double ir_i = P[PR_IRHO * n + i], ir_j = P[PR_IRHO * n + j];
  const double uL = sf::mul(mnL, ir_i), uR = sf::mul(mnR, ir_j);
  const double lam = lambda_pair<MX>(D, uL, p_i, ir_i, P[PR_IP * n + i], P[PR_A * n + i], P[PR_PME * n + i], uR, p_j,
                                     ir_j, P[PR_IP * n + j], P[PR_A * n + j], P[PR_PME * n + j]);
  const double d = sf::mul(cnm, lam);
  S.dL[e] = d;
  S.dL[t] = d;
  // f(U) c_ij with c_ij = |c_ij| n_ij, from m.c = |c| m.n and v.c = |c| v.n
  double cv[DIM], gi[M], gj[M];
#pragma unroll
  for (int q = 0; q < DIM; ++q) cv[q] = sf::mul(cnm, nv[q]);
  flux_n<DIM>(Ui, cv, sf::mul(cnm, mnL), sf::mul(cnm, uL), p_i, gi);
  flux_n<DIM>(Uj, cv, sf::mul(cnm, mnR), sf::mul(cnm, uR), p_j, gj);
  // W = 2 Ubar = U_i + U_j - (f(U_j) - f(U_i)) c_ij / d_ij, halved where it is used
  const double r = MX ? to_f64(1.f / to_f32(d)) : rcp64(d);
  double W[M];
#pragma unroll
  for (int q = 0; q < M; ++q) {
    S.G[q * nnz + e] = gj[q];
    S.G[q * nnz + t] = -gi[q];
    W[q] = fma(-r, gj[q] - gi[q], Ui[q] + Uj[q]);
  }
  double Ub[M];
  Ub[0] = sf::mul_pow2(W[0], -1);
  Ub[DIM + 1] = sf::mul_pow2(W[DIM + 1], -1);
  double mw2 = sf::mul(W[1], W[1]), irb;  // |2 m(Ubar)|^2; 0.125 mw2 = |m(Ubar)|^2 / 2
#pragma unroll
  for (int q = 1; q < DIM; ++q) mw2 = fma(W[1 + q], W[1 + q], mw2);
  const double hm2 = sf::mul_pow2(mw2, -3);
  double stb;
  if constexpr (MX) {
    // eps(Ubar) in FP64 (E - |m|^2 / (2 rho) cancels at high Mach numbers) with 1/rho(Ubar) from one
    // Newton step on the FP32 reciprocal; rho(Ubar)^{-gamma} in FP32
    const float rbf = to_f32(Ub[0]);
    const double y = to_f64(1.f / rbf);
    irb = y * fma(-Ub[0], y, 2.0);
    const float rg = powf(rbf, -D.gamma_f);
    stb = to_f64(rg * to_f32(fma(-hm2, irb, Ub[DIM + 1])));
    if (!finite_f32(rg)) {
      const double rgb = rho_neg_gamma(D, Ub[0], &irb);
      stb = rgb * fma(-hm2, irb, Ub[DIM + 1]);
    }
  } else {
    const double rgb = rho_neg_gamma(D, Ub[0], &irb);  // sets irb = 1 / rho(Ubar) before its use below
    stb = sf::mul(rgb, fma(-hm2, irb, Ub[DIM + 1]));
  }
  S.barR[e] = Ub[0];
  S.barR[t] = Ub[0];
  S.barS[e] = stb;
  S.barS[t] = stb;
}

// Two 512-thread blocks per SM (64 registers, a few bytes of spills): the integer-pipe products of the
// sweep want resident warps to hide their latency (2.77 ms per launch at Q2 1024^2, against 3.04 with one
// block of 512 at 82 registers).
template <int DIM, bool MX, class Src>
__global__ void __launch_bounds__(kThreads, 2) k_edge(Src src) {
  edge_body<DIM, MX, Src>(src);
}

// Sweep A, one thread per row i, after the edge sweep:
//  - the row sums of d_ij^L and f(U_j) c_ij from the edge sweep; boundary states and viscosities (Sec. 4.1;
//    Sec. 4.2, eq. (eq:dij_low_order_modified));
//  - the low-order update of Sec. 4.2, eq. (cijdijschememodified), and the CFL check (CFLcond);
//  - the entropy-viscosity indicator N_i = R_i / D_i (Sec. 5.2);
//  - the one-hop aggregates of the local bounds (Sec. 5.4, eq. (eq:local_bounds)): min/max of rho_j,
//    rho(Ubar_jk), rho_k and min of s~ over node j's stencil, with the bar states of
//    eq. (UsualBarState); and rho, s~ of node i's boundary bar states (eq. (BoundaryBarState)).
// With order LOW (or no limiter pass) it also writes U_out = alpha U_base + (1 - alpha) U^L.
// The mixed path (MX) computes the indicator in FP32 (its sums from FP64 flux differences) and the
// boundary wave-speed bounds with lambda_pair<true>; the low-order update stays FP64.
template <int DIM, bool MX, class Src>
__device__ __forceinline__ void low_body(const Src& src, int sliced, int write_out) {
  constexpr int M = DIM + 2;
  __shared__ Ctx sctx;
  int lb;
  const Ctx& c = src.get(&sctx, &lb);
  if (finished(c)) return;
  const Dev& D = c.D;
  const Scratch& S = c.S;
  const double* U = c.U;
  const int i = row_node(D, lb * blockDim.x + threadIdx.x, sliced && !(write_out && c.Uhost));
  if (i < 0) return;
  const double tau = stage_tau(c);
  size_t n = D.n;
  const double* P = S.prim;
  double Ui[M];
  load_state<DIM>(U, D.n, i, Ui);
  const double irho_i = P[PR_IRHO * n + i], p_i = P[PR_P * n + i], ip_i = P[PR_IP * n + i],
               a_i = P[PR_A * n + i], pme_i = P[PR_PME * n + i], f_i = P[PR_F * n + i], st_i = P[PR_ST * n + i];
  using Acc = std::conditional_t<MX, float, double>;  // arithmetic of the indicator's sums
  // RHS^L = sum_j f(U_j) c_ij - sum_j d_ij (U_j - U_i) + boundary terms, accumulated as its two sums
  // (sg, sdu); the indicator's Fsum reuses sg
  double sg[M], sdu[M];
  Acc Fsum[M];
#pragma unroll
  for (int q = 0; q < M; ++q) {
    sg[q] = sdu[q] = 0.0;
    Fsum[q] = Acc(0);
  }
  Acc psum = Acc(0);
  double dsum = 0.0;
  double lo = Ui[0], hi = Ui[0], sl = st_i;
  const size_t nnz = D.nnz;
  const int e1 = D.sten_end[i];
  for (int e = D.rbeg[i]; e < e1; e += kEll) {  // I(i)
    const int j = D.col[e], t = D.tr[e];
    const double d = S.dL[e];
    dsum += d;
    double Uj[M];
    load_state<DIM>(U, D.n, j, Uj);
#pragma unroll
    for (int q = 0; q < M; ++q) {
      const double ge = S.G[q * nnz + e];
      sg[q] += ge;
      sdu[q] = fma(d, Uj[q] - Ui[q], sdu[q]);
      // Fsum = sum_j (f(U_j) - f(U_i)) c_ij: here the f(U_i) c_ij terms, sg is added after the loop (the
      // two sums are exact negatives of each other term by term on a stencil holding one state); the
      // mixed path sums the FP64 differences in FP32
      if constexpr (MX)
        Fsum[q] += to_f32(ge + S.G[q * nnz + t]);
      else
        Fsum[q] += S.G[q * nnz + t];
    }
    if constexpr (MX)
      psum += to_f32(S.G[e]) * (to_f32(P[PR_F * n + j]) - to_f32(f_i));
    else
      psum = fma(S.G[e], P[PR_F * n + j] - f_i, psum);  // (m_j . c_ij) (f_j - f_i)
    lo = pmin(lo, pmin(Uj[0], S.barR[e]));
    hi = pmax(hi, pmax(Uj[0], S.barR[e]));
    sl = pmin(sl, pmin(P[PR_ST * n + j], S.barS[e]));
  }
  if constexpr (!MX) {
#pragma unroll
    for (int q = 0; q < M; ++q) Fsum[q] += sg[q];
  }
  for (int b = D.b_ptr[i]; b < D.b_ptr[i + 1]; ++b) {
    double nv[DIM], UB[M];
#pragma unroll
    for (int k = 0; k < DIM; ++k) nv[k] = D.bn[(size_t)k * D.nb + b];
    boundary_state<DIM>(D, b, Ui, c.bdata, nv, UB);
    double irB = 1.0 / UB[0];
    double pB = sf::mul(D.gm1, internal_energy<DIM>(UB));
    const double mnL = dot<DIM>(Ui + 1, nv), mnR = dot<DIM>(UB + 1, nv);
    const double uL = sf::mul(mnL, irho_i), uR = sf::mul(mnR, irB);
    double cnm = D.bnorm[b];
    double ipB, aB, pmeB;
    prim_of<MX>(D, UB[0], irB, pB, &ipB, &aB, &pmeB);
    double d = sf::mul(cnm, lambda_pair<MX>(D, uL, p_i, irho_i, ip_i, a_i, pme_i, uR, pB, irB, ipB, aB, pmeB));
    S.dB[b] = d;
    dsum += d;
    double fi[M], fB[M];
    flux_n<DIM>(Ui, nv, mnL, uL, p_i, fi);
    flux_n<DIM>(UB, nv, mnR, uR, pB, fB);
    double t = cnm / sf::mul_pow2(d, 1);
    double Ub[M];
#pragma unroll
    for (int q = 0; q < M; ++q) {
      sg[q] = fma(cnm, fB[q], sg[q]);
      sdu[q] = fma(d, UB[q] - Ui[q], sdu[q]);
      if constexpr (MX)
        Fsum[q] -= to_f32(cnm * fi[q]);
      else
        Fsum[q] = fma(-cnm, fi[q], Fsum[q]);
      Ub[q] = fma(-t, fB[q] - fi[q], 0.5 * (Ui[q] + UB[q]));
    }
    S.bbar[b] = Ub[0];
    S.bbar[(size_t)D.nb + b] = sf::mul(pow(Ub[0], -D.gamma), internal_energy<DIM>(Ub));
  }
  const double inv_mi = D.inv_mi[i];
  if (sf::mul(sf::mul(sf::mul_pow2(tau, 1), dsum), inv_mi) > 1.0 + 1e-12) atomicOr(S.flags, (unsigned)GDG_FLAG_CFL);
  double rhs[M];
#pragma unroll
  for (int q = 0; q < M; ++q) rhs[q] = sg[q] - sdu[q];
  double UL[M];
#pragma unroll
  for (int q = 0; q < M; ++q) UL[q] = fma(-sf::mul(tau, inv_mi), rhs[q], Ui[q]);
  if (write_out) {
#pragma unroll
    for (int q = 0; q < M; ++q) store_out(c, (size_t)q * n + i, rk_out(c, (size_t)q * n + i, UL[q]));
    return;
  }
#pragma unroll
  for (int q = 0; q < M; ++q) {
    S.UL[(size_t)q * n + i] = UL[q];
    S.RHSL[(size_t)q * n + i] = rhs[q];
  }
  S.agg[i] = lo;
  S.agg[n + i] = hi;
  S.agg[2 * n + i] = sl;
  // entropy-viscosity indicator: Fsum_k = sum_j (f_k(U_j) - f_k(U_i)) c_ij - f_k(U_i) sum_k c_i^{d,k}, which
  // equals sum_j f_k(U_j) c_ij by the partition of unity (Lemma LemPart) and vanishes exactly on a
  // stencil holding one state; grad Phi_i = rho_i f'(s_i) grad_U s(U_i), f' = f / (gamma + 1),
  // grad_U s = grad_U p / p - (gamma / rho) e_rho, grad_U p = (gamma - 1)[|v|^2 / 2, -v, 1]
  if constexpr (MX) {
    const float irf = to_f32(irho_i), ipf = to_f32(ip_i), gm1 = 2.f * D.gm1h_f;
    const float pref = to_f32(f_i) * D.inv_gp1_f * to_f32(Ui[0]);
    float v[DIM], v2 = 0.f;
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
      v[k] = to_f32(Ui[1 + k]) * irf;
      v2 += v[k] * v[k];
    }
    float grad[M];
    grad[0] = pref * fmaf(D.gm1h_f * v2, ipf, -(D.gamma_f * irf));
#pragma unroll
    for (int k = 0; k < DIM; ++k) grad[1 + k] = pref * (-gm1 * v[k] * ipf);
    grad[DIM + 1] = pref * (gm1 * ipf);
    float R = psum, Dn = fabsf(psum);
#pragma unroll
    for (int q = 0; q < M; ++q) {
      R -= grad[q] * Fsum[q];
      Dn += fabsf(grad[q]) * fabsf(Fsum[q]);
    }
    S.N[i] = Dn > 0.f ? to_f64(R / Dn) : 0.0;
  } else {
    // rho f / (gamma + 1) from rho itself and 1/p from k_prim, so that no division is needed here
    const double pref = sf::mul(sf::mul(f_i, D.inv_gp1), Ui[0]);
    const double ip = ip_i;
    double vk[DIM];
#pragma unroll
    for (int k = 0; k < DIM; ++k) vk[k] = sf::mul(Ui[1 + k], irho_i);
    double v2 = sf::mul(vk[0], vk[0]);
#pragma unroll
    for (int k = 1; k < DIM; ++k) v2 = fma(vk[k], vk[k], v2);
    double grad[M];
    grad[0] = sf::mul(pref, fma(sf::mul(sf::mul(D.gm1, 0.5), v2), ip, -sf::mul(D.gamma, irho_i)));
#pragma unroll
    for (int k = 0; k < DIM; ++k) grad[1 + k] = sf::mul(pref, sf::mul(sf::mul(-D.gm1, vk[k]), ip));
    grad[DIM + 1] = sf::mul(pref, sf::mul(D.gm1, ip));
    double R = psum, Dn = fabs(psum);
#pragma unroll
    for (int q = 0; q < M; ++q) {
      R = fma(-grad[q], Fsum[q], R);
      Dn = fma(fabs(grad[q]), fabs(Fsum[q]), Dn);
    }
    S.N[i] = Dn > 0.0 ? sf::mul(R, rcp64(Dn)) : 0.0;
  }
}

template <int DIM, bool MX, class Src>
__global__ void __launch_bounds__(kThreads) k_low(Src src, int sliced, int write_out) {
  low_body<DIM, MX, Src>(src, sliced, write_out);
}

template <int DIM, bool MX, class Src>
cudaError_t low_launch(int kern, const Src& src, long long blocks, int threads, int sliced, int arg, cudaStream_t s) {
  if (blocks <= 0) return cudaSuccess;
  if (threads < 32 || threads > kThreads || threads % 32) return cudaErrorInvalidValue;
  const unsigned g = (unsigned)blocks;
  switch (kern) {
    case KN_PRIM: k_prim<DIM, MX, Src><<<g, threads, 0, s>>>(src); break;
    case KN_MAXDT: k_maxdt<DIM, MX, Src><<<g, threads, 0, s>>>(src, sliced); break;
    case KN_TAU: k_tau<DIM, MX, Src><<<g, threads, 0, s>>>(src, sliced); break;
    case KN_EDGE: k_edge<DIM, MX, Src><<<g, threads, 0, s>>>(src); break;
    case KN_LOW: k_low<DIM, MX, Src><<<g, threads, 0, s>>>(src, sliced, arg); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <class Src>
cudaError_t low_dispatch(int kern, int dim, bool mx, const Src& src, long long blocks, int threads, int sliced,
                         int arg, cudaStream_t s) {
  switch (dim * 2 + (mx ? 1 : 0)) {
    case 2: return low_launch<1, false, Src>(kern, src, blocks, threads, sliced, arg, s);
    case 3: return low_launch<1, true, Src>(kern, src, blocks, threads, sliced, arg, s);
    case 4: return low_launch<2, false, Src>(kern, src, blocks, threads, sliced, arg, s);
    case 5: return low_launch<2, true, Src>(kern, src, blocks, threads, sliced, arg, s);
    case 6: return low_launch<3, false, Src>(kern, src, blocks, threads, sliced, arg, s);
    case 7: return low_launch<3, true, Src>(kern, src, blocks, threads, sliced, arg, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

#ifndef GDG_BODIES_ONLY  // (a file that includes this one for its kernel bodies defines it)
// Launchers of this file's kernels, dispatched on the dimension and the precision (called by
// launch_kernel*).
cudaError_t launch_low_file(int kern, int dim, const Ctx& c, long long blocks, int threads, int sliced, int arg,
                            cudaStream_t s) {
  return low_dispatch(kern, dim, c.D.mixed != 0, One{c}, blocks, threads, sliced, arg, s);
}

cudaError_t launch_low_file_many(int kern, int dim, bool mixed, const Many& m, long long blocks, int threads,
                                 int sliced, int arg, cudaStream_t s) {
  return low_dispatch(kern, dim, mixed, m, blocks, threads, sliced, arg, s);
}

#endif  // GDG_BODIES_ONLY

}  // namespace gdg
