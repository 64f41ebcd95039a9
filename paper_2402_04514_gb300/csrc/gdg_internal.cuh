// Internal declarations of the gdg library: device-side problem layout, scratch, the Euler helpers
// shared by the sweep kernels, and the kernel launchers.  Not part of the C ABI (include/gdg.h).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/gdg.h"
#include "softfp64.cuh"

namespace gdg {

// Per-node primitive record written by k_prim and read for every neighbour in the sweeps.
enum { PR_IRHO = 0, PR_P, PR_A, PR_PME, PR_F, PR_ST, PR_IP, NPRIM };

// Constants of the Newton roots x^{-1/q} (rootinv, below).
struct RootQ {
  int q;
  double iq, c2;  // 1 / q and (q + 1) / (2 q^2)
};
__host__ __device__ inline RootQ root_q(int q) {
  RootQ r;
  r.q = q;
  r.iq = 1.0 / q;
  r.c2 = 0.5 * r.iq * (1.0 + r.iq);
  return r;
}

// Per-entry arrays are stored as sliced ELL.  The elements are taken in groups of kEll consecutive
// elements; slice (g, l) holds the rows of local index l of the group's elements, entry k of the row of
// the group's e-th element at slice_base(g, l) + kEll * k + e, and every slice is padded to its longest
// row.  A warp that takes one local index of kEll consecutive elements (the element sweep's thread map)
// then reads entry k of its 32 rows as one contiguous 256-byte segment.  Within a row the stencil entries
// c_ij != 0 come first, then the m_ij-only entries.  Padding slots are never read.
constexpr int kEll = 32;

// Everything a kernel needs, passed by value.  Per-entry arrays are device pointers in the sliced-ELL
// order above (row i's entries at rbeg[i], rbeg[i] + kEll, ... below rend[i]); per-node arrays in node
// order (rows element-contiguous); boundary entries are sorted by node (b_ptr indexes them).
struct Dev {
  int n, nnz, nb, n_loc;      // nnz: the length of the per-entry arrays, padding included
  int nel;                    // elements (n / n_loc)
  unsigned long long nl_mul;  // floor(x / n_loc) = (x * nl_mul) >> nl_shift for 0 <= x < 2^31 (div_nl)
  int nl_shift;
  // rows
  const int* rbeg;      // [n] position of row i's first entry
  const int* rend;      // [n] end of row i: rbeg[i] + kEll * (row length)
  const int* sten_end;  // [n] end of row i's stencil entries: I(i) is rbeg[i], rbeg[i] + kEll, ... below it
  const int* col;       // [nnz]
  const int* tr;        // [nnz] position of the transposed entry (j, i)
  const double* cnorm;  // [nnz] |c_ij| (0 when c_ij = 0)
  const double* cn;     // [dim][nnz] n_ij = c_ij / |c_ij|
  const double* mij;    // [nnz] consistent mass m_ij (0 across elements)
  const double* mu;     // [nnz] c_k h_ij^{p_k} for collocated pairs, else 0 (Sec. 5.1, eq. (ViscMin))
  // nodes
  const double* mi;     // [n]
  const double* inv_mi; // [n]
  const double* inv_km; // [n] 1 / (kappa_i m_i), Sec. 5.4, eq. (ConvexScheme)
  const double* rminus; // [n] r_h^- (Sec. 5.4)
  const double* rplus;  // [n] r_h^+
  const double* muB;    // [n] c_k h_i^{p_k} (boundary minimal-viscosity factor)
  const int* b_ptr;     // [n+1]
  // boundary entries (sorted by node)
  const double* bnorm;  // [nb] |c_i^{d,k}|
  const double* bn;     // [dim][nb] unit normals
  const int* btype;     // [nb]
  const int* borig;     // [nb] index of the entry in the caller's order (for Dirichlet data)
  const double* MKinv;  // [n / n_loc][n_loc][n_loc]
  // canonical stencil edges: entries (i, j) with c_ij != 0 and i < j, in entry order
  int ne;
  const int* edge_e;    // [ne] entry index of (i, j)
  const int* edge_i;    // [ne] row i
  // equation of state and method constants
  double gamma, gm1;    // gamma, gamma - 1
  double gm1h;          // (gamma - 1) / 2
  double e_exp;         // e = (gamma - 1) / (2 gamma)
  double inv_e;         // 1 / e
  int ie;               // 1 / e when it is an integer (7 for gamma = 1.4, 5 for gamma = 5/3), else 0
  double k13;           // (gamma + 1) / (2 gamma)
  int gp, gq;           // gamma = gp / gq with gq <= 8 (7/5, 5/3, ...); gq = 0 when gamma is not such a ratio
  int gk, gc;           // k = ceil(gp / gq) and c = k gq - gp (0 <= c < gq) when gq > 0
  int ie_root;          // 1 / e when it is an integer <= 16 (p^{-e} by a Newton root), else 0
  RootQ root_gq, root_ie, root_gpq;  // rootinv constants for gq, ie_root, gp + gq (q = 1, unused, where undefined)
  double inv_gp1;       // 1 / (gamma + 1)
  double c_ev;
  int order, passes, bounds_mode;
  double ls_tol;
  int ls_maxit;
  // mixed precision (GDG_PRECISION_MIXED): the switch and FP32 copies of the constants it uses
  int mixed;
  float gamma_f, gm1h_f, e_exp_f, inv_e_f, k13_f, inv_gp1_f, c_ev_f;
};

// The multiplier and shift of div_nl for n_loc in 1..32: with s = ceil(log2 n_loc) and
// M = ceil(2^(31+s) / n_loc) < 2^32, x M / 2^(31+s) exceeds x / n_loc by less than 2^-s < 1 / n_loc for
// x < 2^31, which never reaches the next integer, so the shifted product is floor(x / n_loc).
inline void set_nl_division(Dev& D, int nl) {
  int s = 0;
  while ((1 << s) < nl) ++s;
  D.nl_shift = 31 + s;
  D.nl_mul = ((1ULL << D.nl_shift) + (unsigned long long)nl - 1) / (unsigned long long)nl;
}
__device__ __forceinline__ int div_nl(const Dev& D, int x) {
  return (int)(((unsigned long long)(unsigned)x * D.nl_mul) >> D.nl_shift);
}

// The row of slot t of a one-thread-per-row kernel (row_slots below), -1 past the mesh.
__device__ __forceinline__ int row_node(const Dev& D, int t, int sliced) {
  if (!sliced) return t < D.n ? t : -1;
  const int sl = t / kEll;
  const int g = div_nl(D, sl);
  const int E = g * kEll + (t & (kEll - 1));
  return E < D.nel ? E * D.n_loc + (sl - g * D.n_loc) : -1;
}

// Equation-of-state constants of Dev for gamma (host side; gdg_setup and the wave-speed check).
inline void set_eos(Dev& D, double gamma) {
  D.gamma = gamma;
  D.gm1 = gamma - 1.0;
  D.gm1h = 0.5 * D.gm1;
  D.e_exp = (gamma - 1.0) / (2.0 * gamma);
  D.inv_e = 1.0 / D.e_exp;
  const double r = __builtin_round(D.inv_e);
  D.ie = (__builtin_fabs(D.inv_e - r) < 1e-12 * D.inv_e && r >= 1 && r <= 64) ? (int)r : 0;
  D.k13 = (gamma + 1.0) / (2.0 * gamma);
  D.gp = D.gq = 0;
  for (int q = 1; q <= 8 && D.gq == 0; ++q) {
    const double pg = __builtin_round(gamma * q);
    if (__builtin_fabs(gamma * q - pg) < 1e-12 * pg && pg <= 64) {
      D.gp = (int)pg;
      D.gq = q;
    }
  }
  D.gk = D.gq > 0 ? (D.gp + D.gq - 1) / D.gq : 0;
  D.gc = D.gk * D.gq - D.gp;
  D.ie_root = (D.ie > 0 && D.ie <= 16) ? D.ie : 0;
  D.root_gq = root_q(D.gq > 0 ? D.gq : 1);
  D.root_ie = root_q(D.ie_root > 0 ? D.ie_root : 1);
  D.root_gpq = root_q(D.gq > 0 ? D.gp + D.gq : 1);
  D.inv_gp1 = 1.0 / (gamma + 1.0);
  D.gamma_f = (float)gamma;
  D.gm1h_f = (float)(0.5 * D.gm1);
  D.e_exp_f = (float)D.e_exp;
  D.inv_e_f = (float)D.inv_e;
  D.k13_f = (float)D.k13;
  D.inv_gp1_f = (float)D.inv_gp1;
}

struct Scratch {
  double* prim;    // [NPRIM][n]
  double* dL;      // [nnz]
  double* G;       // [m][nnz] f(U_j) c_ij of stencil entries (from the edge sweep)
  double* barR;    // [nnz] rho of the bar state Ubar_ij (symmetric in i, j)
  double* barS;    // [nnz] s~ of the bar state
  double* dB;      // [nb]
  double* bbar;    // [2][nb] rho and s~ of the boundary bar states
  double* UL;      // [m][n]
  double* RHSL;    // [m][n] low-order right-hand side (sum of fluxes and viscous terms)
  double* N;       // [n]
  double* agg;     // [3][n] one-hop aggregates (rho min, rho max, s~ min)
  double* A;       // [m][nnz]
  double* AB;      // [m][nb]
  double* bounds;  // [3][n] rho_min, rho_max, s~_min
  double* l1;      // [nnz] per-row limiter coefficients, pass 1 (before symmetrisation)
  double* l1B;     // [nb]
  double* l2;      // [nnz] pass 2
  double* l2B;     // [nb]
  double* U1;      // [m][n]
  unsigned char* rem;  // [n] 1 where row i has a pass-2 remainder (a symmetrised pass-1 factor below 1)
  unsigned int* flags;
  unsigned int* lsq_n;  // [2] lengths of the deferred line-search queues of passes 1 and 2
  int2* lsq;            // [nnz + nb] deferred line searches of the current pass (ls_defer)
  unsigned long long* tau_bits;  // min of positive doubles via their bit patterns
};

#define GDG_DISPATCH(dim, fn, ...)        \
  switch (dim) {                          \
    case 1: return fn<1>(__VA_ARGS__);    \
    case 2: return fn<2>(__VA_ARGS__);    \
    case 3: return fn<3>(__VA_ARGS__);    \
    default: return cudaErrorInvalidValue; \
  }

// Time state of one instance for the fused SSP-RK3 step (gdg_ssprk3_step and batches): the step's bound
// min_i m_i / (2 |d_ii|) (Sec. 3.3, eq. (MaxCFLdt)) is reduced into tau_bits, and every kernel of the step
// takes tau = min(cfl * bound, t_end - t) (0 once t >= t_end) from it, so the step needs no host round
// trip.  k_clock advances t by tau at the end of the step.
struct Clock {
  unsigned long long tau_bits;  // bit pattern of the bound (positive doubles order like uint64); kTauNone: none
  double t, t_end, cfl;
  double tau;                   // tau of the last completed step
  long long steps;              // completed steps
};
constexpr unsigned long long kTauNone = 0x7f7f7f7f7f7f7f7fULL;

// Everything one kernel of a stage needs for one instance.
struct Ctx {
  Dev D;
  Scratch S;
  const double* U;      // stage input U_in [m][n]
  double* Ucopy;        // where the primitive sweep stores the U_in it read (a stage fed from host memory), or null
  double* Uhost;        // a second copy of U_out in mapped host memory (the last stage of a host-fed step), or null
  const double* Ubase;  // SSP-RK base (read only where alpha != 0)
  double* Uout;         // stage output; may equal Ubase (each node reads its base before writing itself)
  const double* bdata;  // Dirichlet data [m][nb] or null
  double alpha;         // U_out = alpha U_base + (1 - alpha) FE(U_in)  (Ubase2 null), or
  const double* Ubase2; //        alpha U_base + alpha2 U_base2 + w_fe FE(U_in)  (a second base term)
  double alpha2, w_fe;
  double tau;           // the stage's tau when clk is null
  Clock* clk;           // device clock of the fused step, or null
  double tau_scale;     // the stage's tau is tau_scale * dt of the step (fused steps)
  double dt_factor;     // dt = min(cfl * dt_factor * bound, t_end - t): the method's SSP coefficient
};

// The stage's output at flat index idx from its forward-Euler value fe (Shu-Osher combination).  Sums of
// products are written as explicit fused operations: left to the compiler, which product it fuses can
// differ between two instantiations of one kernel, and a batch member must give the bits of its solve
// alone.
__device__ __forceinline__ double rk_out(const Ctx& c, size_t idx, double fe) {
  if (c.Ubase2) return fma(c.w_fe, fe, fma(c.alpha2, c.Ubase2[idx], sf::mul(c.alpha, c.Ubase[idx])));
  return c.alpha != 0.0 ? fma(1.0 - c.alpha, fe, sf::mul(c.alpha, c.Ubase[idx])) : fe;
}

// Writes one value of the stage's output, and its host copy where the stage has one.
__device__ __forceinline__ void store_out(const Ctx& c, size_t idx, double v) {
  c.Uout[idx] = v;
  if (c.Uhost) c.Uhost[idx] = v;
}

// An instance whose clock has reached t_end: every kernel of the fused step returns at once, so the
// step leaves its state untouched (bit for bit) and costs only the launches.
__device__ __forceinline__ bool finished(const Ctx& c) { return c.clk && !(c.clk->t < c.clk->t_end); }

// dt of a fused step from its clock: min(cfl * dt_factor * bound, t_end - t), 0 without a bound.
__device__ __forceinline__ double clock_dt(const Clock* k, double dt_factor, bool* clipped) {
  const unsigned long long b = k->tau_bits;
  *clipped = false;
  if (b == kTauNone) return 0.0;
  const double v = k->cfl * dt_factor * __longlong_as_double((long long)b);
  const double rem = k->t_end - k->t;
  *clipped = !(v < rem);
  return *clipped ? (rem > 0.0 ? rem : 0.0) : v;
}

__device__ __forceinline__ double stage_tau(const Ctx& c) {
  if (!c.clk) return c.tau;
  bool clipped;
  return c.tau_scale * clock_dt(c.clk, c.dt_factor, &clipped);
}

// Where a kernel finds its context.  One: a single instance, the context is the kernel parameter and
// the local block is blockIdx.x.  Many: a batch; the block's instance is the last k with
// start[k] <= blockIdx.x (binary search over the batch's per-kernel block offsets), its context is
// copied from the device table into shared memory, and the local block is blockIdx.x - start[k].  Every
// thread of the block must call get() before any thread leaves.
struct One {
  Ctx c;
  __device__ __forceinline__ const Ctx& get(Ctx*, int* lb, int* nblk = nullptr) const {
    *lb = blockIdx.x;
    if (nblk) *nblk = gridDim.x;
    return c;
  }
  // the length of the deferred line-search queue of a pass, read before the context is loaded
  __device__ __forceinline__ unsigned queue_length(int pass, int* lb) const {
    *lb = blockIdx.x;
    return c.S.lsq_n[pass];
  }
};

struct Many {
  const Ctx* ctx;   // device [ninst]
  const int* start; // device [ninst + 1] first block of each instance, then the total
  int ninst;
  __device__ __forceinline__ int instance() const {
    int lo = 0, hi = ninst - 1;
    const int bx = (int)blockIdx.x;
    while (lo < hi) {  // the last instance starting at or before bx (instances without blocks are skipped)
      const int mid = (lo + hi + 1) >> 1;
      if (start[mid] <= bx) lo = mid; else hi = mid - 1;
    }
    return lo;
  }
  __device__ __forceinline__ unsigned queue_length(int pass, int* lb) const {
    const int k = instance();
    *lb = (int)blockIdx.x - start[k];
    return ctx[k].S.lsq_n[pass];
  }
  __device__ __forceinline__ const Ctx& get(Ctx* smem, int* lb, int* nblk = nullptr) const {
    const int lo = instance();
    const int bx = (int)blockIdx.x;
    *lb = bx - start[lo];
    if (nblk) *nblk = start[lo + 1] - start[lo];
    const int* src = reinterpret_cast<const int*>(ctx + lo);
    int* dst = reinterpret_cast<int*>(smem);
    for (int w = threadIdx.x; w < (int)(sizeof(Ctx) / sizeof(int)); w += blockDim.x) dst[w] = src[w];
    __syncthreads();
    return *smem;
  }
};

// Kernels of the sweep and their launch shapes.
enum Kern { KN_PRIM = 0, KN_MAXDT, KN_EDGE, KN_LOW, KN_HIGH, KN_LIMIT2, KN_FINAL, KN_LSFIX, KN_TAU, KN_AXPY,
            KN_COUNT };
constexpr int kRowMaxThreads = 512;  // one-thread-per-row / per-edge kernels: 128, 256 or 512 threads
constexpr int kHighMaxBlock = 288;   // element sweep: whole elements, at most this many nodes per block
constexpr int kHighDefaultCap = 288;  // the element block of an untuned schedule
constexpr int kLsfixThreads = 128;

// The launch schedule: threads per block of each one-thread-per-row kernel (KN_EDGE: per edge), the
// largest element block of the element sweep (whole elements, <= kHighMaxBlock nodes), and how many
// queue slots per thread the deferred line-search grid is sized for.  The defaults are what an untuned
// handle or batch runs; gdg_autotune / gdg_batch_autotune pick others by timing.
// slices: the row kernels (bit KN_*) whose threads take their rows in ELL slice order (row_node).
struct Sched {
  int bt[KN_COUNT];
  int high_cap;
  int lsfix_slots;
  int slices;
};
constexpr int kSliceable = (1 << KN_MAXDT) | (1 << KN_LOW) | (1 << KN_LIMIT2) | (1 << KN_FINAL) | (1 << KN_TAU);
inline Sched default_sched() {
  Sched sc;
  for (int k = 0; k < KN_COUNT; ++k) sc.bt[k] = 256;
  sc.high_cap = kHighDefaultCap;
  sc.lsfix_slots = 4;
  sc.slices = kSliceable;
  return sc;
}

// Row slots of a one-thread-per-row kernel: in node order slot t is row t; in ELL slice order slot t is
// lane t % kEll of slice t / kEll = g n_loc + l, the row of local index l of element g kEll + t % kEll, so
// that a warp's per-entry loads are contiguous (the nodes' own arrays are then read n_loc apart).
__host__ __device__ inline long long row_slots(const Dev& D, bool sliced) {
  return sliced ? (long long)((D.nel + kEll - 1) / kEll) * kEll * D.n_loc : (long long)D.n;
}
// Elements per block of the element sweep: the largest power of two <= kEll whose nodes fit the cap (so
// that a block is an aligned part of one ELL group), at least one.
__host__ __device__ inline int high_elems_per_block(int n_loc, int cap) {
  if (n_loc <= 0) return 0;
  int eb = kEll;
  while (eb > 1 && eb * n_loc > cap) eb >>= 1;
  return eb;
}
__host__ __device__ inline int high_threads(int n_loc, int eb) { return (eb * n_loc + 31) / 32 * 32; }
inline long long kernel_blocks(int k, const Dev& D, const Sched& sc) {
  switch (k) {
    case KN_EDGE: return ((long long)D.ne + sc.bt[k] - 1) / sc.bt[k];
    case KN_HIGH: {  // the groups of kEll elements, each in kEll / eb blocks
      const int eb = high_elems_per_block(D.n_loc, sc.high_cap);
      return eb > 0 ? ((long long)D.nel + kEll - 1) / kEll * (kEll / eb) : 0;
    }
    case KN_LSFIX: {
      // The queue length is only known on the device.  The grid covers the entries at lsfix_slots per
      // thread (a deferred search per thread unless more than that share of the entries defer, when the
      // threads take a few each), and its blocks beyond the queue return before loading their context.
      const long long per_block = (long long)kLsfixThreads * sc.lsfix_slots;
      return D.n == 0 ? 0 : ((long long)D.nnz + D.nb + per_block - 1) / per_block;
    }
    default: return (row_slots(D, (sc.slices >> k) & 1) + sc.bt[k] - 1) / sc.bt[k];
  }
}

// Kernel launchers of each file, dim in 1..3: one instance (context by value) or a batch (Many; blocks =
// the batch's total for that kernel).  arg: write_out for KN_LOW (the stage ends after U^L), last for
// KN_LIMIT2 (one limiter pass only), the pass (0 or 1) for KN_LSFIX.  threads: the block size of a
// one-thread-per-row kernel; sliced: its rows in ELL slice order; eb: elements per block of KN_HIGH;
// mixed: the precision of every member (single instances take it from their context).
cudaError_t launch_low_file(int kern, int dim, const Ctx& c, long long blocks, int threads, int sliced, int arg,
                            cudaStream_t s);
cudaError_t launch_low_file_many(int kern, int dim, bool mixed, const Many& m, long long blocks, int threads,
                                 int sliced, int arg, cudaStream_t s);
cudaError_t launch_high_file(int dim, const Ctx& c, long long blocks, int eb, cudaStream_t s);
cudaError_t launch_high_file_many(int dim, bool mixed, const Many& m, int n_loc, long long blocks, int eb,
                                  cudaStream_t s);
cudaError_t launch_limit_file(int kern, int dim, const Ctx& c, long long blocks, int threads, int sliced, int arg,
                              cudaStream_t s);
cudaError_t launch_limit_file_many(int kern, int dim, const Many& m, long long blocks, int threads, int sliced,
                                   int arg, cudaStream_t s);
// A batch in persistent mode (persistent.cu): one cooperative launch per stage runs every kernel of the
// stage for every member as phases separated by grid-wide barriers.  The arguments: the stage's contexts,
// the virtual block offsets of every phase ([KN_COUNT][ninst + 1], kernel_blocks of each member for the
// persistent block size) and their totals, and the step's structure.  grid returns the co-resident
// grid the launch used.
struct PersistArgs {
  const Ctx* ctx;
  const int* start;
  int ninst, stage, eb, low_only, order, passes, slices;
  int nblk[KN_COUNT];
};
cudaError_t launch_stage_persistent(int dim, bool mixed, const PersistArgs& a, int block, int* grid,
                                    cudaStream_t s);

// End of a fused step: advances the clock(s) by the step's dt (kernels_limit.cu).
cudaError_t launch_clock_one(Clock* clk, double dt_factor, cudaStream_t s);
cudaError_t launch_clock_many(const Ctx* ctx, int ninst, cudaStream_t s);

// One kernel of the sweep for one instance, shaped by the schedule.
inline cudaError_t launch_one(int kern, int dim, const Ctx& c, int arg, const Sched& sc, cudaStream_t s) {
  const long long blocks = kernel_blocks(kern, c.D, sc);
  switch (kern) {
    case KN_HIGH: return launch_high_file(dim, c, blocks, high_elems_per_block(c.D.n_loc, sc.high_cap), s);
    case KN_LIMIT2:
    case KN_FINAL:
    case KN_AXPY:
    case KN_LSFIX: return launch_limit_file(kern, dim, c, blocks, sc.bt[kern], (sc.slices >> kern) & 1, arg, s);
    default: return launch_low_file(kern, dim, c, blocks, sc.bt[kern], (sc.slices >> kern) & 1, arg, s);
  }
}

// ------------------------------------------------------------------------------------------------
// Device helpers (Euler equations of Sec. 2.2 and the pieces of Sec. 3-5 used by several kernels).

// a * b on the integer pipe (Soft, csrc/softfp64.cuh) or on the FP64 pipe: the same bits either way.  The
// deferred line searches take the FP64 pipe: their few active lanes per warp hide less of the integer
// routine's latency than they gain from the freed FP64 slots (k_lsfix 0.37 -> 0.41 ms per launch at Q2
// 1024^2 with the integer products).
template <bool Soft>
__device__ __forceinline__ double mulp(double a, double b) {
  if constexpr (Soft)
    return sf::mul(a, b);
  else
    return a * b;
}

// x^k for an integer k >= 0 by binary powering without a trailing square (k = 5, 7, 12 take 3, 4, 4
// multiplications).
template <bool Soft = true>
__device__ __forceinline__ double ipow(double x, int k) {
  if (k <= 0) return 1.0;
  while (!(k & 1)) {
    x = mulp<Soft>(x, x);
    k >>= 1;
  }
  double r = x;
  while (k >>= 1) {
    x = mulp<Soft>(x, x);
    if (k & 1) r = mulp<Soft>(r, x);
  }
  return r;
}

// FP64 -> FP32 by integer operations only (no instruction on the FP64 pipe, where the hardware conversion
// costs about 1.6 FMA issue slots): exponent rebias and the significand truncated to 23 bits (relative
// error < 2^-23) for values in the FP32 normal range, +-0 -> +-0.  Every other value (below the FP32
// normal range, above it, inf, NaN) gives NaN, so that a certificate or a seed computed from it fails its
// own check and the caller takes its FP64 path.
__device__ __forceinline__ float d2f_fast(double x) {
  const unsigned hi = (unsigned)__double2hiint(x);
  const unsigned lo = (unsigned)__double2loint(x);
  const int e = (int)((hi >> 20) & 0x7ffu) - 1023 + 127;
  unsigned r = (hi & 0x80000000u) | ((unsigned)e << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
  if (e <= 0 || e >= 255) r = (((hi & 0x7fffffffu) | lo) == 0u) ? (hi & 0x80000000u) : 0x7fc00000u;
  return __uint_as_float(r);
}

// d2f_fast for an increment x that the FP64 line search adds to a state component u0 as fma(s, x, u0).
// A nonzero x below the FP32 normal range (|x| < 2^-126) gives +-0 instead of NaN when that fma cannot see
// it, which the caller asserts with fz: s_f 2^-71 < |u0| in FP32 (s_f = s in FP32, relative error below
// 3 2^-23; |u0| truncated, so at most |u0|) gives s 2^-72 < |u0|, hence s |x| < s 2^-126 < 2^-54 |u0|,
// less than half an ulp of u0, and fma(s, x, u0) = u0 = fma(s, 0, u0): the FP64 search evaluates the same
// point as for x = 0.  Without fz, and above the FP32 range, the result is NaN, which fails a certificate.
// (Antidiffusive fluxes of a uniform neighbourhood are rounding residuals, some of them products of two
// residuals far below 2^-126.)
__device__ __forceinline__ float d2f_incr(double x, bool fz) {
  const unsigned hi = (unsigned)__double2hiint(x);
  const unsigned lo = (unsigned)__double2loint(x);
  const int e = (int)((hi >> 20) & 0x7ffu) - 1023 + 127;
  unsigned r = (hi & 0x80000000u) | ((unsigned)e << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
  if (e <= 0 || e >= 255) r = (e <= 0 && fz) ? (hi & 0x80000000u) : 0x7fc00000u;
  return __uint_as_float(r);
}

// FP32 -> FP64 by integer operations only: exact for normal numbers, zeros, infinities and NaN; an FP32
// subnormal gives NaN (no caller produces one where a result is needed: the seeds below are normal, and
// a NaN certificate fails).
__device__ __forceinline__ double f2d_fast(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned sg = u & 0x80000000u, e = (u >> 23) & 0xffu, mt = u & 0x7fffffu;
  unsigned hi = sg | ((e + 896u) << 20) | (mt >> 3);
  if (e == 255u) hi = sg | 0x7ff00000u | (mt >> 3);
  if (e == 0u) hi = mt ? 0x7ff80000u : sg;
  return __hiloint2double((int)hi, (int)(mt << 29));
}

// |x| and min / max of non-negative doubles through their bit patterns (IEEE order of non-negative
// numbers is the integer order), and x == +-0; all on the integer pipe.
__device__ __forceinline__ double abs_bits(double x) {
  return __longlong_as_double(__double_as_longlong(x) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ bool is_zero_bits(double x) { return (__double_as_longlong(x) << 1) == 0; }
__device__ __forceinline__ bool is_one_bits(double x) { return __double_as_longlong(x) == 0x3ff0000000000000LL; }

// FP64 reciprocal from the FP32 reciprocal y0 of x in FP32 (relative error e = 1 - x y0 below 2^-22):
// 1/x = y0 / (1 - e) = y0 (1 + e + e^2 + ...), summed through e^2 in one fused update, leaves
// e^3 < 2^-66 plus the rounding of the last FMA, so the result is within 2 ulp of 1/x.  Costs 3 FP64
// operations instead of a full FP64 division on a chip whose FP64 pipe is the bottleneck.  Arguments
// outside the FP32 normal range take the IEEE division.
__device__ __forceinline__ double rcp64(double x) {
  float xf = d2f_fast(x);
  float ax = fabsf(xf);
  if (!(ax > 1e-37f && ax < 1e37f)) return 1.0 / x;
  const double y = f2d_fast(__frcp_rn(xf));
  const double e = fma(-x, y, 1.0);
  return fma(y, fma(e, e, e), y);
}

// sqrt(x) for x in the FP32 normal range by two Heron corrections s <- s + (x - s^2) h from s0 = x y0,
// with y0 the FP32 reciprocal square root (relative error below 2^-21) and h = y0 / 2 held fixed: each
// correction multiplies the relative error by about that of h and adds half its square
// (2^-21 -> 2^-41 -> 2^-61), so the result is within an ulp or so of sqrt(x).  5 FP64 operations instead of
// CUDA's square root with its special-case handling.  Other arguments take sqrt.
__device__ __forceinline__ double sqrt64(double x) {
  const float xf = d2f_fast(x);
  if (!(xf > 1e-37f && xf < 1e37f)) return sqrt(x);
  const float yf = rsqrtf(xf);
  const double h = f2d_fast(0.5f * yf);
  double s = sf::mul(x, f2d_fast(yf));
  s = fma(fma(-s, s, x), h, s);
  return fma(fma(-s, s, x), h, s);
}

// y = x^{-1/q} for x > 0 and 1 <= q <= 16.  From the FP32 seed y0 = exp2(-log2(x) / q), with
// t = 1 - x y0^q and x^{-1/q} = y0 (1 - t)^{-1/q}, one step y0 (1 + t/q + (q+1)/(2q^2) t^2) sums the
// binomial series through t^2; the rest, |binom(-1/q, 3)| |t|^3 (1 + O(t)) with |binom(-1/q, 3)| <= 1
// (0.09 for q >= 5), is below 2^-56 when |t| <= 2^-19, which the seed's 2^-22 relative error (times q)
// gives for arguments near 1.  Far
// from 1 log2f's absolute error grows with |log2 x| and the seed can be worse; then one Newton step
// y <- y + y (1 - x y^q) / q squares the remaining error.  Arguments outside the FP32 normal range use pow.
template <bool Soft = true>
__device__ __forceinline__ double rootinv(double x, const RootQ& r) {
  float xf = d2f_fast(x);
  if (!(xf > 1e-37f && xf < 1e37f)) return pow(x, -r.iq);
  double y = f2d_fast(exp2f(-log2f(xf) / (float)r.q));
  const double t = fma(-x, ipow<Soft>(y, r.q), 1.0);
  y = fma(mulp<Soft>(y, t), fma(r.c2, t, r.iq), y);
  // |t| > 2^-19, compared on the bit patterns (integer pipe)
  if ((__double_as_longlong(t) & 0x7fffffffffffffffLL) > 0x3ec0000000000000LL) {
    const double t2 = fma(-x, ipow<Soft>(y, r.q), 1.0);
    y = fma(y * t2, r.iq, y);
  }
  return y;
}

// rho^{-gamma} and 1/rho together.  With gamma = p/q (p > q): y = rho^{-1/q}, 1/rho = y^q and
// rho^{-gamma} = y^p, as y^q y^{p-q} (Share: fewer multiplications, one longer chain; faster in the edge
// sweep) or by its own powering (measured faster in k_prim).
template <bool Share = true>
__device__ __forceinline__ double rho_neg_gamma(const Dev& D, double rho, double* inv_rho) {
  if (D.gq > 0) {
    const double y = rootinv(rho, D.root_gq);
    const double yq = ipow(y, D.gq);
    *inv_rho = yq;
    return Share ? sf::mul(yq, ipow(y, D.gp - D.gq)) : ipow(y, D.gp);
  }
  *inv_rho = rcp64(rho);
  return pow(rho, -D.gamma);
}

// rho^gamma and 1/rho together.  With gamma = p/q, k = ceil(p/q) and c = kq - p (0 <= c < q):
// rho^gamma = rho^k y^c and 1/rho = y^q = y^c y^{q-c}.
template <bool Soft = true>
__device__ __forceinline__ double rho_pow_gamma(const Dev& D, double rho, double* inv_rho) {
  if (D.gq > 0) {
    const double y = rootinv<Soft>(rho, D.root_gq);
    const double yc = ipow<Soft>(y, D.gc);
    *inv_rho = mulp<Soft>(yc, ipow<Soft>(y, D.gq - D.gc));
    return mulp<Soft>(ipow<Soft>(rho, D.gk), yc);
  }
  *inv_rho = rcp64(rho);
  return pow(rho, D.gamma);
}

// min / max of positive doubles through their bit patterns (IEEE order of positive numbers is the
// integer order), which keeps the bound aggregates off the FP64 pipe.
__device__ __forceinline__ double pmin(double a, double b) {
  long long x = __double_as_longlong(a), y = __double_as_longlong(b);
  return __longlong_as_double(x < y ? x : y);
}
__device__ __forceinline__ double pmax(double a, double b) {
  long long x = __double_as_longlong(a), y = __double_as_longlong(b);
  return __longlong_as_double(x > y ? x : y);
}

// lambda_max^+ of the Riemann problem along n (Sec. 3.1, eq. (eq:dij_low_order)), from the normal
// velocities u, pressures p (and 1/p), sound speeds a and p^{-e} of both states: the two-rarefaction pressure
// p~ bounds the star pressure from above for 1 < gamma <= 5/3; the outer wave speeds at p~ bound the
// exact ones.
__device__ __forceinline__ double lambda_max(const Dev& D, double uL, double pL, double ipL, double aL,
                                             double pmeL, double uR, double pR, double ipR, double aR,
                                             double pmeR) {
  // max(x, 0), the tests x > 0 and the final maximum of two non-negative values on the integer pipe
  // (a positive double is a positive int64)
  auto pos = [](double x) { return __double_as_longlong(x) > 0 ? x : 0.0; };
  double num = pos(fma(-D.gm1h, uR - uL, aL + aR));
  double r = sf::mul(num, rcp64(fma(aL, pmeL, sf::mul(aR, pmeR))));
  double pt = D.ie > 0 ? ipow(r, D.ie) : pow(r, D.inv_e);
  double xL = pt - pL, xR = pt - pR;
  double sL = __double_as_longlong(xL) > 0 ? sqrt64(fma(sf::mul(D.k13, xL), ipL, 1.0)) : 1.0;
  double sR = __double_as_longlong(xR) > 0 ? sqrt64(fma(sf::mul(D.k13, xR), ipR, 1.0)) : 1.0;
  double l1 = fma(-aL, sL, uL);
  double l3 = fma(aR, sR, uR);
  return pmax(pos(-l1), pos(l3));
}

// ------------------------------------------------------------------------------------------------
// Mixed precision (GDG_PRECISION_MIXED; the contract is documented at the enum in include/gdg.h).

// FP64 -> FP32 on the integer pipe, for arithmetic: the significand truncated to 23 bits (relative error
// below 2^-23, and to_f32(-x) = -to_f32(x), which keeps antisymmetric quantities antisymmetric); values
// below the FP32 normal range flush to +-0, values above it give +-inf, NaN stays NaN.
__device__ __forceinline__ float to_f32(double x) {
  const unsigned hi = (unsigned)__double2hiint(x);
  const unsigned lo = (unsigned)__double2loint(x);
  const unsigned sg = hi & 0x80000000u, ah = hi & 0x7fffffffu;
  const int e = (int)(ah >> 20) - 1023 + 127;
  unsigned r = sg | ((unsigned)e << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
  if (e <= 0) r = sg;
  if (e >= 255) r = (ah > 0x7ff00000u || (ah == 0x7ff00000u && lo != 0u)) ? 0x7fc00000u : (sg | 0x7f800000u);
  return __uint_as_float(r);
}

// FP32 -> FP64 on the integer pipe: exact for normal numbers, zeros, infinities and NaN; FP32 subnormals
// flush to +-0.
__device__ __forceinline__ double to_f64(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned sg = u & 0x80000000u, e = (u >> 23) & 0xffu, mt = u & 0x7fffffu;
  unsigned hi = sg | ((e + 896u) << 20) | (mt >> 3), lo = mt << 29;
  if (e == 255u) hi = sg | 0x7ff00000u | (mt >> 3);
  if (e == 0u) {
    hi = sg;
    lo = 0u;
  }
  return __hiloint2double((int)hi, (int)lo);
}

__device__ __forceinline__ bool finite_f32(float x) { return (__float_as_uint(x) & 0x7f800000u) != 0x7f800000u; }

__device__ __forceinline__ float ipowf(float x, int k) {
  if (k <= 0) return 1.f;
  while (!(k & 1)) {
    x *= x;
    k >>= 1;
  }
  float r = x;
  while (k >>= 1) {
    x *= x;
    if (k & 1) r *= x;
  }
  return r;
}

// The FP32 primitives the mixed path's wave-speed bound takes from a node: 1/p, a = sqrt(gamma p / rho)
// and p^{-e} (Sec. 2.2), from the FP64 rho and p.
struct PrimF {
  float ip, a, pme;
};
__device__ __forceinline__ PrimF prim_mx(const Dev& D, double rho, double p) {
  const float rf = to_f32(rho), pf = to_f32(p);
  PrimF o;
  o.ip = 1.f / pf;
  o.a = sqrtf(D.gamma_f * pf / rf);
  o.pme = powf(pf, -D.e_exp_f);
  return o;
}

// Margin of the mixed path's wave-speed bound, relative to S = |u_L| + |u_R| + a_L s_L + a_R s_R, which
// is at least lambda (-lambda_1 <= |u_L| + a_L s_L, lambda_3 <= |u_R| + a_R s_R).  Every FP32 operation
// and input of lambda_max_mx is within a few ulp (2^-23) of its FP64 counterpart; the largest
// amplification is the power 1/e of p~ (7 for gamma = 1.4, 5 for 5/3), which reaches s_L, s_R through a
// square root, so that the FP32 bound differs from the FP64 one by less than 2^-17 S (the largest
// difference seen over several million states, including near-vacuum and near-equal pairs, is 2^-19.9 S).
// The margin is twice that bound.
constexpr float kMxMargin = 1.52587890625e-05f;  // 2^-16

// lambda_max^+ of the FP64 path's formula (lambda_max) evaluated in FP32 and raised by kMxMargin S.  The
// denominators and S are summed without contraction, so that the bound is symmetric under
// (L, R, n) -> (R, L, -n) bit for bit like the FP64 one.  raw / scale (optional) receive the value
// before the margin and S.
__device__ __forceinline__ float lambda_max_mx(const Dev& D, float uL, float pL, const PrimF& L, float uR, float pR,
                                               const PrimF& R, float* raw = nullptr, float* scale = nullptr) {
  const float num = fmaxf(L.a + R.a - D.gm1h_f * (uR - uL), 0.f);
  const float den = __fadd_rn(__fmul_rn(L.a, L.pme), __fmul_rn(R.a, R.pme));
  const float r = num / den;
  const float pt = D.ie > 0 ? ipowf(r, D.ie) : powf(r, D.inv_e_f);
  const float xL = pt - pL, xR = pt - pR;
  const float sL = xL > 0.f ? sqrtf(1.f + D.k13_f * xL * L.ip) : 1.f;
  const float sR = xR > 0.f ? sqrtf(1.f + D.k13_f * xR * R.ip) : 1.f;
  const float l1 = uL - L.a * sL;
  const float l3 = uR + R.a * sR;
  const float lam = fmaxf(fmaxf(-l1, 0.f), fmaxf(l3, 0.f));
  const float S = __fadd_rn(__fadd_rn(fabsf(uL), fabsf(uR)), __fadd_rn(__fmul_rn(L.a, sL), __fmul_rn(R.a, sR)));
  if (raw) *raw = lam;
  if (scale) *scale = S;
  return fmaf(kMxMargin, S, lam);
}

// The FP64 primitives of k_prim's FP64 path from rho (as 1/rho) and p.
__device__ __forceinline__ void prim_fp64(const Dev& D, double irho, double p, double* ip, double* a, double* pme) {
  *ip = 1.0 / p;
  *a = sqrt64(sf::mul(sf::mul(D.gamma, p), irho));
  *pme = D.ie_root > 0 ? rootinv(p, D.root_ie) : pow(p, -D.e_exp);
}

// 1/p, a and p^{-e} of a state that k_prim does not see (a boundary state), as each path computes them.
template <bool MX>
__device__ __forceinline__ void prim_of(const Dev& D, double rho, double irho, double p, double* ip, double* a,
                                        double* pme) {
  if constexpr (MX) {
    const PrimF f = prim_mx(D, rho, p);
    *ip = to_f64(f.ip);
    *a = to_f64(f.a);
    *pme = to_f64(f.pme);
  } else {
    *ip = 1.0 / p;
    *a = sqrt64(sf::mul(sf::mul(D.gamma, p), irho));
    *pme = pow(p, -D.e_exp);
  }
}

// The wave-speed bound of either path from a pair of nodes' stored primitives (normal velocities u, FP64
// p and 1/rho, and 1/p, a, p^{-e} as the path's k_prim wrote them).  The mixed path falls back to the FP64
// formula when its FP32 bound is infinite or NaN (states near the ends of the FP32 range).
template <bool MX>
__device__ __forceinline__ double lambda_pair(const Dev& D, double uL, double pL, double irL, double ipL, double aL,
                                              double pmeL, double uR, double pR, double irR, double ipR, double aR,
                                              double pmeR) {
  if constexpr (MX) {
    const PrimF Lf{to_f32(ipL), to_f32(aL), to_f32(pmeL)}, Rf{to_f32(ipR), to_f32(aR), to_f32(pmeR)};
    const float lam = lambda_max_mx(D, to_f32(uL), to_f32(pL), Lf, to_f32(uR), to_f32(pR), Rf);
    if (finite_f32(lam)) return to_f64(lam);
    prim_fp64(D, irL, pL, &ipL, &aL, &pmeL);
    prim_fp64(D, irR, pR, &ipR, &aR, &pmeR);
  }
  return lambda_max(D, uL, pL, ipL, aL, pmeL, uR, pR, ipR, aR, pmeR);
}

// f(U) n for a unit vector n, given m.n = mn, v.n = un and p: [m.n, m un + p n, (E + p) un].
template <int DIM>
__device__ __forceinline__ void flux_n(const double* U, const double* n, double mn, double un, double p,
                                       double* out) {
  out[0] = mn;
#pragma unroll
  for (int k = 0; k < DIM; ++k) out[1 + k] = fma(U[1 + k], un, sf::mul(p, n[k]));
  out[DIM + 1] = sf::mul(U[DIM + 1] + p, un);
}

// a . b for DIM-vectors, as an explicit chain: the first product rounded on its own (integer pipe), each
// later one fused into the sum.  Written out so that the compiler has no choice of which products to fuse:
// where it has one, two instantiations of a kernel can round differently.
template <int DIM>
__device__ __forceinline__ double dot(const double* a, const double* b) {
  double s = sf::mul(a[0], b[0]);
#pragma unroll
  for (int k = 1; k < DIM; ++k) s = fma(a[k], b[k], s);
  return s;
}

template <int DIM>
__device__ __forceinline__ double internal_energy(const double* U) {
  const double m2 = dot<DIM>(U + 1, U + 1);
  return U[DIM + 1] - sf::mul_pow2(m2, -1) / U[0];
}

// In- and outflow boundary state (Sec. 4.1) from the interior state Ui, the data Ud and the outward unit
// normal n: supersonic inflow (v.n < -a) takes the data, supersonic outflow (v.n >= a) the interior state
// (eq. (eq:supersonic_inoutflow)); in between, the characteristic variables of eq. (eq:characteristics),
// R = {v_n - 2a/(g-1), p/rho^g, v - (v.n) n, v_n + 2a/(g-1)}, are the data's where the characteristic speed
// at the interior state {v_n - a, v_n, v_n, v_n + a} is <= 0 and the interior state's otherwise, and the
// state is rebuilt from them.  Where the blend admits no state (a <= 0, a vacuum) the interior state is
// used.  Boundary entries only: plain FP64 with CUDA's sqrt and pow.
template <int DIM>
__device__ __forceinline__ void inoutflow_state(double g, const double* Ui, const double* Ud, const double* n,
                                                double* UB) {
  constexpr int M = DIM + 2;
  double vi[DIM], vd[DIM], m2i = 0.0, m2d = 0.0, vni = 0.0, vnd = 0.0;
#pragma unroll
  for (int k = 0; k < DIM; ++k) {
    vi[k] = Ui[1 + k] / Ui[0];
    vd[k] = Ud[1 + k] / Ud[0];
    m2i += Ui[1 + k] * Ui[1 + k];
    m2d += Ud[1 + k] * Ud[1 + k];
    vni += vi[k] * n[k];
    vnd += vd[k] * n[k];
  }
  const double pi = (g - 1.0) * (Ui[DIM + 1] - 0.5 * m2i / Ui[0]);
  const double ai = sqrt(g * pi / Ui[0]);
  if (vni < -ai) {
#pragma unroll
    for (int q = 0; q < M; ++q) UB[q] = Ud[q];
    return;
  }
  if (vni >= ai) {
#pragma unroll
    for (int q = 0; q < M; ++q) UB[q] = Ui[q];
    return;
  }
  const double pd = (g - 1.0) * (Ud[DIM + 1] - 0.5 * m2d / Ud[0]);
  const double ad = sqrt(g * pd / Ud[0]);
  const bool in = vni <= 0.0;  // the middle characteristics come in
  const double R1 = vnd - 2.0 * ad / (g - 1.0);
  const double R4 = vni + 2.0 * ai / (g - 1.0);
  const double R2 = in ? pd / pow(Ud[0], g) : pi / pow(Ui[0], g);
  const double vns = in ? vnd : vni;
  const double vn = 0.5 * (R1 + R4);
  const double a = 0.25 * (g - 1.0) * (R4 - R1);
  if (!(a > 0.0)) {
#pragma unroll
    for (int q = 0; q < M; ++q) UB[q] = Ui[q];
    return;
  }
  const double rho = pow(a * a / (g * R2), 1.0 / (g - 1.0));
  const double p = R2 * pow(rho, g);
  double v2 = 0.0;
  UB[0] = rho;
#pragma unroll
  for (int k = 0; k < DIM; ++k) {
    const double vk = vn * n[k] + ((in ? vd[k] : vi[k]) - vns * n[k]);
    UB[1 + k] = rho * vk;
    v2 += vk * vk;
  }
  UB[DIM + 1] = p / (g - 1.0) + 0.5 * rho * v2;
}

// Slip (Sec. 4.1, eq. (eq:slip_boundary)), Dirichlet or in/outflow boundary state of entry b.
template <int DIM>
__device__ __forceinline__ void boundary_state(const Dev& D, int b, const double* Ui, const double* bdata,
                                               const double* n, double* UB) {
  constexpr int M = DIM + 2;
  if (D.btype[b] == GDG_BC_DIRICHLET) {
    int o = D.borig[b];
#pragma unroll
    for (int q = 0; q < M; ++q) UB[q] = bdata[(size_t)q * D.nb + o];
  } else if (D.btype[b] == GDG_BC_INOUTFLOW) {
    const int o = D.borig[b];
    double Ud[M];
#pragma unroll
    for (int q = 0; q < M; ++q) Ud[q] = bdata[(size_t)q * D.nb + o];
    inoutflow_state<DIM>(D.gamma, Ui, Ud, n, UB);
  } else {
    const double mn2 = sf::mul_pow2(dot<DIM>(Ui + 1, n), 1);  // 2 m.n
    UB[0] = Ui[0];
#pragma unroll
    for (int k = 0; k < DIM; ++k) UB[1 + k] = fma(-mn2, n[k], Ui[1 + k]);
    UB[DIM + 1] = Ui[DIM + 1];
  }
}

// Per-row context of the line searches from one state U0 (the row's U^L or U^(1)) against the row's
// bounds: psi(0) in FP64 once per row, and FP32 copies of U0's parts, of psi(0) and of the distances of
// rho(U0) to its bounds for the FP32 certificates.  The searches run along P = w A (w = the row's
// 1 / (kappa_i m_i), times 1 - l1 in pass 2), so a point t of the search is U0 + (t w) A.
template <int DIM>
struct LsRow {
  double U0[DIM + 2];
  double rmin, rmax, smin, psi0;
  float r0, ir0, m0[DIM], m0sq, sg0, psi0f, dlo, dhi;
  float fl;  // min(rho0, |m0_k|, psi0f) in FP32, 0 unless all are positive: the bound of d2f_incr's guard
};

template <int DIM>
__device__ __forceinline__ void ls_row(const Dev& D, LsRow<DIM>& c, const double* U0, double rmin, double rmax,
                                       double smin) {
  double m2 = 0.0;
#pragma unroll
  for (int q = 0; q < DIM + 2; ++q) c.U0[q] = U0[q];
#pragma unroll
  for (int k = 0; k < DIM; ++k) m2 += U0[1 + k] * U0[1 + k];
  c.rmin = rmin;
  c.rmax = rmax;
  c.smin = smin;
  double ir;
  double rg = (U0[0] > 0.0) ? rho_pow_gamma(D, U0[0], &ir) : 0.0;
  c.psi0 = (U0[0] > 0.0) ? fma(-smin, rg, fma(-sf::mul_pow2(m2, -1), ir, U0[DIM + 1])) : -1.0;
  c.r0 = d2f_fast(U0[0]);
  c.ir0 = __frcp_rn(c.r0);
#pragma unroll
  for (int k = 0; k < DIM; ++k) c.m0[k] = d2f_fast(U0[1 + k]);
  c.m0sq = d2f_fast(m2);
  c.sg0 = d2f_fast(smin * rg);
  c.psi0f = d2f_fast(c.psi0);
  // distances to the density bounds for the FP32 density certificate, kept only when they exceed 1e-6
  // rho(U0): the FP64 comparisons of the closed form round relative to rho, so a certificate on a smaller
  // gap could disagree with them (a zero distance sends every search of the row to the FP64 form)
  const float dlo = d2f_fast(U0[0] - rmin), dhi = d2f_fast(rmax - U0[0]), gap = 1e-6f * c.r0;
  c.dlo = dlo > gap ? dlo : 0.f;
  c.dhi = dhi > gap ? dhi : 0.f;
  // |E0| >= psi(0) >= psi0f, so that psi0f bounds |E0| from below where it is positive
  float fl = c.psi0f;
#pragma unroll
  for (int k = 0; k < DIM; ++k) fl = fminf(fl, fabsf(c.m0[k]));
  fl = fminf(fl, c.r0);
  c.fl = fl > 0.f ? fl : 0.f;  // NaN (a value outside the FP32 range) also gives 0
}

// psi(s) = eps(U0 + s A) - s_min rho(s)^gamma (the entropy constraint of the set B_i, Sec. 5.4,
// eq. (BiSet), times rho^gamma); concave in s.
template <int DIM>
__device__ __forceinline__ double ls_psi(const Dev& D, const double* U0, const double* A, double s, double smin) {
  double V[DIM + 2];
#pragma unroll
  for (int q = 0; q < DIM + 2; ++q) V[q] = fma(s, A[q], U0[q]);
  if (!(V[0] > 0.0)) return -1.0;
  double m2 = 0.0;
#pragma unroll
  for (int k = 0; k < DIM; ++k) m2 += V[1 + k] * V[1 + k];
  double irho;
  double rg = rho_pow_gamma<false>(D, V[0], &irho);
  return fma(-smin, rg, fma(-sf::mul_pow2(m2, -1), irho, V[DIM + 1]));
}

// d psi / d s
template <int DIM>
__device__ __forceinline__ double ls_dpsi(const Dev& D, const double* U0, const double* A, double s, double smin) {
  double V[DIM + 2];
#pragma unroll
  for (int q = 0; q < DIM + 2; ++q) V[q] = fma(s, A[q], U0[q]);
  double mA = 0.0, m2 = 0.0;
#pragma unroll
  for (int k = 0; k < DIM; ++k) {
    mA += V[1 + k] * A[1 + k];
    m2 += V[1 + k] * V[1 + k];
  }
  double irho;
  double rg = rho_pow_gamma<false>(D, V[0], &irho);
  double deps = A[DIM + 1] - mA * irho + 0.5 * m2 * A[0] * irho * irho;
  return deps - smin * D.gamma * rg * irho * A[0];
}

// psi(s) and d psi / d s together (the two share the state, rho^gamma and 1/rho), each computed as
// ls_psi and ls_dpsi compute it.
template <int DIM>
__device__ __forceinline__ double ls_psi_dpsi(const Dev& D, const double* U0, const double* A, double s, double smin,
                                              double* dpsi) {
  double V[DIM + 2];
#pragma unroll
  for (int q = 0; q < DIM + 2; ++q) V[q] = fma(s, A[q], U0[q]);
  double mA = 0.0, m2 = 0.0;
#pragma unroll
  for (int k = 0; k < DIM; ++k) {
    mA += V[1 + k] * A[1 + k];
    m2 += V[1 + k] * V[1 + k];
  }
  double irho;
  double rg = rho_pow_gamma<false>(D, V[0], &irho);
  double deps = A[DIM + 1] - mA * irho + 0.5 * m2 * A[0] * irho * irho;
  *dpsi = deps - smin * D.gamma * rg * irho * A[0];
  if (!(V[0] > 0.0)) return -1.0;
  return fma(-smin, rg, fma(-sf::mul_pow2(m2, -1), irho, V[DIM + 1]));
}

// Certifies psi(s) >= 0 from psi(0) and the increment dpsi = psi(s) - psi(0) evaluated in FP32 in
// differenced form, so that its error scales with |s A| rather than with |U0|:
//   dpsi = s A_E - dK - dG,  dK = (rho0 (2 m0.b + |b|^2) - a |m0|^2) / (2 rho0 (rho0 + a)),
//   dG = s_min rho0^gamma expm1(gamma log1p(a / rho0)),   a = s A_rho, b = s A_m.
// sf is s in FP32 with relative error at most 3 2^-23.  Every other FP32 operation and conversion has
// relative error <= 2^-23 (the two quotients by the denominator and a / rho0 are products with correctly
// rounded reciprocals, two roundings of at most 2^-24 each; a denominator above 1e36 fails the
// certificate, so that its reciprocal stays a normal number) and log1pf / expm1f a few ulp.  The
// quotients never take FP32 division's slow path, which a zero numerator (A = 0) would otherwise take.
// So the FP32 dpsi is within 2e-6 S of the exact
// increment, S = |s A_E| + S_K + |dG| and S_K the magnitude of dK's terms.  With t = psi0f + dpsi in FP32
// (psi0f = psi(0) truncated to FP32, relative error < 2^-23), certifying only when
// t > 1e-4 S + 1e-6 |psi0f| leaves a factor of 50 on every error term, so psi(s) > 0 exactly.  Requires
// a > -rho0 / 2 (otherwise the caller evaluates psi in FP64); any NaN (an input outside the FP32 normal
// range) fails the final comparison.
template <int DIM>
__device__ __forceinline__ bool ls_certified(const Dev& D, const LsRow<DIM>& c, const double* A, float sf) {
  // components of A below the FP32 range count as 0 where the FP64 search cannot see them (d2f_incr)
  const bool fz = sf * 0x1p-71f < c.fl;
  float a = sf * d2f_incr(A[0], fz);
  if (!(a > -0.5f * c.r0)) return false;
  float mb = 0.f, bb = 0.f, nb2 = 0.f;
#pragma unroll
  for (int k = 0; k < DIM; ++k) {
    float b = sf * d2f_incr(A[1 + k], fz);
    mb = fmaf(c.m0[k], b, mb);
    bb = fmaf(b, b, bb);
    nb2 = fmaf(fabsf(c.m0[k]), fabsf(b), nb2);
  }
  float eE = sf * d2f_incr(A[DIM + 1], fz);
  float r1 = c.r0 + a;
  float den = 2.f * c.r0 * r1;
  if (!(den < 1e36f)) return false;
  const float iden = __frcp_rn(den);
  float dK = (c.r0 * (2.f * mb + bb) - a * c.m0sq) * iden;
  float SK = (c.r0 * (2.f * nb2 + bb) + fabsf(a) * c.m0sq) * iden;
  float dG = c.sg0 * expm1f(D.gamma_f * log1pf(a * c.ir0));
  float dpsi = eE - dK - dG;
  float scale = fabsf(eE) + SK + fabsf(dG);
  float t = c.psi0f + dpsi;
  return t > 1e-4f * scale + 1e-6f * fabsf(c.psi0f);
}

// Largest l in [0, 1] with U0 + l P in B_i, P = w A (Sec. 5.4, eq. (ConvexScheme), Lemma
// ConsInvariants), in two parts.  The head takes the closed form for the density bounds and decides the
// common cases: the entropy constraint holds at l_rho (proved by the FP32 certificate, else by psi in FP64),
// or psi(0) < 0 (roundoff) and l = 0.  It returns false when psi(l_rho) < 0 <= psi(0); then the tail runs
// a bracketed iteration on the concave psi from [0, l_rho]: the chord root stays feasible, the tangent root
// from the infeasible end stays infeasible, and a bisection follows every iteration that has not halved the
// bracket; it stops when the bracket is at most ls_tol wide and returns the feasible end.  The FP32 certificate only skips FP64
// evaluations whose outcome it proves; the result is that of the FP64 search.
template <int DIM>
__device__ __forceinline__ bool line_search_head(const Dev& D, const LsRow<DIM>& c, const double* A, double w,
                                                 float wf, double* l_out, double* fb_out) {
  // Density bounds.  The common case, rho(U0) + w A_rho inside [rho_min, rho_max] so that l_rho = 1, is
  // proved in FP32 (wf = w in FP32): the products and conversions have relative error below 4e-7, so a
  // relative margin of 1e-6 on both sides leaves the exact distance to the bound above 8e-7 times a gap
  // of at least 1e-6 rho (ls_row), far beyond the FP64 rounding of the closed form's comparisons, which
  // therefore agree with it.  An A_rho below the FP32 range counts as 0 under the guard of d2f_incr, which
  // also makes rho(U0) + w A_rho round to rho(U0) in the closed form.
  const float pr = wf * d2f_incr(A[0], wf * 0x1p-71f < c.fl);
  const bool inside = pr >= 0.f ? pr * 1.000001f < c.dhi * 0.999999f : -pr * 1.000001f < c.dlo * 0.999999f;
  double l = 1.0;
  float sf = wf;
  if (!inside) {
    const double Pr = w * A[0];
    if (c.U0[0] + Pr < c.rmin) l = (c.rmin - c.U0[0]) / Pr;
    if (c.U0[0] + Pr > c.rmax) l = (c.rmax - c.U0[0]) / Pr;
    if (!(l > 0.0)) l = 0.0;
    if (l > 1.0) l = 1.0;
    sf = d2f_fast(l * w);
  }
  *l_out = l;
  if (ls_certified<DIM>(D, c, A, sf)) return true;
  const double fb = ls_psi<DIM>(D, c.U0, A, l * w, c.smin);
  *fb_out = fb;
  if (fb >= 0.0) return true;
  if (c.psi0 < 0.0) {
    *l_out = 0.0;
    return true;
  }
  return false;
}

template <int DIM>
__device__ double line_search_tail(const Dev& D, const LsRow<DIM>& c, const double* A, double w,
                                                double l, double fb) {
  const double* U0 = c.U0;
  const double smin = c.smin;
  double fa = c.psi0;
  double a = 0.0, b = l;
  // the slope at b, kept while b stays: the tangent point, which usually becomes the next b, is evaluated
  // with its slope; a b set by the chord or the bisection takes it afresh at the next iteration
  double dfb = 0.0;
  bool fresh = false;
  for (int it = 0; it < D.ls_maxit && b - a > D.ls_tol; ++it) {
    const double width = b - a;
    double ts = a + (b - a) * fa / (fa - fb);
    if (!fresh) dfb = w * ls_dpsi<DIM>(D, U0, A, b * w, smin);
    fresh = true;
    double tn = dfb < 0.0 ? b - fb / dfb : b;
    if (ts > a && ts < b) {
      double fs = ls_psi<DIM>(D, U0, A, ts * w, smin);
      if (fs >= 0.0) { a = ts; fa = fs; } else { b = ts; fb = fs; fresh = false; }
    }
    if (tn > a && tn < b) {
      double dn;
      double fn = ls_psi_dpsi<DIM>(D, U0, A, tn * w, smin, &dn);
      if (fn >= 0.0) { a = tn; fa = fn; } else { b = tn; fb = fn; dfb = w * dn; fresh = true; }
    }
    // Near the root psi is evaluated below its rounding resolution (a change of t by an ulp leaves
    // U0 + t P unchanged), and the chord and tangent points then creep towards one end while the other
    // stays put: when the bracket has not halved, bisect, so that it always shrinks to ls_tol.
    if (b - a > 0.5 * width) {
      double tm = a + 0.5 * (b - a);
      if (!(tm > a && tm < b)) break;
      double fm = ls_psi<DIM>(D, U0, A, tm * w, smin);
      if (fm >= 0.0) { a = tm; fa = fm; } else { b = tm; fb = fm; fresh = false; }
    }
  }
  return a;
}

// The searches that need the tail are rare (well under 1% of the entries) but take ~10 iterations, and a
// lane that iterates holds up its whole warp; the sweep kernels therefore queue them (entry, row) and
// k_lsfix runs the tails with every lane busy.  Queue item: x = CSR entry e, or -(b + 1) for boundary
// entry b; y = row i.
__device__ __forceinline__ void ls_defer(const Scratch& S, int pass, int code, int i) {
  const unsigned k = atomicAdd(S.lsq_n + pass, 1u);
  S.lsq[k] = make_int2(code, i);
}

template <int DIM>
__device__ __forceinline__ void load_state(const double* U, int n, int i, double* out) {
#pragma unroll
  for (int q = 0; q < DIM + 2; ++q) out[q] = U[(size_t)q * n + i];
}

}  // namespace gdg
