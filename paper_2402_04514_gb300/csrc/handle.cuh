// Private to the library: the handle behind gdg_handle (gdg_abi.cu) and the helpers that gdg_abi.cu and
// batch.cu share to build stage contexts and time kernel launches.
#pragma once

#include <vector>

#include "gdg_internal.cuh"

struct gdg_handle {
  int device = 0;
  int dim = 0, degree = 0, n_loc = 0;
  int64_t n = 0, nnz = 0, nb = 0;
  double gamma = 1.4, omega = 1.0;
  gdg_params params{};
  bool has_dirichlet = false;
  void* arena = nullptr;
  size_t arena_bytes = 0;
  gdg::Dev D{};
  gdg::Scratch S{};
  // host copies needed after setup
  std::vector<int> row_ptr, col, tr, borig, bnode_sorted;
  std::vector<int> eorig;  // caller's index of each CSR entry q (rows are stencil-first on the device)
  std::vector<int> epos;   // position of CSR entry q in the device's sliced-ELL arrays
  int64_t nnz_ell = 0;     // length of the device's per-entry arrays (padding included)
  std::vector<uint8_t> coloc;
  std::vector<double> mi;
  // device pointers of the parameter-dependent arrays
  double *d_mu = nullptr, *d_rminus = nullptr, *d_rplus = nullptr, *d_muB = nullptr;
  // kernel timing (gdg_profile)
  struct Rec {
    int kernel;
    cudaEvent_t a, b;
  };
  bool profiling = false;
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  gdg::Sched sched = gdg::default_sched();  // launch shapes (gdg_autotune)
  gdg::Clock* clk = nullptr;     // device clock of the fused step (in the arena)
};

namespace gdg_detail {

inline cudaEvent_t take_event(gdg_handle* h) {
  if (!h->pool.empty()) {
    cudaEvent_t e = h->pool.back();
    h->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

// Runs one launcher, bracketed by events when profiling.
template <class F>
inline cudaError_t timed(gdg_handle* h, int kernel, cudaStream_t s, F&& launch) {
  if (!h->profiling) return launch();
  cudaEvent_t a = take_event(h), b = take_event(h);
  if (!a || !b) return cudaErrorMemoryAllocation;
  cudaEventRecord(a, s);
  cudaError_t e = launch();
  cudaEventRecord(b, s);
  h->recs.push_back({kernel, a, b});
  return e;
}

}  // namespace gdg_detail

using gdg_detail::take_event;
using gdg_detail::timed;


inline gdg::Ctx make_ctx(const gdg_handle* h, const double* U, const double* Ubase, double* Uout,
                         const double* bdata, double alpha, double tau, gdg::Clock* clk) {
  gdg::Ctx c{};
  c.D = h->D;
  c.S = h->S;
  c.U = U;
  c.Ucopy = nullptr;
  c.Uhost = nullptr;
  c.Ubase = Ubase;
  c.Uout = Uout;
  c.bdata = bdata;
  c.alpha = alpha;
  c.Ubase2 = nullptr;
  c.alpha2 = 0.0;
  c.w_fe = 0.0;
  c.tau = tau;
  c.clk = clk;
  c.tau_scale = 1.0;
  c.dt_factor = 1.0;
  return c;
}


// Launch-shape autotuning shared by handles and batches (gdg_autotune, gdg_batch_autotune).  Coordinate
// descent over three groups of knobs, each candidate timed over `trials` fused steps from the same saved
// state (restore() puts state and clocks back before every candidate and at the end):
//   1. threads per block of the one-thread-per-row/edge kernels, 128, 256 or 512, chosen per kernel
//      (all row kernels take the candidate together; each keeps its own fastest); then the row order
//      (node order or ELL slice order) of the kernels with per-entry loops, each keeping the faster;
//   2. the element sweep's block: 32, 16, 8 or 4 elements of one ELL group (the cap eb * n_loc), those
//      that fit kHighMaxBlock nodes;
//   3. the queue slots per thread of the deferred line-search grid, 1, 4 or 16.
// apply(sc) installs a schedule, step() runs one fused step with kernel timing on, kernel_ms(ms) returns
// the mean ms per launch of each GDG_K_* kernel since the last call.
template <class Apply, class Step, class Read, class Restore>
int autotune_schedule(gdg::Sched& sched, int n_loc, int trials, Apply apply, Step step, Read kernel_ms,
                      Restore restore) {
  if (trials < 1) trials = 1;
  static const int row_kern[][2] = {{gdg::KN_PRIM, GDG_K_PRIM},   {gdg::KN_EDGE, GDG_K_EDGE},
                                    {gdg::KN_TAU, GDG_K_TAU},     {gdg::KN_LOW, GDG_K_LOW},
                                    {gdg::KN_LIMIT2, GDG_K_LIMIT2}, {gdg::KN_FINAL, GDG_K_FINAL}};
  gdg::Sched sc = sched;
  double ms[GDG_NKERNELS];
  auto trial = [&](const gdg::Sched& cand, double* out) -> int {
    if (int rc = restore(); rc != GDG_OK) return rc;
    if (int rc = apply(cand); rc != GDG_OK) return rc;
    if (int rc = step(); rc != GDG_OK) return rc;  // warm-up: first launches of new shapes
    if (int rc = kernel_ms(out); rc != GDG_OK) return rc;
    for (int t = 0; t < trials; ++t)
      if (int rc = step(); rc != GDG_OK) return rc;
    return kernel_ms(out);
  };
  // 1. row kernels
  const int bts[3] = {128, 256, 512};
  double best_row[6];
  for (int r = 0; r < 6; ++r) best_row[r] = 1e300;
  for (int bt : bts) {
    gdg::Sched cand = sc;
    for (auto& rk : row_kern) cand.bt[rk[0]] = bt;
    if (int rc = trial(cand, ms); rc != GDG_OK) return rc;
    for (int r = 0; r < 6; ++r)
      if (ms[row_kern[r][1]] > 0.0 && ms[row_kern[r][1]] < best_row[r]) {
        best_row[r] = ms[row_kern[r][1]];
        sc.bt[row_kern[r][0]] = bt;
      }
  }
  // 1b. row order of the kernels with per-entry loops: node order or ELL slice order, each kernel keeps
  //     the faster (k_maxdt is not part of a fused step and keeps its order)
  {
    static const int order_kern[][2] = {{gdg::KN_TAU, GDG_K_TAU}, {gdg::KN_LOW, GDG_K_LOW},
                                        {gdg::KN_LIMIT2, GDG_K_LIMIT2}, {gdg::KN_FINAL, GDG_K_FINAL}};
    double t_on[4], t_off[4];
    gdg::Sched cand = sc;
    for (auto& ok : order_kern) cand.slices |= 1 << ok[0];
    if (int rc = trial(cand, ms); rc != GDG_OK) return rc;
    for (int r = 0; r < 4; ++r) t_on[r] = ms[order_kern[r][1]];
    for (auto& ok : order_kern) cand.slices &= ~(1 << ok[0]);
    if (int rc = trial(cand, ms); rc != GDG_OK) return rc;
    for (int r = 0; r < 4; ++r) {
      t_off[r] = ms[order_kern[r][1]];
      if (t_off[r] > 0.0 && t_off[r] < t_on[r])
        sc.slices &= ~(1 << order_kern[r][0]);
      else
        sc.slices |= 1 << order_kern[r][0];
    }
  }
  // 2. element sweep block: eb = 32, 16, 8, 4 elements (parts of one ELL group), the cap eb * n_loc
  double best = 1e300;
  int best_cap = sc.high_cap;
  for (int eb = gdg::kEll; eb >= 4; eb >>= 1) {
    const int cap = eb * n_loc;
    if (cap > gdg::kHighMaxBlock) continue;
    gdg::Sched cand = sc;
    cand.high_cap = cap;
    if (int rc = trial(cand, ms); rc != GDG_OK) return rc;
    if (ms[GDG_K_HIGH] > 0.0 && ms[GDG_K_HIGH] < best) {
      best = ms[GDG_K_HIGH];
      best_cap = cap;
    }
  }
  sc.high_cap = best_cap;
  // 3. deferred line-search grid
  best = 1e300;
  int best_slots = sc.lsfix_slots;
  for (int slots : {1, 4, 16}) {
    gdg::Sched cand = sc;
    cand.lsfix_slots = slots;
    if (int rc = trial(cand, ms); rc != GDG_OK) return rc;
    if (ms[GDG_K_LSFIX] < best) {
      best = ms[GDG_K_LSFIX];
      best_slots = slots;
    }
  }
  sc.lsfix_slots = best_slots;
  if (int rc = restore(); rc != GDG_OK) return rc;
  if (int rc = apply(sc); rc != GDG_OK) return rc;
  sched = sc;
  return GDG_OK;
}

// Public <-> internal schedule.
inline void sched_to_public(const gdg::Sched& sc, gdg_schedule* out) {
  out->prim_threads = sc.bt[gdg::KN_PRIM];
  out->edge_threads = sc.bt[gdg::KN_EDGE];
  out->tau_threads = sc.bt[gdg::KN_TAU];
  out->low_threads = sc.bt[gdg::KN_LOW];
  out->limit2_threads = sc.bt[gdg::KN_LIMIT2];
  out->final_threads = sc.bt[gdg::KN_FINAL];
  out->maxdt_threads = sc.bt[gdg::KN_MAXDT];
  out->high_block_cap = sc.high_cap;
  out->lsfix_slots = sc.lsfix_slots;
  static const int map[][2] = {{gdg::KN_MAXDT, GDG_K_MAXDT}, {gdg::KN_LOW, GDG_K_LOW}, {gdg::KN_LIMIT2, GDG_K_LIMIT2},
                               {gdg::KN_FINAL, GDG_K_FINAL}, {gdg::KN_TAU, GDG_K_TAU}};
  out->row_slices = 0;
  for (auto& mp : map)
    if ((sc.slices >> mp[0]) & 1) out->row_slices |= 1 << mp[1];
}

inline bool sched_from_public(const gdg_schedule* in, gdg::Sched* sc) {
  const int32_t t[7] = {in->prim_threads, in->edge_threads,  in->tau_threads,  in->low_threads,
                        in->limit2_threads, in->final_threads, in->maxdt_threads};
  for (int32_t v : t)
    if (v != 128 && v != 256 && v != 512) return false;
  if (in->high_block_cap < 1 || in->high_block_cap > gdg::kHighMaxBlock) return false;
  if (in->lsfix_slots < 1 || in->lsfix_slots > 1024) return false;
  const int public_sliceable = (1 << GDG_K_MAXDT) | (1 << GDG_K_LOW) | (1 << GDG_K_LIMIT2) | (1 << GDG_K_FINAL) |
                               (1 << GDG_K_TAU);
  if (in->row_slices & ~public_sliceable) return false;
  *sc = gdg::default_sched();
  sc->bt[gdg::KN_PRIM] = in->prim_threads;
  sc->bt[gdg::KN_EDGE] = in->edge_threads;
  sc->bt[gdg::KN_TAU] = in->tau_threads;
  sc->bt[gdg::KN_LOW] = in->low_threads;
  sc->bt[gdg::KN_LIMIT2] = in->limit2_threads;
  sc->bt[gdg::KN_FINAL] = in->final_threads;
  sc->bt[gdg::KN_MAXDT] = in->maxdt_threads;
  sc->high_cap = in->high_block_cap;
  sc->lsfix_slots = in->lsfix_slots;
  static const int map[][2] = {{gdg::KN_MAXDT, GDG_K_MAXDT}, {gdg::KN_LOW, GDG_K_LOW}, {gdg::KN_LIMIT2, GDG_K_LIMIT2},
                               {gdg::KN_FINAL, GDG_K_FINAL}, {gdg::KN_TAU, GDG_K_TAU}};
  sc->slices = 0;
  for (auto& mp : map)
    if ((in->row_slices >> mp[1]) & 1) sc->slices |= 1 << mp[0];
  return true;
}
