// Batches (gdg_batch_*): many independent instances (gdg handles, each with its own mesh, scratch, state
// buffers and clock) advanced by fused SSP-RK3 steps in which every kernel of the sweep is one launch over
// all instances.  A block of such a launch finds its instance from the batch's per-kernel block offsets
// (gdg::Many); each instance keeps its own time step (its clock), so instances of different sizes, speeds
// and end times share the launches.  The paper treats one problem at a time; batching is this library's.
#include <algorithm>
#include <cmath>
#include <vector>

#include "gdg_internal.cuh"
#include "handle.cuh"

struct gdg_batch {
  int device = 0, dim = 0, n_loc = 0, order = 0, passes = 0, count = 0;
  bool mixed = false;                  // precision of every member (GDG_PRECISION_MIXED)
  gdg::Sched sched = gdg::default_sched();  // launch shapes (gdg_batch_autotune)
  std::vector<gdg_handle*> hs;
  void* mem = nullptr;                 // device: context tables and block offsets
  gdg::Ctx* ctx[3] = {nullptr, nullptr, nullptr};  // [count] contexts of the three stages
  int* start[gdg::KN_COUNT] = {};      // [count + 1] block offsets of each kernel
  long long blocks[gdg::KN_COUNT] = {};
  // persistent mode (gdg_batch_set_persistent): one cooperative launch per stage of pblock threads, the
  // element sweep in blocks of peb elements; pstart [KN_COUNT][count + 1] the virtual block offsets
  bool persistent = false;
  int pblock = 0, peb = 0;
  int* pstart = nullptr;
  long long pblocks[gdg::KN_COUNT] = {};
  // kernel timing, as gdg_profile
  struct Rec {
    int kernel;
    cudaEvent_t a, b;
  };
  bool profiling = false;
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  // the step as a CUDA graph (captured on the first step on a non-default stream, replayed after)
  cudaGraphExec_t exec = nullptr;
  bool graph_failed = false;
};

namespace {

int cuda_fail_b(cudaError_t) {
  cudaGetLastError();
  return GDG_ECUDA;
}

cudaError_t launch_many(const gdg_batch* b, int kern, int stage, int arg, cudaStream_t s) {
  const gdg::Many m{b->ctx[stage], b->start[kern], b->count};
  const long long blocks = b->blocks[kern];
  switch (kern) {
    case gdg::KN_HIGH:
      return gdg::launch_high_file_many(b->dim, b->mixed, m, b->n_loc, blocks,
                                        gdg::high_elems_per_block(b->n_loc, b->sched.high_cap), s);
    case gdg::KN_LIMIT2:
    case gdg::KN_FINAL:
    case gdg::KN_LSFIX:
      return gdg::launch_limit_file_many(kern, b->dim, m, blocks, b->sched.bt[kern], (b->sched.slices >> kern) & 1,
                                         arg, s);
    default:
      return gdg::launch_low_file_many(kern, b->dim, b->mixed, m, blocks, b->sched.bt[kern],
                                       (b->sched.slices >> kern) & 1, arg, s);
  }
}

// Block offsets of every kernel under a schedule into a host table, and the totals.
int offsets(const gdg_batch* b, const gdg::Sched& sc, std::vector<int>& start, long long* blocks) {
  start.assign((size_t)gdg::KN_COUNT * (b->count + 1), 0);
  for (int kern = 0; kern < gdg::KN_COUNT; ++kern) {
    long long acc = 0;
    int* st = &start[(size_t)kern * (b->count + 1)];
    for (int k = 0; k < b->count; ++k) {
      st[k] = (int)acc;
      acc += gdg::kernel_blocks(kern, b->hs[k]->D, sc);
    }
    st[b->count] = (int)acc;
    if (acc > 0x7fffffffLL) return GDG_ENOTSUP;  // more blocks than a grid holds
    blocks[kern] = acc;
  }
  return GDG_OK;
}

// Block offsets of every kernel under the batch's schedule, and those of the persistent mode (every
// phase in blocks of pblock threads, the element sweep in the largest block of whole ELL-group parts that
// fits them), uploaded into the batch's tables (synchronous).
int upload_offsets(gdg_batch* b) {
  std::vector<int> start, pstart;
  if (int rc = offsets(b, b->sched, start, b->blocks); rc != GDG_OK) return rc;
  b->peb = gdg::high_elems_per_block(b->n_loc, gdg::kHighMaxBlock);
  b->pblock = gdg::high_threads(b->n_loc, b->peb);
  gdg::Sched ps = b->sched;
  for (int k = 0; k < gdg::KN_COUNT; ++k) ps.bt[k] = b->pblock;
  ps.high_cap = b->peb * b->n_loc;
  if (int rc = offsets(b, ps, pstart, b->pblocks); rc != GDG_OK) return rc;
  if (cudaMemcpy(b->start[0], start.data(), sizeof(int) * start.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b->pstart, pstart.data(), sizeof(int) * pstart.size(), cudaMemcpyHostToDevice) != cudaSuccess)
    return cuda_fail_b(cudaErrorUnknown);
  if (b->exec) {  // the captured step has the old shapes
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  return GDG_OK;
}

template <class F>
cudaError_t btimed(gdg_batch* b, int kernel, cudaStream_t s, F&& launch) {
  if (!b->profiling) return launch();
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  for (cudaEvent_t* e : {&e0, &e1}) {
    if (!b->pool.empty()) {
      *e = b->pool.back();
      b->pool.pop_back();
    } else if (cudaEventCreate(e) != cudaSuccess) {
      return cudaErrorMemoryAllocation;
    }
  }
  cudaEventRecord(e0, s);
  cudaError_t e = launch();
  cudaEventRecord(e1, s);
  b->recs.push_back({kernel, e0, e1});
  return e;
}

void release(gdg_batch* b) {
  for (auto& r : b->recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto e : b->pool) cudaEventDestroy(e);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->mem) cudaFree(b->mem);
  delete b;
}

// The launches of one fused SSP-RK3 step of every member.
int step_launches(gdg_batch* b, cudaStream_t s) {
  const bool low_only = b->order == GDG_ORDER_LOW || (b->order == GDG_ORDER_LIMITED && b->passes == 0);
  cudaError_t e;
  for (int stage = 0; stage < 3; ++stage) {
    auto go = [&](int id, int kern, int arg) {
      return btimed(b, id, s, [&] { return launch_many(b, kern, stage, arg, s); });
    };
    if ((e = go(GDG_K_PRIM, gdg::KN_PRIM, 0)) != cudaSuccess) return cuda_fail_b(e);
    if ((e = go(GDG_K_EDGE, gdg::KN_EDGE, 0)) != cudaSuccess) return cuda_fail_b(e);
    if (stage == 0 && (e = go(GDG_K_TAU, gdg::KN_TAU, 0)) != cudaSuccess) return cuda_fail_b(e);
    if ((e = go(GDG_K_LOW, gdg::KN_LOW, low_only ? 1 : 0)) != cudaSuccess) return cuda_fail_b(e);
    if (low_only) continue;
    if ((e = go(GDG_K_HIGH, gdg::KN_HIGH, 0)) != cudaSuccess) return cuda_fail_b(e);
    if (b->order == GDG_ORDER_HIGH) continue;
    if ((e = go(GDG_K_LSFIX, gdg::KN_LSFIX, 0)) != cudaSuccess) return cuda_fail_b(e);
    if ((e = go(GDG_K_LIMIT2, gdg::KN_LIMIT2, b->passes == 1 ? 1 : 0)) != cudaSuccess) return cuda_fail_b(e);
    if (b->passes == 1) continue;
    if ((e = go(GDG_K_LSFIX, gdg::KN_LSFIX, 1)) != cudaSuccess) return cuda_fail_b(e);
    if ((e = go(GDG_K_FINAL, gdg::KN_FINAL, 0)) != cudaSuccess) return cuda_fail_b(e);
  }
  e = btimed(b, GDG_K_CLOCK, s, [&] { return gdg::launch_clock_many(b->ctx[0], b->count, s); });
  return e == cudaSuccess ? GDG_OK : cuda_fail_b(e);
}

// One fused SSP-RK3 step of every member in persistent mode: one cooperative launch per stage (the last
// one also advances the clocks).
int persistent_step(gdg_batch* b, cudaStream_t s) {
  const bool low_only = b->order == GDG_ORDER_LOW || (b->order == GDG_ORDER_LIMITED && b->passes == 0);
  for (int stage = 0; stage < 3; ++stage) {
    gdg::PersistArgs a{};
    a.ctx = b->ctx[stage];
    a.start = b->pstart;
    a.ninst = b->count;
    a.stage = stage;
    a.eb = b->peb;
    a.low_only = low_only ? 1 : 0;
    a.order = b->order;
    a.passes = b->passes;
    a.slices = b->sched.slices;
    for (int k = 0; k < gdg::KN_COUNT; ++k) a.nblk[k] = (int)b->pblocks[k];
    int grid = 0;
    cudaError_t e = gdg::launch_stage_persistent(b->dim, b->mixed, a, b->pblock, &grid, s);
    if (e != cudaSuccess) return e == cudaErrorNotSupported ? GDG_ENOTSUP : cuda_fail_b(e);
  }
  return GDG_OK;
}

}  // namespace

extern "C" {

int gdg_batch_create(gdg_handle* const* handles, int32_t count, double* const* U, double* const* T1,
                     double* const* T2, const double* const* bdata, gdg_batch** out) {
  if (!out) return GDG_EINVAL;
  *out = nullptr;
  if (!handles || count < 1 || !U || !T1 || !T2) return GDG_EINVAL;
  const gdg_handle* h0 = handles[0];
  if (!h0) return GDG_EINVAL;
  int dev = 0;
  cudaGetDevice(&dev);
  for (int k = 0; k < count; ++k) {
    const gdg_handle* h = handles[k];
    if (!h || h->device != dev || h->dim != h0->dim || h->n_loc != h0->n_loc || h->D.order != h0->D.order ||
        h->D.passes != h0->D.passes || h->D.mixed != h0->D.mixed)
      return GDG_EINVAL;
    if (h->n > 0 && (!U[k] || !T1[k] || !T2[k] || U[k] == T1[k] || U[k] == T2[k] || T1[k] == T2[k]))
      return GDG_EINVAL;
    if (h->has_dirichlet && !(bdata && bdata[k])) return GDG_EINVAL;
    for (int q = 0; q < k; ++q)
      if (handles[q] == h) return GDG_EINVAL;  // an instance's scratch and clock serve one member
  }
  gdg_batch* b = new (std::nothrow) gdg_batch;
  if (!b) return GDG_ENOMEM;
  b->device = dev;
  b->dim = h0->dim;
  b->n_loc = h0->n_loc;
  b->order = h0->D.order;
  b->passes = h0->D.passes;
  b->mixed = h0->D.mixed != 0;
  b->count = count;
  b->hs.assign(handles, handles + count);
  // host tables: contexts of the three stages (Shu-Osher SSP-RK3, the last stage in place) and the
  // block offsets of every kernel
  std::vector<gdg::Ctx> ctx((size_t)3 * count);
  for (int k = 0; k < count; ++k) {
    gdg_handle* h = handles[k];
    const double* bd = bdata ? bdata[k] : nullptr;
    ctx[k] = make_ctx(h, U[k], nullptr, T1[k], bd, 0.0, 0.0, h->clk);
    ctx[(size_t)count + k] = make_ctx(h, T1[k], U[k], T2[k], bd, 0.75, 0.0, h->clk);
    ctx[(size_t)2 * count + k] = make_ctx(h, T2[k], U[k], U[k], bd, 1.0 / 3.0, 0.0, h->clk);
  }
  const size_t ctx_bytes = sizeof(gdg::Ctx) * ctx.size();
  const size_t start_bytes = sizeof(int) * (size_t)gdg::KN_COUNT * (count + 1);
  cudaError_t e = cudaMalloc(&b->mem, ctx_bytes + 2 * start_bytes);
  if (e != cudaSuccess) {
    b->mem = nullptr;
    cudaGetLastError();
    release(b);
    return GDG_ENOMEM;
  }
  char* base = (char*)b->mem;
  if ((e = cudaMemcpy(base, ctx.data(), ctx_bytes, cudaMemcpyHostToDevice)) != cudaSuccess) {
    release(b);
    return cuda_fail_b(e);
  }
  for (int st = 0; st < 3; ++st) b->ctx[st] = (gdg::Ctx*)base + (size_t)st * count;
  for (int kern = 0; kern < gdg::KN_COUNT; ++kern)
    b->start[kern] = (int*)(base + ctx_bytes) + (size_t)kern * (count + 1);
  b->pstart = (int*)(base + ctx_bytes + start_bytes);
  if (int rc = upload_offsets(b); rc != GDG_OK) {
    release(b);
    return rc;
  }
  *out = b;
  return GDG_OK;
}

int gdg_batch_step(gdg_batch* b, void* stream) {
  if (!b) return GDG_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  if (b->persistent) return persistent_step(b, s);
  // Every step launches the same kernels with the same arguments (the members' time steps live on the
  // device), so the step is captured once as a CUDA graph and replayed: one launch instead of ~26.  Not
  // on the legacy default stream (which cannot be captured) nor while profiling.
  if (b->profiling || s == nullptr || b->graph_failed) return step_launches(b, s);
  if (!b->exec) {
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      b->graph_failed = true;
      return step_launches(b, s);
    }
    const int rc = step_launches(b, s);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(s, &g);
    if (e == cudaSuccess && rc == GDG_OK && g) e = cudaGraphInstantiate(&b->exec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (rc != GDG_OK || e != cudaSuccess || !b->exec) {
      cudaGetLastError();
      b->exec = nullptr;
      b->graph_failed = true;
      return step_launches(b, s);
    }
  }
  const cudaError_t e = cudaGraphLaunch(b->exec, s);
  return e == cudaSuccess ? GDG_OK : cuda_fail_b(e);
}

int gdg_batch_profile(gdg_batch* b, int32_t enable) {
  if (!b) return GDG_EINVAL;
  for (auto& r : b->recs) {
    b->pool.push_back(r.a);
    b->pool.push_back(r.b);
  }
  b->recs.clear();
  b->profiling = enable != 0;
  return GDG_OK;
}

int gdg_batch_profile_read(gdg_batch* b, double* total_ms, int64_t* launches) {
  if (!b || !total_ms || !launches) return GDG_EINVAL;
  for (int k = 0; k < GDG_NKERNELS; ++k) {
    total_ms[k] = 0.0;
    launches[k] = 0;
  }
  int rc = GDG_OK;
  for (auto& r : b->recs) {
    float ms = 0.f;
    cudaError_t e = cudaEventSynchronize(r.b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, r.a, r.b);
    if (e != cudaSuccess) rc = cuda_fail_b(e);
    total_ms[r.kernel] += ms;
    launches[r.kernel] += 1;
    b->pool.push_back(r.a);
    b->pool.push_back(r.b);
  }
  b->recs.clear();
  return rc;
}

int gdg_batch_autotune(gdg_batch* b, int32_t trials, void* stream) {
  if (!b) return GDG_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  // the members' states (the third stage's output U of each member) and clocks
  std::vector<double*> U(b->count);
  std::vector<size_t> bytes(b->count), off(b->count);
  size_t total = 0;
  for (int k = 0; k < b->count; ++k) {
    const gdg_handle* h = b->hs[k];
    bytes[k] = sizeof(double) * (size_t)(h->dim + 2) * h->n;
    off[k] = total;
    total += bytes[k];
  }
  // member k's U is the stage-3 output: read it back from the context table
  std::vector<gdg::Ctx> c3(b->count);
  cudaError_t e = cudaMemcpy(c3.data(), b->ctx[2], sizeof(gdg::Ctx) * b->count, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail_b(e);
  for (int k = 0; k < b->count; ++k) U[k] = c3[k].Uout;
  char* save = nullptr;
  if ((e = cudaMalloc(&save, std::max<size_t>(total, 1))) != cudaSuccess) {
    cudaGetLastError();
    return GDG_ENOMEM;
  }
  std::vector<gdg::Clock> clk0(b->count), tune(b->count);
  std::vector<unsigned> flags0(b->count);
  for (int k = 0; k < b->count && e == cudaSuccess; ++k) {
    if (bytes[k]) e = cudaMemcpyAsync(save + off[k], U[k], bytes[k], cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(&clk0[k], b->hs[k]->clk, sizeof(gdg::Clock), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(&flags0[k], b->hs[k]->S.flags, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cudaFree(save);
    return cuda_fail_b(e);
  }
  for (int k = 0; k < b->count; ++k) {  // members that already reached t_end would time no-op steps
    tune[k] = clk0[k];
    tune[k].t_end = INFINITY;
    tune[k].tau_bits = gdg::kTauNone;
  }
  auto put_back = [&](const std::vector<gdg::Clock>& ck) -> int {
    cudaError_t r = cudaSuccess;
    for (int k = 0; k < b->count && r == cudaSuccess; ++k) {
      if (bytes[k]) r = cudaMemcpyAsync(U[k], save + off[k], bytes[k], cudaMemcpyDeviceToDevice, s);
      if (r == cudaSuccess)
        r = cudaMemcpyAsync(b->hs[k]->clk, &ck[k], sizeof(gdg::Clock), cudaMemcpyHostToDevice, s);
      if (r == cudaSuccess)
        r = cudaMemcpyAsync(b->hs[k]->S.flags, &flags0[k], sizeof(unsigned), cudaMemcpyHostToDevice, s);
    }
    if (r == cudaSuccess) r = cudaStreamSynchronize(s);
    return r == cudaSuccess ? GDG_OK : cuda_fail_b(r);
  };
  const bool prof0 = b->profiling;
  gdg_batch_profile(b, 1);
  int rc = autotune_schedule(
      b->sched, b->n_loc, trials,
      [&](const gdg::Sched& sc) {
        b->sched = sc;
        return upload_offsets(b);
      },
      [&] { return gdg_batch_step(b, stream); },
      [&](double* ms) {
        double tot[GDG_NKERNELS];
        int64_t cnt[GDG_NKERNELS];
        const int r = gdg_batch_profile_read(b, tot, cnt);
        for (int k = 0; k < GDG_NKERNELS; ++k) ms[k] = cnt[k] ? tot[k] / (double)cnt[k] : 0.0;
        return r;
      },
      [&] { return put_back(tune); });
  gdg_batch_profile(b, prof0 ? 1 : 0);
  const int rc2 = put_back(clk0);
  cudaFree(save);
  return rc != GDG_OK ? rc : rc2;
}

int gdg_batch_set_persistent(gdg_batch* b, int32_t on) {
  if (!b || (on != 0 && on != 1)) return GDG_EINVAL;
  b->persistent = on != 0;
  return GDG_OK;
}

int gdg_batch_get_schedule(gdg_batch* b, gdg_schedule* out) {
  if (!b || !out) return GDG_EINVAL;
  sched_to_public(b->sched, out);
  return GDG_OK;
}

int gdg_batch_set_schedule(gdg_batch* b, const gdg_schedule* in) {
  if (!b || !in) return GDG_EINVAL;
  gdg::Sched sc;
  if (!sched_from_public(in, &sc)) return GDG_EINVAL;
  b->sched = sc;
  return upload_offsets(b);
}

void gdg_batch_destroy(gdg_batch* b) {
  if (b) release(b);
}

}  // extern "C"
