// Serving (gdg_server_*): a request loop with continuous batching.  Requests (a mesh, an initial state,
// an end time) are accepted at any time.  A preparation thread admits them in arrival order as soon as
// their device footprint (gdg_footprint + state buffers) fits the HBM budget, sets them up and uploads
// their state.  The loop thread adds prepared requests to the batch of their element type (instances in
// one batch share the block shape), advances every batch by one fused SSP-RK3 step per iteration (each
// member with its own time step and end time), and retires members that reached their end time:
// their state is copied to the host, their device memory released, their slot and budget freed for the
// next arrivals.  State stays on the device from admission to completion.  The paper treats one problem
// at a time; serving is this library's.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <tuple>
#include <vector>

#include "gdg_internal.cuh"
#include "handle.cuh"

namespace {

struct Request {
  int64_t id = 0;
  // owned copies of the caller's inputs
  gdg_problem prob{};
  std::vector<int64_t> row_ptr;
  std::vector<int32_t> col, b_node, b_type;
  std::vector<double> cij, mi, MK, b_c, U0, bdata;
  std::vector<uint8_t> coloc;
  double t_end = 0.0, cfl = 0.5;
  int64_t footprint = 0;  // arena + three state buffers + Dirichlet data
  // device side
  gdg_handle* h = nullptr;
  double* dmem = nullptr;  // U, T1, T2 (and bdata) in one allocation
  double *U = nullptr, *T1 = nullptr, *T2 = nullptr, *bd = nullptr;
  // outcome
  std::vector<double> result;
  int status = GDG_OK;
  int32_t flags = 0;
  int64_t steps = 0;
  double t_submit = 0.0, t_start = 0.0, t_done = 0.0, t_final = 0.0;
  bool done = false;
};

using Key = std::tuple<int, int, int, int, int>;  // dim, n_loc, order, passes, precision: a batch's members share them

struct Lane {
  std::vector<Request*> members;
  gdg_batch* batch = nullptr;
  bool dirty = false;
};

double seconds_since(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace

struct gdg_server {
  int device = 0;
  int64_t budget = 0;
  std::chrono::steady_clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv_prep, cv_loop, cv_done;
  std::deque<Request*> queue;   // submitted, waiting for budget
  std::deque<Request*> ready;   // set up, waiting to join a batch
  std::map<int64_t, std::unique_ptr<Request>> all;
  int64_t next_id = 1, in_use = 0, active = 0, iterations = 0;
  bool stop = false, prep_busy = false;
  std::thread prep, loop;
  cudaStream_t prep_stream = nullptr, loop_stream = nullptr;
  int* done_dev = nullptr;      // [cap] finished flags of one lane's members
  int* done_host = nullptr;     // pinned copy
  int cap = 0;
};

namespace {

void release_device(Request* r) {
  if (r->h) gdg_destroy(r->h);
  r->h = nullptr;
  if (r->dmem) cudaFree(r->dmem);
  r->dmem = nullptr;
}

// Setup of one admitted request on the preparation thread: handle, state buffers, upload, clock.
int prepare(gdg_server* s, Request* r) {
  int rc = gdg_setup(&r->prob, &r->h);
  if (rc != GDG_OK) return rc;
  const size_t mn = (size_t)(r->prob.dim + 2) * r->prob.n, mb = (size_t)(r->prob.dim + 2) * r->prob.nb;
  const size_t words = 3 * mn + (r->bdata.empty() ? 0 : mb);
  if (cudaMalloc(&r->dmem, sizeof(double) * std::max<size_t>(words, 1)) != cudaSuccess) {
    cudaGetLastError();
    r->dmem = nullptr;
    return GDG_ENOMEM;
  }
  r->U = r->dmem;
  r->T1 = r->U + mn;
  r->T2 = r->T1 + mn;
  r->bd = r->bdata.empty() ? nullptr : r->T2 + mn;
  cudaError_t e = cudaMemcpyAsync(r->U, r->U0.data(), sizeof(double) * mn, cudaMemcpyHostToDevice, s->prep_stream);
  if (e == cudaSuccess && r->bd)
    e = cudaMemcpyAsync(r->bd, r->bdata.data(), sizeof(double) * mb, cudaMemcpyHostToDevice, s->prep_stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return GDG_ECUDA;
  }
  rc = gdg_clock_set(r->h, 0.0, r->t_end, r->cfl, s->prep_stream);  // synchronises the preparation stream
  if (rc != GDG_OK) return rc;
  // the host copies of the inputs are no longer needed
  std::vector<int64_t>().swap(r->row_ptr);
  std::vector<int32_t>().swap(r->col);
  std::vector<int32_t>().swap(r->b_node);
  std::vector<int32_t>().swap(r->b_type);
  std::vector<double>().swap(r->cij);
  std::vector<double>().swap(r->mi);
  std::vector<double>().swap(r->MK);
  std::vector<double>().swap(r->b_c);
  std::vector<double>().swap(r->U0);
  std::vector<double>().swap(r->bdata);
  std::vector<uint8_t>().swap(r->coloc);
  return GDG_OK;
}

void prep_main(gdg_server* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    // FIFO admission: the oldest request waits until its footprint fits the budget
    s->cv_prep.wait(lk, [&] {
      return (s->stop && s->queue.empty()) ||
             (!s->queue.empty() && s->in_use + s->queue.front()->footprint <= s->budget);
    });
    if (s->queue.empty()) return;
    Request* r = s->queue.front();
    s->queue.pop_front();
    s->in_use += r->footprint;
    s->prep_busy = true;
    lk.unlock();
    const int rc = prepare(s, r);
    lk.lock();
    s->prep_busy = false;
    if (rc != GDG_OK) {
      release_device(r);
      s->in_use -= r->footprint;
      r->status = rc;
      r->t_start = r->t_done = seconds_since(s->t0);
      r->done = true;
      s->cv_done.notify_all();
      s->cv_prep.notify_all();
    } else {
      s->ready.push_back(r);
    }
    s->cv_loop.notify_all();
  }
}

// finished[k] = 1 when member k's clock has reached its end time
__global__ void k_finished(gdg::Clock* const* clks, int n, int* finished) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) finished[k] = !(clks[k]->t < clks[k]->t_end);
}

struct LaneDev {
  gdg::Clock** clks = nullptr;  // device [cap]
  int cap = 0;
  cudaStream_t stream = nullptr;  // each batch runs on its own stream, so batches of different kinds overlap
};

// Steps per completion check: a member that finished in between only takes no-op steps (its kernels
// return at once), and the loop synchronises with the device once per kSteps steps.
constexpr int kSteps = 4;

int rebuild(Lane& L, LaneDev& LD, cudaStream_t s) {
  if (L.batch) gdg_batch_destroy(L.batch);
  L.batch = nullptr;
  L.dirty = false;
  const int n = (int)L.members.size();
  if (n == 0) return GDG_OK;
  std::vector<gdg_handle*> hs(n);
  std::vector<double*> U(n), T1(n), T2(n);
  std::vector<const double*> bd(n);
  std::vector<gdg::Clock*> clks(n);
  for (int k = 0; k < n; ++k) {
    Request* r = L.members[k];
    hs[k] = r->h;
    U[k] = r->U;
    T1[k] = r->T1;
    T2[k] = r->T2;
    bd[k] = r->bd;
    clks[k] = r->h->clk;
  }
  int rc = gdg_batch_create(hs.data(), n, U.data(), T1.data(), T2.data(), bd.data(), &L.batch);
  if (rc != GDG_OK) return rc;
  if (n > LD.cap) {
    if (LD.clks) cudaFree(LD.clks);
    LD.cap = std::max(n, 2 * LD.cap);
    if (cudaMalloc(&LD.clks, sizeof(gdg::Clock*) * LD.cap) != cudaSuccess) {
      cudaGetLastError();
      LD.clks = nullptr;
      LD.cap = 0;
      return GDG_ENOMEM;
    }
  }
  if (cudaMemcpyAsync(LD.clks, clks.data(), sizeof(gdg::Clock*) * n, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return GDG_ECUDA;
  }
  return GDG_OK;
}

void fail_member(gdg_server* s, Request* r, int rc) {
  release_device(r);
  std::lock_guard<std::mutex> lk(s->mu);
  s->in_use -= r->footprint;
  s->active -= 1;
  r->status = rc;
  r->t_done = seconds_since(s->t0);
  r->done = true;
  s->cv_done.notify_all();
  s->cv_prep.notify_all();
}

void loop_main(gdg_server* s) {
  cudaSetDevice(s->device);
  std::map<Key, Lane> lanes;
  std::map<Key, LaneDev> lanedev;
  for (;;) {
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_loop.wait(lk, [&] {
        return !s->ready.empty() || s->active > 0 || (s->stop && s->queue.empty() && !s->prep_busy);
      });
      const double now = seconds_since(s->t0);
      while (!s->ready.empty()) {
        Request* r = s->ready.front();
        s->ready.pop_front();
        const Key key{r->prob.dim, r->prob.n_loc, r->prob.params.order, r->prob.params.limiter_passes,
                      r->prob.params.precision};
        Lane& L = lanes[key];
        L.members.push_back(r);
        L.dirty = true;
        r->t_start = now;
        s->active += 1;
      }
      if (s->active == 0) {
        if (s->stop && s->queue.empty() && !s->prep_busy) break;
        continue;
      }
      s->iterations += 1;
    }
    // one step of every batch, then the finished members of each
    std::vector<std::pair<Lane*, LaneDev*>> live;
    for (auto& kv : lanes) {
      Lane& L = kv.second;
      LaneDev& LD = lanedev[kv.first];
      if (L.members.empty()) continue;
      if (!LD.stream && cudaStreamCreateWithFlags(&LD.stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        LD.stream = nullptr;
        for (Request* r : L.members) fail_member(s, r, GDG_ECUDA);
        L.members.clear();
        continue;
      }
      if (L.dirty) {
        const int rc = rebuild(L, LD, LD.stream);
        if (rc != GDG_OK) {  // the batch could not be formed: its members fail
          for (Request* r : L.members) fail_member(s, r, rc);
          L.members.clear();
          continue;
        }
      }
      int rc = GDG_OK;
      for (int q = 0; q < kSteps && rc == GDG_OK; ++q) rc = gdg_batch_step(L.batch, LD.stream);
      if (rc != GDG_OK) {
        for (Request* r : L.members) fail_member(s, r, rc);
        L.members.clear();
        L.dirty = true;
        continue;
      }
      live.emplace_back(&L, &LD);
    }
    int total = 0;
    for (auto& p : live) total += (int)p.first->members.size();
    if (total > s->cap) {
      if (s->done_dev) cudaFree(s->done_dev);
      if (s->done_host) cudaFreeHost(s->done_host);
      s->cap = std::max(total, 2 * s->cap);
      if (cudaMalloc(&s->done_dev, sizeof(int) * s->cap) != cudaSuccess ||
          cudaMallocHost(&s->done_host, sizeof(int) * s->cap) != cudaSuccess) {
        cudaGetLastError();
        s->done_dev = nullptr;
        s->done_host = nullptr;
        s->cap = 0;
      }
    }
    int off = 0;
    bool ok = s->done_dev != nullptr || total == 0;
    for (auto& p : live) {
      const int n = (int)p.first->members.size();
      cudaStream_t ls = p.second->stream;
      if (ok && n > 0) {
        k_finished<<<(n + 127) / 128, 128, 0, ls>>>(p.second->clks, n, s->done_dev + off);
        ok = cudaMemcpyAsync(s->done_host + off, s->done_dev + off, sizeof(int) * n, cudaMemcpyDeviceToHost, ls) ==
             cudaSuccess;
      }
      off += n;
    }
    for (auto& p : live) ok = (cudaStreamSynchronize(p.second->stream) == cudaSuccess) && ok;
    off = 0;
    for (auto& p : live) {
      Lane& L = *p.first;
      const int n = (int)L.members.size();
      std::vector<Request*> keep;
      for (int k = 0; k < n; ++k) {
        Request* r = L.members[k];
        if (!ok) {
          fail_member(s, r, GDG_ECUDA);
          continue;
        }
        if (!s->done_host[off + k]) {
          keep.push_back(r);
          continue;
        }
        // retire: result to the host, device memory released
        const size_t mn = (size_t)(r->prob.dim + 2) * r->prob.n;
        r->result.resize(mn);
        int rc = GDG_OK;
        if (mn && (cudaMemcpyAsync(r->result.data(), r->U, sizeof(double) * mn, cudaMemcpyDeviceToHost,
                                   s->loop_stream) != cudaSuccess ||
                   cudaStreamSynchronize(s->loop_stream) != cudaSuccess)) {
          cudaGetLastError();
          rc = GDG_ECUDA;
        }
        int32_t flags = 0;
        double t = 0.0, tau = 0.0;
        int64_t steps = 0;
        if (rc == GDG_OK) rc = gdg_status(r->h, &flags, 0, s->loop_stream);
        if (rc == GDG_OK) rc = gdg_clock_get(r->h, &t, &tau, &steps, s->loop_stream);
        release_device(r);
        std::lock_guard<std::mutex> lk(s->mu);
        s->in_use -= r->footprint;
        s->active -= 1;
        r->status = rc;
        r->flags = flags;
        r->steps = steps;
        r->t_final = t;
        r->t_done = seconds_since(s->t0);
        r->done = true;
        s->cv_done.notify_all();
        s->cv_prep.notify_all();
      }
      off += n;
      if (keep.size() != L.members.size()) {
        L.members.swap(keep);
        L.dirty = true;
      }
    }
  }
  for (auto& kv : lanes)
    if (kv.second.batch) gdg_batch_destroy(kv.second.batch);
  for (auto& kv : lanedev) {
    if (kv.second.clks) cudaFree(kv.second.clks);
    if (kv.second.stream) cudaStreamDestroy(kv.second.stream);
  }
}

}  // namespace

extern "C" {

int gdg_server_create(int64_t hbm_budget_bytes, gdg_server** out) {
  if (!out) return GDG_EINVAL;
  *out = nullptr;
  gdg_server* s = new (std::nothrow) gdg_server;
  if (!s) return GDG_ENOMEM;
  cudaGetDevice(&s->device);
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    cudaGetLastError();
    delete s;
    return GDG_ECUDA;
  }
  s->budget = hbm_budget_bytes > 0 ? hbm_budget_bytes : (int64_t)(0.8 * (double)free_b);
  if (cudaStreamCreateWithFlags(&s->prep_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s->loop_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    if (s->prep_stream) cudaStreamDestroy(s->prep_stream);
    delete s;
    return GDG_ECUDA;
  }
  s->t0 = std::chrono::steady_clock::now();
  s->prep = std::thread(prep_main, s);
  s->loop = std::thread(loop_main, s);
  *out = s;
  return GDG_OK;
}

int gdg_server_submit(gdg_server* s, const gdg_problem* P, const double* U0, const double* bdata, double t_end,
                      double cfl, int64_t* id_out) {
  if (!s || !P || !id_out || !(t_end >= 0.0) || !std::isfinite(t_end) || !(cfl > 0.0) || !std::isfinite(cfl))
    return GDG_EINVAL;
  if (P->n > 0 && !U0) return GDG_EINVAL;
  int64_t arena = 0;
  if (int rc = gdg_footprint(P, &arena); rc != GDG_OK) return rc;
  std::unique_ptr<Request> r(new (std::nothrow) Request);
  if (!r) return GDG_ENOMEM;
  const int m = P->dim + 2;
  const int64_t n = P->n, nnz = P->nnz, nb = P->nb, nel = P->n / std::max(1, P->n_loc);
  bool dirichlet = false;
  for (int64_t b = 0; b < nb && P->b_type; ++b) dirichlet = dirichlet || P->b_type[b] != GDG_BC_SLIP;  // data needed
  if (dirichlet && !bdata) return GDG_EINVAL;
  r->footprint = arena + (int64_t)sizeof(double) * (3 * m * n + (dirichlet ? m * nb : 0)) + 4096;
  if (r->footprint > s->budget) return GDG_ENOMEM;  // could never be admitted
  auto cp = [](auto& dst, const auto* src, int64_t count) {
    if (src && count > 0) dst.assign(src, src + count);
  };
  cp(r->row_ptr, P->row_ptr, n + 1);
  cp(r->col, P->col_idx, nnz);
  cp(r->cij, P->cij, (int64_t)P->dim * nnz);
  cp(r->coloc, P->coloc, nnz);
  cp(r->mi, P->mi, n);
  cp(r->MK, P->MK, nel * P->n_loc * P->n_loc);
  cp(r->b_node, P->b_node, nb);
  cp(r->b_c, P->b_c, (int64_t)P->dim * nb);
  cp(r->b_type, P->b_type, nb);
  cp(r->U0, U0, m * n);
  if (dirichlet) cp(r->bdata, bdata, m * nb);
  r->prob = *P;
  r->prob.row_ptr = r->row_ptr.empty() ? nullptr : r->row_ptr.data();
  r->prob.col_idx = r->col.empty() ? nullptr : r->col.data();
  r->prob.cij = r->cij.empty() ? nullptr : r->cij.data();
  r->prob.coloc = r->coloc.empty() ? nullptr : r->coloc.data();
  r->prob.mi = r->mi.empty() ? nullptr : r->mi.data();
  r->prob.MK = r->MK.empty() ? nullptr : r->MK.data();
  r->prob.b_node = r->b_node.empty() ? nullptr : r->b_node.data();
  r->prob.b_c = r->b_c.empty() ? nullptr : r->b_c.data();
  r->prob.b_type = r->b_type.empty() ? nullptr : r->b_type.data();
  r->t_end = t_end;
  r->cfl = cfl;
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stop) return GDG_EINVAL;
  r->id = s->next_id++;
  r->t_submit = seconds_since(s->t0);
  *id_out = r->id;
  s->queue.push_back(r.get());
  s->all.emplace(r->id, std::move(r));
  s->cv_prep.notify_all();
  return GDG_OK;
}

int gdg_server_wait(gdg_server* s, int64_t id, double timeout_s, double* U_out, gdg_request_info* info) {
  if (!s) return GDG_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->all.find(id);
  if (it == s->all.end()) return GDG_EINVAL;
  Request* r = it->second.get();
  auto pred = [&] { return r->done; };
  if (timeout_s < 0) {
    s->cv_done.wait(lk, pred);
  } else if (!s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), pred)) {
    return GDG_ETIMEOUT;
  }
  if (U_out && r->status == GDG_OK && !r->result.empty())
    std::memcpy(U_out, r->result.data(), sizeof(double) * r->result.size());
  if (info) {
    info->t_submit = r->t_submit;
    info->t_start = r->t_start;
    info->t_done = r->t_done;
    info->t_final = r->t_final;
    info->steps = r->steps;
    info->status = r->status;
    info->flags = r->flags;
    info->device_bytes = r->footprint;
  }
  const int rc = r->status;
  s->all.erase(it);
  return rc;
}

int gdg_server_stats(gdg_server* s, gdg_server_info* info) {
  if (!s || !info) return GDG_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  info->queued = (int64_t)s->queue.size() + (int64_t)s->ready.size() + (s->prep_busy ? 1 : 0);
  info->active = s->active;
  info->bytes_in_use = s->in_use;
  info->budget = s->budget;
  info->iterations = s->iterations;
  info->now = seconds_since(s->t0);
  return GDG_OK;
}

void gdg_server_destroy(gdg_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_prep.notify_all();
  s->cv_loop.notify_all();
  if (s->prep.joinable()) s->prep.join();
  s->cv_loop.notify_all();
  if (s->loop.joinable()) s->loop.join();
  for (auto& kv : s->all) release_device(kv.second.get());
  if (s->done_dev) cudaFree(s->done_dev);
  if (s->done_host) cudaFreeHost(s->done_host);
  cudaStreamDestroy(s->prep_stream);
  cudaStreamDestroy(s->loop_stream);
  delete s;
}

}  // extern "C"
