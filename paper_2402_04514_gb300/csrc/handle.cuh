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
  int sms = 1;                   // multiprocessors of the device (grid of the deferred line searches)
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
  c.Ubase = Ubase;
  c.Uout = Uout;
  c.bdata = bdata;
  c.alpha = alpha;
  c.tau = tau;
  c.clk = clk;
  return c;
}

