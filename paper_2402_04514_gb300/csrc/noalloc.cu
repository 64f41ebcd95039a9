// gdg_max_dt_noalloc: the time step of the handle-based gdg_max_dt, for callers that must not
// allocate device memory.  The per-block partial minima live in a fixed file-scope device array
// instead of handle scratch; the per-node primitives are recomputed on the fly from U.
#include <cuda.h>

#include <cmath>
#include <mutex>

#include "gdg_internal.cuh"

namespace gdg {
namespace {

constexpr int kThreads = 256;
constexpr int kMaxBlocks = GDG_NOALLOC_MAX_NODES / kThreads;
static_assert(GDG_NOALLOC_MAX_NODES % kThreads == 0, "node limit must be a multiple of the block size");

// Scratch of every call: one partial minimum per block.  Every GPU that loads the library holds these
// 128 KB until the process exits.
static __device__ __align__(256) double g_noalloc_partial[kMaxBlocks];

// Address of g_noalloc_partial on each device, filled by the first call made with that device current,
// with the id of the context it was looked up in: after a device reset the runtime creates a new context
// and loads the module again, so a cached address is used only while the current context has that id.
std::mutex g_setup_mutex;
double* g_partial_ptr[64] = {nullptr};
unsigned long long g_partial_ctx[64] = {0};

// The driver's context calls, reached through the runtime (the library links only cudart).
using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

// Id of the current context (0 when it cannot be read: then every call looks the address up again).
unsigned long long current_context_id() {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<CtxGetCurrentFn>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<CtxGetIdFn>(f);
    cudaGetLastError();
  }
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS)
    return 0;
  return id;
}

struct NodePrim {
  double irho, p, ip, a, pme;
};

__device__ __forceinline__ NodePrim node_prim(const Dev& D, const double* U, int dim) {
  NodePrim r;
  double m2 = 0.0;
  for (int k = 0; k < dim; ++k) m2 += U[1 + k] * U[1 + k];
  r.irho = 1.0 / U[0];
  r.p = D.gm1 * (U[dim + 1] - 0.5 * m2 * r.irho);
  r.ip = 1.0 / r.p;
  r.a = sqrt(D.gamma * r.p * r.irho);
  r.pme = D.ie_root > 0 ? rootinv(r.p, D.root_ie) : pow(r.p, -D.e_exp);
  return r;
}

// Per node: -d_ii = sum_j |c_ij| lambda_max^+(U_i, U_j, n_ij) + sum_k |c_i^k| lambda_max^+(U_i, U^k, n_i^k)
// (Sec. 3.1, eq. (eq:dij_low_order_supplement)); then the block minimum of m_i / (2 |d_ii|) into
// partial[blockIdx.x].  A Dirichlet entry without data makes the node's value NaN.
template <int DIM>
__global__ void __launch_bounds__(kThreads) k_noalloc_partial(Dev D, gdg_dev_mesh M, const double* __restrict__ U,
                                                              const double* __restrict__ bdata,
                                                              double* __restrict__ partial) {
  constexpr int Mc = DIM + 2;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const size_t n = (size_t)M.n;
  double val = INFINITY;
  if (i < M.n) {
    double Ui[Mc];
    for (int q = 0; q < Mc; ++q) Ui[q] = U[q * n + i];
    NodePrim Pi = node_prim(D, Ui, DIM);
    double dsum = 0.0;
    for (int e = M.row_ptr[i]; e < M.row_ptr[i + 1]; ++e) {
      double c[DIM], c2 = 0.0;
      for (int k = 0; k < DIM; ++k) {
        c[k] = M.cij[(size_t)k * M.nnz + e];
        c2 += c[k] * c[k];
      }
      if (c2 == 0.0) continue;
      const double cn = sqrt(c2), icn = 1.0 / cn;
      const int j = M.col_idx[e];
      double Uj[Mc];
      for (int q = 0; q < Mc; ++q) Uj[q] = U[q * n + j];
      NodePrim Pj = node_prim(D, Uj, DIM);
      double uL = 0.0, uR = 0.0;
      for (int k = 0; k < DIM; ++k) {
        uL += Ui[1 + k] * c[k];
        uR += Uj[1 + k] * c[k];
      }
      uL *= icn * Pi.irho;
      uR *= icn * Pj.irho;
      dsum += cn * lambda_max(D, uL, Pi.p, Pi.ip, Pi.a, Pi.pme, uR, Pj.p, Pj.ip, Pj.a, Pj.pme);
    }
    for (int b = M.b_ptr[i]; b < M.b_ptr[i + 1]; ++b) {
      double nv[DIM], c2 = 0.0;
      for (int k = 0; k < DIM; ++k) {
        nv[k] = M.b_c[(size_t)k * M.nb + b];
        c2 += nv[k] * nv[k];
      }
      const double cn = sqrt(c2);
      for (int k = 0; k < DIM; ++k) nv[k] /= cn;
      double UB[Mc];
      if (M.b_type[b] == GDG_BC_DIRICHLET || M.b_type[b] == GDG_BC_INOUTFLOW) {
        if (!bdata) {
          dsum = NAN;
          break;
        }
        if (M.b_type[b] == GDG_BC_DIRICHLET) {
          for (int q = 0; q < Mc; ++q) UB[q] = bdata[(size_t)q * M.nb + b];
        } else {
          double Ud[Mc];
          for (int q = 0; q < Mc; ++q) Ud[q] = bdata[(size_t)q * M.nb + b];
          inoutflow_state<DIM>(D.gamma, Ui, Ud, nv, UB);
        }
      } else {
        double mn = 0.0;
        for (int k = 0; k < DIM; ++k) mn += Ui[1 + k] * nv[k];
        UB[0] = Ui[0];
        for (int k = 0; k < DIM; ++k) UB[1 + k] = Ui[1 + k] - 2.0 * mn * nv[k];
        UB[DIM + 1] = Ui[DIM + 1];
      }
      NodePrim PB = node_prim(D, UB, DIM);
      double uL = 0.0, uR = 0.0;
      for (int k = 0; k < DIM; ++k) {
        uL += Ui[1 + k] * nv[k];
        uR += UB[1 + k] * nv[k];
      }
      dsum += cn * lambda_max(D, uL * Pi.irho, Pi.p, Pi.ip, Pi.a, Pi.pme, uR * PB.irho, PB.p, PB.ip, PB.a, PB.pme);
    }
    if (dsum > 0.0) val = M.mi[i] / (2.0 * dsum);
    if (dsum != dsum) val = NAN;
  }
  __shared__ double red[kThreads / 32];
  __shared__ int bad[kThreads / 32];
  int isnan_ = val != val;
  double v = isnan_ ? INFINITY : val;
  for (int off = 16; off > 0; off >>= 1) {
    v = fmin(v, __shfl_xor_sync(0xffffffffu, v, off));
    isnan_ |= __shfl_xor_sync(0xffffffffu, isnan_, off);
  }
  if ((threadIdx.x & 31) == 0) {
    red[threadIdx.x >> 5] = v;
    bad[threadIdx.x >> 5] = isnan_;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = INFINITY;
    int anybad = 0;
    for (int w = 0; w < kThreads / 32; ++w) {
      m = fmin(m, red[w]);
      anybad |= bad[w];
    }
    partial[blockIdx.x] = anybad ? NAN : m;
  }
}

// tau = cfl * min over the first `count` partial minima (count = 0 gives +inf).
__global__ void k_noalloc_final(const double* __restrict__ partial, int count, double cfl, double* tau_out) {
  __shared__ double red[32];
  __shared__ int bad[32];
  double v = INFINITY;
  int isnan_ = 0;
  for (int b = threadIdx.x; b < count; b += blockDim.x) {
    double x = partial[b];
    if (x != x) isnan_ = 1; else v = fmin(v, x);
  }
  for (int off = 16; off > 0; off >>= 1) {
    v = fmin(v, __shfl_xor_sync(0xffffffffu, v, off));
    isnan_ |= __shfl_xor_sync(0xffffffffu, isnan_, off);
  }
  if ((threadIdx.x & 31) == 0) {
    red[threadIdx.x >> 5] = v;
    bad[threadIdx.x >> 5] = isnan_;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = INFINITY;
    int anybad = 0;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) {
      m = fmin(m, red[w]);
      anybad |= bad[w];
    }
    *tau_out = anybad ? NAN : (m < INFINITY ? cfl * m : INFINITY);
  }
}

// Looks up (once per device and context, under a lock) the device address of g_noalloc_partial.
int partial_buffer(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return GDG_ECUDA;
  if (dev < 0 || dev >= 64) return GDG_ENOTSUP;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  unsigned long long ctx = current_context_id();
  if (!g_partial_ptr[dev] || ctx == 0 || ctx != g_partial_ctx[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_partial) != cudaSuccess || !p) {
      cudaGetLastError();
      return GDG_ECUDA;
    }
    g_partial_ptr[dev] = static_cast<double*>(p);
    g_partial_ctx[dev] = ctx ? ctx : current_context_id();  // the lookup creates the context if it had none
  }
  *out = g_partial_ptr[dev];
  return GDG_OK;
}

template <int DIM>
cudaError_t launch_partial(const Dev& D, const gdg_dev_mesh& M, const double* U, const double* bdata, double* partial,
                           int blocks, cudaStream_t s) {
  k_noalloc_partial<DIM><<<blocks, kThreads, 0, s>>>(D, M, U, bdata, partial);
  return cudaGetLastError();
}

cudaError_t dispatch_partial(int dim, const Dev& D, const gdg_dev_mesh& M, const double* U, const double* bdata,
                             double* partial, int blocks, cudaStream_t s) {
  GDG_DISPATCH(dim, launch_partial, D, M, U, bdata, partial, blocks, s);
}

}  // namespace
}  // namespace gdg

extern "C" int gdg_max_dt_noalloc(const gdg_dev_mesh* mesh, const double* U, const double* bdata, double cfl,
                                  double* tau_out, void* stream) {
  if (!mesh || !tau_out || !(cfl > 0.0)) return GDG_EINVAL;
  const gdg_dev_mesh& M = *mesh;
  if (M.dim < 1 || M.dim > 3) return GDG_ENOTSUP;
  if (M.n < 0 || M.nnz < 0 || M.nb < 0 || !(M.gamma > 1.0)) return GDG_EINVAL;
  if (M.n > GDG_NOALLOC_MAX_NODES || M.nnz >= (int64_t(1) << 31) || M.nb >= (int64_t(1) << 31)) return GDG_ENOTSUP;
  if (M.n > 0 && (!U || !M.row_ptr || !M.mi || !M.b_ptr)) return GDG_EINVAL;
  if (M.nnz > 0 && (!M.col_idx || !M.cij)) return GDG_EINVAL;
  if (M.nb > 0 && (!M.b_c || !M.b_type)) return GDG_EINVAL;
  double* partial = nullptr;
  if (int rc = gdg::partial_buffer(&partial); rc != GDG_OK) return rc;
  gdg::Dev D{};
  gdg::set_eos(D, M.gamma);
  cudaStream_t s = (cudaStream_t)stream;
  const int blocks = (int)((M.n + gdg::kThreads - 1) / gdg::kThreads);
  if (blocks > 0 && gdg::dispatch_partial(M.dim, D, M, U, bdata, partial, blocks, s) != cudaSuccess) return GDG_ECUDA;
  gdg::k_noalloc_final<<<1, 1024, 0, s>>>(partial, blocks, cfl, tau_out);
  return cudaGetLastError() == cudaSuccess ? GDG_OK : GDG_ECUDA;
}
