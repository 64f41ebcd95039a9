// Batches in persistent mode: one cooperative launch per SSP-RK3 stage runs every kernel of the stage for
// every member, with a grid-wide barrier where the sweep has a grid-wide dependency.  The kernel bodies are
// the ones of the per-kernel launches (included below), so the results are the same bits; only the
// launch structure differs: 3 launches per step instead of 26.
#include <cooperative_groups.h>

#define GDG_BODIES_ONLY
#include "kernels_low.cu"
#include "kernels_high.cu"
#include "kernels_limit.cu"
#undef GDG_BODIES_ONLY

namespace gdg {

namespace {

// The source of one virtual block of a phase: virtual block vb of the phase's grid belongs to the last
// instance k with start[k] <= vb (the batch's block offsets for that kernel, computed for the persistent
// block size), exactly as Many maps blockIdx.x.  Every thread of the block must call get().
struct Virt {
  const Ctx* ctx;
  const int* start;
  int ninst;
  int vb;
  __device__ __forceinline__ int instance() const {
    int lo = 0, hi = ninst - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (start[mid] <= vb) lo = mid; else hi = mid - 1;
    }
    return lo;
  }
  __device__ __forceinline__ unsigned queue_length(int pass, int* lb) const {
    const int k = instance();
    *lb = vb - start[k];
    return ctx[k].S.lsq_n[pass];
  }
  __device__ __forceinline__ const Ctx& get(Ctx* smem, int* lb, int* nblk = nullptr) const {
    const int k = instance();
    *lb = vb - start[k];
    if (nblk) *nblk = start[k + 1] - start[k];
    const int* src = reinterpret_cast<const int*>(ctx + k);
    int* dst = reinterpret_cast<int*>(smem);
    for (int w = threadIdx.x; w < (int)(sizeof(Ctx) / sizeof(int)); w += blockDim.x) dst[w] = src[w];
    __syncthreads();
    return *smem;
  }
};

// Every virtual block of one phase, spread over the co-resident blocks, then a grid-wide barrier: the
// next phase reads what this one wrote for neighbouring rows of any block.
template <class Body>
__device__ __forceinline__ void phase(const PersistArgs& a, int kern, cooperative_groups::grid_group& grid,
                                      Body&& body) {
  const int* start = a.start + (size_t)kern * (a.ninst + 1);
  for (int vb = blockIdx.x; vb < a.nblk[kern]; vb += gridDim.x) {
    body(Virt{a.ctx, start, a.ninst, vb});
    __syncthreads();  // the next virtual block's context copy reuses the shared context
  }
  grid.sync();
}

// One stage of the fused SSP-RK3 step of every member (the launch sequence of a batch step, gdg_batch_step,
// as phases of one launch); the last stage also advances the members' clocks.
template <int DIM, bool MX>
__global__ void __launch_bounds__(kHighMaxBlock) k_stage_persistent(PersistArgs a) {
  cooperative_groups::grid_group grid = cooperative_groups::this_grid();
  const int sl_low = (a.slices >> KN_LOW) & 1, sl_lim = (a.slices >> KN_LIMIT2) & 1;
  const int sl_fin = (a.slices >> KN_FINAL) & 1, sl_tau = (a.slices >> KN_TAU) & 1;
  phase(a, KN_PRIM, grid, [&](const Virt& v) { prim_body<DIM, MX, Virt>(v); });
  phase(a, KN_EDGE, grid, [&](const Virt& v) { edge_body<DIM, MX, Virt>(v); });
  if (a.stage == 0) phase(a, KN_TAU, grid, [&](const Virt& v) { tau_body<DIM, MX, Virt>(v, sl_tau); });
  phase(a, KN_LOW, grid, [&](const Virt& v) { low_body<DIM, MX, Virt>(v, sl_low, a.low_only); });
  if (!a.low_only) {
    phase(a, KN_HIGH, grid, [&](const Virt& v) { high_sweep<DIM, MX, Virt>(v, a.eb); });
    if (a.order != GDG_ORDER_HIGH) {
      phase(a, KN_LSFIX, grid, [&](const Virt& v) { lsfix_body<DIM, Virt>(v, 0); });
      phase(a, KN_LIMIT2, grid, [&](const Virt& v) { limit2_body<DIM, Virt>(v, sl_lim, a.passes == 1); });
      if (a.passes != 1) {
        phase(a, KN_LSFIX, grid, [&](const Virt& v) { lsfix_body<DIM, Virt>(v, 1); });
        phase(a, KN_FINAL, grid, [&](const Virt& v) { final_body<DIM, Virt>(v, sl_fin); });
      }
    }
  }
  if (a.stage == 2)
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < a.ninst; k += gridDim.x * blockDim.x)
      clock_advance(a.ctx[k].clk, a.ctx[k].dt_factor);
}

template <int DIM, bool MX>
cudaError_t persistent_launch(const PersistArgs& a, int block, int* grid_out, cudaStream_t s) {
  const void* fn = (const void*)k_stage_persistent<DIM, MX>;
  int dev = 0, sms = 0, per_sm = 0, coop = 0;
  cudaError_t e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev)) != cudaSuccess) return e;
  if (!coop) return cudaErrorNotSupported;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, block, 0)) != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int grid = per_sm * sms;  // every block co-resident, as the grid-wide barrier requires
  *grid_out = grid;
  PersistArgs args = a;
  void* params[] = {&args};
  return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(block), params, 0, s);
}

}  // namespace

cudaError_t launch_stage_persistent(int dim, bool mixed, const PersistArgs& a, int block, int* grid,
                                    cudaStream_t s) {
  switch (dim * 2 + (mixed ? 1 : 0)) {
    case 2: return persistent_launch<1, false>(a, block, grid, s);
    case 3: return persistent_launch<1, true>(a, block, grid, s);
    case 4: return persistent_launch<2, false>(a, block, grid, s);
    case 5: return persistent_launch<2, true>(a, block, grid, s);
    case 6: return persistent_launch<3, false>(a, block, grid, s);
    case 7: return persistent_launch<3, true>(a, block, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace gdg
