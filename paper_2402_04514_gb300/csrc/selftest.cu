// Device self-test of the FP64 helpers the sweep uses in place of CUDA's division and power
// (gdg_math_selftest): runs one helper, or CUDA's own reference operation, over a device array.
#include "gdg_internal.cuh"

namespace gdg {
namespace {

__global__ void k_math(int fn, int q, const double* __restrict__ x, double* __restrict__ y, long long n) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double v = x[i];
  switch (fn) {
    case 0: y[i] = rcp64(v); break;
    case 1: y[i] = rootinv(v, root_q(q)); break;
    case 2: y[i] = 1.0 / v; break;
    case 3: y[i] = pow(v, -1.0 / q); break;
    case 4: y[i] = f2d_fast(d2f_fast(v)); break;
    case 5: y[i] = sqrt64(v); break;
    case 6: y[i] = sqrt(v); break;
    default: y[i] = 0.0;
  }
}

// The integer-pipe binary64 product and sum against the FP64 instructions: pairs (x[2i], x[2i+1]).
__global__ void k_math2(int fn, const double* __restrict__ x, double* __restrict__ y, long long n) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double a = x[2 * i], b = x[2 * i + 1];
  switch (fn) {
    case 7: y[i] = sf::mul(a, b); break;
    case 8: y[i] = __dmul_rn(a, b); break;
    case 9: y[i] = sf::add(a, b); break;
    case 10: y[i] = __dadd_rn(a, b); break;
    case 11: y[i] = sf::mul_pow2(a, (int)b); break;
    default: y[i] = 0.0;
  }
}

}  // namespace
}  // namespace gdg

extern "C" int gdg_math_selftest(int32_t fn, int32_t q, const double* x, double* y, int64_t n, void* stream) {
  if (fn < 0 || fn > 11 || q < 1 || q > 16 || n < 0 || (n > 0 && (!x || !y))) return GDG_EINVAL;
  if (n == 0) return GDG_OK;
  int threads = 256;
  long long blocks = (n + threads - 1) / threads;
  if (fn >= 7)
    gdg::k_math2<<<(unsigned)blocks, threads, 0, (cudaStream_t)stream>>>(fn, x, y, n);
  else
    gdg::k_math<<<(unsigned)blocks, threads, 0, (cudaStream_t)stream>>>(fn, q, x, y, n);
  return cudaGetLastError() == cudaSuccess ? GDG_OK : GDG_ECUDA;
}

// ------------------------------------------------------------------------------------------------
// The mixed path's wave-speed bound against the FP64 path's (gdg_wave_speed_check): both from the
// primitives their own k_prim computes, for one-dimensional states (rho, u, p) on each side.
namespace gdg {
namespace {

__global__ void k_wave(Dev D, const double* __restrict__ st, double* __restrict__ out, long long n) {
  long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const double* s = st + 6 * k;
  const double rL = s[0], uL = s[1], pL = s[2], rR = s[3], uR = s[4], pR = s[5];
  const double irL = 1.0 / rL, irR = 1.0 / rR;
  double ipL, aL, pmeL, ipR, aR, pmeR;
  prim_fp64(D, irL, pL, &ipL, &aL, &pmeL);
  prim_fp64(D, irR, pR, &ipR, &aR, &pmeR);
  const double lam64 = lambda_max(D, uL, pL, ipL, aL, pmeL, uR, pR, ipR, aR, pmeR);
  const PrimF Lf = prim_mx(D, rL, pL), Rf = prim_mx(D, rR, pR);
  float raw = 0.f, scale = 0.f;
  lambda_max_mx(D, to_f32(uL), to_f32(pL), Lf, to_f32(uR), to_f32(pR), Rf, &raw, &scale);
  const double lmx = lambda_pair<true>(D, uL, pL, irL, to_f64(Lf.ip), to_f64(Lf.a), to_f64(Lf.pme), uR, pR, irR,
                                       to_f64(Rf.ip), to_f64(Rf.a), to_f64(Rf.pme));
  out[4 * k + 0] = lam64;
  out[4 * k + 1] = lmx;
  out[4 * k + 2] = to_f64(raw);
  out[4 * k + 3] = to_f64(scale);
}

}  // namespace
}  // namespace gdg

extern "C" int gdg_wave_speed_check(double gamma, const double* states, double* out, int64_t n, void* stream) {
  if (!(gamma > 1.0) || n < 0 || (n > 0 && (!states || !out))) return GDG_EINVAL;
  if (n == 0) return GDG_OK;
  gdg::Dev D{};
  gdg::set_eos(D, gamma);
  const int threads = 256;
  const long long blocks = (n + threads - 1) / threads;
  gdg::k_wave<<<(unsigned)blocks, threads, 0, (cudaStream_t)stream>>>(D, states, out, n);
  return cudaGetLastError() == cudaSuccess ? GDG_OK : GDG_ECUDA;
}

// ------------------------------------------------------------------------------------------------
// The FP32 entropy certificate of the line search (gdg_certificate_check): for given U0, A, s_min and s,
// whether ls_certified proves psi(s) >= 0, and psi(s) in FP64.
namespace gdg {
namespace {

template <int DIM>
__global__ void k_cert(Dev D, const double* __restrict__ in, double* __restrict__ out, long long n) {
  constexpr int M = DIM + 2;
  long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const double* r = in + (2 * M + 2) * k;
  double U0[M], A[M];
#pragma unroll
  for (int q = 0; q < M; ++q) {
    U0[q] = r[q];
    A[q] = r[M + q];
  }
  const double smin = r[2 * M], sv = r[2 * M + 1];
  LsRow<DIM> c;
  ls_row<DIM>(D, c, U0, 0.0, INFINITY, smin);
  out[2 * k] = ls_certified<DIM>(D, c, A, d2f_fast(sv)) ? 1.0 : 0.0;
  out[2 * k + 1] = ls_psi<DIM>(D, U0, A, sv, smin);
}

}  // namespace
}  // namespace gdg

extern "C" int gdg_certificate_check(int32_t dim, double gamma, const double* in, double* out, int64_t n,
                                     void* stream) {
  if (dim < 1 || dim > 3 || !(gamma > 1.0) || n < 0 || (n > 0 && (!in || !out))) return GDG_EINVAL;
  if (n == 0) return GDG_OK;
  gdg::Dev D{};
  gdg::set_eos(D, gamma);
  const int threads = 256;
  const unsigned blocks = (unsigned)((n + threads - 1) / threads);
  cudaStream_t s = (cudaStream_t)stream;
  switch (dim) {
    case 1: gdg::k_cert<1><<<blocks, threads, 0, s>>>(D, in, out, n); break;
    case 2: gdg::k_cert<2><<<blocks, threads, 0, s>>>(D, in, out, n); break;
    default: gdg::k_cert<3><<<blocks, threads, 0, s>>>(D, in, out, n); break;
  }
  return cudaGetLastError() == cudaSuccess ? GDG_OK : GDG_ECUDA;
}

// ------------------------------------------------------------------------------------------------
// Throughput of the arithmetic the sweep is made of (gdg_fp64_throughput): every thread runs ILP
// independent chains of one operation; the result is operations per second over the whole GPU.
namespace gdg {
namespace {

constexpr int kIlp = 8;

template <int OP>
__global__ void k_rate(double* out, int iters, double a, double b) {
  double x[kIlp];
#pragma unroll
  for (int k = 0; k < kIlp; ++k) x[k] = 1.0 + 1e-3 * (threadIdx.x & 63) + 0.01 * k;
  float xf[kIlp];
#pragma unroll
  for (int k = 0; k < kIlp; ++k) xf[k] = (float)x[k];
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < kIlp; ++k) {
      if (OP == 0) x[k] = fma(x[k], a, b);                 // DFMA
      if (OP == 1) x[k] = a / x[k] + b;                    // FP64 division
      if (OP == 2) x[k] = sqrt(x[k]) + b;                  // FP64 square root
      if (OP == 3) x[k] = pow(x[k], a) + b;                // FP64 power
      if (OP == 4) xf[k] = fmaf(xf[k], (float)a, (float)b);  // FFMA
      if (OP == 5) x[k] = rcp64(x[k]) + b;                 // reciprocal of this library
      if (OP == 6) x[k] = rootinv(x[k], root_q(5)) + b;            // x^{-1/5} of this library
      if (OP == 7) x[k] = (double)((float)x[k] * 0.5f) + b;  // FP64 -> FP32 -> FP64 conversion pair
      if (OP == 8) x[k] = x[k] * a;                                  // DMUL
      if (OP == 9) x[k] = sf::mul(x[k], a);                          // product on the integer pipe
      if (OP == 10) x[k] = k < kIlp / 2 ? sf::mul(x[k], a) : x[k] * a;  // half the chains on each pipe
      if (OP == 11) x[k] = x[k] + (k & 1 ? b : -b);                  // DADD
      if (OP == 12) x[k] = sf::add(x[k], k & 1 ? b : -b);            // sum on the integer pipe
      if (OP == 13) x[k] = k < kIlp / 4 ? sf::add(x[k], k & 1 ? b : -b) : x[k] + (k & 1 ? b : -b);  // a quarter
    }
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kIlp; ++k) s += x[k] + xf[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <int OP>
cudaError_t run_rate(int blocks, int threads, int iters, double* buf, cudaStream_t s, float* ms) {
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double a = (OP == 3) ? 0.3 : (OP >= 8 && OP <= 10) ? 0.9999 : 0.999;
  double b = (OP == 0 || OP == 4 || OP >= 11) ? 1e-3 : 0.5;
  k_rate<OP><<<blocks, threads, 0, s>>>(buf, iters, a, b);  // warm-up
  cudaEventRecord(e0, s);
  k_rate<OP><<<blocks, threads, 0, s>>>(buf, iters, a, b);
  cudaEventRecord(e1, s);
  cudaError_t err = cudaEventSynchronize(e1);
  cudaEventElapsedTime(ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return err == cudaSuccess ? cudaGetLastError() : err;
}

}  // namespace
}  // namespace gdg

extern "C" int gdg_fp64_throughput(int32_t op, double* ops_per_s, void* stream) {
  if (op < 0 || op > 13 || !ops_per_s) return GDG_EINVAL;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int threads = 256, blocks = sms * 8;
  const int iters[14] = {4096, 256, 256, 32, 16384, 512, 128, 1024, 4096, 2048, 4096, 4096, 2048, 4096};
  double* buf = nullptr;
  if (cudaMalloc(&buf, sizeof(double) * blocks * threads) != cudaSuccess) return GDG_ENOMEM;
  float ms = 0.f;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  switch (op) {
    case 0: e = gdg::run_rate<0>(blocks, threads, iters[0], buf, s, &ms); break;
    case 1: e = gdg::run_rate<1>(blocks, threads, iters[1], buf, s, &ms); break;
    case 2: e = gdg::run_rate<2>(blocks, threads, iters[2], buf, s, &ms); break;
    case 3: e = gdg::run_rate<3>(blocks, threads, iters[3], buf, s, &ms); break;
    case 4: e = gdg::run_rate<4>(blocks, threads, iters[4], buf, s, &ms); break;
    case 5: e = gdg::run_rate<5>(blocks, threads, iters[5], buf, s, &ms); break;
    case 6: e = gdg::run_rate<6>(blocks, threads, iters[6], buf, s, &ms); break;
    case 7: e = gdg::run_rate<7>(blocks, threads, iters[7], buf, s, &ms); break;
    case 8: e = gdg::run_rate<8>(blocks, threads, iters[8], buf, s, &ms); break;
    case 9: e = gdg::run_rate<9>(blocks, threads, iters[9], buf, s, &ms); break;
    case 10: e = gdg::run_rate<10>(blocks, threads, iters[10], buf, s, &ms); break;
    case 11: e = gdg::run_rate<11>(blocks, threads, iters[11], buf, s, &ms); break;
    case 12: e = gdg::run_rate<12>(blocks, threads, iters[12], buf, s, &ms); break;
    default: e = gdg::run_rate<13>(blocks, threads, iters[13], buf, s, &ms); break;
  }
  cudaFree(buf);
  if (e != cudaSuccess) return GDG_ECUDA;
  *ops_per_s = (double)blocks * threads * gdg::kIlp * iters[op] / (ms * 1e-3);
  return GDG_OK;
}
