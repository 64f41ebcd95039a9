// C ABI of the gdg library (include/gdg.h): problem validation, derived per-entry / per-node data,
// one device arena per handle, and the kernel sequence of a stage.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "gdg_internal.cuh"

#include "handle.cuh"

using gdg::Dev;
using gdg::Scratch;

namespace {

template <class F>
void parallel_for(int64_t count, F&& f) {
  unsigned hw = std::thread::hardware_concurrency();
  int nt = (int)std::min<int64_t>(std::max(1u, std::min(hw, 32u)), std::max<int64_t>(1, count / 65536));
  if (nt <= 1) {
    f(0, count);
    return;
  }
  std::vector<std::thread> th;
  int64_t chunk = (count + nt - 1) / nt;
  for (int t = 0; t < nt; ++t) {
    int64_t b = t * chunk, e = std::min(count, b + chunk);
    if (b < e) th.emplace_back([&f, b, e] { f(b, e); });
  }
  for (auto& x : th) x.join();
}

bool check_params(const gdg_params& p) {
  if (p.order < GDG_ORDER_LOW || p.order > GDG_ORDER_LIMITED) return false;
  if (p.limiter_passes < 0 || p.limiter_passes > 2) return false;
  if (p.bounds_mode < 0 || p.bounds_mode > 1) return false;
  if (!(p.c_k >= 0) || !(p.c_ev >= 0) || !(p.c_r >= 0) || !std::isfinite(p.p_k) || !std::isfinite(p.p_r))
    return false;
  if (!(p.ls_tol > 0) || p.ls_maxit < 0) return false;
  if (p.precision != GDG_PRECISION_FP64 && p.precision != GDG_PRECISION_MIXED) return false;
  if (p.relax_measure != GDG_RELAX_NODE && p.relax_measure != GDG_RELAX_ELEMENT) return false;
  return true;
}

// Invert a symmetric positive definite block by Cholesky; returns false if not SPD.
bool spd_inverse(const double* A, int nl, double* Ainv) {
  std::vector<double> L(nl * nl, 0.0);
  for (int j = 0; j < nl; ++j) {
    double s = A[j * nl + j];
    for (int k = 0; k < j; ++k) s -= L[j * nl + k] * L[j * nl + k];
    if (!(s > 0.0)) return false;
    L[j * nl + j] = std::sqrt(s);
    for (int i = j + 1; i < nl; ++i) {
      double t = A[i * nl + j];
      for (int k = 0; k < j; ++k) t -= L[i * nl + k] * L[j * nl + k];
      L[i * nl + j] = t / L[j * nl + j];
    }
  }
  for (int c = 0; c < nl; ++c) {  // solve L L^T x = e_c
    std::vector<double> y(nl, 0.0);
    for (int i = 0; i < nl; ++i) {
      double s = (i == c) ? 1.0 : 0.0;
      for (int k = 0; k < i; ++k) s -= L[i * nl + k] * y[k];
      y[i] = s / L[i * nl + i];
    }
    for (int i = nl - 1; i >= 0; --i) {
      double s = y[i];
      for (int k = i + 1; k < nl; ++k) s -= L[k * nl + i] * y[k];
      y[i] = s / L[i * nl + i];
    }
    for (int i = 0; i < nl; ++i) Ainv[i * nl + c] = y[i];
  }
  for (int i = 0; i < nl; ++i)  // symmetrise
    for (int j = i + 1; j < nl; ++j) {
      double v = 0.5 * (Ainv[i * nl + j] + Ainv[j * nl + i]);
      Ainv[i * nl + j] = Ainv[j * nl + i] = v;
    }
  return true;
}

struct Arena {
  size_t off = 0;
  template <class T>
  size_t take(size_t count) {
    size_t o = off;
    off += (count * sizeof(T) + 255) / 256 * 256;
    if (count == 0) off += 256;
    return o;
  }
};

// The device arena of a handle: every array with its element type and count (m = dim + 2 components,
// nnz the length of the sliced-ELL per-entry arrays, ne canonical stencil edges, nel the elements rounded
// up to whole ELL groups, of nl nodes).  gdg_setup allocates it; gdg_footprint sizes it.
#define GDG_ARENA(X)                                                                                       \
  X(rbeg, int, n) X(rend, int, n) X(sten, int, n) X(col, int, nnz) X(tr, int, nnz) X(cnorm, double, nnz) X(cn, double, dim * nnz)   \
  X(mij, double, nnz) X(mu, double, nnz) X(mi, double, n) X(imi, double, n) X(ikm, double, n)             \
  X(rm, double, n) X(rp, double, n) X(muB, double, n) X(bptr, int, n + 1) X(bnorm, double, nb)           \
  X(bn, double, dim * nb) X(btype, int, nb) X(borig, int, nb) X(minv, double, nel * nl * nl)             \
  X(ee, int, ne) X(ei, int, ne) X(G, double, m * nnz) X(barR, double, nnz) X(barS, double, nnz)          \
  X(prim, double, gdg::NPRIM * n) X(dL, double, nnz) X(dB, double, nb) X(bbar, double, 2 * nb)            \
  X(UL, double, m * n) X(RHSL, double, m * n) X(N, double, n) X(agg, double, 3 * n) X(A, double, m * nnz) \
  X(AB, double, m * nb) X(bounds, double, 3 * n) X(l1, double, nnz) X(l1B, double, nb) X(l2, double, nnz) \
  X(l2B, double, nb) X(U1, double, m * n) X(rem, unsigned char, n) X(flags, unsigned, 4)                 \
  X(tau, unsigned long long, 1)                                                                          \
  X(lsq, int2, nnz + nb) X(clk, gdg::Clock, 1)

struct Layout {
#define GDG_F(name, T, cnt) size_t o_##name;
  GDG_ARENA(GDG_F)
#undef GDG_F
  size_t total;
};

// Sliced-ELL layout of the per-entry arrays (kEll in gdg_internal.cuh): the start of every slice (group g of
// kEll consecutive elements, local index l) from the row lengths, each slice padded to its longest row,
// and the total length.
struct EllLayout {
  std::vector<int64_t> sbase;  // [groups * nl + 1]
  int64_t total = 0;
};
template <class Len>
EllLayout ell_layout(int64_t n, int nl, Len len) {
  const int64_t nel = n / nl, ngrp = (nel + gdg::kEll - 1) / gdg::kEll;
  EllLayout L;
  L.sbase.assign((size_t)(ngrp * nl + 1), 0);
  for (int64_t g = 0; g < ngrp; ++g)
    for (int l = 0; l < nl; ++l) {
      int64_t w = 0;
      for (int e = 0; e < gdg::kEll; ++e) {
        const int64_t E = g * gdg::kEll + e;
        if (E < nel) w = std::max<int64_t>(w, len(E * nl + l));
      }
      const int64_t sl = g * nl + l;
      L.sbase[sl + 1] = L.sbase[sl] + gdg::kEll * w;
    }
  L.total = L.sbase[ngrp * nl];
  return L;
}

int64_t padded_elements(int64_t nel) { return (nel + gdg::kEll - 1) / gdg::kEll * gdg::kEll; }

Layout make_layout(int dim, int64_t n, int64_t nnz, int64_t nb, int nl, int64_t ne, int64_t nel) {
  const int64_t m = dim + 2;
  Layout Lo;
  Arena ar;
#define GDG_F(name, T, cnt) Lo.o_##name = ar.take<T>((size_t)(cnt));
  GDG_ARENA(GDG_F)
#undef GDG_F
  Lo.total = ar.off;
  return Lo;
}

int cuda_fail(cudaError_t e) { return e == cudaErrorMemoryAllocation ? GDG_ENOMEM : GDG_ECUDA; }

// Parameter-dependent per-entry / per-node data: c_k h^{p_k} (Sec. 5.1) and r_h^{+-} (Sec. 5.4).
struct ParamArrays {
  std::vector<double> mu, rm, rp, muB;
};

int param_arrays(const gdg_handle* h, const gdg_params& p, ParamArrays& A) {
  const int64_t n = h->n;
  const double dinv = 1.0 / h->dim;
  A.mu.assign(h->nnz_ell, 0.0);
  A.rm.resize(n);
  A.rp.resize(n);
  A.muB.resize(n);
  for (int64_t i = 0; i < n; ++i) {
    double hi = std::pow(h->mi[i] / h->omega, dinv);
    double hr = hi;  // the relaxation's mesh size: the node's (as printed) or its element's
    if (p.relax_measure == GDG_RELAX_ELEMENT) {
      double mel = 0.0;
      for (int64_t q = i / h->n_loc * h->n_loc; q < (i / h->n_loc + 1) * h->n_loc; ++q) mel += h->mi[q];
      hr = std::pow(mel / h->omega, dinv);
    }
    double rel = p.c_r * std::pow(hr, p.p_r);
    A.rm[i] = 1.0 - rel;
    A.rp[i] = 1.0 + rel;
    A.muB[i] = p.c_k * std::pow(hi, p.p_k);
    if (p.order == GDG_ORDER_LIMITED && p.bounds_mode == 0 && !(A.rm[i] > 0.0)) return GDG_ESETUP;
    for (int e = h->row_ptr[i]; e < h->row_ptr[i + 1]; ++e) {
      if (!h->coloc[e]) continue;
      int j = h->col[e];
      double hij = std::pow(0.5 * (h->mi[i] + h->mi[j]) / h->omega, dinv);
      A.mu[h->epos[e]] = p.c_k * std::pow(hij, p.p_k);
    }
  }
  return GDG_OK;
}

int upload_param_arrays(gdg_handle* h, const ParamArrays& A) {
  const int64_t n = h->n, nnz = h->nnz_ell;
  cudaError_t e;
  if ((nnz > 0 && (e = cudaMemcpy(h->d_mu, A.mu.data(), sizeof(double) * nnz, cudaMemcpyHostToDevice)) != cudaSuccess) ||
      (n > 0 && (e = cudaMemcpy(h->d_rminus, A.rm.data(), sizeof(double) * n, cudaMemcpyHostToDevice)) != cudaSuccess) ||
      (n > 0 && (e = cudaMemcpy(h->d_rplus, A.rp.data(), sizeof(double) * n, cudaMemcpyHostToDevice)) != cudaSuccess) ||
      (n > 0 && (e = cudaMemcpy(h->d_muB, A.muB.data(), sizeof(double) * n, cudaMemcpyHostToDevice)) != cudaSuccess))
    return cuda_fail(e);
  const gdg_params& p = h->params;
  Dev& D = h->D;
  D.c_ev = p.c_ev;
  D.order = p.order;
  D.passes = p.limiter_passes;
  D.bounds_mode = p.bounds_mode;
  D.ls_tol = p.ls_tol;
  D.ls_maxit = p.ls_maxit;
  D.mixed = p.precision == GDG_PRECISION_MIXED;
  D.c_ev_f = (float)p.c_ev;
  return GDG_OK;
}

}  // namespace

extern "C" {

void gdg_default_params(int32_t degree, gdg_params* out) {
  if (!out) return;
  out->order = GDG_ORDER_LIMITED;
  out->limiter_passes = 2;
  out->bounds_mode = 0;
  out->c_k = 1.0;
  out->p_k = (degree % 2 == 0) ? 0.5 : 0.0;
  out->c_ev = degree <= 1 ? 1.0 : (degree == 2 ? 0.5 : 0.25);
  out->c_r = 4.0;
  out->p_r = 1.5;
  out->ls_tol = 1e-14;
  out->ls_maxit = 50;
  out->precision = GDG_PRECISION_FP64;
  out->relax_measure = GDG_RELAX_NODE;
}

const char* gdg_error_string(int code) {
  switch (code) {
    case GDG_OK: return "GDG_OK";
    case GDG_EINVAL: return "GDG_EINVAL: invalid argument";
    case GDG_ENOMEM: return "GDG_ENOMEM: out of memory";
    case GDG_ECUDA: return "GDG_ECUDA: CUDA runtime error";
    case GDG_ESETUP: return "GDG_ESETUP: problem data violates a documented requirement";
    case GDG_EADMISSIBLE: return "GDG_EADMISSIBLE: inadmissible state";
    case GDG_ECFL: return "GDG_ECFL: CFL condition violated";
    case GDG_ETIMEOUT: return "GDG_ETIMEOUT: bounded device wait gave up";
    case GDG_ENOTSUP: return "GDG_ENOTSUP: unsupported configuration";
    default: return "gdg: unknown status code";
  }
}

int gdg_setup(const gdg_problem* P, gdg_handle** out) {
  if (!out) return GDG_EINVAL;
  *out = nullptr;
  if (!P || !P->row_ptr || (P->n > 0 && (!P->mi || !P->MK))) return GDG_EINVAL;
  if (P->nnz > 0 && (!P->col_idx || !P->cij || !P->coloc)) return GDG_EINVAL;
  if (P->nb > 0 && (!P->b_node || !P->b_c || !P->b_type)) return GDG_EINVAL;
  if (P->dim < 1 || P->dim > 3) return GDG_ENOTSUP;
  if (P->n_loc < 1 || P->n_loc > 32 || P->degree < 1) return GDG_ENOTSUP;
  if (P->n < 0 || P->nnz < 0 || P->nb < 0) return GDG_EINVAL;
  if (P->n >= (int64_t(1) << 31) || P->nnz >= (int64_t(1) << 31) || P->nb >= (int64_t(1) << 31))
    return GDG_ENOTSUP;
  if (P->n % P->n_loc != 0) return GDG_ESETUP;
  if (!(P->gamma > 1.0) || !(P->omega_measure > 0.0)) return GDG_ESETUP;
  if (!check_params(P->params)) return GDG_EINVAL;

  gdg_handle* h = new (std::nothrow) gdg_handle();
  if (!h) return GDG_ENOMEM;
  auto fail = [&](int code) {
    gdg_destroy(h);
    return code;
  };
  cudaGetDevice(&h->device);
  const int dim = P->dim, nl = P->n_loc, m = dim + 2;
  const int64_t n = P->n, nnz = P->nnz, nb = P->nb;
  h->dim = dim;
  h->degree = P->degree;
  h->n_loc = nl;
  h->n = n;
  h->nnz = nnz;
  h->nb = nb;
  h->gamma = P->gamma;
  h->omega = P->omega_measure;
  h->params = P->params;

  // ---- CSR structure ----
  if (P->row_ptr[0] != 0 || P->row_ptr[n] != nnz) return fail(GDG_ESETUP);
  h->row_ptr.resize(n + 1);
  for (int64_t i = 0; i <= n; ++i) {
    if (i > 0 && P->row_ptr[i] < P->row_ptr[i - 1]) return fail(GDG_ESETUP);
    h->row_ptr[i] = (int)P->row_ptr[i];
  }
  // Device entry order: within each row the stencil entries (c_ij != 0) come first, then the
  // m_ij-only entries, each group in the caller's order, so the stencil loops of the sweeps run over a
  // contiguous prefix of the row with no per-entry test.  eorig[q] is the caller's index of entry q.
  h->eorig.resize(nnz);
  std::vector<int> sten_end(n);
  {
    auto nz = [&](int64_t q) {  // the test |c_ij| > 0 of the stencil edges below
      double c2 = 0;
      for (int k = 0; k < dim; ++k) c2 += P->cij[(size_t)k * nnz + q] * P->cij[(size_t)k * nnz + q];
      return c2 > 0.0;
    };
    parallel_for(n, [&](int64_t b, int64_t e) {
      for (int64_t i = b; i < e; ++i) {
        int k = h->row_ptr[i];
        for (int q = h->row_ptr[i]; q < h->row_ptr[i + 1]; ++q)
          if (nz(q)) h->eorig[k++] = q;
        sten_end[i] = k;
        for (int q = h->row_ptr[i]; q < h->row_ptr[i + 1]; ++q)
          if (!nz(q)) h->eorig[k++] = q;
      }
    });
  }
  std::vector<double> cijv((size_t)dim * nnz);
  h->col.resize(nnz);
  h->coloc.resize(nnz);
  parallel_for(nnz, [&](int64_t b, int64_t e) {
    for (int64_t q = b; q < e; ++q) {
      const int64_t o = h->eorig[q];
      h->col[q] = P->col_idx[o];
      h->coloc[q] = P->coloc[o];
      for (int k = 0; k < dim; ++k) cijv[(size_t)k * nnz + q] = P->cij[(size_t)k * nnz + o];
    }
  });
  const double* cij = cijv.data();
  h->mi.assign(P->mi, P->mi + n);
  {
    std::vector<char> rowbad(n, 0);
    parallel_for(n, [&](int64_t b, int64_t e) {
      std::vector<int> tmp;
      for (int64_t i = b; i < e; ++i) {
        if (!(h->mi[i] > 0.0)) { rowbad[i] = 1; continue; }
        uint32_t mask = 0;
        int same = 0;
        tmp.assign(h->col.begin() + h->row_ptr[i], h->col.begin() + h->row_ptr[i + 1]);
        std::sort(tmp.begin(), tmp.end());
        if (std::adjacent_find(tmp.begin(), tmp.end()) != tmp.end()) { rowbad[i] = 1; continue; }
        for (int q = h->row_ptr[i]; q < h->row_ptr[i + 1]; ++q) {
          int j = h->col[q];
          if (j < 0 || j >= n || j == i) { rowbad[i] = 1; break; }
          if (j / nl == i / nl) {
            mask |= 1u << (j % nl);
            ++same;
          }
        }
        if (same != nl - 1 || (mask & (1u << (i % nl)))) rowbad[i] = 1;
      }
    });
    for (int64_t i = 0; i < n; ++i)
      if (rowbad[i]) return fail(GDG_ESETUP);
  }
  // transpose map, exact skew symmetry (Lemma PropSkew), collocation symmetry
  h->tr.assign(nnz, -1);
  {
    std::vector<char> bad(n, 0);
    parallel_for(n, [&](int64_t b, int64_t e) {
      for (int64_t i = b; i < e; ++i)
        for (int q = h->row_ptr[i]; q < h->row_ptr[i + 1]; ++q) {
          int j = h->col[q], t = -1;
          for (int r = h->row_ptr[j]; r < h->row_ptr[j + 1]; ++r)
            if (h->col[r] == i) { t = r; break; }
          if (t < 0 || h->coloc[t] != h->coloc[q]) { bad[i] = 1; continue; }
          for (int k = 0; k < dim; ++k)
            if (cij[(size_t)k * nnz + t] != -cij[(size_t)k * nnz + q]) bad[i] = 1;
          h->tr[q] = t;
        }
    });
    for (int64_t i = 0; i < n; ++i)
      if (bad[i]) return fail(GDG_ESETUP);
  }
  // boundary entries sorted by node
  std::vector<int> border(nb);
  for (int64_t b = 0; b < nb; ++b) {
    if (P->b_node[b] < 0 || P->b_node[b] >= n) return fail(GDG_ESETUP);
    if (P->b_type[b] != GDG_BC_SLIP && P->b_type[b] != GDG_BC_DIRICHLET && P->b_type[b] != GDG_BC_INOUTFLOW)
      return fail(GDG_ESETUP);
    if (P->b_type[b] != GDG_BC_SLIP) h->has_dirichlet = true;  // Dirichlet and in/outflow entries need data
    double c2 = 0;
    for (int k = 0; k < dim; ++k) c2 += P->b_c[(size_t)k * nb + b] * P->b_c[(size_t)k * nb + b];
    if (!(c2 > 0.0)) return fail(GDG_ESETUP);
    border[b] = (int)b;
  }
  std::stable_sort(border.begin(), border.end(), [&](int a, int b) { return P->b_node[a] < P->b_node[b]; });
  std::vector<int> b_ptr(n + 1, 0);
  for (int64_t b = 0; b < nb; ++b) b_ptr[P->b_node[b] + 1]++;
  for (int64_t i = 0; i < n; ++i) b_ptr[i + 1] += b_ptr[i];
  h->borig = border;
  // partition of unity (Lemma LemPart)
  {
    std::vector<char> bad(n, 0);
    parallel_for(n, [&](int64_t b, int64_t e) {
      for (int64_t i = b; i < e; ++i)
        for (int k = 0; k < dim; ++k) {
          double s = 0, a = 0;
          for (int q = h->row_ptr[i]; q < h->row_ptr[i + 1]; ++q) {
            double c = cij[(size_t)k * nnz + q];
            s += c;
            a += std::fabs(c);
          }
          for (int t = b_ptr[i]; t < b_ptr[i + 1]; ++t) {
            double c = P->b_c[(size_t)k * nb + border[t]];
            s += c;
            a += std::fabs(c);
          }
          if (std::fabs(s) > 1e-12 * a) bad[i] = 1;
        }
    });
    for (int64_t i = 0; i < n; ++i)
      if (bad[i]) return fail(GDG_ESETUP);
  }
  // element mass blocks: row sums equal m_i (Sec. 5.3), SPD, inverse
  const int64_t nel = n / nl;
  std::vector<double> MKinv((size_t)nel * nl * nl);
  {
    std::vector<char> bad(nel, 0);
    parallel_for(nel, [&](int64_t b, int64_t e) {
      for (int64_t K = b; K < e; ++K) {
        const double* A = P->MK + (size_t)K * nl * nl;
        for (int a = 0; a < nl; ++a) {
          double s = 0;
          for (int c = 0; c < nl; ++c) s += A[a * nl + c];
          double mi = h->mi[K * nl + a];
          if (std::fabs(s - mi) > 1e-12 * mi) bad[K] = 1;
          for (int c = 0; c < nl; ++c)
            if (A[a * nl + c] != A[c * nl + a]) bad[K] = 1;
        }
        if (!spd_inverse(A, nl, MKinv.data() + (size_t)K * nl * nl)) bad[K] = 1;
      }
    });
    for (int64_t K = 0; K < nel; ++K)
      if (bad[K]) return fail(GDG_ESETUP);
  }
  // per-entry data: |c_ij|, n_ij, m_ij
  std::vector<double> cnorm(nnz), cn((size_t)dim * nnz), mij(nnz, 0.0);
  parallel_for(n, [&](int64_t b, int64_t e) {
    for (int64_t i = b; i < e; ++i)
      for (int q = h->row_ptr[i]; q < h->row_ptr[i + 1]; ++q) {
        double c2 = 0;
        for (int k = 0; k < dim; ++k) c2 += cij[(size_t)k * nnz + q] * cij[(size_t)k * nnz + q];
        double cm = std::sqrt(c2);
        cnorm[q] = cm;
        for (int k = 0; k < dim; ++k) cn[(size_t)k * nnz + q] = cm > 0 ? cij[(size_t)k * nnz + q] / cm : 0.0;
        int j = h->col[q];
        if (j / nl == i / nl) mij[q] = P->MK[((size_t)(i / nl) * nl + i % nl) * nl + j % nl];
      }
  });
  // per-node: 1/m_i, 1/(kappa_i m_i) with kappa_i = 1/(row length + boundary entries of i)
  std::vector<double> inv_mi(n), inv_km(n);
  for (int64_t i = 0; i < n; ++i) {
    inv_mi[i] = 1.0 / h->mi[i];
    double terms = (h->row_ptr[i + 1] - h->row_ptr[i]) + (b_ptr[i + 1] - b_ptr[i]);
    inv_km[i] = terms > 0 ? terms / h->mi[i] : 0.0;
  }
  // ---- sliced-ELL positions of the entries (gdg_internal.cuh, kEll) ----
  const EllLayout EL = ell_layout(n, nl, [&](int64_t i) { return (int64_t)(h->row_ptr[i + 1] - h->row_ptr[i]); });
  if (EL.total >= (int64_t(1) << 31)) return fail(GDG_ENOTSUP);
  const int64_t NE = EL.total;
  h->nnz_ell = NE;
  h->epos.resize(nnz);
  std::vector<int> rbeg(n), rend(n), sten_ell(n);
  parallel_for(n, [&](int64_t b, int64_t e) {
    for (int64_t i = b; i < e; ++i) {
      const int64_t E = i / nl, l = i % nl;
      const int64_t p0 = EL.sbase[(size_t)((E / gdg::kEll) * nl + l)] + E % gdg::kEll;
      rbeg[i] = (int)p0;
      rend[i] = (int)(p0 + gdg::kEll * (int64_t)(h->row_ptr[i + 1] - h->row_ptr[i]));
      sten_ell[i] = (int)(p0 + gdg::kEll * (int64_t)(sten_end[i] - h->row_ptr[i]));
      for (int q = h->row_ptr[i]; q < h->row_ptr[i + 1]; ++q)
        h->epos[q] = (int)(p0 + gdg::kEll * (int64_t)(q - h->row_ptr[i]));
    }
  });
  // the per-entry arrays in ELL order; padding slots stay zero and no kernel reads them
  std::vector<int> col_e((size_t)NE, 0), tr_e((size_t)NE, 0);
  std::vector<double> cnorm_e((size_t)NE, 0.0), cn_e((size_t)dim * NE, 0.0), mij_e((size_t)NE, 0.0);
  parallel_for(nnz, [&](int64_t b, int64_t e) {
    for (int64_t q = b; q < e; ++q) {
      const int64_t pq = h->epos[q];
      col_e[pq] = h->col[q];
      tr_e[pq] = h->epos[h->tr[q]];
      cnorm_e[pq] = cnorm[q];
      mij_e[pq] = mij[q];
      for (int k = 0; k < dim; ++k) cn_e[(size_t)k * NE + pq] = cn[(size_t)k * nnz + q];
    }
  });
  // M_K^{-1} grouped like the entries: (K, a, b) at ((K / kEll * nl + a) * nl + b) * kEll + K % kEll
  const int64_t nel_pad = padded_elements(nel);
  std::vector<double> minv_g((size_t)nel_pad * nl * nl, 0.0);
  parallel_for(nel, [&](int64_t b, int64_t e) {
    for (int64_t K = b; K < e; ++K)
      for (int a = 0; a < nl; ++a)
        for (int c = 0; c < nl; ++c)
          minv_g[(((size_t)(K / gdg::kEll) * nl + a) * nl + c) * gdg::kEll + K % gdg::kEll] =
              MKinv[((size_t)K * nl + a) * nl + c];
  });
  // canonical stencil edges (i < j, c_ij != 0) in ELL order: consecutive threads of the edge sweep take
  // the same entry of the rows of consecutive elements, so their per-entry writes are contiguous
  std::vector<std::pair<int, int>> edges;
  edges.reserve(nnz / 2 + 1);
  for (int64_t i = 0; i < n; ++i)
    for (int q = h->row_ptr[i]; q < h->row_ptr[i + 1]; ++q)
      if (cnorm[q] > 0.0 && h->col[q] > i) edges.emplace_back(h->epos[q], (int)i);
  std::sort(edges.begin(), edges.end());
  std::vector<int> edge_e(edges.size()), edge_i(edges.size());
  for (size_t k = 0; k < edges.size(); ++k) {
    edge_e[k] = edges[k].first;
    edge_i[k] = edges[k].second;
  }
  const int64_t ne = (int64_t)edge_e.size();
  std::vector<double> bnorm(nb), bn((size_t)dim * nb);
  std::vector<int> btype(nb);
  for (int64_t t = 0; t < nb; ++t) {
    int b = border[t];
    double c2 = 0;
    for (int k = 0; k < dim; ++k) c2 += P->b_c[(size_t)k * nb + b] * P->b_c[(size_t)k * nb + b];
    bnorm[t] = std::sqrt(c2);
    for (int k = 0; k < dim; ++k) bn[(size_t)k * nb + t] = P->b_c[(size_t)k * nb + b] / bnorm[t];
    btype[t] = P->b_type[b];
  }

  ParamArrays pa;
  if (int rc = param_arrays(h, h->params, pa); rc != GDG_OK) return fail(rc);

  // ---- device arena ----
  const Layout Lo = make_layout(dim, n, NE, nb, nl, ne, nel_pad);
#define GDG_F(name, T, cnt) const size_t o_##name = Lo.o_##name;
  GDG_ARENA(GDG_F)
#undef GDG_F
  h->arena_bytes = Lo.total;
  cudaError_t ce = cudaMalloc(&h->arena, h->arena_bytes);
  if (ce != cudaSuccess) {
    h->arena = nullptr;
    cudaGetLastError();
    return fail(cuda_fail(ce));
  }
  // zero the whole arena once: entries no kernel writes (d^L, A of m_ij-only entries) read as 0
  if ((ce = cudaMemset(h->arena, 0, h->arena_bytes)) != cudaSuccess) return fail(cuda_fail(ce));
  char* base = (char*)h->arena;
  auto ptr = [&](size_t o) { return (void*)(base + o); };
  auto up = [&](size_t o, const void* src, size_t bytes) {
    if (bytes == 0) return cudaSuccess;
    return cudaMemcpy(ptr(o), src, bytes, cudaMemcpyHostToDevice);
  };
  if ((ce = up(o_rbeg, rbeg.data(), sizeof(int) * n)) != cudaSuccess ||
      (ce = up(o_rend, rend.data(), sizeof(int) * n)) != cudaSuccess ||
      (ce = up(o_sten, sten_ell.data(), sizeof(int) * n)) != cudaSuccess ||
      (ce = up(o_col, col_e.data(), sizeof(int) * NE)) != cudaSuccess ||
      (ce = up(o_tr, tr_e.data(), sizeof(int) * NE)) != cudaSuccess ||
      (ce = up(o_cnorm, cnorm_e.data(), sizeof(double) * NE)) != cudaSuccess ||
      (ce = up(o_cn, cn_e.data(), sizeof(double) * dim * NE)) != cudaSuccess ||
      (ce = up(o_mij, mij_e.data(), sizeof(double) * NE)) != cudaSuccess ||
      (ce = up(o_mi, h->mi.data(), sizeof(double) * n)) != cudaSuccess ||
      (ce = up(o_imi, inv_mi.data(), sizeof(double) * n)) != cudaSuccess ||
      (ce = up(o_ikm, inv_km.data(), sizeof(double) * n)) != cudaSuccess ||
      (ce = up(o_bptr, b_ptr.data(), sizeof(int) * (n + 1))) != cudaSuccess ||
      (ce = up(o_bnorm, bnorm.data(), sizeof(double) * nb)) != cudaSuccess ||
      (ce = up(o_bn, bn.data(), sizeof(double) * dim * nb)) != cudaSuccess ||
      (ce = up(o_btype, btype.data(), sizeof(int) * nb)) != cudaSuccess ||
      (ce = up(o_borig, border.data(), sizeof(int) * nb)) != cudaSuccess ||
      (ce = up(o_minv, minv_g.data(), sizeof(double) * minv_g.size())) != cudaSuccess ||
      (ce = up(o_ee, edge_e.data(), sizeof(int) * ne)) != cudaSuccess ||
      (ce = up(o_ei, edge_i.data(), sizeof(int) * ne)) != cudaSuccess ||
      (ce = cudaMemset(ptr(o_flags), 0, 16)) != cudaSuccess)
    return fail(cuda_fail(ce));

  Dev& D = h->D;
  D.n = (int)n;
  D.nnz = (int)NE;
  D.nb = (int)nb;
  D.n_loc = nl;
  D.nel = (int)nel;
  gdg::set_nl_division(D, nl);
  D.rbeg = (const int*)ptr(o_rbeg);
  D.rend = (const int*)ptr(o_rend);
  D.sten_end = (const int*)ptr(o_sten);
  D.col = (const int*)ptr(o_col);
  D.tr = (const int*)ptr(o_tr);
  D.cnorm = (const double*)ptr(o_cnorm);
  D.cn = (const double*)ptr(o_cn);
  D.mij = (const double*)ptr(o_mij);
  D.mu = (const double*)ptr(o_mu);
  D.mi = (const double*)ptr(o_mi);
  D.inv_mi = (const double*)ptr(o_imi);
  D.inv_km = (const double*)ptr(o_ikm);
  D.rminus = (const double*)ptr(o_rm);
  D.rplus = (const double*)ptr(o_rp);
  D.muB = (const double*)ptr(o_muB);
  D.b_ptr = (const int*)ptr(o_bptr);
  D.bnorm = (const double*)ptr(o_bnorm);
  D.bn = (const double*)ptr(o_bn);
  D.btype = (const int*)ptr(o_btype);
  D.borig = (const int*)ptr(o_borig);
  D.MKinv = (const double*)ptr(o_minv);
  D.ne = (int)ne;
  D.edge_e = (const int*)ptr(o_ee);
  D.edge_i = (const int*)ptr(o_ei);
  gdg::set_eos(D, P->gamma);
  h->d_mu = (double*)ptr(o_mu);
  h->d_rminus = (double*)ptr(o_rm);
  h->d_rplus = (double*)ptr(o_rp);
  h->d_muB = (double*)ptr(o_muB);

  Scratch& S = h->S;
  S.prim = (double*)ptr(o_prim);
  S.dL = (double*)ptr(o_dL);
  S.G = (double*)ptr(o_G);
  S.barR = (double*)ptr(o_barR);
  S.barS = (double*)ptr(o_barS);
  S.dB = (double*)ptr(o_dB);
  S.bbar = (double*)ptr(o_bbar);
  S.UL = (double*)ptr(o_UL);
  S.RHSL = (double*)ptr(o_RHSL);
  S.N = (double*)ptr(o_N);
  S.agg = (double*)ptr(o_agg);
  S.A = (double*)ptr(o_A);
  S.AB = (double*)ptr(o_AB);
  S.bounds = (double*)ptr(o_bounds);
  S.l1 = (double*)ptr(o_l1);
  S.l1B = (double*)ptr(o_l1B);
  S.l2 = (double*)ptr(o_l2);
  S.l2B = (double*)ptr(o_l2B);
  S.U1 = (double*)ptr(o_U1);
  S.rem = (unsigned char*)ptr(o_rem);
  S.flags = (unsigned*)ptr(o_flags);
  S.lsq_n = S.flags + 2;
  S.lsq = (int2*)ptr(o_lsq);
  h->clk = (gdg::Clock*)ptr(o_clk);
  {
    gdg::Clock c0{};
    c0.tau_bits = gdg::kTauNone;
    c0.t = 0.0;
    c0.t_end = INFINITY;
    c0.cfl = 0.5;
    if ((ce = cudaMemcpy(h->clk, &c0, sizeof(c0), cudaMemcpyHostToDevice)) != cudaSuccess) return fail(cuda_fail(ce));
  }
  S.tau_bits = (unsigned long long*)ptr(o_tau);

  if (int rc = upload_param_arrays(h, pa); rc != GDG_OK) return fail(rc);
  *out = h;
  return GDG_OK;
}

int gdg_footprint(const gdg_problem* P, int64_t* bytes) {
  if (!P || !bytes || P->dim < 1 || P->dim > 3 || P->n < 0 || P->nnz < 0 || P->nb < 0 || P->n_loc < 1)
    return GDG_EINVAL;
  if ((P->n > 0 && (!P->row_ptr || !P->col_idx)) || (P->nnz > 0 && !P->cij)) return GDG_EINVAL;
  int64_t ne = 0;
  for (int64_t i = 0; i < P->n; ++i)
    for (int64_t q = P->row_ptr[i]; q < P->row_ptr[i + 1]; ++q) {
      if (q < 0 || q >= P->nnz) return GDG_EINVAL;
      bool nz = false;
      for (int k = 0; k < P->dim; ++k) nz = nz || P->cij[(size_t)k * P->nnz + q] != 0.0;
      if (nz && P->col_idx[q] > i) ++ne;
    }
  if (P->n % P->n_loc != 0) return GDG_EINVAL;
  const EllLayout EL = ell_layout(P->n, P->n_loc, [&](int64_t i) { return P->row_ptr[i + 1] - P->row_ptr[i]; });
  *bytes = (int64_t)make_layout(P->dim, P->n, EL.total, P->nb, P->n_loc, ne, padded_elements(P->n / P->n_loc)).total;
  return GDG_OK;
}

int gdg_set_params(gdg_handle* h, const gdg_params* params) {
  if (!h || !params || !check_params(*params)) return GDG_EINVAL;
  ParamArrays pa;
  if (int rc = param_arrays(h, *params, pa); rc != GDG_OK) return rc;
  h->params = *params;
  return upload_param_arrays(h, pa);
}

int gdg_max_dt(gdg_handle* h, const double* U, const double* bdata, double cfl, double* tau_out, void* stream) {
  if (!h || (!U && h->n > 0) || !tau_out || !(cfl > 0)) return GDG_EINVAL;
  if (h->has_dirichlet && !bdata) return GDG_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  if ((e = cudaMemsetAsync(h->S.tau_bits, 0x7f, sizeof(unsigned long long), s)) != cudaSuccess) return cuda_fail(e);
  const gdg::Ctx c = make_ctx(h, U, nullptr, nullptr, bdata, 0.0, 0.0, nullptr);
  if ((e = timed(h, GDG_K_PRIM, s, [&] { return gdg::launch_one(gdg::KN_PRIM, h->dim, c, 0, h->sched, s); })) !=
      cudaSuccess)
    return cuda_fail(e);
  if ((e = timed(h, GDG_K_MAXDT, s, [&] { return gdg::launch_one(gdg::KN_MAXDT, h->dim, c, 0, h->sched, s); })) !=
      cudaSuccess)
    return cuda_fail(e);
  unsigned long long bits = 0;
  if ((e = cudaMemcpyAsync(&bits, h->S.tau_bits, sizeof(bits), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return cuda_fail(e);
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e);
  double v;
  std::memcpy(&v, &bits, sizeof(v));
  *tau_out = (bits == 0x7f7f7f7f7f7f7f7fULL) ? INFINITY : cfl * v;
  return GDG_OK;
}

// The kernels of one stage (Sec. 6.1): primitives, edge sweep, [the fused step's tau bound], sweep A,
// then, as the order and the number of limiter passes ask, the element sweep, the deferred line searches
// of pass 1, sweep C, those of pass 2 and sweep D.
// prim_ctx, when given, is the context of the primitive sweep alone (a stage whose input it reads from
// host memory and stores where c.U points).
static int run_stage(gdg_handle* h, const gdg::Ctx& c, bool with_tau, cudaStream_t s,
                     const gdg::Ctx* prim_ctx = nullptr) {
  const int dim = h->dim;
  const gdg::Dev& D = h->D;
  cudaError_t e;
  auto go = [&](int id, int kern, int arg) {
    return timed(h, id, s, [&] { return gdg::launch_one(kern, dim, c, arg, h->sched, s); });
  };
  const bool low_only = D.order == GDG_ORDER_LOW || (D.order == GDG_ORDER_LIMITED && D.passes == 0);
  if (prim_ctx) {
    e = timed(h, GDG_K_PRIM, s, [&] { return gdg::launch_one(gdg::KN_PRIM, dim, *prim_ctx, 0, h->sched, s); });
    if (e != cudaSuccess) return cuda_fail(e);
  } else if ((e = go(GDG_K_PRIM, gdg::KN_PRIM, 0)) != cudaSuccess) {
    return cuda_fail(e);
  }
  if ((e = go(GDG_K_EDGE, gdg::KN_EDGE, 0)) != cudaSuccess) return cuda_fail(e);
  if (with_tau && (e = go(GDG_K_TAU, gdg::KN_TAU, 0)) != cudaSuccess) return cuda_fail(e);
  if ((e = go(GDG_K_LOW, gdg::KN_LOW, low_only ? 1 : 0)) != cudaSuccess) return cuda_fail(e);
  if (low_only) return GDG_OK;
  if ((e = go(GDG_K_HIGH, gdg::KN_HIGH, 0)) != cudaSuccess) return cuda_fail(e);
  if (D.order == GDG_ORDER_HIGH) return GDG_OK;
  if ((e = go(GDG_K_LSFIX, gdg::KN_LSFIX, 0)) != cudaSuccess) return cuda_fail(e);
  if ((e = go(GDG_K_LIMIT2, gdg::KN_LIMIT2, D.passes == 1 ? 1 : 0)) != cudaSuccess) return cuda_fail(e);
  if (D.passes == 1) return GDG_OK;
  if ((e = go(GDG_K_LSFIX, gdg::KN_LSFIX, 1)) != cudaSuccess) return cuda_fail(e);
  if ((e = go(GDG_K_FINAL, gdg::KN_FINAL, 0)) != cudaSuccess) return cuda_fail(e);
  return GDG_OK;
}

int gdg_stage(gdg_handle* h, const double* U_in, const double* U_base, double alpha, double tau,
              const double* bdata, double* U_out, void* stream) {
  if (!h || ((!U_in || !U_out) && h->n > 0) || !(tau >= 0) || !std::isfinite(tau)) return GDG_EINVAL;
  if (h->n > 0 && U_out == U_in) return GDG_EINVAL;
  if (alpha != 0.0 && !U_base && h->n > 0) return GDG_EINVAL;
  if (h->has_dirichlet && !bdata) return GDG_EINVAL;
  const gdg::Ctx c = make_ctx(h, U_in, U_base, U_out, bdata, alpha, tau, nullptr);
  return run_stage(h, c, false, (cudaStream_t)stream);
}

int gdg_clock_set(gdg_handle* h, double t, double t_end, double cfl, void* stream) {
  if (!h || !std::isfinite(t) || !(t_end >= t) || !(cfl > 0) || !std::isfinite(cfl)) return GDG_EINVAL;
  gdg::Clock c0{};
  c0.tau_bits = gdg::kTauNone;
  c0.t = t;
  c0.t_end = t_end;
  c0.cfl = cfl;
  c0.tau = 0.0;
  c0.steps = 0;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  if ((e = cudaMemcpyAsync(h->clk, &c0, sizeof(c0), cudaMemcpyHostToDevice, s)) != cudaSuccess) return cuda_fail(e);
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e);
  return GDG_OK;
}

int gdg_clock_get(gdg_handle* h, double* t, double* tau, int64_t* steps, void* stream) {
  if (!h) return GDG_EINVAL;
  gdg::Clock c0{};
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  if ((e = cudaMemcpyAsync(&c0, h->clk, sizeof(c0), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return cuda_fail(e);
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e);
  if (t) *t = c0.t;
  if (tau) *tau = c0.tau;
  if (steps) *steps = c0.steps;
  return GDG_OK;
}

// The three stages of the fused SSP-RK3 step on U (device).  With in_mapped, the first stage's primitive
// sweep reads the step's input from that kernel-addressable host memory and stores it in U first; with
// out_mapped (only together with in_mapped), the last stage's writers also write the new state there, and
// so does the primitive sweep when the clock has finished and the step changes nothing.
static int ssprk3_stages(gdg_handle* h, double* U, double* T1, double* T2, const double* bdata,
                         const double* in_mapped, double* out_mapped, cudaStream_t s) {
  // Shu-Osher form of SSP-RK3 (Sec. 6.2): U1 = FE(U); U2 = 3/4 U + 1/4 FE(U1); U <- 1/3 U + 2/3 FE(U2),
  // the last in place (each node reads its base value before writing it)
  const gdg::Ctx c1 = make_ctx(h, U, nullptr, T1, bdata, 0.0, 0.0, h->clk);
  const gdg::Ctx c2 = make_ctx(h, T1, U, T2, bdata, 0.75, 0.0, h->clk);
  gdg::Ctx c3 = make_ctx(h, T2, U, U, bdata, 1.0 / 3.0, 0.0, h->clk);
  gdg::Ctx p1 = c1;
  if (in_mapped) {
    p1.U = in_mapped;
    p1.Ucopy = U;
    p1.Uhost = out_mapped;
    c3.Uhost = out_mapped;
  }
  if (int rc = run_stage(h, c1, true, s, in_mapped ? &p1 : nullptr); rc != GDG_OK) return rc;
  if (int rc = run_stage(h, c2, false, s); rc != GDG_OK) return rc;
  if (int rc = run_stage(h, c3, false, s); rc != GDG_OK) return rc;
  cudaError_t e = timed(h, GDG_K_CLOCK, s, [&] { return gdg::launch_clock_one(h->clk, 1.0, s); });
  return e == cudaSuccess ? GDG_OK : cuda_fail(e);
}

int gdg_ssprk3_step(gdg_handle* h, double* U, double* T1, double* T2, const double* bdata, void* stream) {
  if (!h || ((!U || !T1 || !T2) && h->n > 0)) return GDG_EINVAL;
  if (h->n > 0 && (U == T1 || U == T2 || T1 == T2)) return GDG_EINVAL;
  if (h->has_dirichlet && !bdata) return GDG_EINVAL;
  return ssprk3_stages(h, U, T1, T2, bdata, nullptr, nullptr, (cudaStream_t)stream);
}

// The address kernels on the current device use for host memory p, when p lies in page-locked memory
// mapped into the device's address space (cudaHostAlloc, cudaMallocHost, cudaHostRegister with mapping);
// null for any other memory.
static double* mapped_host(const double* p) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();  // not a pointer the runtime knows: plain host memory
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? static_cast<double*>(a.devicePointer) : nullptr;
}

int gdg_ssprk3_step_host(gdg_handle* h, const double* U_host_in, double* U_host_out, double* U, double* T1,
                         double* T2, const double* bdata, void* stream) {
  if (!h || ((!U_host_in || !U_host_out || !U || !T1 || !T2) && h->n > 0)) return GDG_EINVAL;
  if (h->n > 0 && (U == T1 || U == T2 || T1 == T2)) return GDG_EINVAL;
  if (h->has_dirichlet && !bdata) return GDG_EINVAL;
  if (h->n == 0) return ssprk3_stages(h, U, T1, T2, bdata, nullptr, nullptr, (cudaStream_t)stream);
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes = sizeof(double) * (size_t)(h->dim + 2) * h->n;
  const double* in_dev = mapped_host(U_host_in);
  double* out_dev = in_dev ? mapped_host(U_host_out) : nullptr;
  cudaError_t e;
  if (!in_dev && (e = cudaMemcpyAsync(U, U_host_in, bytes, cudaMemcpyDefault, s)) != cudaSuccess)
    return cuda_fail(e);
  if (int rc = ssprk3_stages(h, U, T1, T2, bdata, in_dev, out_dev, s); rc != GDG_OK) return rc;
  if (!out_dev && (e = cudaMemcpyAsync(U_host_out, U, bytes, cudaMemcpyDefault, s)) != cudaSuccess)
    return cuda_fail(e);
  return GDG_OK;
}

// SSPRK(5,4): the optimal five-stage fourth-order SSP method (Spiteri-Ruuth coefficients; the method the
// paper's experiments use, Sec. 6.2) in Shu-Osher form.  Stage j's forward-Euler step is
// (beta / alpha) dt; u_3 enters u_4 and u_5 with the same step, so one evaluation F3 = FE(u_3) serves both.
namespace {
constexpr double kA[5][5] = {{1.0, 0, 0, 0, 0},
                             {0.444370493651235, 0.555629506348765, 0, 0, 0},
                             {0.620101851488403, 0.0, 0.379898148511597, 0, 0},
                             {0.178079954393132, 0.0, 0.0, 0.821920045606868, 0},
                             {0.0, 0.0, 0.517231671970585, 0.096059710526147, 0.386708617503269}};
constexpr double kB[5][5] = {{0.391752226571890, 0, 0, 0, 0},
                             {0.0, 0.368410593050371, 0, 0, 0},
                             {0.0, 0.0, 0.251891774271694, 0, 0},
                             {0.0, 0.0, 0.0, 0.544974750228521, 0},
                             {0.0, 0.0, 0.0, 0.063692468666290, 0.226007483236906}};
// the SSP coefficient min alpha / beta: dt = cfl * C * bound keeps every stage's step within cfl * bound
double ssp54_coefficient() {
  double c = 1e300;
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j <= i; ++j)
      if (kB[i][j] != 0.0) c = std::min(c, kA[i][j] / kB[i][j]);
  return c;
}
}  // namespace

int gdg_ssprk54_step(gdg_handle* h, double* U, double* T1, double* T2, double* T3, const double* bdata,
                     void* stream) {
  if (!h || ((!U || !T1 || !T2 || !T3) && h->n > 0)) return GDG_EINVAL;
  if (h->n > 0 && (U == T1 || U == T2 || U == T3 || T1 == T2 || T1 == T3 || T2 == T3)) return GDG_EINVAL;
  if (h->has_dirichlet && !bdata) return GDG_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const double C = ssp54_coefficient();
  auto ctx = [&](const double* in, const double* base, double alpha, double* out, double scale) {
    gdg::Ctx c = make_ctx(h, in, base, out, bdata, alpha, 0.0, h->clk);
    c.tau_scale = scale;
    c.dt_factor = C;
    return c;
  };
  // u1 = FE(u) -> T1;  u2 = a u + b FE(u1) -> T2;  u3 = a u + b FE(u2) -> T1;  F3 = FE(u3) -> T3;
  // u4 = a u + b F3 -> T1;  u5 = a u2 + b F3 + c FE(u4) -> T2 (in place on u2);  U <- u5
  const gdg::Ctx s1 = ctx(U, nullptr, 0.0, T1, kB[0][0] / kA[0][0]);
  const gdg::Ctx s2 = ctx(T1, U, kA[1][0], T2, kB[1][1] / kA[1][1]);
  const gdg::Ctx s3 = ctx(T2, U, kA[2][0], T1, kB[2][2] / kA[2][2]);
  const gdg::Ctx s4 = ctx(T1, nullptr, 0.0, T3, kB[3][3] / kA[3][3]);
  const gdg::Ctx c4 = ctx(T3, U, kA[3][0], T1, 0.0);
  gdg::Ctx s5 = ctx(T1, T2, kA[4][2], T2, kB[4][4] / kA[4][4]);
  s5.Ubase2 = T3;
  s5.alpha2 = kA[4][3];
  s5.w_fe = kA[4][4];
  const gdg::Ctx cp = ctx(T2, nullptr, 0.0, U, 0.0);
  auto axpy = [&](const gdg::Ctx& c) {
    return timed(h, GDG_K_AXPY, s, [&] { return gdg::launch_one(gdg::KN_AXPY, h->dim, c, 0, h->sched, s); });
  };
  if (int rc = run_stage(h, s1, true, s); rc != GDG_OK) return rc;
  if (int rc = run_stage(h, s2, false, s); rc != GDG_OK) return rc;
  if (int rc = run_stage(h, s3, false, s); rc != GDG_OK) return rc;
  if (int rc = run_stage(h, s4, false, s); rc != GDG_OK) return rc;
  cudaError_t e;
  if ((e = axpy(c4)) != cudaSuccess) return cuda_fail(e);
  if (int rc = run_stage(h, s5, false, s); rc != GDG_OK) return rc;
  if ((e = axpy(cp)) != cudaSuccess) return cuda_fail(e);
  e = timed(h, GDG_K_CLOCK, s, [&] { return gdg::launch_clock_one(h->clk, C, s); });
  return e == cudaSuccess ? GDG_OK : cuda_fail(e);
}

int gdg_autotune(gdg_handle* h, double* U, double* T1, double* T2, const double* bdata, int32_t trials,
                 void* stream) {
  if (!h || ((!U || !T1 || !T2) && h->n > 0)) return GDG_EINVAL;
  if (h->n > 0 && (U == T1 || U == T2 || T1 == T2)) return GDG_EINVAL;
  if (h->has_dirichlet && !bdata) return GDG_EINVAL;
  if (h->n == 0) return GDG_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes = sizeof(double) * (size_t)(h->dim + 2) * h->n;
  double* save = nullptr;
  cudaError_t e = cudaMalloc(&save, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return GDG_ENOMEM;
  }
  gdg::Clock clk0{};
  unsigned flags0 = 0;
  if ((e = cudaMemcpyAsync(save, U, bytes, cudaMemcpyDeviceToDevice, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(&clk0, h->clk, sizeof(clk0), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(&flags0, h->S.flags, sizeof(flags0), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess) {
    cudaFree(save);
    return cuda_fail(e);
  }
  gdg::Clock tune_clk = clk0;  // an instance that already reached t_end would time no-op steps
  tune_clk.t_end = INFINITY;
  tune_clk.tau_bits = gdg::kTauNone;
  auto put_back = [&](const gdg::Clock& ck) -> int {
    cudaError_t r;
    if ((r = cudaMemcpyAsync(U, save, bytes, cudaMemcpyDeviceToDevice, s)) != cudaSuccess ||
        (r = cudaMemcpyAsync(h->clk, &ck, sizeof(ck), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (r = cudaMemcpyAsync(h->S.flags, &flags0, sizeof(flags0), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (r = cudaStreamSynchronize(s)) != cudaSuccess)
      return cuda_fail(r);
    return GDG_OK;
  };
  const bool prof0 = h->profiling;
  gdg_profile(h, 1);
  int rc = autotune_schedule(
      h->sched, h->n_loc, trials,
      [&](const gdg::Sched& sc) {
        h->sched = sc;
        return GDG_OK;
      },
      [&] { return gdg_ssprk3_step(h, U, T1, T2, bdata, stream); },
      [&](double* ms) {
        double tot[GDG_NKERNELS];
        int64_t cnt[GDG_NKERNELS];
        const int r = gdg_profile_read(h, tot, cnt);
        for (int k = 0; k < GDG_NKERNELS; ++k) ms[k] = cnt[k] ? tot[k] / (double)cnt[k] : 0.0;
        return r;
      },
      [&] { return put_back(tune_clk); });
  gdg_profile(h, prof0 ? 1 : 0);
  const int rc2 = put_back(clk0);
  cudaFree(save);
  return rc != GDG_OK ? rc : rc2;
}

int gdg_get_schedule(gdg_handle* h, gdg_schedule* out) {
  if (!h || !out) return GDG_EINVAL;
  sched_to_public(h->sched, out);
  return GDG_OK;
}

int gdg_set_schedule(gdg_handle* h, const gdg_schedule* in) {
  if (!h || !in) return GDG_EINVAL;
  gdg::Sched sc;
  if (!sched_from_public(in, &sc)) return GDG_EINVAL;
  h->sched = sc;
  return GDG_OK;
}

int gdg_status(gdg_handle* h, int32_t* flags, int32_t clear, void* stream) {
  if (!h || !flags) return GDG_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned v = 0;
  cudaError_t e;
  if ((e = cudaMemcpyAsync(&v, h->S.flags, sizeof(v), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return cuda_fail(e);
  if (clear && (e = cudaMemsetAsync(h->S.flags, 0, sizeof(unsigned), s)) != cudaSuccess) return cuda_fail(e);
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e);
  *flags = (int32_t)v;
  return GDG_OK;
}

int gdg_debug_export(gdg_handle* h, const char* name, double* dst, int64_t count, void* stream) {
  if (!h || !name || !dst) return GDG_EINVAL;
  const int64_t n = h->n, nnz = h->nnz, nb = h->nb, m = h->dim + 2, NE = h->nnz_ell;
  const double* src = nullptr;
  int64_t want = -1;
  int kind = 0;  // 0 plain copy, 1 symmetrised per-entry limiter, 2 boundary order
  bool per_entry = false;
  std::string nm(name);
  if (nm == "dL") { src = h->S.dL; want = nnz; per_entry = true; }
  else if (nm == "dB") { src = h->S.dB; want = nb; kind = 2; }
  else if (nm == "N") { src = h->S.N; want = n; }
  else if (nm == "UL") { src = h->S.UL; want = m * n; }
  else if (nm == "U1") { src = h->S.U1; want = m * n; }
  else if (nm == "A") { src = h->S.A; want = m * nnz; per_entry = true; }
  else if (nm == "rho_min") { src = h->S.bounds; want = n; }
  else if (nm == "rho_max") { src = h->S.bounds + n; want = n; }
  else if (nm == "s_min") { src = h->S.bounds + 2 * n; want = n; }
  else if (nm == "l1") { src = h->S.l1; want = nnz; kind = 1; }
  else if (nm == "l2") { src = h->S.l2; want = nnz; kind = 1; }
  else if (nm == "ls_deferred") { want = 2; kind = 3; }
  else return GDG_EINVAL;
  if (count != want) return GDG_EINVAL;
  cudaError_t e;
  if ((e = cudaStreamSynchronize((cudaStream_t)stream)) != cudaSuccess) return cuda_fail(e);
  if (kind == 3) {  // lengths of the deferred line-search queues of the last stage's two limiter passes
    unsigned q[2];
    if ((e = cudaMemcpy(q, h->S.lsq_n, sizeof(q), cudaMemcpyDeviceToHost)) != cudaSuccess) return cuda_fail(e);
    dst[0] = q[0];
    dst[1] = q[1];
    return GDG_OK;
  }
  // per-entry arrays live in sliced-ELL order on the device (their length NE per component)
  const int64_t dev_count = (per_entry || kind == 1) ? want / std::max<int64_t>(nnz, 1) * NE : want;
  std::vector<double> tmp(dev_count);
  if (dev_count > 0 &&
      (e = cudaMemcpy(tmp.data(), src, sizeof(double) * dev_count, cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_fail(e);
  if (kind == 0 && per_entry) {  // device entry order back to the caller's
    for (int64_t r = 0; r < want / std::max<int64_t>(nnz, 1); ++r)
      for (int64_t q = 0; q < nnz; ++q) dst[r * nnz + h->eorig[q]] = tmp[r * NE + h->epos[q]];
  } else if (kind == 0) {
    std::memcpy(dst, tmp.data(), sizeof(double) * want);
  } else if (kind == 1) {
    for (int64_t q = 0; q < want; ++q) dst[h->eorig[q]] = std::min(tmp[h->epos[q]], tmp[h->epos[h->tr[q]]]);
  } else {
    for (int64_t t = 0; t < want; ++t) dst[h->borig[t]] = tmp[t];
  }
  return GDG_OK;
}

int gdg_profile(gdg_handle* h, int32_t enable) {
  if (!h) return GDG_EINVAL;
  for (auto& r : h->recs) {
    h->pool.push_back(r.a);
    h->pool.push_back(r.b);
  }
  h->recs.clear();
  h->profiling = enable != 0;
  return GDG_OK;
}

int gdg_profile_read(gdg_handle* h, double* total_ms, int64_t* launches) {
  if (!h || !total_ms || !launches) return GDG_EINVAL;
  for (int k = 0; k < GDG_NKERNELS; ++k) {
    total_ms[k] = 0.0;
    launches[k] = 0;
  }
  int rc = GDG_OK;
  for (auto& r : h->recs) {
    float ms = 0.f;
    cudaError_t e = cudaEventSynchronize(r.b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, r.a, r.b);
    if (e != cudaSuccess) rc = cuda_fail(e);
    total_ms[r.kernel] += ms;
    launches[r.kernel] += 1;
    h->pool.push_back(r.a);
    h->pool.push_back(r.b);
  }
  h->recs.clear();
  return rc;
}

int gdg_get_info(gdg_handle* h, gdg_info* out) {
  if (!h || !out) return GDG_EINVAL;
  out->n = h->n;
  out->nnz = h->nnz;
  out->nb = h->nb;
  out->dim = h->dim;
  out->n_loc = h->n_loc;
  out->device_bytes = (int64_t)h->arena_bytes;
  return GDG_OK;
}

void gdg_destroy(gdg_handle* h) {
  if (!h) return;
  for (auto& r : h->recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto e : h->pool) cudaEventDestroy(e);
  if (h->arena) cudaFree(h->arena);
  delete h;
}

}  // extern "C"
