/* Oracle: one forward-Euler stage of the convex-limited graph-based dG scheme, plain FP64 C.
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).  Every function follows one passage of the paper
 * (arXiv 2402.04514, cited by section and equation label) and is a plain loop over rows in the order
 * the paper states the method.  Where the paper leaves a choice open, the reading taken is stated at
 * the function.
 *
 * Notation: m = d + 2 components; I(i) = {j : c_ij != 0} (Sec. 2.3); the CSR row of i also holds the
 * other nodes of i's element, which the consistent mass m_ij couples in Sec. 5, eq. (HighScheme).
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define MAXM 5
#define MAXNL 32 /* nodes per element (Q2 in 3D has 27); the Python wrapper rejects more */

/* The row loops carry ORC_PARALLEL_* markers.  They are empty in the default build, the one the tests pin.
 * Built with -fopenmp (the multi-core timing build of the CPU baseline) they share the rows of a loop
 * among threads; every row writes only its own entries, so both builds give bit-identical results. */
#ifdef _OPENMP
#define ORC_PRAGMA(x) _Pragma(#x)
#define ORC_PARALLEL_FOR ORC_PRAGMA(omp parallel for schedule(dynamic, 1024))
#define ORC_PARALLEL_PRIVATE(...) ORC_PRAGMA(omp parallel for schedule(dynamic, 1024) private(__VA_ARGS__))
#else
#define ORC_PARALLEL_FOR
#define ORC_PARALLEL_PRIVATE(...)
#endif

static double dot(const double* a, const double* b, int d) {
  double s = 0.0;
  for (int k = 0; k < d; ++k) s += a[k] * b[k];
  return s;
}

static void gather(const double* U, long n, long i, int m, double* out) {
  for (int c = 0; c < m; ++c) out[c] = U[c * n + i];
}

/* Sec. 2.2, eq. (PressurEuler): eps(U) = E - |m|^2 / (2 rho) (internal energy per unit volume). */
static double internal_energy(const double* U, int d) {
  double m2 = 0.0;
  for (int k = 0; k < d; ++k) m2 += U[1 + k] * U[1 + k];
  return U[d + 1] - 0.5 * m2 / U[0];
}

/* Sec. 2.2, eq. (PressurEuler): p = (gamma - 1) eps. */
static double pressure(const double* U, int d, double g) { return (g - 1.0) * internal_energy(U, d); }

/* Sec. 5.4: s~(U) = rho^{-gamma} eps(U), the rescaled specific entropy of eq. (EntropyEuler). */
static double s_tilde(const double* U, int d, double g) { return pow(U[0], -g) * internal_energy(U, d); }

/* Sec. 2.2, eq. (eq:euler_flux): the flux f(U) in R^{m x d} applied to a d-vector c,
 * f(U) c = [ m.c ; m (v.c) + p c ; (E + p) v.c ]. */
static void flux_dot(const double* U, const double* c, int d, double g, double* out) {
  double mc = dot(U + 1, c, d);
  double vc = mc / U[0];
  double p = pressure(U, d, g);
  out[0] = mc;
  for (int k = 0; k < d; ++k) out[1 + k] = U[1 + k] * vc + p * c[k];
  out[d + 1] = (U[d + 1] + p) * vc;
}

/* Upper bound lambda_max^+ on the maximum wave speed of the projected Riemann problem of Sec. 2.1,
 * eq. (eq:riemann_problem), used by Sec. 3.1, eq. (eq:dij_low_order).  The paper defers the formula to
 * Guermond-Popov (2016); the reading taken is the two-rarefaction pressure bound
 *   p~ = ( max(a_L + a_R - (gamma-1)/2 (u_R - u_L), 0) / (a_L p_L^{-e} + a_R p_R^{-e}) )^{1/e},
 *   e = (gamma-1)/(2 gamma),
 * which bounds the star pressure from above for 1 < gamma <= 5/3, and the extreme wave speeds at p~
 * (both monotone in p):
 *   lambda_1 = u_L - a_L sqrt(1 + (gamma+1)/(2 gamma) (p~ - p_L)^+ / p_L),
 *   lambda_3 = u_R + a_R sqrt(1 + (gamma+1)/(2 gamma) (p~ - p_R)^+ / p_R),
 *   lambda_max^+ = max((lambda_1)^-, (lambda_3)^+),  u = v.n,  a = sqrt(gamma p / rho). */
double orc_lambda_max(const double* UL, const double* UR, const double* nrm, int d, double g) {
  double rhoL = UL[0], rhoR = UR[0];
  double uL = dot(UL + 1, nrm, d) / rhoL;
  double uR = dot(UR + 1, nrm, d) / rhoR;
  double pL = pressure(UL, d, g), pR = pressure(UR, d, g);
  double aL = sqrt(g * pL / rhoL), aR = sqrt(g * pR / rhoR);
  double e = (g - 1.0) / (2.0 * g);
  double num = aL + aR - 0.5 * (g - 1.0) * (uR - uL);
  if (num < 0.0) num = 0.0;
  double den = aL * pow(pL, -e) + aR * pow(pR, -e);
  double pt = pow(num / den, 1.0 / e);
  double k = (g + 1.0) / (2.0 * g);
  double l1 = uL - aL * sqrt(1.0 + k * fmax(pt - pL, 0.0) / pL);
  double l3 = uR + aR * sqrt(1.0 + k * fmax(pt - pR, 0.0) / pR);
  return fmax(fmax(-l1, 0.0), fmax(l3, 0.0));
}

void orc_lambda_max_batch(long count, const double* UL, const double* UR, const double* nrm, int d,
                          double g, double* out) {
  int m = d + 2;
  for (long q = 0; q < count; ++q) out[q] = orc_lambda_max(UL + q * m, UR + q * m, nrm + q * d, d, g);
}

/* |c| and n = c / |c| of the entry's c_ij (0 when c_ij = 0, i.e. j is not in I(i)). */
static double entry_c(const orc_problem* P, long e, double* c, double* nrm) {
  int d = P->dim;
  for (int k = 0; k < d; ++k) c[k] = P->cij[k * P->nnz + e];
  double cn = sqrt(dot(c, c, d));
  if (cn > 0.0)
    for (int k = 0; k < d; ++k) nrm[k] = c[k] / cn;
  return cn;
}

/* Sec. 4.1: boundary state U_i^{d,k} of boundary entry b: slip, eq. (eq:slip_boundary)
 * (m^d = m - 2 (m.n) n, rho and E copied), or the given Dirichlet data. */
/* Sec. 4.1, in- and outflow: supersonic inflow (v.n < -a) takes the data, supersonic outflow (v.n >= a) the
 * interior state (eq. (eq:supersonic_inoutflow)); in between, the characteristic variables of
 * eq. (eq:characteristics) R = {v_n - 2a/(g-1), p/rho^g, v - (v.n) n, v_n + 2a/(g-1)} of the boundary state
 * are those of the data where the characteristic speed {v_n - a, v_n, v_n, v_n + a} at the interior state
 * is <= 0 (incoming) and those of the interior state otherwise.  The state is rebuilt from R:
 * v_n = (R1 + R4)/2, a = (g-1)(R4 - R1)/4, rho = (a^2 / (g R2))^(1/(g-1)), p = R2 rho^g.  The paper leaves
 * the case where the blend gives no admissible state (a <= 0: a vacuum) to a cited construction; here the
 * boundary state is then the interior state. */
static void prim_of(const double* U, int d, double g, double* v, double* p, double* a) {
  for (int k = 0; k < d; ++k) v[k] = U[1 + k] / U[0];
  *p = (g - 1.0) * internal_energy(U, d);
  *a = sqrt(g * *p / U[0]);
}

void orc_inoutflow_state(const double* Ui, const double* Ud, const double* nrm, int d, double g, double* UB) {
  int m = d + 2;
  double vi[3], vd[3], pi, pd, ai, ad;
  prim_of(Ui, d, g, vi, &pi, &ai);
  double vni = dot(vi, nrm, d);
  if (vni < -ai) {
    for (int q = 0; q < m; ++q) UB[q] = Ud[q];
    return;
  }
  if (vni >= ai) {
    for (int q = 0; q < m; ++q) UB[q] = Ui[q];
    return;
  }
  prim_of(Ud, d, g, vd, &pd, &ad);
  double vnd = dot(vd, nrm, d);
  /* subsonic: v_n - a < 0 (incoming: data), v_n + a > 0 (outgoing: interior); v_n decides the middle ones */
  const double* vsrc = vni <= 0.0 ? vd : vi;
  double R1 = vnd - 2.0 * ad / (g - 1.0);
  double R4 = vni + 2.0 * ai / (g - 1.0);
  double R2 = vni <= 0.0 ? pd / pow(Ud[0], g) : pi / pow(Ui[0], g);
  double vnsrc = dot(vsrc, nrm, d);
  double vt[3];
  for (int k = 0; k < d; ++k) vt[k] = vsrc[k] - vnsrc * nrm[k];
  double vn = 0.5 * (R1 + R4);
  double a = 0.25 * (g - 1.0) * (R4 - R1);
  if (!(a > 0.0)) {
    for (int q = 0; q < m; ++q) UB[q] = Ui[q];
    return;
  }
  double rho = pow(a * a / (g * R2), 1.0 / (g - 1.0));
  double p = R2 * pow(rho, g);
  double v2 = 0.0;
  UB[0] = rho;
  for (int k = 0; k < d; ++k) {
    double vk = vn * nrm[k] + vt[k];
    UB[1 + k] = rho * vk;
    v2 += vk * vk;
  }
  UB[d + 1] = p / (g - 1.0) + 0.5 * rho * v2;
}

static double boundary_state(const orc_problem* P, const double* U, const double* bdata, long b,
                             double* Ui, double* UB, double* c, double* nrm) {
  int d = P->dim, m = d + 2;
  for (int k = 0; k < d; ++k) c[k] = P->b_c[k * P->nb + b];
  double cn = sqrt(dot(c, c, d));
  for (int k = 0; k < d; ++k) nrm[k] = c[k] / cn;
  gather(U, P->n, P->b_node[b], m, Ui);
  if (P->b_type[b] == ORC_DIRICHLET) {
    for (int q = 0; q < m; ++q) UB[q] = bdata[q * P->nb + b];
  } else if (P->b_type[b] == ORC_INOUTFLOW) {
    double Ud[5];
    for (int q = 0; q < m; ++q) Ud[q] = bdata[q * P->nb + b];
    orc_inoutflow_state(Ui, Ud, nrm, d, P->gamma, UB);
  } else {
    double mn = dot(Ui + 1, nrm, d);
    UB[0] = Ui[0];
    for (int k = 0; k < d; ++k) UB[1 + k] = Ui[1 + k] - 2.0 * mn * nrm[k];
    UB[d + 1] = Ui[d + 1];
  }
  return cn;
}

/* Boundary entries of each node: bptr[i]..bptr[i+1] index into bidx (a counting sort of b_node). */
static void boundary_index(const orc_problem* P, long* bptr, long* bidx) {
  memset(bptr, 0, sizeof(long) * (P->n + 1));
  for (long b = 0; b < P->nb; ++b) bptr[P->b_node[b] + 1]++;
  for (long i = 0; i < P->n; ++i) bptr[i + 1] += bptr[i];
  long* fill = malloc(sizeof(long) * (P->n + 1));
  memcpy(fill, bptr, sizeof(long) * (P->n + 1));
  for (long b = 0; b < P->nb; ++b) bidx[fill[P->b_node[b]]++] = b;
  free(fill);
}

/* Sec. 3.1, eq. (eq:dij_low_order): d_ij^L = |c_ij| lambda_max^+(U_i, U_j, n_ij) for j in I(i); the
 * boundary viscosities of Sec. 4.2, eq. (eq:dij_low_order_modified), with the interior state on the
 * left (that equation and eq. (eq:dij_low_order) write the two states in opposite orders; the order of
 * eq. (eq:dij_low_order) is taken); d_ii by eq. (eq:dij_low_order_supplement). */
static void low_order_viscosities(const orc_problem* P, const double* U, const double* bdata, double* dL,
                                  double* dB, double* UB, double* dii) {
  int d = P->dim, m = d + 2;
  long n = P->n;
  double Ui[MAXM], Uj[MAXM], Ub[MAXM], c[3], nrm[3];
  ORC_PARALLEL_PRIVATE(Ui, Uj, Ub, c, nrm)
  for (long i = 0; i < n; ++i) {
    gather(U, n, i, m, Ui);
    dii[i] = 0.0;
    for (long e = P->row_ptr[i]; e < P->row_ptr[i + 1]; ++e) {
      double cn = entry_c(P, e, c, nrm);
      dL[e] = 0.0;
      if (cn == 0.0) continue;
      gather(U, n, P->col_idx[e], m, Uj);
      dL[e] = cn * orc_lambda_max(Ui, Uj, nrm, d, P->gamma);
      dii[i] -= dL[e];
    }
  }
  for (long b = 0; b < P->nb; ++b) {
    double cn = boundary_state(P, U, bdata, b, Ui, Ub, c, nrm);
    for (int q = 0; q < m; ++q) UB[q * P->nb + b] = Ub[q];
    dB[b] = cn * orc_lambda_max(Ui, Ub, nrm, d, P->gamma);
    dii[P->b_node[b]] -= dB[b];
  }
}

int orc_max_dt(const orc_problem* P, const double* U, const double* bdata, double cfl, double* tau) {
  int m = P->dim + 2;
  double* dL = malloc(sizeof(double) * (P->nnz > 0 ? P->nnz : 1));
  double* dB = malloc(sizeof(double) * (P->nb > 0 ? P->nb : 1));
  double* UB = malloc(sizeof(double) * m * (P->nb > 0 ? P->nb : 1));
  double* dii = malloc(sizeof(double) * P->n);
  low_order_viscosities(P, U, bdata, dL, dB, UB, dii);
  /* Sec. 3.3, eq. (MaxCFLdt): tau = Cr min_i ( -m_i / (2 d_ii) ) */
  double t = INFINITY;
  for (long i = 0; i < P->n; ++i)
    if (dii[i] < 0.0) t = fmin(t, -P->mi[i] / (2.0 * dii[i]));
  *tau = cfl * t;
  free(dL);
  free(dB);
  free(UB);
  free(dii);
  return 0;
}

/* Sec. 3.3, eqs. (UsualBarState), (BoundaryBarState):
 * Ubar = (U_i + U_j)/2 - |c| / (2 d) (f(U_j) - f(U_i)) n. */
static void bar_state(const double* Ui, const double* Uj, const double* nrm, double cn, double dij, int d,
                      double g, double* out) {
  int m = d + 2;
  double fi[MAXM], fj[MAXM];
  flux_dot(Ui, nrm, d, g, fi);
  flux_dot(Uj, nrm, d, g, fj);
  for (int q = 0; q < m; ++q) out[q] = 0.5 * (Ui[q] + Uj[q]) - cn / (2.0 * dij) * (fj[q] - fi[q]);
}

/* psi(t) = eps(U0 + t P) - s_min rho(t)^gamma: the constraint s~ >= s_min of the set B_i of Sec. 5.4,
 * eq. (BiSet), multiplied by rho^gamma.  psi is concave in t (eps is concave in U, rho^gamma convex),
 * so its feasible set is an interval that contains 0 when U0 is in B_i. */
static double psi(const double* U0, const double* Pv, double t, int d, double g, double smin) {
  double V[MAXM];
  for (int q = 0; q < d + 2; ++q) V[q] = U0[q] + t * Pv[q];
  if (V[0] <= 0.0) return -1.0;
  return internal_energy(V, d) - smin * pow(V[0], g);
}

static double dpsi(const double* U0, const double* Pv, double t, int d, double g, double smin) {
  double V[MAXM];
  for (int q = 0; q < d + 2; ++q) V[q] = U0[q] + t * Pv[q];
  double rho = V[0];
  double mP = dot(V + 1, Pv + 1, d), m2 = dot(V + 1, V + 1, d);
  double deps = Pv[d + 1] - mP / rho + 0.5 * m2 * Pv[0] / (rho * rho);
  return deps - smin * g * pow(rho, g - 1.0) * Pv[0];
}

/* Sec. 5.4, eq. (ConvexScheme) and Lemma ConsInvariants: the largest l in [0, 1] with U0 + l P in
 * B_i.  The paper does not state the line search; the reading taken: the density constraints give l
 * in closed form; for the entropy constraint, keep l_rho if psi(l_rho) >= 0, otherwise bracket the
 * root of psi in [0, l_rho] and iterate with the chord (feasible, psi being concave) and the tangent
 * from the infeasible end (infeasible), bisecting whenever an iteration has not halved the bracket,
 * until the bracket is at most tol wide; return the feasible end. */
static double line_search(const double* U0, const double* Pv, double rmin, double rmax, double smin,
                          int d, double g, double tol, int maxit) {
  double l = 1.0;
  if (U0[0] + Pv[0] < rmin) l = (rmin - U0[0]) / Pv[0];
  if (U0[0] + Pv[0] > rmax) l = (rmax - U0[0]) / Pv[0];
  if (!(l > 0.0)) l = 0.0;
  if (l > 1.0) l = 1.0;
  double fb = psi(U0, Pv, l, d, g, smin);
  if (fb >= 0.0) return l;
  double fa = psi(U0, Pv, 0.0, d, g, smin);
  if (fa < 0.0) return 0.0;
  double a = 0.0, b = l;
  for (int it = 0; it < maxit && b - a > tol; ++it) {
    double width = b - a;
    double ts = a + (b - a) * fa / (fa - fb); /* chord root */
    double dfb = dpsi(U0, Pv, b, d, g, smin);
    double tn = dfb < 0.0 ? b - fb / dfb : b; /* tangent root from the infeasible end */
    if (ts > a && ts < b) {
      double fs = psi(U0, Pv, ts, d, g, smin);
      if (fs >= 0.0) { a = ts; fa = fs; } else { b = ts; fb = fs; }
    }
    if (tn > a && tn < b) {
      double fn = psi(U0, Pv, tn, d, g, smin);
      if (fn >= 0.0) { a = tn; fa = fn; } else { b = tn; fb = fn; }
    }
    /* Near the root psi is evaluated below its rounding resolution (a change of t by an ulp leaves U0 + t P
     * unchanged), and the chord and tangent points then creep towards one end while the other stays put:
     * when the bracket has not halved, bisect, so that it always shrinks to tol. */
    if (b - a > 0.5 * width) {
      double tm = a + 0.5 * (b - a);
      if (!(tm > a && tm < b)) break;
      double fm = psi(U0, Pv, tm, d, g, smin);
      if (fm >= 0.0) { a = tm; fa = fm; } else { b = tm; fb = fm; }
    }
  }
  return a;
}

int orc_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

double orc_line_search(const double* U0, const double* Pv, double rmin, double rmax, double smin, int d,
                       double g, double tol, int maxit) {
  return line_search(U0, Pv, rmin, rmax, smin, d, g, tol, maxit);
}

static long transpose_entry(const orc_problem* P, long i, long j) {
  for (long e = P->row_ptr[j]; e < P->row_ptr[j + 1]; ++e)
    if (P->col_idx[e] == i) return e;
  return -1;
}

/* Solve M_K X = B for the m right-hand sides of one element by Gaussian elimination with partial
 * pivoting.  For discontinuous elements the consistent mass of Sec. 5, eq. (HighScheme), is block
 * diagonal, so the high-order update is one such solve per element. */
static void element_solve(const double* MK, int nl, int m, double* B /* [nl][m]: in B, out X */) {
  double A[MAXNL * MAXNL];
  memcpy(A, MK, sizeof(double) * nl * nl);
  for (int c = 0; c < nl; ++c) {
    int piv = c;
    for (int r = c + 1; r < nl; ++r)
      if (fabs(A[r * nl + c]) > fabs(A[piv * nl + c])) piv = r;
    if (piv != c) {
      for (int k = 0; k < nl; ++k) { double t = A[c * nl + k]; A[c * nl + k] = A[piv * nl + k]; A[piv * nl + k] = t; }
      for (int q = 0; q < m; ++q) { double t = B[c * m + q]; B[c * m + q] = B[piv * m + q]; B[piv * m + q] = t; }
    }
    for (int r = c + 1; r < nl; ++r) {
      double f = A[r * nl + c] / A[c * nl + c];
      for (int k = c; k < nl; ++k) A[r * nl + k] -= f * A[c * nl + k];
      for (int q = 0; q < m; ++q) B[r * m + q] -= f * B[c * m + q];
    }
  }
  for (int c = nl - 1; c >= 0; --c) {
    for (int q = 0; q < m; ++q) {
      double s = B[c * m + q];
      for (int k = c + 1; k < nl; ++k) s -= A[c * nl + k] * B[k * m + q];
      B[c * m + q] = s / A[c * nl + c];
    }
  }
}

#define ALLOC(p, cnt) double* p = calloc((size_t)((cnt) > 0 ? (cnt) : 1), sizeof(double))
#define OUT(dst, src, cnt) if (T && T->dst) memcpy(T->dst, src, sizeof(double) * (size_t)(cnt))

int orc_stage(const orc_problem* P, const double* Uin, const double* Ubase, double alpha, double tau,
              const double* bdata, double* Uout, orc_trace* T) {
  const int d = P->dim, m = d + 2, nl = P->n_loc;
  const long n = P->n, nnz = P->nnz, nb = P->nb;
  const double g = P->gamma;
  int flags = 0;
  double Ui[MAXM], Uj[MAXM], Ub[MAXM], c[3], nrm[3], fv[MAXM];

  long* bptr = malloc(sizeof(long) * (n + 1));
  long* bidx = malloc(sizeof(long) * (nb > 0 ? nb : 1));
  boundary_index(P, bptr, bidx);

  /* Admissible set A, Sec. 2.2, eq. (AddSet): rho > 0 and eps > 0. */
  for (long i = 0; i < n; ++i) {
    gather(Uin, n, i, m, Ui);
    if (!(Ui[0] > 0.0) || !(internal_energy(Ui, d) > 0.0)) flags |= ORC_F_INADMISSIBLE;
  }

  /* ---- boundary states and low-order viscosities (Sec. 4.1; Sec. 3.1; Sec. 4.2) ---- */
  ALLOC(dL, nnz); ALLOC(dB, nb); ALLOC(UB, m * nb); ALLOC(dii, n);
  low_order_viscosities(P, Uin, bdata, dL, dB, UB, dii);
  for (long i = 0; i < n; ++i) /* Sec. 3.3, CFL condition (CFLcond) */
    if (-2.0 * tau * dii[i] / P->mi[i] > 1.0 + 1e-12) flags |= ORC_F_CFL;
  OUT(dL, dL, nnz); OUT(dB, dB, nb); OUT(dii, dii, n); OUT(UB, UB, m * nb);

  /* ---- low-order update: Sec. 4.2, eq. (cijdijschememodified), i.e. Sec. 3.1, eq. (cijdijscheme)
   * with one boundary term per boundary part ---- */
  ALLOC(UL, m * n);
  ORC_PARALLEL_PRIVATE(Ui, Uj, Ub, c, nrm, fv)
  for (long i = 0; i < n; ++i) {
    double acc[MAXM] = {0};
    gather(Uin, n, i, m, Ui);
    for (long e = P->row_ptr[i]; e < P->row_ptr[i + 1]; ++e) {
      if (entry_c(P, e, c, nrm) == 0.0) continue; /* j not in I(i) */
      gather(Uin, n, P->col_idx[e], m, Uj);
      flux_dot(Uj, c, d, g, fv);
      for (int q = 0; q < m; ++q) acc[q] += fv[q] - dL[e] * (Uj[q] - Ui[q]);
    }
    for (long t = bptr[i]; t < bptr[i + 1]; ++t) {
      long b = bidx[t];
      for (int k = 0; k < d; ++k) c[k] = P->b_c[k * nb + b];
      for (int q = 0; q < m; ++q) Ub[q] = UB[q * nb + b];
      flux_dot(Ub, c, d, g, fv);
      for (int q = 0; q < m; ++q) acc[q] += fv[q] - dB[b] * (Ub[q] - Ui[q]);
    }
    for (int q = 0; q < m; ++q) UL[q * n + i] = Ui[q] - tau / P->mi[i] * acc[q];
  }
  OUT(UL, UL, m * n);

  /* bar states for the trace and the local bounds */
  ALLOC(ubar, m * nnz); ALLOC(ubarB, m * nb);
  ORC_PARALLEL_PRIVATE(Ui, Uj, c, nrm)
  for (long i = 0; i < n; ++i) {
    gather(Uin, n, i, m, Ui);
    for (long e = P->row_ptr[i]; e < P->row_ptr[i + 1]; ++e) {
      double cn = entry_c(P, e, c, nrm);
      if (cn == 0.0) continue;
      gather(Uin, n, P->col_idx[e], m, Uj);
      double out[MAXM];
      bar_state(Ui, Uj, nrm, cn, dL[e], d, g, out);
      for (int q = 0; q < m; ++q) ubar[q * nnz + e] = out[q];
    }
  }
  for (long b = 0; b < nb; ++b) {
    double out[MAXM];
    double cn = boundary_state(P, Uin, bdata, b, Ui, Ub, c, nrm);
    bar_state(Ui, Ub, nrm, cn, dB[b], d, g, out);
    for (int q = 0; q < m; ++q) ubarB[q * nb + b] = out[q];
  }
  OUT(ubar, ubar, m * nnz); OUT(ubarB, ubarB, m * nb);

  double* UFE = UL;
  ALLOC(N, n); ALLOC(dH, nnz); ALLOC(dBH, nb); ALLOC(UH, m * n); ALLOC(dUH, m * n);
  ALLOC(A, m * nnz); ALLOC(AB, m * nb); ALLOC(rmin, n); ALLOC(rmax, n); ALLOC(smin, n);
  ALLOC(l1, nnz); ALLOC(l1B, nb); ALLOC(l2, nnz); ALLOC(l2B, nb); ALLOC(U1, m * n); ALLOC(U2, m * n);
  ALLOC(lraw, nnz); ALLOC(lrawB, nb);

  if (P->order != ORC_LOW) {
    /* ---- entropy-viscosity indicator N_i (Sec. 5.2) ----
     * Readings: f(s) = exp(s / (gamma + 1)), so rho f = ((gamma-1)(rho E - |m|^2/2))^{1/(gamma+1)} (the
     * Harten family; f' > 0 and f'/c_p - f'' > 0 with c_p = gamma in these units); grad Phi_i is taken
     * at U_i, grad Phi_i = rho_i f'(s_i) grad_U s(U_i); the free index j in D_i is read as
     *   D_i = |sum_j psi_i(U_j).c_ij| + sum_k |[grad Phi_i]_k| |sum_j f_k(U_j) c_ij|
     * with the shifted entropy flux psi_i(U) = m (f(U) - f(U_i)), so |R_i| <= D_i; N_i = 0 when
     * D_i = 0; the sums run over I(i) (no boundary terms).  The flux sums sum_j f_k(U_j) c_ij are
     * evaluated as sum_j (f_k(U_j) - f_k(U_i)) c_ij - f_k(U_i) sum_k c_i^{d,k}, equal by the partition
     * of unity (Lemma LemPart): a node whose stencil holds a single state then gets R_i = D_i = 0
     * exactly instead of a ratio of rounding errors. */
    ORC_PARALLEL_PRIVATE(Ui, Uj, c, nrm, fv)
    for (long i = 0; i < n; ++i) {
      gather(Uin, n, i, m, Ui);
      double pi = pressure(Ui, d, g);
      double fi = exp(log(pow(Ui[0], -g) * pi) / (g + 1.0));
      double grad[MAXM];
      double pref = Ui[0] * fi / (g + 1.0); /* rho_i f'(s_i) */
      double v2 = 0.0;
      for (int k = 0; k < d; ++k) v2 += (Ui[1 + k] / Ui[0]) * (Ui[1 + k] / Ui[0]);
      /* grad_U s = grad_U p / p - (gamma / rho) e_rho,  grad_U p = (gamma-1) [|v|^2/2, -v, 1] */
      grad[0] = pref * ((g - 1.0) * 0.5 * v2 / pi - g / Ui[0]);
      for (int k = 0; k < d; ++k) grad[1 + k] = pref * (-(g - 1.0) * (Ui[1 + k] / Ui[0]) / pi);
      grad[d + 1] = pref * ((g - 1.0) / pi);
      double Fsum[MAXM] = {0}, psum = 0.0, fiv[MAXM];
      for (long e = P->row_ptr[i]; e < P->row_ptr[i + 1]; ++e) {
        if (entry_c(P, e, c, nrm) == 0.0) continue;
        gather(Uin, n, P->col_idx[e], m, Uj);
        double fj = exp(log(pow(Uj[0], -g) * pressure(Uj, d, g)) / (g + 1.0));
        flux_dot(Uj, c, d, g, fv);
        flux_dot(Ui, c, d, g, fiv);
        for (int q = 0; q < m; ++q) Fsum[q] += fv[q] - fiv[q];
        psum += dot(Uj + 1, c, d) * (fj - fi);
      }
      for (long t = bptr[i]; t < bptr[i + 1]; ++t) {
        for (int k = 0; k < d; ++k) c[k] = P->b_c[k * nb + bidx[t]];
        flux_dot(Ui, c, d, g, fiv);
        for (int q = 0; q < m; ++q) Fsum[q] -= fiv[q];
      }
      double R = psum, D = fabs(psum);
      for (int q = 0; q < m; ++q) {
        R -= grad[q] * Fsum[q];
        D += fabs(grad[q]) * fabs(Fsum[q]);
      }
      N[i] = D > 0.0 ? R / D : 0.0;
    }
    OUT(N, N, n);

    /* ---- high-order viscosity: Sec. 5, eq. (HighOrderViscosity), d^H = max(d^min, d^ev), with
     * Sec. 5.1, eq. (ViscMin), and d^ev of Sec. 5.2 ---- */
    ORC_PARALLEL_FOR
    for (long i = 0; i < n; ++i) {
      for (long e = P->row_ptr[i]; e < P->row_ptr[i + 1]; ++e) {
        long j = P->col_idx[e];
        double dmin = 0.0;
        if (P->coloc[e]) { /* c_k h_ij^{p_k} d_ij^L,  h_ij = (0.5 (m_i + m_j) / |Omega|)^{1/d} */
          double hij = pow(0.5 * (P->mi[i] + P->mi[j]) / P->omega, 1.0 / d);
          dmin = P->c_k * pow(hij, P->p_k) * dL[e];
        }
        double dev = dL[e] * fmin(P->c_ev * fmax(fabs(N[i]), fabs(N[j])), 1.0);
        dH[e] = fmax(dmin, dev);
      }
    }
    /* The paper does not define the high-order boundary viscosity; the reading taken treats the ghost
     * node as collocated with x_i (h_ij -> h_i, N_j -> N_i):
     * d^{d,H} = max(c_k h_i^{p_k}, min(c_ev |N_i|, 1)) d^{d,L}. */
    for (long b = 0; b < nb; ++b) {
      long i = P->b_node[b];
      double hi = pow(P->mi[i] / P->omega, 1.0 / d);
      dBH[b] = fmax(P->c_k * pow(hi, P->p_k), fmin(P->c_ev * fabs(N[i]), 1.0)) * dB[b];
    }
    OUT(dH, dH, nnz); OUT(dBH, dBH, nb);

    /* ---- high-order update, Sec. 5, eq. (HighScheme): sum_j m_ij (U_j^H - U_j)/tau + RHS_i^H = 0 ---- */
    ALLOC(rhs, m * n);
    ORC_PARALLEL_PRIVATE(Ui, Uj, Ub, c, nrm, fv)
    for (long i = 0; i < n; ++i) {
      gather(Uin, n, i, m, Ui);
      double acc[MAXM] = {0};
      for (long e = P->row_ptr[i]; e < P->row_ptr[i + 1]; ++e) {
        if (entry_c(P, e, c, nrm) == 0.0) continue;
        gather(Uin, n, P->col_idx[e], m, Uj);
        flux_dot(Uj, c, d, g, fv);
        for (int q = 0; q < m; ++q) acc[q] += fv[q] - dH[e] * (Uj[q] - Ui[q]);
      }
      for (long t = bptr[i]; t < bptr[i + 1]; ++t) {
        long b = bidx[t];
        for (int k = 0; k < d; ++k) c[k] = P->b_c[k * nb + b];
        for (int q = 0; q < m; ++q) Ub[q] = UB[q * nb + b];
        flux_dot(Ub, c, d, g, fv);
        for (int q = 0; q < m; ++q) acc[q] += fv[q] - dBH[b] * (Ub[q] - Ui[q]);
      }
      for (int q = 0; q < m; ++q) rhs[q * n + i] = acc[q];
    }
    double Bblk[MAXNL * MAXM];
    ORC_PARALLEL_PRIVATE(Bblk)
    for (long K = 0; K < n / nl; ++K) {
      for (int a = 0; a < nl; ++a)
        for (int q = 0; q < m; ++q) Bblk[a * m + q] = -tau * rhs[q * n + K * nl + a];
      element_solve(P->MK + K * nl * nl, nl, m, Bblk);
      for (int a = 0; a < nl; ++a)
        for (int q = 0; q < m; ++q) {
          dUH[q * n + K * nl + a] = Bblk[a * m + q];
          UH[q * n + K * nl + a] = Uin[q * n + K * nl + a] + Bblk[a * m + q];
        }
    }
    free(rhs);
    OUT(UH, UH, m * n);
    UFE = UH;
  }

  if (P->order == ORC_LIMITED) {
    /* ---- relaxed local bounds, Sec. 5.4, eq. (eq:local_bounds), r_h^{+-} = 1 +- c_r h_i^{p_r},
     * h_i = (m_i / |Omega|)^{1/d} ----
     * Reading: the outer minimum runs over I(i) and i itself, the inner one over I(j) and j itself;
     * only node i's own boundary bar states enter. */
    ORC_PARALLEL_PRIVATE(Uj, Ub, c, nrm)
    for (long i = 0; i < n; ++i) {
      double lo = INFINITY, hi = -INFINITY, sl = INFINITY;
      for (long t = bptr[i]; t < bptr[i + 1]; ++t) {
        long b = bidx[t];
        for (int q = 0; q < m; ++q) Ub[q] = ubarB[q * nb + b];
        lo = fmin(lo, Ub[0]); hi = fmax(hi, Ub[0]); sl = fmin(sl, s_tilde(Ub, d, g));
      }
      long r0 = P->row_ptr[i], r1 = P->row_ptr[i + 1];
      for (long ej = r0 - 1; ej < r1; ++ej) { /* ej = r0 - 1 stands for j = i */
        long j = i;
        if (ej >= r0) {
          if (entry_c(P, ej, c, nrm) == 0.0) continue;
          j = P->col_idx[ej];
        }
        gather(Uin, n, j, m, Uj);
        lo = fmin(lo, Uj[0]); hi = fmax(hi, Uj[0]); sl = fmin(sl, s_tilde(Uj, d, g));
        for (long ek = P->row_ptr[j]; ek < P->row_ptr[j + 1]; ++ek) {
          if (entry_c(P, ek, c, nrm) == 0.0) continue;
          double Uk[MAXM], Ubk[MAXM];
          gather(Uin, n, P->col_idx[ek], m, Uk);
          for (int q = 0; q < m; ++q) Ubk[q] = ubar[q * nnz + ek];
          lo = fmin(lo, fmin(Uk[0], Ubk[0]));
          hi = fmax(hi, fmax(Uk[0], Ubk[0]));
          sl = fmin(sl, fmin(s_tilde(Uk, d, g), s_tilde(Ubk, d, g)));
        }
      }
      /* r_h^{+-} = 1 +- c_r h_i^{p_r}, h_i = (m_i / |Omega|)^{1/d} (eq. (ViscMinConst2)'s passage); with
       * relax_measure = 1 the measure of i's element, the sum of its nodes' lumped masses, replaces m_i
       * (the reading under which the limited scheme reproduces the paper's Q2 and Q3 vortex errors) */
      double meas = P->mi[i];
      if (P->relax_measure == 1) {
        meas = 0.0;
        for (long a = (i / nl) * nl; a < (i / nl + 1) * nl; ++a) meas += P->mi[a];
      }
      double hh = pow(pow(meas / P->omega, 1.0 / d), P->p_r);
      double rm = 1.0 - P->c_r * hh, rp = 1.0 + P->c_r * hh;
      if (P->bounds_mode == 1) {
        rmin[i] = 0.0; rmax[i] = INFINITY; smin[i] = 0.0;
      } else {
        rmin[i] = rm * lo; rmax[i] = rp * hi; smin[i] = rm * sl;
      }
    }
    OUT(rho_min, rmin, n); OUT(rho_max, rmax, n); OUT(s_min, smin, n);

    /* ---- antidiffusive fluxes, Sec. 5.3, eq. (HighLowOrderIdentity) with the fluxes of
     * eq. (skewSymmetric) and eq. (HighSchemeAlgebraic):
     *   A_ij = tau (d_ij^H - d_ij^L)(U_j - U_i) - (m_ij - delta_ij m_i)(dU_j^H - dU_i^H),
     *   A_i^{d,k} = tau (d^{d,H} - d^{d,L})(U^{d,k} - U_i). ---- */
    ORC_PARALLEL_FOR
    for (long i = 0; i < n; ++i) {
      long K = i / nl;
      for (long e = P->row_ptr[i]; e < P->row_ptr[i + 1]; ++e) {
        long j = P->col_idx[e];
        double mij = (j / nl == K) ? P->MK[K * nl * nl + (i % nl) * nl + (j % nl)] : 0.0;
        for (int q = 0; q < m; ++q)
          A[q * nnz + e] = tau * (dH[e] - dL[e]) * (Uin[q * n + j] - Uin[q * n + i]) -
                           mij * (dUH[q * n + j] - dUH[q * n + i]);
      }
    }
    for (long b = 0; b < nb; ++b) {
      long i = P->b_node[b];
      for (int q = 0; q < m; ++q) AB[q * nb + b] = tau * (dBH[b] - dB[b]) * (UB[q * nb + b] - Uin[q * n + i]);
    }
    OUT(A, A, m * nnz); OUT(AB, AB, m * nb);

    /* ---- convex limiting, Sec. 5.4, eq. (ConvexScheme): kappa_i = 1 / (number of terms),
     * P_ij = A_ij / (kappa_i m_i), one line search per term; l_ij = min(l_ij^(i), l_ji^(j)) gives the
     * symmetry Lemma ConsInvariants needs; eq. (LimitedScheme) forms the update.  Sec. 6.1 runs the
     * limiter twice: pass 2 limits the remainder (1 - l) A from the pass-1 state against the same
     * bounds.  Reading: the number of terms is the row length of i plus i's boundary entries. ---- */
    memcpy(U1, UL, sizeof(double) * m * n);
    memcpy(U2, UL, sizeof(double) * m * n);
    ALLOC(Arem, m * nnz); ALLOC(ABrem, m * nb);
    memcpy(Arem, A, sizeof(double) * m * nnz);
    memcpy(ABrem, AB, sizeof(double) * m * nb);
    double* Ufrom = UL;
    double* Uto = U1;
    for (int pass = 0; pass < P->limiter_passes; ++pass) {
      double* lsym = pass == 0 ? l1 : l2;
      double* lsymB = pass == 0 ? l1B : l2B;
      ORC_PARALLEL_FOR
      for (long i = 0; i < n; ++i) {
        long nterms = (P->row_ptr[i + 1] - P->row_ptr[i]) + (bptr[i + 1] - bptr[i]);
        double kappa = 1.0 / (double)nterms;
        double U0[MAXM], Pv[MAXM];
        gather(Ufrom, n, i, m, U0);
        for (long e = P->row_ptr[i]; e < P->row_ptr[i + 1]; ++e) {
          for (int q = 0; q < m; ++q) Pv[q] = Arem[q * nnz + e] / (kappa * P->mi[i]);
          lraw[e] = line_search(U0, Pv, rmin[i], rmax[i], smin[i], d, g, P->ls_tol, P->ls_maxit);
        }
        for (long t = bptr[i]; t < bptr[i + 1]; ++t) {
          long b = bidx[t];
          for (int q = 0; q < m; ++q) Pv[q] = ABrem[q * nb + b] / (kappa * P->mi[i]);
          lrawB[b] = line_search(U0, Pv, rmin[i], rmax[i], smin[i], d, g, P->ls_tol, P->ls_maxit);
        }
      }
      ORC_PARALLEL_FOR
      for (long i = 0; i < n; ++i)
        for (long e = P->row_ptr[i]; e < P->row_ptr[i + 1]; ++e)
          lsym[e] = fmin(lraw[e], lraw[transpose_entry(P, i, P->col_idx[e])]);
      memcpy(lsymB, lrawB, sizeof(double) * nb);
      ORC_PARALLEL_FOR
      for (long i = 0; i < n; ++i) {
        double acc[MAXM] = {0};
        for (long e = P->row_ptr[i]; e < P->row_ptr[i + 1]; ++e)
          for (int q = 0; q < m; ++q) acc[q] += lsym[e] * Arem[q * nnz + e];
        for (long t = bptr[i]; t < bptr[i + 1]; ++t)
          for (int q = 0; q < m; ++q) acc[q] += lsymB[bidx[t]] * ABrem[q * nb + bidx[t]];
        for (int q = 0; q < m; ++q) Uto[q * n + i] = Ufrom[q * n + i] + acc[q] / P->mi[i];
      }
      for (long e = 0; e < nnz; ++e)
        for (int q = 0; q < m; ++q) Arem[q * nnz + e] *= (1.0 - lsym[e]);
      for (long b = 0; b < nb; ++b)
        for (int q = 0; q < m; ++q) ABrem[q * nb + b] *= (1.0 - lsymB[b]);
      Ufrom = U1;
      Uto = U2;
    }
    OUT(U1, U1, m * n);
    OUT(l1, l1, nnz); OUT(l1B, l1B, nb); OUT(l2, l2, nnz); OUT(l2B, l2B, nb);
    UFE = P->limiter_passes == 0 ? UL : (P->limiter_passes == 1 ? U1 : U2);
    free(Arem);
    free(ABrem);
  }

  /* ---- Shu-Osher combination of the SSP Runge-Kutta stages (SSPRK3 in Sec. 6.2) ---- */
  for (long q = 0; q < (long)m * n; ++q)
    Uout[q] = (alpha != 0.0 && Ubase) ? alpha * Ubase[q] + (1.0 - alpha) * UFE[q] : UFE[q];

  free(bptr); free(bidx);
  free(dL); free(dB); free(UB); free(dii); free(UL); free(ubar); free(ubarB);
  free(N); free(dH); free(dBH); free(UH); free(dUH); free(A); free(AB);
  free(rmin); free(rmax); free(smin); free(l1); free(l1B); free(l2); free(l2B); free(U1); free(U2);
  free(lraw); free(lrawB);
  return flags;
}
