/* Oracle for one forward-Euler stage of the convex-limited graph-based dG scheme for the compressible
 * Euler equations (Kronbichler, Maier, Tomas, arXiv 2402.04514).
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow FP64 CPU restatement of the paper's algorithm,
 * written loop by loop in the paper's order, used to check the CUDA library.  Only tests/,
 * __graft_entry__.smoke() and bench.py's cpu_baseline / reference arm may build, load or call it;
 * the library never does.  It shares no code, header or helper with the library.
 *
 * Layouts: states are component-major, U[c * n + i], c = 0 (rho), 1..d (momentum), d+1 (E).
 * c_ij is [dim][nnz] (cij[k * nnz + e]); boundary normals b_c are [dim][nb]; Dirichlet data bdata is
 * [m][nb].  Rows are element-contiguous with n_loc nodes per element; MK holds the consistent mass
 * block of each element, [n / n_loc][n_loc][n_loc].
 */
#ifndef ORC_ORACLE_H
#define ORC_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_LOW = 0, ORC_HIGH = 1, ORC_LIMITED = 2 };
enum { ORC_SLIP = 0, ORC_DIRICHLET = 1, ORC_INOUTFLOW = 2 };
/* stage flags (bitmask) */
enum { ORC_F_INADMISSIBLE = 1, ORC_F_CFL = 2 };

typedef struct {
  int dim, degree, n_loc;
  long n, nnz, nb;
  const long* row_ptr;
  const int* col_idx;
  const double* cij;
  const unsigned char* coloc;
  const double* mi;
  const double* MK;
  const int* b_node;
  const double* b_c;
  const int* b_type;
  double gamma, omega;
  int order;          /* ORC_LOW, ORC_HIGH, ORC_LIMITED */
  int limiter_passes; /* 0, 1 or 2 (Sec. 6.1: the limiter runs twice) */
  int bounds_mode;    /* 0: relaxed local bounds (Eq. (5.8)); 1: rho >= 0, s~ >= 0 only (test knob) */
  double c_k, p_k, c_ev, c_r, p_r;
  double ls_tol;
  int ls_maxit;
  int relax_measure;  /* 0: h_i = (m_i / |Omega|)^{1/d} in r_h (Sec. 5.4 as printed); 1: h_i of i's element */
} orc_problem;

/* Optional outputs of a stage; every pointer may be NULL. */
typedef struct {
  double* dL;    /* [nnz] low-order graph viscosity d_ij^L (0 where c_ij = 0) */
  double* dB;    /* [nb]  boundary viscosity d_i^{d,k} */
  double* dii;   /* [n]   Eq. (3.4) */
  double* UB;    /* [m][nb] boundary states U_i^{d,k} */
  double* ubar;  /* [m][nnz] bar states (0 where c_ij = 0) */
  double* ubarB; /* [m][nb] boundary bar states */
  double* UL;    /* [m][n] low-order update */
  double* N;     /* [n] normalised entropy residual N_i */
  double* dH;    /* [nnz] high-order viscosity */
  double* dBH;   /* [nb] high-order boundary viscosity */
  double* UH;    /* [m][n] high-order update */
  double* A;     /* [m][nnz] antidiffusive fluxes A_ij */
  double* AB;    /* [m][nb] boundary fluxes A_i^{d,k} */
  double* rho_min; double* rho_max; double* s_min; /* [n] relaxed local bounds */
  double* l1; double* l1B; /* [nnz], [nb] symmetrised limiter coefficients, pass 1 */
  double* l2; double* l2B; /* pass 2 */
  double* U1;    /* [m][n] state after pass 1 */
} orc_trace;

/* Threads a stage's row loops use: 1 in the default build, OpenMP's thread count in the -fopenmp build. */
int orc_threads(void);
/* Upper bound on the maximum wave speed of the 1D Riemann problem (U_L, U_R) along unit n. */
double orc_lambda_max(const double* UL, const double* UR, const double* nrm, int dim, double gamma);
/* The line search of the limiter (Sec. 5.4): the largest l in [0, 1] with U0 + l Pv inside the bounds
 * rho in [rmin, rmax], p / rho^g >= smin (see oracle.c for the iteration). */
double orc_line_search(const double* U0, const double* Pv, double rmin, double rmax, double smin, int dim,
                       double gamma, double tol, int maxit);
/* Boundary state of an in/outflow entry (Sec. 4.1, eqs. (eq:supersonic_inoutflow), (eq:characteristics))
 * from the interior state Ui, the given data Ud and the outward unit normal nrm; written to UB. */
void orc_inoutflow_state(const double* Ui, const double* Ud, const double* nrm, int dim, double gamma, double* UB);
void orc_lambda_max_batch(long count, const double* UL, const double* UR, const double* nrm, int dim,
                          double gamma, double* out); /* UL/UR [count][m], nrm [count][dim] */

/* Eq. (3.9): tau = cfl * min_i(-m_i / (2 d_ii)).  Returns stage flags. */
int orc_max_dt(const orc_problem* P, const double* U, const double* bdata, double cfl, double* tau);

/* U_out = alpha * U_base + (1 - alpha) * FE(U_in); U_base may be NULL when alpha == 0.
 * Returns stage flags (ORC_F_*). */
int orc_stage(const orc_problem* P, const double* U_in, const double* U_base, double alpha, double tau,
              const double* bdata, double* U_out, orc_trace* T);

#ifdef __cplusplus
}
#endif
#endif
