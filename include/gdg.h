/* gdg: GB300-native forward-Euler stage of the invariant-domain-preserving graph-based
 * discontinuous Galerkin scheme for the compressible Euler equations (Kronbichler, Maier, Tomas,
 * arXiv 2402.04514).  C ABI; all compute runs in CUDA kernels for sm_103a, in FP64.
 *
 * One stage (gdg_stage) computes, on the algebraic stencil of Sec. 2.3:
 *   - the low-order update, Sec. 3.1, eq. (cijdijscheme), with the graph viscosity of
 *     eq. (eq:dij_low_order) and the multi-valued boundary terms of Sec. 4.2,
 *     eq. (cijdijschememodified);
 *   - the high-order update of Sec. 5, eq. (HighScheme), with the viscosity of eq. (HighOrderViscosity)
 *     (minimal viscosity, Sec. 5.1, eq. (ViscMin); entropy viscosity, Sec. 5.2) and the consistent
 *     element mass;
 *   - the relaxed local bounds of Sec. 5.4, eq. (eq:local_bounds), and two passes of the convex-limiting
 *     line search of eq. (ConvexScheme) that blend the two (Sec. 6.1);
 *   - the Shu-Osher combination U_out = alpha U_base + (1 - alpha) U_FE of an SSP Runge-Kutta stage.
 * gdg_max_dt computes the time step of Sec. 3.3, eq. (MaxCFLdt).
 *
 * Conventions
 *   States are FP64, component-major: U[c * n + i], c = 0 (rho), 1..dim (momentum), dim+1 (E).
 *   Vector-valued per-entry data is [dim][count] (component-major).
 *   Every pointer named "device" is a CUDA device pointer on the handle's device; "host" pointers are
 *   read during the call only and stay owned by the caller.
 *   Return codes are gdg_status_code values; gdg_error_string() names them.
 *   stream is a cudaStream_t passed as void* (NULL = the legacy default stream).
 */
#ifndef GDG_H
#define GDG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  GDG_OK = 0,
  GDG_EINVAL = 1,       /* bad argument (NULL pointer, size out of range, aliasing) */
  GDG_ENOMEM = 2,       /* device or host allocation failed */
  GDG_ECUDA = 3,        /* a CUDA runtime call failed */
  GDG_ESETUP = 4,       /* problem data violates a requirement listed at gdg_problem */
  GDG_EADMISSIBLE = 5,  /* a state handed to a stage is not admissible (rho <= 0 or eps <= 0) */
  GDG_ECFL = 6,         /* a stage ran with tau above the CFL limit of eq. (CFLcond) */
  GDG_ETIMEOUT = 7,     /* reserved: a bounded device-side wait gave up */
  GDG_ENOTSUP = 8       /* configuration not supported (dim > 3, n_loc > 32, nnz >= 2^31, ...) */
} gdg_status_code;

enum { GDG_ORDER_LOW = 0, GDG_ORDER_HIGH = 1, GDG_ORDER_LIMITED = 2 };
/* boundary entry types (Sec. 4.1): slip wall, Dirichlet data, in/outflow (supersonic and subsonic,
 * from the characteristic variables of eq. (eq:characteristics); needs data like Dirichlet entries) */
enum { GDG_BC_SLIP = 0, GDG_BC_DIRICHLET = 1, GDG_BC_INOUTFLOW = 2 };
/* sticky device flags, read by gdg_status */
enum { GDG_FLAG_INADMISSIBLE = 1, GDG_FLAG_CFL = 2 };
/* arithmetic of the sweep (gdg_params.precision).  GDG_PRECISION_FP64: every step in FP64.
 * GDG_PRECISION_MIXED: a faster path whose results differ from the FP64 path by up to about 1e-5 of
 * max |U| per stage: the coefficients of the scheme (the primitives behind lambda_max^+ of Sec. 3.1, the
 * wave-speed bound itself, raised by a margin that covers its FP32 rounding so that d_ij^L still bounds
 * the FP64 value from above, the entropy-viscosity indicator of Sec. 5.2, the entropy of the bar states
 * in the bounds of Sec. 5.4, the high-order correction dU^H of Sec. 5 and the antidiffusive fluxes A_ij
 * of Sec. 5.3) are computed in FP32 and held as FP64 values, while the low-order fluxes and row sums,
 * every state update and the limiter's acceptance tests stay FP64.  d_ij^L and the limiter coefficients
 * stay symmetric and A_ij antisymmetric bit for bit, so the limited and low-order schemes conserve to
 * FP64 rounding and the limiter enforces the local bounds exactly as in the FP64 path (the unlimited
 * high order, a test setting, conserves only to the FP32 accuracy of dU^H).  States must have rho, p
 * and the velocities inside the FP32 normal range (about 1e-37 .. 1e37); a wave-speed bound that comes
 * out infinite or NaN in FP32 is recomputed in FP64. */
enum { GDG_PRECISION_FP64 = 0, GDG_PRECISION_MIXED = 1 };

/* Method parameters.  gdg_default_params fills the paper's values: c_k = 1 and p_k = 1/2 (k even),
 * 0 (k odd) of Sec. 5.1; c_ev = 1, 0.5, 0.25 for k = 1, 2, >= 3 (Sec. 5.2); c_r = 4, p_r = 1.5
 * (Sec. 5.4, eq. (ViscMinConst2)); two limiter passes (Sec. 6.1); line-search bracket tolerance
 * 1e-14 with at most 50 iterations. */
typedef struct {
  int32_t order;          /* GDG_ORDER_LOW: eq. (cijdijscheme) only; GDG_ORDER_HIGH: eq. (HighScheme)
                             without limiting; GDG_ORDER_LIMITED: eq. (LimitedScheme) */
  int32_t limiter_passes; /* 0, 1 or 2 */
  int32_t bounds_mode;    /* 0: relaxed local bounds of eq. (eq:local_bounds); 1: only rho >= 0 and
                             s~ >= 0 (a test knob: the limiter then keeps every admissible U^H) */
  double c_k, p_k, c_ev, c_r, p_r;
  double ls_tol;
  int32_t ls_maxit;
  int32_t precision;      /* GDG_PRECISION_FP64 (default) or GDG_PRECISION_MIXED */
  int32_t relax_measure;  /* the mesh size h_i of the relaxation r_h^+- = 1 +- c_r h_i^{p_r} (Sec. 5.4):
                             GDG_RELAX_NODE (default): h_i = (m_i / |Omega|)^{1/d} as eq. (ViscMinConst2)'s
                             passage prints it; GDG_RELAX_ELEMENT: h_i = (|K_i| / |Omega|)^{1/d} with |K_i|
                             the measure (the sum of the lumped masses) of i's element, with which the
                             limited scheme reproduces the paper's Q2 and Q3 vortex table */
} gdg_params;
enum { GDG_RELAX_NODE = 0, GDG_RELAX_ELEMENT = 1 };

/* One mesh instance (all host pointers, copied by gdg_setup).
 * Requirements (gdg_setup returns GDG_ESETUP when one fails):
 *   - rows are element-contiguous: element e owns nodes [e n_loc, (e+1) n_loc), n % n_loc == 0;
 *   - row i lists every other node of its element (the consistent mass couples them all) and every j
 *     with c_ij != 0; no diagonal entry; no duplicates; entries with c_ij = 0 carry only m_ij;
 *   - c_ji == -c_ij exactly for every entry (Lemma PropSkew) and the transpose of every entry exists;
 *   - partition of unity sum_j c_ij + sum_k c_i^{d,k} = 0 (Lemma LemPart) to 1e-12 relative;
 *   - coloc[e] = 1 iff x_i == x_j (face partners across an element face), symmetric;
 *   - m_i > 0 and sum_j MK[e][a][j] == m_i to 1e-12 relative (Sec. 5.3 absorbs the consistent mass into
 *     the fluxes using sum_j (m_ij - delta_ij m_i) = 0); every MK block symmetric positive definite;
 *   - boundary entries: 0 <= b_node < n, |c_i^{d,k}| > 0, b_type GDG_BC_SLIP, GDG_BC_DIRICHLET or
 *     GDG_BC_INOUTFLOW;
 *   - gamma > 1, omega_measure = |Omega| > 0; for the limited order with bounds_mode 0,
 *     r_h^- = 1 - c_r h_i^{p_r} > 0 at every node (h_i = (m_i / |Omega|)^{1/dim}). */
typedef struct {
  int32_t dim;            /* 1, 2 or 3 (m = dim + 2 components) */
  int32_t degree;         /* polynomial degree k of the Q^k elements */
  int32_t n_loc;          /* nodes per element, (k+1)^dim for Q^k, at most 32 */
  int64_t n;              /* nodes */
  int64_t nnz;            /* CSR entries (< 2^31) */
  int64_t nb;             /* boundary entries (i, k) of Sec. 4.2 */
  const int64_t* row_ptr; /* host [n+1] */
  const int32_t* col_idx; /* host [nnz] */
  const double* cij;      /* host [dim][nnz]: c_ij of eq. (eq:cij_def1) */
  const uint8_t* coloc;   /* host [nnz] */
  const double* mi;       /* host [n]: lumped mass m_i of eq. (eq:mass_matrices) */
  const double* MK;       /* host [n / n_loc][n_loc][n_loc]: consistent element mass blocks m_ij */
  const int32_t* b_node;  /* host [nb] */
  const double* b_c;      /* host [dim][nb]: c_i^{d,k} of Sec. 4.2 */
  const int32_t* b_type;  /* host [nb] */
  double gamma;           /* ratio of specific heats, eq. (PressurEuler) */
  double omega_measure;   /* |Omega| (Sec. 5.1 and 5.4 dimensionless mesh sizes) */
  gdg_params params;
} gdg_problem;

typedef struct gdg_handle gdg_handle;

typedef struct {
  int64_t n, nnz, nb;
  int32_t dim, n_loc;
  int64_t device_bytes;   /* device memory held by the handle (setup copies and scratch) */
} gdg_info;

void gdg_default_params(int32_t degree, gdg_params* out);

/* Validates and copies the problem to the current CUDA device, derives the per-entry and per-node
 * data of the sweep (unit normals, transpose map, element mass inverses, relaxation factors) and
 * allocates all scratch.  *out is owned by the caller and released with gdg_destroy.
 * Errors: GDG_EINVAL (NULL), GDG_ENOTSUP, GDG_ESETUP, GDG_ENOMEM, GDG_ECUDA; *out is NULL on error. */
int gdg_setup(const gdg_problem* prob, gdg_handle** out);

/* Device bytes gdg_setup would allocate for prob (its arena: setup copies and scratch; the caller's
 * state buffers are not included), without touching the device.  Reads row_ptr, col_idx and cij only.
 * Errors: GDG_EINVAL. */
int gdg_footprint(const gdg_problem* prob, int64_t* bytes);

/* Replaces the method parameters of a handle (same validation as gdg_setup). */
int gdg_set_params(gdg_handle* h, const gdg_params* params);

/* Sec. 3.3, eq. (MaxCFLdt): *tau_out = cfl * min_i (-m_i / (2 d_ii)), d_ii of
 * eq. (eq:dij_low_order_supplement) at the state U (device [m][n]).  bdata (device [m][nb], in the
 * order of gdg_problem's boundary entries) holds the data of the Dirichlet and in/outflow entries; it
 * may be NULL when every entry is a slip wall.  Synchronises the stream.  Flags an inadmissible U. */
int gdg_max_dt(gdg_handle* h, const double* U, const double* bdata, double cfl, double* tau_out,
               void* stream);

/* One forward-Euler stage with step tau followed by the SSP Runge-Kutta combination:
 *   U_out = alpha * U_base + (1 - alpha) * FE(U_in)        (U_base may be NULL when alpha == 0).
 * U_in, U_base, U_out: device [m][n]; U_out must not alias U_in (GDG_EINVAL); it may equal U_base (each
 * node reads its base value before its output is written).  bdata as in gdg_max_dt, evaluated at the
 * stage time.  Asynchronous on stream; allocates nothing; inadmissible input and a CFL violation set
 * sticky flags (gdg_status), never trap. */
int gdg_stage(gdg_handle* h, const double* U_in, const double* U_base, double alpha, double tau,
              const double* bdata, double* U_out, void* stream);

/* One whole SSP-RK3 step (Sec. 6.2, Shu-Osher form) with the time step chosen and kept on the device:
 *   tau = min(cfl * min_i (-m_i / (2 d_ii(U))), t_end - t)     (Sec. 3.3, eq. (MaxCFLdt); 0 once t >= t_end)
 *   U1 = FE_tau(U) -> T1;  U2 = 3/4 U + 1/4 FE_tau(U1) -> T2;  U <- 1/3 U + 2/3 FE_tau(U2)  (in place)
 * then t += tau.  cfl, t and t_end are the handle's clock (gdg_clock_set; t = 0, t_end = +inf, cfl = 0.5
 * after gdg_setup).  The bound is reduced from the first stage's edge sweep, so the step does no work
 * twice and never waits for the host: it is asynchronous on stream and allocates nothing.  U, T1, T2:
 * device [m][n], distinct (GDG_EINVAL otherwise); T1 and T2 are workspace.  bdata: Dirichlet data as in
 * gdg_stage, used unchanged at the three stage times (for time-dependent data call gdg_stage).
 * Flags as gdg_stage. */
int gdg_ssprk3_step(gdg_handle* h, double* U, double* T1, double* T2, const double* bdata, void* stream);

/* gdg_ssprk3_step for a state kept in host memory: reads the step's input from U_host_in (host [m][n]),
 * runs the step on the device in U, T1, T2 (device [m][n], distinct; all three overwritten, U left holding
 * the new state) and writes the new state to U_host_out (host [m][n]; may equal U_host_in).
 * When U_host_in is page-locked memory mapped into the device's address space (cudaHostAlloc,
 * cudaMallocHost, or cudaHostRegister with mapping), the first stage's primitive sweep reads it over the
 * host link and stores it in U itself, so that the transfer overlaps that sweep's arithmetic; if
 * U_host_out is such memory too, the last stage's sweeps write each node's new state there as they write
 * it to U, overlapping the transfer back with the rest of the stage.  Other buffers are copied by
 * cudaMemcpyAsync before and after the step.
 * Asynchronous on stream for page-locked buffers: U_host_out is complete, and U_host_in may change, only
 * once the stream has been synchronized (pageable buffers make the copies wait for the host as
 * cudaMemcpyAsync does).  Clock, bdata (device), flags and errors as gdg_ssprk3_step; with a finished clock
 * the state is copied through unchanged. */
int gdg_ssprk3_step_host(gdg_handle* h, const double* U_host_in, double* U_host_out, double* U, double* T1,
                         double* T2, const double* bdata, void* stream);

/* One SSPRK(5,4) step: the five-stage fourth-order SSP Runge-Kutta method the paper's experiments use
 * (Sec. 6.2; the optimal coefficients of Spiteri and Ruuth, SSP coefficient C = 1.508), in Shu-Osher form
 * from limited forward-Euler stages, with dt = min(cfl * C * min_i (-m_i / (2 d_ii(U))), t_end - t) chosen
 * on the device as in gdg_ssprk3_step (each stage's forward-Euler step is at most cfl times the bound of
 * eq. (MaxCFLdt)).  Five stage sweeps and two elementwise combinations; the result is written back to U.
 * U, T1, T2, T3: device [m][n], distinct (GDG_EINVAL otherwise); T1..T3 are workspace.  Clock, bdata,
 * flags, asynchrony and allocation as gdg_ssprk3_step. */
int gdg_ssprk54_step(gdg_handle* h, double* U, double* T1, double* T2, double* T3, const double* bdata,
                     void* stream);

/* Sets the clock of gdg_ssprk3_step and gdg_ssprk54_step: current time t, final time t_end >= t (+inf: no end), CFL number
 * cfl > 0; resets the step count.  Synchronises the stream. */
int gdg_clock_set(gdg_handle* h, double t, double t_end, double cfl, void* stream);

/* Reads the clock: current time, tau of the last step, completed steps (any pointer may be NULL; steps
 * taken after t reached t_end change nothing and are not counted).  Synchronises the stream. */
int gdg_clock_get(gdg_handle* h, double* t, double* tau, int64_t* steps, void* stream);

/* Reads (and with clear != 0 resets) the sticky device flags GDG_FLAG_*; synchronises the stream. */
int gdg_status(gdg_handle* h, int32_t* flags, int32_t clear, void* stream);

/* Copies an intermediate of the last stage to host memory (for tests and diagnostics): name is one of
 * "dL" [nnz], "dB" [nb], "N" [n], "UL" [m][n], "rho_min" [n], "rho_max" [n], "s_min" [n], "l1" [nnz],
 * "l2" [nnz] (written only where min(l1_ij, l1_ji) < 1, the entries whose pass-2 factor multiplies a
 * nonzero remainder), "U1" [m][n], "A" [m][nnz]; entries follow gdg_problem's order (boundary data its
 * own).
 * "ls_deferred" [2] gives the number of line searches of each limiter pass that needed the bracketed
 * iteration (run by a separate kernel over a queue).  count must equal the array size.  Synchronises
 * the stream. */
int gdg_debug_export(gdg_handle* h, const char* name, double* host_dst, int64_t count, void* stream);

/* Kernel timing for measurement.  With gdg_profile(h, 1) every kernel launch of gdg_stage,
 * gdg_ssprk3_step and gdg_max_dt is bracketed by CUDA events recorded on the launching stream (no synchronisation is
 * added).  gdg_profile_read synchronises, accumulates the elapsed time of each kernel of the sweep
 * (indices GDG_K_*) into total_ms[GDG_NKERNELS] and launches[GDG_NKERNELS], and clears the records.
 * gdg_profile(h, 0) stops recording and drops pending records. */
enum { GDG_K_PRIM = 0, GDG_K_MAXDT = 1, GDG_K_LOW = 2, GDG_K_HIGH = 3, GDG_K_LIMIT2 = 4, GDG_K_FINAL = 5,
       GDG_K_EDGE = 6, GDG_K_LSFIX = 7, GDG_K_TAU = 8, GDG_K_CLOCK = 9, GDG_K_AXPY = 10, GDG_NKERNELS = 11 };
int gdg_profile(gdg_handle* h, int32_t enable);
int gdg_profile_read(gdg_handle* h, double* total_ms, int64_t* launches);

/* Self-test of the FP64 helpers that replace CUDA's division, power and square root on the sweep's hot
 * loops: fn 0 = reciprocal from an FP32 seed, 1 = x^{-1/q} from an FP32 seed, 2 = CUDA's 1.0 / x,
 * 3 = CUDA's pow(x, -1.0 / q), 4 = the integer-only FP64 -> FP32 -> FP64 conversion pair of the FP32
 * certificates (truncation to 23 significand bits in the FP32 normal range, zeros kept, NaN otherwise),
 * 5 = square root from the FP32 reciprocal square root, 6 = CUDA's sqrt; x, y: device [n];
 * 1 <= q <= 16.  fn 7..10 take pairs: x is [2n] and y[i] is computed from x[2i] and x[2i+1] by 7 = the
 * integer-pipe binary64 product of the sweep kernels, 8 = CUDA's __dmul_rn, 9 = the integer-pipe sum,
 * 10 = CUDA's __dadd_rn, 11 = the integer-pipe scaling x[2i] * 2^k with k = x[2i+1], an integer in
 * [-1022, 1023] (q is not used).  Asynchronous on stream.  The tests compare 0 with 2, 1 with 3
 * and 5 with 6 in ulps, 4 with the truncation done on the host, 7 with 8 and 9 with 10 bit for bit. */
int gdg_math_selftest(int32_t fn, int32_t q, const double* x, double* y, int64_t n, void* stream);

/* Check of the mixed-precision wave-speed bound (GDG_PRECISION_MIXED) against the FP64 one, for gamma
 * and n one-dimensional Riemann problems states[k] = (rho_L, u_L, p_L, rho_R, u_R, p_R) (device [n][6],
 * u the normal velocities): out[k] = (lambda_max^+ as the FP64 path computes it, the mixed path's
 * bound with its margin, the same without the margin, the margin's scale S) (device [n][4]), from the
 * per-node primitives each path computes.  The mixed bound must not fall below the FP64 one.
 * Asynchronous on stream.  Errors: GDG_EINVAL (gamma <= 1, n < 0, NULL arrays with n > 0). */
int gdg_wave_speed_check(double gamma, const double* states, double* out, int64_t n, void* stream);

/* Check of the FP32 certificate that lets the line search of Sec. 5.4 skip an FP64 evaluation of the
 * entropy constraint psi(s) = eps(U0 + s A) - s_min rho(U0 + s A)^gamma: for n rows
 * in[k] = (U0[m], A[m], s_min, s) (device [n][2m + 2], m = dim + 2), out[k] = (1 if the certificate proves
 * psi(s) >= 0 else 0, psi(s) in FP64) (device [n][2]).  A certified row must have psi(s) >= 0.
 * Asynchronous on stream.  Errors: GDG_EINVAL (dim outside 1..3, gamma <= 1, n < 0, NULL arrays). */
int gdg_certificate_check(int32_t dim, double gamma, const double* in, double* out, int64_t n, void* stream);

/* Measured throughput (operations per second over the GPU, timed with CUDA events) of the arithmetic
 * the sweep is made of: op 0 = FP64 FMA, 1 = FP64 division, 2 = FP64 sqrt, 3 = FP64 pow, 4 = FP32 FMA,
 * 5 = this library's FP64 reciprocal, 6 = this library's x^{-1/5}, 7 = an FP64 -> FP32 -> FP64
 * conversion pair, 8 = FP64 multiplication, 9 = the integer-pipe binary64 product of the sweep kernels,
 * 10 = half of the chains on each of the two, 11 = FP64 addition, 12 = the integer-pipe sum, 13 = a
 * quarter of the chains on the integer pipe.  Allocates and frees a scratch
 * buffer; synchronises the stream.  Used for the FP64 roofline of the measurement script. */
int gdg_fp64_throughput(int32_t op, double* ops_per_s, void* stream);

/* Time step without any device allocation.  The paper has no counterpart: this is a service for
 * callers that may not allocate device memory themselves.  Examples are:
 *   - code that runs while a CUDA stream is being captured into a graph, where cudaMalloc and
 *     cudaFree are not allowed;
 *   - plug-ins inside an application whose device memory belongs to its own pool or budget (a caching
 *     allocator, a serving process with a fixed HBM share), where a private cudaMalloc bypasses that
 *     accounting and can fail or fragment the pool;
 *   - latency-sensitive paths that cannot afford the implicit synchronisation of cudaMalloc.
 * Such callers cannot create a gdg_handle (gdg_setup allocates), so this entry takes the mesh as device
 * arrays they own and computes the same tau as gdg_max_dt: cfl * min_i (-m_i / (2 d_ii)).
 *
 * Inputs (device pointers owned by the caller, read only):
 *   row_ptr [n+1] and col_idx [nnz] (int32 CSR, as in gdg_problem), cij [dim][nnz], mi [n];
 *   boundary entries ordered by node: those of node i are b_ptr[i] .. b_ptr[i+1]-1 (int32 [n+1]), with
 *   b_c [dim][nb] and b_type [nb] in that order, and bdata [m][nb] (the data of the Dirichlet and
 *   in/outflow entries in the same order; may be NULL when every entry is a slip wall).
 * The arrays are trusted, not checked: they must satisfy the rules gdg_setup checks on the host (row_ptr
 * non-decreasing from 0 to nnz, 0 <= col_idx < n with no diagonal entry, b_ptr non-decreasing from 0 to
 * nb, m_i > 0, c_ij = -c_ji, U admissible).  Reading them on the device to check would cost the caller a
 * synchronisation; an index out of range is an out-of-bounds read.
 * NaN: a node whose sum is NaN (an inadmissible state, or a Dirichlet / in-flow entry without data) makes
 * tau NaN.  gdg_max_dt instead refuses a call without the data (GDG_EINVAL) and drops an inadmissible
 * node from its minimum (fmin ignores NaN), reporting the state through gdg_status, which this entry,
 * having no handle, cannot do.
 * Output: *tau_out, a device double, written on stream (asynchronous; the call does not synchronise).
 *
 * Scratch: a fixed array of GDG_NOALLOC_MAX_NODES / 256 doubles (128 KB) in the library's own device
 * memory, which every GPU that loads the library holds until the process exits.  Meshes with more than
 * GDG_NOALLOC_MAX_NODES nodes are rejected with GDG_ENOTSUP before any work.  All calls share that
 * array, so calls whose kernels overlap on the GPU (on different streams, or from several threads)
 * race and must be serialised by the caller.  The array needs no clearing: each call writes every
 * slot it reads.  The first call on a device, with that device current, looks up the array's device
 * address (cudaGetSymbolAddress) and caches it with the id of the current context; make that first call
 * before any stream capture.  After a device reset (a new primary context) the next call looks the
 * address up again, so it too must come before any capture.
 * Errors: GDG_EINVAL (NULL pointer, cfl <= 0, gamma <= 1), GDG_ENOTSUP (dim, sizes), GDG_ECUDA. */
#define GDG_NOALLOC_MAX_NODES 4194304
typedef struct {
  int32_t dim;
  int64_t n, nnz, nb;
  const int32_t* row_ptr;
  const int32_t* col_idx;
  const double* cij;
  const double* mi;
  const int32_t* b_ptr;
  const double* b_c;
  const int32_t* b_type;
  double gamma;
} gdg_dev_mesh;
int gdg_max_dt_noalloc(const gdg_dev_mesh* mesh, const double* U, const double* bdata, double cfl,
                       double* tau_out, void* stream);

/* Launch schedule: threads per block of the one-thread-per-row (per-edge) kernels (128, 256 or 512),
 * the node cap of the element sweep's blocks (1..288: a block holds the largest power of two of
 * elements, at most 32, whose nodes fit the cap, one element at least) and the queue slots per thread of
 * the deferred line-search grid (1..1024), and the row order of the kernels with per-entry loops.
 * Defaults: 256 threads, 288 nodes, 4 slots, slice order.  gdg_autotune picks them for one handle by
 * timing: it saves U and the clock, runs 3 + 2 + 4 + 3 candidate schedules of (trials + 1)
 * gdg_ssprk3_step each from that saved state (coordinate descent: row-kernel block sizes, their row
 * order, then the element block, then the queue grid; each kernel keeps its fastest candidate),
 * and restores U, the clock and the status flags.  It allocates one temporary state copy and
 * synchronises the stream.  Arguments as gdg_ssprk3_step.  The schedule changes speed only: results are
 * bit-identical under every schedule.  gdg_get_schedule / gdg_set_schedule read or install one (e.g. a
 * schedule tuned on one instance for others of the same kind).  Errors: GDG_EINVAL (bad values),
 * GDG_ENOMEM, GDG_ECUDA. */
typedef struct {
  int32_t prim_threads, edge_threads, tau_threads, low_threads, limit2_threads, final_threads, maxdt_threads;
  int32_t high_block_cap;
  int32_t lsfix_slots;
  int32_t row_slices;  // bits 1 << GDG_K_{MAXDT,LOW,LIMIT2,FINAL,TAU}: that kernel's threads take their rows in
                       // the entry storage's slice order (a warp takes one local index of 32 consecutive
                       // elements) instead of node order; default: all five
} gdg_schedule;
int gdg_autotune(gdg_handle* h, double* U, double* T1, double* T2, const double* bdata, int32_t trials,
                 void* stream);
int gdg_get_schedule(gdg_handle* h, gdg_schedule* out);
int gdg_set_schedule(gdg_handle* h, const gdg_schedule* in);

/* Batches: many independent instances advanced together.  The paper solves one problem at a time; a
 * batch runs the per-stage sweep of Sec. 6.1 for all its members in the same kernel launches (one
 * launch per kernel and stage over all instances; each block finds its instance from per-kernel block
 * offsets), so small meshes share the GPU instead of each paying its own launches and host round trips.
 *
 * gdg_batch_create: handles[count] (distinct, same device, dim, n_loc, order and limiter passes; each
 * keeps its own mesh, scratch and clock), with the state U[k] and the workspace T1[k], T2[k] of member
 * k (device [m][n_k], distinct, caller-owned, not copied: the batch keeps the pointers) and Dirichlet
 * data bdata[k] (device [m][nb_k]; the array or an entry may be NULL where a member has no Dirichlet
 * entry).  Copies two small tables to the device (contexts and block offsets; freed by
 * gdg_batch_destroy).  The handles must outlive the batch.  Errors: GDG_EINVAL, GDG_ENOMEM, GDG_ENOTSUP
 * (more than 2^31 - 1 blocks in one kernel), GDG_ECUDA.
 *
 * gdg_batch_step: one gdg_ssprk3_step of every member, each with the time step of its own clock
 * (gdg_clock_set on its handle; a member whose clock reached t_end is left untouched).  Asynchronous on
 * stream; allocates nothing; results are those of gdg_ssprk3_step on each handle alone.
 *
 * gdg_batch_profile / gdg_batch_profile_read: as gdg_profile / gdg_profile_read, for the batch's
 * launches. */
typedef struct gdg_batch gdg_batch;
int gdg_batch_create(gdg_handle* const* handles, int32_t count, double* const* U, double* const* T1,
                     double* const* T2, const double* const* bdata, gdg_batch** out);
int gdg_batch_step(gdg_batch* b, void* stream);
/* gdg_batch_set_persistent: on = 1 runs each later gdg_batch_step as one cooperative launch per stage
 * (3 launches per step instead of 26), whose phases (the kernels of the stage, Sec. 6.1, for every
 * member) are separated by grid-wide barriers at the sweep's grid-wide dependencies, with one block per
 * co-resident slot of the GPU (cudaLaunchCooperativeKernel); on = 0 returns to one launch per kernel.
 * The results are the same bits either way.  Persistent steps are not captured into the batch's graph
 * and record no kernel times (gdg_batch_profile).  Errors: GDG_EINVAL; at step time GDG_ENOTSUP where
 * the device has no cooperative launch. */
int gdg_batch_set_persistent(gdg_batch* b, int32_t on);
int gdg_batch_profile(gdg_batch* b, int32_t enable);
int gdg_batch_profile_read(gdg_batch* b, double* total_ms, int64_t* launches);
/* gdg_batch_autotune: as gdg_autotune for the whole batch (every member's state and clock saved and
 * restored; one temporary copy of all members' states).  gdg_batch_get_schedule / _set_schedule as for
 * a handle. */
int gdg_batch_autotune(gdg_batch* b, int32_t trials, void* stream);
int gdg_batch_get_schedule(gdg_batch* b, gdg_schedule* out);
int gdg_batch_set_schedule(gdg_batch* b, const gdg_schedule* in);
void gdg_batch_destroy(gdg_batch* b);

/* Serving: a request loop with continuous batching, for streams of independent solves that arrive over
 * time (the paper solves one problem at a time).  gdg_server_create starts two host threads on the
 * current device.  A preparation thread takes submitted requests in arrival order, each as soon as its
 * device footprint (gdg_footprint plus three state buffers and its Dirichlet data) fits the HBM budget,
 * runs gdg_setup and uploads its state.  A loop thread adds prepared requests to the batch of their
 * kind (dim, n_loc, order, limiter passes), advances every batch by one fused SSP-RK3 step per iteration
 * (gdg_batch_step: each member with its own time step, up to its own end time) and retires the members
 * that reached their end time: state to the host, device memory freed, budget released for the next
 * arrivals.  A request's state stays on the device from admission to completion, and requests that
 * arrive while others run join the running batches at the next iteration.  Results are those of the
 * request run alone with gdg_ssprk3_step to t_end.
 *
 * gdg_server_create: hbm_budget_bytes > 0 caps the device memory of admitted requests (<= 0: 80% of the
 *   free device memory).  Errors: GDG_ENOMEM, GDG_ECUDA.
 * gdg_server_submit: copies prob (as gdg_setup reads it), U0 (host [m][n]) and bdata (host [m][nb],
 *   Dirichlet data used at every stage; NULL when no entry is Dirichlet), to be solved from t = 0 to t_end
 *   at CFL number cfl; returns at once with *id.  Errors: GDG_EINVAL, GDG_ENOMEM (the request alone
 *   exceeds the budget).  Setup errors are reported by gdg_server_wait.
 * gdg_server_wait: blocks until request id is done or timeout_s seconds passed (timeout_s < 0: no limit;
 *   GDG_ETIMEOUT then, and the request stays pending), copies its final state to U_out (host [m][n], may
 *   be NULL) and its timings to *info (may be NULL), forgets the request and returns its status.
 * gdg_server_stats: a snapshot of the queue, the active members and the memory in use.
 * gdg_server_destroy: finishes every submitted request, stops the threads, frees everything (results
 *   not waited for are dropped).
 * Times are seconds since gdg_server_create on a monotonic clock. */
typedef struct gdg_server gdg_server;
typedef struct {
  double t_submit;      /* submitted */
  double t_start;       /* set up and joined a batch */
  double t_done;        /* final state on the host */
  double t_final;       /* simulated time reached (t_end) */
  int64_t steps;        /* SSP-RK3 steps taken */
  int32_t status;       /* GDG_OK or the error of its setup or run */
  int32_t flags;        /* sticky device flags GDG_FLAG_* */
  int64_t device_bytes; /* footprint counted against the budget */
} gdg_request_info;
typedef struct {
  int64_t queued;       /* submitted, not yet in a batch */
  int64_t active;       /* in a batch on the device */
  int64_t bytes_in_use; /* footprint of admitted requests */
  int64_t budget;
  int64_t iterations;   /* loop iterations (one step of every batch each) */
  double now;
} gdg_server_info;
int gdg_server_create(int64_t hbm_budget_bytes, gdg_server** out);
int gdg_server_submit(gdg_server* s, const gdg_problem* prob, const double* U0, const double* bdata, double t_end,
                      double cfl, int64_t* id);
int gdg_server_wait(gdg_server* s, int64_t id, double timeout_s, double* U_out, gdg_request_info* info);
int gdg_server_stats(gdg_server* s, gdg_server_info* info);
void gdg_server_destroy(gdg_server* s);

int gdg_get_info(gdg_handle* h, gdg_info* out);
void gdg_destroy(gdg_handle* h);
const char* gdg_error_string(int code);

#ifdef __cplusplus
}
#endif
#endif
