/*
 * fks.h - flexible shifted-Krylov solver for GB300 (sm_103a), C ABI.
 *
 * Solves the shifted systems of Section 2, Eq. multipleshifted,
 *     (K + sigma_j M) x_j = b,   j = 1..n_f,
 * for a real symmetric positive definite stiffness K and a storage (mass)
 * matrix M, from ONE flexible Arnoldi basis (Algorithm 3) built with the
 * shifted preconditioners (K + tau_k M)^{-1}, applied inexactly by an inner
 * iterative solve (Section 4, Eq. zmmoditer), followed by a per-shift
 * least-squares solve (Algorithm 4, FGMRES) and the assembly x_j = Z_m y_j.
 * Grid operators (fks_op_grid: lumped, diagonal M) use geometric-multigrid
 * cycles for the inner solve; general sparse operators (fks_op_csr) use
 * BiCGSTAB cycles.
 *
 * Conventions (all entry points):
 *  - Every call returns fks_status; fks_last_error() gives the message of the
 *    last failing call on the calling thread. No C++ exception crosses the ABI.
 *  - The caller owns every array it passes. The library owns its contexts,
 *    operators, device workspaces and streams it creates.
 *  - Invalid arguments return FKS_ERR_ARG before any device work is queued.
 *  - Data pointers passed to fks_solve / fks_op_apply may be host or device
 *    memory (detected with cudaPointerGetAttributes); device pointers are used in
 *    place on the given stream, host pointers are copied.
 *  - A context is used by one thread at a time.
 *  - Complex numbers are fks_c128 (layout of C99 double complex).
 *  - The grid is cell-centred, x fastest: cell (i, j, k) is at flat index
 *    (k * ny + j) * nx + i; 2D grids have nz = 1.
 */
#ifndef FKS_H
#define FKS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct { double re, im; } fks_c128;

typedef enum {
  FKS_OK = 0,                  /* every shift converged                            */
  FKS_NOT_CONVERGED = 1,       /* some shift reached m_max without converging      */
  FKS_BREAKDOWN_EXACT = 2,     /* h_{k+1,k} = 0: the iterate is exact (Section 3)  */
  FKS_INNER_NOT_CONVERGED = 3, /* an inner solve hit its cycle cap (result valid)  */
  FKS_ERR_ARG = -1,
  FKS_ERR_OOM = -2,
  FKS_ERR_CUDA = -3,
  FKS_ERR_TIMEOUT = -4,
  FKS_ERR_CANCELLED = -5
} fks_status;

typedef struct fks_ctx fks_ctx;
typedef struct fks_op fks_op;

/* Create a context bound to CUDA device `device`. */
fks_status fks_create(fks_ctx** out, int device);
void fks_destroy(fks_ctx* ctx);
/* Message of the last failing call on this thread ("" if none). */
const char* fks_last_error(void);
/* Library version string. */
const char* fks_version(void);

/*
 * Structured-grid operator (Section 5.1, Eq. phasor1, discretised by cell-centred
 * two-point-flux finite volumes):
 *   interior face between cells c, c' on axis a: t = (A_a / h_a) 2 K_c K_c' / (K_c + K_c')
 *   zero-head face (bit set in dirichlet_mask):  t = 2 K_c A_a / h_a
 *   no-flow face (bit clear):                    t = 0
 *   (K x)_c = sum_faces t (x_c - x_nb) + sum_zero_head_faces t x_c,
 *   M = diag(S_s,c * hx * hy * hz)   (lumped storage, the cell volume times S_s)
 * with A_a the face area prod_{b != a} h_b.
 *  dim            2 or 3
 *  ncell[3]       (nx, ny, nz); nz ignored (taken as 1) when dim == 2; each >= 1
 *  h[3]           cell size per axis (> 0)
 *  cond           [n] hydraulic conductivity per cell, > 0, host memory
 *  ss             [n] specific storage S_s per cell, > 0, host memory
 *  dirichlet_mask bit 2a: low face of axis a is zero-head; bit 2a+1: high face
 *  out            receives the operator (owned by the library; free with fks_op_destroy)
 * The multigrid hierarchy is built here: axis a is halved while n_a is even and
 * n_a > 4. If that hierarchy ends above 1024 cells (the largest coarsest level
 * solved exactly), it is built again with odd axes > 4 also halved, to
 * (n_a + 1) / 2 cells (the last coarse cell having one child), while a level
 * has more than 1024 cells. FKS_ERR_ARG only if that needs more than 16 levels.
 */
fks_status fks_op_grid(fks_ctx* ctx, int dim, const int64_t ncell[3], const double h[3],
                       const double* cond, const double* ss, uint32_t dirichlet_mask,
                       fks_op** out);
/*
 * General sparse operator: K and M given as CSR matrices (finite-element
 * stiffness and consistent mass of Section 5.1, or any real K, M for which
 * K + tau M has a nonzero diagonal). The inner solve (K + tau_k M)^{-1} v_k is
 * then the same defect correction z <- z + C(v - (K + tau_k M) z) from z = 0 as
 * for grids (Section 4, Eq. zmmoditer), where one cycle C is `inner_steps`
 * BiCGSTAB steps (the Krylov inner method of Section 6) with the Jacobi
 * preconditioner diag(K + tau_k M)^{-1}, started from zero; ||p_k|| is the
 * complex128 defect, computed exactly.
 *  n                       number of unknowns, 1 <= n < 2^31
 *  k_rowptr[n+1], k_col[nnz_K], k_val[nnz_K]   CSR of K (int64 row pointers,
 *                          int32 column indices, any order within a row,
 *                          duplicates summed), host memory
 *  m_rowptr, m_col, m_val  CSR of M, same conventions
 *  out                     receives the operator (free with fks_op_destroy)
 * K and M are stored on the device on the union of their patterns (a K and an M
 * value per entry). Rows out of order, a column index outside 0..n-1 or a
 * non-finite value return FKS_ERR_ARG. fks_op_autotune, fks_op_set_fusion and
 * fks_precond_apply_noalloc are grid-only (FKS_ERR_ARG on a CSR operator).
 */
fks_status fks_op_csr(fks_ctx* ctx, int64_t n, const int64_t* k_rowptr, const int32_t* k_col,
                      const double* k_val, const int64_t* m_rowptr, const int32_t* m_col,
                      const double* m_val, fks_op** out);
/*
 * Smoothed-aggregation algebraic multigrid as the BiCGSTAB preconditioner of a
 * CSR operator's inner solve: Section 6 inverts each K + tau_k M with BiCGSTAB
 * preconditioned by smoothed-aggregation AMG. With enable != 0 every BiCGSTAB
 * step applies one V-cycle of K + tau_k M's hierarchy where the Jacobi
 * diagonal was applied; enable = 0 returns to Jacobi. The hierarchy:
 *  - strength graph: the stored connections of A_l (level 0: the entries where
 *    K or M is nonzero), so the aggregates depend on the pattern only and are
 *    shared by every tau;
 *  - standard two-pass aggregation (ascending nodes; pass 2 joins a node to the
 *    aggregate of its first neighbour placed by pass 1);
 *  - tentative prolongator from the near-null-space vector (1 on level 0),
 *    smoothed P = (I - omega D^{-1} A) T with omega = 4 / (3 rho), rho the
 *    Gershgorin bound max_i sum_j |a_ij| / |a_ii|;
 *  - A_{l+1} = P^T A_l P (plain transpose); the coarsest level (at most
 *    max_coarse unknowns, or level max_levels - 1) is solved by its dense inverse;
 *  - V-cycle: nu damped-Jacobi sweeps (weight omega) from zero, residual,
 *    restriction by P^T, coarse correction by P, nu sweeps.
 *  max_levels  1..16 (0: 10);  max_coarse 1..4096 (0: 256);  nu 1..8 (0: 2)
 * Hierarchies are built on the host when a solve first needs a tau (or by
 * fks_op_amg_setup) and kept on the operator per (tau, precision) until the
 * next fks_op_amg call, which must not run while a solve on this operator is in
 * flight. The default inner_steps becomes 4. FKS_ERR_ARG on a grid operator or
 * out-of-range arguments; a later solve returns FKS_ERR_ARG when a level has a
 * zero diagonal entry or the coarsest level is singular or above 4096 unknowns.
 */
fks_status fks_op_amg(fks_op* op, int enable, int max_levels, int64_t max_coarse, int nu);
/* Build (or find) the hierarchies of K + tau_q M for the n_tau taus (host array,
 * 1..16) in the cycle precision (FKS_PREC_FP64: complex128 values,
 * FKS_PREC_MIXED: complex64). setup_ms (may be NULL) receives the host time
 * spent, including the uploads. */
fks_status fks_op_amg_setup(fks_op* op, const fks_c128* tau, int n_tau, int precision, double* setup_ms);
/* The hierarchy's shape once one has been built: *n_levels, sizes[l] (at least
 * n_levels entries, may be NULL) and, level after level, the aggregate of every
 * unknown of every level but the coarsest in agg (may be NULL; agg_cap entries
 * at least sum of sizes[0 .. n_levels - 2]). FKS_ERR_ARG before the first build. */
fks_status fks_op_amg_info(fks_op* op, int* n_levels, int64_t* sizes, int sizes_cap, int32_t* agg,
                           int64_t agg_cap);
/*
 * Host only (no GPU, no device memory): the hierarchy fks_op_amg would build
 * for one complex matrix A0, given as CSR in host memory (int64 row pointers,
 * int32 columns ascending within each row, complex128 values; its pattern is
 * the strength graph, so pass only the entries that are structurally nonzero).
 * Returns *n_levels and per level (arrays of sizes_cap >= n_levels entries, each
 * may be NULL): unknowns, entries of A_l, entries of P_l (0 on the coarsest)
 * and the Jacobi weight omega_l; agg as in fks_op_amg_info. max_levels and
 * max_coarse as in fks_op_amg (0: default). FKS_ERR_ARG on malformed input, a
 * zero diagonal entry, a singular or too large coarsest level.
 */
fks_status fks_amg_host_shape(int64_t n, const int64_t* rowptr, const int32_t* col, const fks_c128* val,
                              int max_levels, int64_t max_coarse, int* n_levels, int64_t* sizes,
                              int64_t* nnz_a, int64_t* nnz_p, double* omega, int sizes_cap, int32_t* agg,
                              int64_t agg_cap);
void fks_op_destroy(fks_op* op);
/* Number of cells n of the operator (0 on a NULL operator). */
int64_t fks_op_size(const fks_op* op);

enum { FKS_FGMRES = 0, FKS_FFOM = 1 };
enum { FKS_PREC_FP64 = 0, FKS_PREC_MIXED = 1, FKS_PREC_MIXED_BF16 = 2 };

typedef struct {
  double tol;            /* relative tolerance on ||b - (K + sigma_j M) x_j|| / ||b||, > 0     */
  int m_max;             /* maximum Arnoldi steps, 1..128                                     */
  int variant;           /* FKS_FGMRES (least squares) or FKS_FFOM (square solve)             */
  int precision;         /* FKS_PREC_FP64: complex128 throughout; FKS_PREC_MIXED: inner
                            multigrid cycles in complex64, defect correction and everything
                            else in complex128; FKS_PREC_MIXED_BF16 (grid operators): as
                            FKS_PREC_MIXED with the multigrid coefficients (faces, storage)
                            rounded to bf16 and stored so for the per-level smoother and
                            restriction kernels (fp32 arithmetic; the complex128 defect
                            correction uses the exact operator)                               */
  double inner_tol;      /* eps: stop the inner solve when ||p_k|| <= eps ||v_k||; <= 0 means
                            min(1e-6, tol / 100)                                              */
  int inner_max_cycles;  /* cap on multigrid cycles per inner solve (<= 0 means 50)           */
  const int32_t* tau_schedule; /* host [sched_len]: index into tau for step k, cycled         */
  int sched_len;         /* >= 1                                                              */
  int replay_mode;       /* 1: run exactly replay_inner_cycles / freeze at replay_mj          */
  const int32_t* replay_inner_cycles; /* host [m_max * n_rhs], step-major per source          */
  const int32_t* replay_mj;           /* host [n_f * n_rhs]                                   */
  int launch_mode;       /* 0: the step loop runs as one CUDA graph with conditional WHILE nodes
                            (no host round trip per step); 1: host-driven loop (one host sync per
                            inner cycle; per-kernel timing with fks_profile_select works here)  */
  int inner_steps;       /* CSR operators: BiCGSTAB steps per inner cycle (<= 0 means 8, or 4
                            with AMG; at most 64); ignored by grid operators                  */
  int assembly;          /* x_j = Z y_j (Algorithm 4): 0 = tensor cores (Z and Y cut into eight
                            7-bit bf16 slices, exact fp32 accumulation of the slice products
                            over chunks of at most 64 steps, the chunks added in 64-bit
                            integers; error at the level of an FP64 GEMM; any step count up
                            to 128); 1 = FP64 FMA kernel                                       */
  double inner_relax;    /* l > 0: relaxed inner tolerance, step k uses
                            min(1e-3, max(eps, l * tol / R_{k-1})) with R_{k-1} the largest
                            ||beta e_1 - H_bar(sigma_j) y|| / beta of the shifts still iterating
                            after step k-1 (R_0 = 1); the idea Section 4 closes with (after
                            Simoncini and Szyld). Convergence is still decided by the bound of
                            Eq. trueresidual with the measured ||p_k||. <= 0: eps at every step */
  int restart_len;       /* > 0: restarted FFOM (Section 2.2.2): cycles of at most restart_len
                            steps (<= m_max), each restarted on the common residual direction
                            v_{k+1} of the shifts not yet certified (FOM residuals are
                            collinear, Eq. fomresidualsimplified), x_j += C_j d_j; the tau
                            schedule continues across cycles; each shift carries the part of
                            its error the finished cycles' estimates did not see (Eq.
                            trueresidual) and is certified when that plus its current bound is
                            <= tol. Needs variant FKS_FFOM and no replay; the workspace holds
                            restart_len + 1 basis vectors per source instead of m_max + 1.
                            m_j counts steps over all cycles; fks_info reports steps and
                            breakdown only. 0: no restarts                                     */
  int max_restarts;      /* cycles after the first (<= 0: 20); shifts still open then are
                            FKS_NOT_CONVERGED                                                  */
} fks_options;

/* Optional per-solve diagnostics, host arrays owned by the caller (any may be NULL). */
typedef struct {
  int32_t* steps;         /* [n_rhs] Arnoldi steps taken                                     */
  int32_t* inner_cycles;  /* [m_max * n_rhs] inner cycles of step k (source-major)           */
  double* pnorm;          /* [m_max * n_rhs] ||p_k|| = ||v_k - (K + tau_k M) z_k||           */
  int32_t* breakdown;     /* [n_rhs] 1 if h_{k+1,k} vanished                                 */
  /* Monitors (Section 3); each may be NULL, host or device:
   * gmres_alpha [n_f * n_rhs]: Prop. 3's alpha = ||eta H_m(sigma_j; T)^{-*} e_m||,
   *   eta = h_{m+1,m}(sigma_j - tau_m), at the shift's freeze step m = m_j, so
   *   ||r_fom - r_gmres|| <= alpha (1 + alpha) / (1 + alpha^2) ||r_fom||; a large
   *   alpha flags FGMRES stagnation (infinite when H_m(sigma_j; T) is singular)
   * hbar [(m_max + 1) * m_max * n_rhs]: the flexible Hessenberg H_bar of each
   *   source, column-major: h_{i,k} at r (m_max + 1) m_max + (k - 1)(m_max + 1) + i - 1
   *   (zero beyond the steps taken)
   * tau_k [m_max * n_rhs]: the preconditioner shift of each step (T_m's diagonal)
   * Together with steps they give Prop. 1's Ritz values (fks_ritz). */
  double* gmres_alpha;
  fks_c128* hbar;
  fks_c128* tau_k;
} fks_info;

/*
 * Solve (K + sigma_j M) x_j = b_r for every shift j and every source r
 * (Algorithms 3 and 4). The n_rhs sources run as independent Arnoldi processes
 * advanced together (no block Krylov). Zero initial guess; beta = ||b_r||.
 *  b          [n * n_rhs] source-major (column r contiguous)
 *  sigma      [n_f] shifts; tau [n_tau] distinct preconditioner shifts
 *  X          [n * n_f * n_rhs] out: x_j of source r at ((r * n_f) + j) * n
 *  res_est    [n_f * n_rhs] out: ||beta e_1 - H_bar(sigma_j; T) y_j|| / beta
 *  res_bound  [n_f * n_rhs] out: (res_est * beta + sum_i |y_i| ||p_i||) / beta (Eq. trueresidual)
 *  res_true   [n_f * n_rhs] out: ||b - (K + sigma_j M) x_j|| / beta (computed), may be NULL
 *  m_j        [n_f * n_rhs] out: steps used by shift j
 *  shift_status [n_f * n_rhs] out: FKS_OK / FKS_NOT_CONVERGED / FKS_BREAKDOWN_EXACT
 *  stream     cudaStream_t to run on (NULL: the legacy default stream)
 * Shift j is converged when the bound of Eq. trueresidual is <= tol * beta; it
 * is then frozen (Algorithm 4's "if not converged"). Returns FKS_OK when all
 * shifts of all sources converged, FKS_NOT_CONVERGED or FKS_BREAKDOWN_EXACT
 * otherwise, or an error. Outputs are complete when the call returns.
 */
fks_status fks_solve(fks_op* op, const fks_c128* b, int n_rhs, const fks_c128* sigma, int n_f,
                     const fks_c128* tau, int n_tau, const fks_options* opt, fks_c128* X,
                     double* res_est, double* res_bound, double* res_true, int32_t* m_j,
                     int32_t* shift_status, fks_info* info, void* stream);

/*
 * y = (K + s M) x for n_vec vectors (the operator apply of Section 2), x and y
 * [n * n_vec] vector-major, host or device. Used by the solver's residual check.
 */
fks_status fks_op_apply(fks_op* op, fks_c128 s, const fks_c128* x, fks_c128* y, int n_vec, void* stream);

/*
 * Prop. 1's Ritz values (Section 3, Eq. genritz) of every source of a solve,
 * from its monitors (fks_info hbar, tau_k, steps): the eigenvalues theta of
 * H_m(sigma; T_m) f = theta H_m f with m = steps[r], at sigma = 0. At another
 * shift they are theta + sigma (H_m^{-1} H_m(sigma; T_m) = H_m^{-1} - T_m + sigma I);
 * they approximate lambda + sigma, lambda the eigenvalues of K x = lambda M x.
 * Computed on the GPU, one warp per source: Gauss-Jordan inverse of H_m,
 * Householder reduction of H_m^{-1} - T_m to Hessenberg form, shifted QR.
 *  hbar   [(m_max + 1) * m_max * n_rhs], tau_k [m_max * n_rhs], steps [n_rhs] in
 *         (the layouts of fks_info; 0 <= steps[r] <= m_max)
 *  theta  [m_max * n_rhs] out: source r's m values at r * m_max (unordered),
 *         zero beyond them
 *  status [n_rhs] out: 0 converged; 1 the QR sweep limit (60 m) was reached and
 *         theta holds the unconverged diagonal; 2 H_m is singular (theta zero)
 * Pointers host or device; m_max <= 128. Outputs complete when the call returns.
 */
fks_status fks_ritz(fks_ctx* ctx, const fks_c128* hbar, const fks_c128* tau_k, const int32_t* steps,
                    int n_rhs, int m_max, fks_c128* theta, int32_t* status, void* stream);

/*
 * Sensitivities of the phasor measurements by the adjoint-state method
 * (Section 5: Eq. measurement, Eq. sensitivity, Eq. adjoint, Algorithm 6), for
 * grid operators (fks_op_grid). Sensor m sits in cell x_m and records
 * h = Phi_j(x_m) at shift sigma_j (real and imaginary part: the two
 * coefficients per frequency). With A = K + sigma_j M, A Phi_j = b and the
 * adjoint phasor A Psi_mj = -e_{x_m} (A is complex symmetric, so the adjoint
 * solves are plain fks_solve calls with the right-hand sides -e_{x_m}),
 *   dh/dp = Psi_mj^T (dA/dp) Phi_j   (no conjugation), and per cell c:
 *   j_lnk: dh/dlnK_c = sum over c's interior faces (to nb, transmissibility t)
 *          of t K_nb/(K_c + K_nb) (Psi_c - Psi_nb)(Phi_c - Phi_nb), plus t Psi_c Phi_c
 *          over its zero-head boundary faces (the dK grad Phi . grad Psi term)
 *   j_lns: dh/dlnS_s,c = sigma_j M_cc Psi_c Phi_c   (the i omega dS_s Phi Psi term)
 *  phi    [n_f * n] in: forward phasors Phi_j (one source's X of fks_solve)
 *  psi    [n_m * n_f * n] in: adjoint phasors, measurement-major (the X of an
 *         fks_solve with n_rhs = n_m right-hand sides -e_{x_m})
 *  sigma  [n_f] in: the shifts
 *  j_lnk, j_lns [n_m * n_f * n] out, indexed ((m * n_f) + j) * n + c
 * Pointers host or device; with all four arrays on the device the call runs
 * one kernel on them in place, otherwise it stages one measurement at a time.
 * FKS_ERR_ARG for CSR operators, n_m < 1, n_f outside [1, 65535], NULL
 * arrays or non-finite host sigma. Outputs are complete when the call returns.
 */
fks_status fks_sensitivity(fks_op* op, const fks_c128* phi, const fks_c128* psi, int n_m,
                           const fks_c128* sigma, int n_f, fks_c128* j_lnk, fks_c128* j_lns,
                           void* stream);

/*
 * Inexact preconditioner apply (Section 4, Eq. zmmoditer): z ~ (K + tau M)^{-1} v by
 * multigrid cycles from z = 0 until ||v - (K + tau M) z|| <= eps ||v|| or max_cycles
 * (cycles >= 0 forces exactly that many). precision as in fks_options.
 * v, z [n] host or device; out_cycles, out_pnorm host scalars (may be NULL).
 * z is written in full: z = 0 where no cycle runs (cycles == 0, or v = 0).
 */
fks_status fks_precond_apply(fks_op* op, fks_c128 tau, const fks_c128* v, fks_c128* z, double eps,
                             int max_cycles, int cycles, int precision, int32_t* out_cycles,
                             double* out_pnorm, void* stream);

/*
 * Serving (no counterpart in the paper): a request loop over the solver with
 * continuous (iteration-level) batching. One driver thread issues all of the
 * server's CUDA calls; each lane (own stream, workspace and step-loop graph)
 * runs a batch started for the first queued request that fits the
 * device-memory budget, with spare slots (one slot per source)
 * for later requests that share its operator, shifts, taus and options. The
 * batch's step loop runs one Arnoldi step per launch; between launches the
 * worker admits queued compatible requests into free slots (their sources
 * start at step 1 while the others go on), stops cancelled or timed-out
 * requests, and delivers every source that has finished (assembly, true
 * residual, copies into the request's arrays) as soon as it finishes.
 * Batches on different lanes overlap on the device. Each request's result
 * equals what fks_solve gives it alone. All request arrays are HOST memory
 * owned by the caller and must stay valid until the request is done; X may be
 * NULL (the residuals and statuses are still delivered); options'
 * tau_schedule is copied at submit. Replay mode is not accepted. The server is
 * thread-safe. A workspace that cannot be allocated ends the requests of that
 * batch with FKS_ERR_OOM and releases their slots and budget.
 */
typedef struct fks_server fks_server;
typedef struct {
  fks_op* op;
  const fks_c128* b; int n_rhs;          /* [n * n_rhs]                                        */
  const fks_c128* sigma; int n_f;
  const fks_c128* tau; int n_tau;
  fks_options opt;
  fks_c128* X;                           /* [n * n_f * n_rhs] out                               */
  double* res_est; double* res_bound;    /* [n_f * n_rhs] out                                   */
  double* res_true;                      /* [n_f * n_rhs] out or NULL                           */
  int32_t* m_j; int32_t* shift_status;   /* [n_f * n_rhs] out                                   */
  double timeout_s;                      /* > 0: stop with FKS_ERR_TIMEOUT once the request has run
                                            this long (checked between Arnoldi steps); 0: none      */
} fks_request;
/* lanes: concurrent batches (1..64); mem_budget_bytes: device memory the
 * admitted batches' workspaces may use together (one oversized request still
 * runs when nothing else is in flight). */
fks_status fks_server_create(fks_ctx* ctx, size_t mem_budget_bytes, int lanes, fks_server** out);
/* FKS_ERR_ARG for replayed (replay_mode) or restarted (restart_len) requests:
 * those go through fks_solve. */
fks_status fks_server_submit(fks_server* srv, const fks_request* req, uint64_t* ticket);
/* done = 1 when finished or cancelled; result = the request's status. */
fks_status fks_server_poll(fks_server* srv, uint64_t ticket, int* done, fks_status* result);
fks_status fks_server_wait(fks_server* srv, uint64_t ticket, fks_status* result);
/* Cancels a request: a queued one at once, a running one at its batch's next
 * Arnoldi-step boundary (its sources take no further step and deliver nothing).
 * Its result is FKS_ERR_CANCELLED. FKS_ERR_ARG if it already finished. */
fks_status fks_server_cancel(fks_server* srv, uint64_t ticket);
/* Host wall-clock seconds (steady clock) of submit, start and end of a request. */
fks_status fks_server_times(fks_server* srv, uint64_t ticket, double* submit_s, double* start_s, double* end_s);
/* Kernel launches made by the server's lanes since it was created. */
fks_status fks_server_launches(fks_server* srv, int64_t* launches);
/*
 * Test hook (no counterpart in the paper): the next `count` workspace
 * reservations of any solve or server batch fail as cudaMalloc does when the
 * device is out of memory (FKS_ERR_OOM), so that failure handling can be tested
 * without exhausting a GPU. count = 0 clears it.
 */
void fks_debug_fail_allocs(int count);
/* Stops the workers after their current batches; queued requests are dropped. */
void fks_server_destroy(fks_server* srv);

/*
 * Autotuner (no counterpart in the paper): times one multigrid V-cycle of the
 * operator on this GPU for every choice of which 2D levels use the fused
 * shared-memory tile kernels (levels at most `chosen` cells), which of those
 * run on 16 x 16 rather than 32 x 32 tiles and which small levels run in the
 * single-block tail kernel (64, 256, 1024 or 4096 cells) or, instead of the tail,
 * which lower levels run in the cluster kernel (fks_op_set_cluster), for the
 * cycle precision `precision` and shift `tau`, and keeps the fastest in the
 * operator for later solves; then, for that choice, which of the smallest fused
 * levels run on 8 x 8 tiles.
 * Solves before any tuning fuse levels up to 65536 cells (complex128 cycles) or
 * all levels (complex64 cycles), use 16 x 16 tiles up to 16384 cells and a tail
 * of at most 256 cells and no cluster kernel.
 * `chosen` (host, may be NULL) receives the fusion threshold (fks_op_tiling
 * reads all four).
 */
fks_status fks_op_autotune(fks_op* op, int precision, fks_c128 tau, void* stream, int64_t* chosen);
/* Set that threshold directly (max_cells < 0: every fusable level). The fused and
 * per-sweep kernels perform the same operations in the same order, so results
 * do not depend on it. */
fks_status fks_op_set_fusion(fks_op* op, int precision, int64_t max_cells);
/*
 * Fused 2D levels with at most max_cells cells run on 16 x 16 tiles, larger
 * ones on 32 x 32 (< 0: all on 16 x 16). The tiling does not change results.
 * fks_op_autotune picks it together with the fusion threshold. Grid operators only.
 */
fks_status fks_op_set_tiles(fks_op* op, int precision, int64_t max_cells);
/* Fused 2D levels with at most max_cells cells run on 8 x 8 tiles (before the
 * 16 x 16 rule; < 0: all, 0: none): more CTAs on small levels, at more
 * recomputed halo. The tiling does not change results. Grid operators only. */
fks_status fks_op_set_tiles8(fks_op* op, int precision, int64_t max_cells);
/* Levels with at most max_cells cells (the coarsest always) run in the
 * single-block tail kernel; FKS_ERR_ARG if their vectors do not fit in shared
 * memory. The results do not depend on it. Grid operators only. */
fks_status fks_op_set_tail(fks_op* op, int precision, int64_t max_cells);
/*
 * Cluster V-cycle (Section 4's multigrid inner solve, lower levels): from the
 * first level with at most max_cells cells down to the coarsest, the V-cycle runs
 * in one kernel, one cluster of 8 CTAs per source. Every level of that range
 * is split into 8 bands of rows held in the CTAs' shared memory together with
 * the band's coefficients; rows across a band edge are read from the
 * neighbouring CTA's shared memory and half sweeps are separated by cluster
 * barriers. Replaces the tail kernel when on. It applies to 2D operators whose
 * levels from there on halve in both axes, have a multiple of 8 rows (of 16
 * where a further banded level follows) and a coarsest level of at most 64
 * cells, and whose bands fit in 200 KB of shared memory; if the first level
 * with at most max_cells cells does not, the next coarser one is tried.
 * max_cells <= 0 turns it off. FKS_ERR_ARG if no level qualifies or the GPU
 * cannot schedule the cluster. The results do not depend on it. Grid
 * operators only.
 */
fks_status fks_op_set_cluster(fks_op* op, int precision, int64_t max_cells);
/*
 * Fused 3D levels (Section 4's multigrid inner solve): a 3D level coarsened by
 * 2 in every axis and within the fusion threshold runs its pre-smoothing
 * (four half sweeps, residual, restriction) and its post-smoothing
 * (interpolation, four half sweeps) as one kernel each. A block owns a tile of
 * cells in the x-y plane (8 x 8, 16 x 16 or 32 x 16, by the same thresholds as
 * the 2D tiles) and a chunk of `planes` consecutive planes, and marches through
 * them. This sets the chunk of multigrid level `level` (0 = finest) for
 * `precision`; planes is rounded down to an even number >= 2, and planes <= 0
 * means the whole level. FKS_ERR_ARG for a bad level. The results do not
 * depend on it. Grid operators only.
 */
fks_status fks_op_set_zchunk(fks_op* op, int precision, int level, int planes);
/*
 * Launch overlap (no counterpart in the paper): the multigrid and defect
 * kernels are launched with programmatic dependent launch, so that each one's
 * blocks are scheduled while its predecessor finishes (they wait for the
 * predecessor's results before reading memory). on = 1 (the default) or 0 sets
 * it for the whole process (call it while no solve or server is running); a
 * negative value only queries. Returns the previous setting. Results are the same bits either way; graphs built before a change
 * are rebuilt at their next use. If a graph capture refuses the overlap, the
 * library switches it off by itself.
 */
int fks_set_pdl(int on);
/*
 * Cooperative lower cycle (no counterpart in the paper): from the first
 * multigrid level with at most max_cells cells (not the finest, above the tail
 * kernel's levels) down to the coarsest, the V-cycle's phases run in one
 * cooperative launch with grid-wide barriers between them, on the levels'
 * vectors in device memory, instead of one launch per phase; 0 switches it off
 * (the default). Results are bitwise those of the separate kernels.
 * fks_op_autotune tries it. fks_op_coop_max reads the setting.
 */
fks_status fks_op_set_coop(fks_op* op, int precision, int64_t max_cells);
fks_status fks_op_coop_max(fks_op* op, int precision, int64_t* max_cells);
/* The z-chunk of every multigrid level of `precision` (planes[0 .. levels-1],
 * as fks_op_set_zchunk stores them); *levels receives the level count. */
fks_status fks_op_zchunks(const fks_op* op, int precision, int32_t* planes, int cap, int* levels);
/* The current fusion threshold, 16 x 16 tile threshold, single-block tail
 * threshold (levels of at most tail_max cells run in one block per source),
 * cluster threshold (0: off) and 8 x 8 tile threshold of `precision`; any
 * output may be NULL. */
fks_status fks_op_tiling(const fks_op* op, int precision, int64_t* fuse_max, int64_t* tile16_max,
                         int64_t* tail_max, int64_t* cluster_max, int64_t* tile8_max);

/*
 * Allocation-free variant of fks_precond_apply (the paper has no counterpart).
 * For callers that may not allocate device memory: code inside a host framework
 * whose memory pool owns the GPU's memory, or real-time code that cannot take
 * cudaMalloc's implicit synchronisation. It computes exactly what
 * fks_precond_apply computes, but its multigrid scratch is a fixed 16 MiB
 * device array inside the library (held by every GPU that loads the library
 * until the process exits) and it calls no cudaMalloc, cudaFree or other
 * allocating routine.
 *  - v, z must be device memory (the caller passes inputs and outputs). z may
 *    alias v (an in-place call): v is first copied into the fixed array.
 *  - z is written in full; where no cycle runs (cycles == 0 in replay, or
 *    v = 0), z = 0.
 *  - Limits: at most 65536 cells, coarsest multigrid level at most 256 cells;
 *    larger grids return FKS_ERR_ARG with a message.
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) and keeps it for later calls.
 *  - The call is synchronous on `stream` (it reads the cycle count and ||p||
 *    back to the host before it returns), so it must not be made while that
 *    stream is being captured into a CUDA graph.
 *  - All calls share the one array and leave their contents in it; calls that
 *    overlap on the GPU (other streams, other threads) race and must be
 *    serialised by the caller.
 */
fks_status fks_precond_apply_noalloc(fks_op* op, fks_c128 tau, const fks_c128* v, fks_c128* z, double eps,
                                     int max_cycles, int cycles, int precision, int32_t* out_cycles,
                                     double* out_pnorm, void* stream);

/*
 * Instrumentation (no counterpart in the paper). Kernel classes of the solve:
 */
enum {
  FKS_K_SMOOTH = 0,    /* red-black Gauss-Seidel half sweep (any level)           */
  FKS_K_RESTRICT = 1,  /* residual + restriction to the next coarser level        */
  FKS_K_PROLONG = 2,   /* interpolation + correction from the coarser level       */
  FKS_K_COARSE = 3,    /* coarsest-level dense solve (inside the tail kernel now)  */
  FKS_K_DEFECT = 4,    /* complex128 defect r = v - (K + tau M) z of the inner solve */
  FKS_K_CORRECT = 5,   /* z += e of the inner solve                               */
  FKS_K_MDOT = 6,      /* CGS projection pass h = V^* w                           */
  FKS_K_MAXPY = 7,     /* CGS update pass w -= V h                                */
  FKS_K_GIVENS = 8,    /* per-shift Givens least-squares update                   */
  FKS_K_ASSEMBLE = 9,  /* x_j = Z y_j                                             */
  FKS_K_TRES = 10,     /* true residuals                                          */
  FKS_K_TAIL = 11,     /* the V-cycle of all small levels in one block per source */
  FKS_K_PRE2D = 12,    /* 2D level: four pre-smoothing half sweeps + residual + restriction */
  FKS_K_POST2D = 13,   /* 2D level: prolongation + four post-smoothing half sweeps */
  FKS_K_BICGSTAB = 14, /* CSR operators: one BiCGSTAB cycle of the inner solve    */
  FKS_K_CLUSTER = 15,  /* the V-cycle of the lower 2D levels in one 8-CTA cluster per source */
  FKS_K_PRE3D = 16,    /* 3D level: four pre-smoothing half sweeps + residual + restriction (z-march) */
  FKS_K_POST3D = 17,   /* 3D level: prolongation + four post-smoothing half sweeps (z-march) */
  FKS_K_COOP = 18,     /* the lower levels' V-cycle in one cooperative launch */
  FKS_K_COUNT = 19
};
/*
 * Time every launch of kernel class `kclass` (on level `level`, or every level
 * when level < 0) with CUDA events recorded on the launching stream, from now
 * on; kclass < 0 stops timing. Every kernel launch is counted either way.
 */
fks_status fks_profile_select(fks_op* op, int kclass, int level);
/*
 * Read and reset the counters: launches of the selected class, their summed
 * event time (ms), their summed algorithmic bytes and flops (the per-launch
 * models of each class), and the number of all kernel launches since the last
 * read. Any output pointer may be NULL. Synchronises the recorded events.
 */
fks_status fks_profile_read(fks_op* op, int64_t* launches, double* total_ms, double* alg_bytes,
                            double* alg_flops, int64_t* all_launches);

#ifdef __cplusplus
}
#endif

#endif /* FKS_H */
