/*
 * libsos - HSDE ADMM for sum-of-squares programs on one GB300 GPU (sm_103a).
 *
 * Method: Zheng, Fantuzzi, Papachristodoulou, "Fast ADMM for sum-of-squares
 * programs using partial orthogonality".  An SOS program in the standard form
 * of eq. (7) (weighted blocks as in eq. (37)) is recast as the conic program
 * of eq. (15) over K = R^t x S_+^{N_1} x ... and solved by the three-step ADMM
 * of eq. (20) on its homogeneous self-dual embedding (eq. (18)-(19)).  The
 * affine step uses the eliminations of eq. (23)-(27) and the diagonal-plus-
 * low-rank structure of Prop. 1 / Prop. 3 (Woodbury, eq. (28)).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - All pointers in argument structs are HOST pointers owned by the caller;
 *   sos_setup copies what it needs, so they may be freed after it returns.
 * - The handle is owned by the library and released with sos_destroy.
 * - Exponent arrays are row-major int32 [count x n_vars].
 * - Packed Gram order ("svec"): for each block, the lower triangle column by
 *   column (column j holds rows j..N-1); off-diagonal entries are scaled by
 *   sqrt(2), so <svec X, svec Y> = trace(X Y).
 * - Per instance the primal vector is xi = [u (t free variables); svec X_1;
 *   svec X_2; ...] of length n_x, the dual vector y has length m (one entry
 *   per matched monomial, constraints concatenated in order), and the HSDE
 *   iterates are u = [xi; y; tau], v = [z; s; kappa] (eq. (19)).
 * - Return codes: SOS_OK (0) or a negative SOS_ERR_*; the message of the last
 *   failure on a handle is available from sos_last_error.  A failure during
 *   sos_setup leaves *out NULL; its message is available from
 *   sos_last_error(NULL).
 * - Solver outcomes are reported in sos_result.status, not in return codes.
 * - Every entry point is synchronous with respect to the host unless noted;
 *   device work is issued on the stream given in sos_options.cuda_stream
 *   (NULL: a stream the library creates).
 */
#ifndef LIBSOS_SOS_H
#define LIBSOS_SOS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ---- */
#define SOS_OK 0
#define SOS_ERR_INVALID_ARG (-1)   /* malformed input: bad sizes, a monomial that is not a row, ... */
#define SOS_ERR_CUDA (-2)          /* a CUDA runtime call failed */
#define SOS_ERR_FACTOR (-3)        /* the Woodbury core I + A_L^T P^-1 A_L is not SPD in FP64 */
#define SOS_ERR_TIMEOUT (-4)       /* a bounded device-side wait expired; the context stays usable */
#define SOS_ERR_UNSUPPORTED (-5)   /* option not available for this problem (e.g. block too large) */

/* ---- solver status (sos_result.status) ---- */
#define SOS_RUNNING 0
#define SOS_SOLVED 1
#define SOS_PRIMAL_INFEASIBLE 2
#define SOS_DUAL_INFEASIBLE 3
#define SOS_MAX_ITER 4
#define SOS_NUMERICAL 5

/* ---- precision forms (sos_options.precision) ----
 * The Woodbury core (factor and solve), tau/kappa and every residual are FP64
 * in all forms. */
#define SOS_PREC_FP64 0   /* plain: FP64 iterates, FP64 PSD projections */
#define SOS_PREC_MIXED 1  /* FP64 iterates, PSD projections computed in FP32 */
#define SOS_PREC_FP32 2   /* FP32 iterates and FP32 projections */

typedef struct sos_handle sos_handle;

/* One Gram block X_b of a constraint.  basis_exps lists the N monomials of
 * its basis v (eq. (4) for the full basis).  With n_weight_terms == 0 the
 * block contributes v^T X v (eq. (5)); otherwise it contributes
 * p(x) v^T X v with p = sum_k weight_coef[k] x^weight_exps[k] (eq. (38)). */
typedef struct {
  int32_t N;
  const int32_t* basis_exps;   /* [N x n_vars] */
  int32_t n_weight_terms;
  const int32_t* weight_exps;  /* [n_weight_terms x n_vars] */
  const double* weight_coef;   /* [n_weight_terms] */
} sos_block;

/* One polynomial identity of eq. (7):
 *   g_0(x) - sum_i u_i g_i(x) = sum_b (weighted) Gram forms of its blocks,
 * matched coefficient-wise on the n_rows monomials row_exps (eq. (11)).
 * term k adds term_coef[k] x^term_exps[k] to g_{term_poly[k]}
 * (term_poly 0 = g_0 -> b, 1..t = g_i -> column i-1 of A_1). */
typedef struct {
  int32_t n_rows;
  const int32_t* row_exps;     /* [n_rows x n_vars], distinct */
  int64_t n_terms;
  const int32_t* term_poly;    /* [n_terms] in 0..t */
  const int32_t* term_exps;    /* [n_terms x n_vars] */
  const double* term_coef;     /* [n_terms] */
  int32_t n_blocks;
  const sos_block* blocks;     /* [n_blocks] */
  int32_t matrix_r;            /* 0: the polynomial identity above; r >= 1:
                                  a matrix-valued constraint of size r */
  const int32_t* term_pair;    /* matrix-valued: [n_terms x 2] entry (i, j),
                                  0 <= i <= j < r, of P_{term_poly[k]} that
                                  term k belongs to; else unused */
} sos_constraint;

/* Matrix-valued constraints (Section V, eq. (47)-(48)), matrix_r = r >= 1:
 *   P_0(x) - sum_h u_h P_h(x) = (I_r (x) v(x))^T Y (I_r (x) v(x)),  Y PSD,
 * with term k adding term_coef[k] x^term_exps[k] to entry term_pair[k] of
 * P_{term_poly[k]} (the matrices are symmetric: give entries i <= j only),
 * row_exps the monomials alpha to match, and exactly one unweighted block
 * whose basis is v (Y is then r N x r N, rows and columns block-major:
 * index i N + a is basis monomial a of block row i).  The library matches
 * coefficients for every triple (alpha, i, j) of Prop. 2 with i <= j (rows
 * ordered by the pairs (i, j) row-major, then alpha): (alpha, i, j) and
 * (alpha, j, i) state the same equation for a symmetric Y, so the row
 * collects both blocks Y_ij and Y_ji and its right side is
 * 2 (P_0)_ij - 2 sum_h u_h (P_h)_ij for i < j (the coefficient of
 * y_i y_j x^alpha in y^T P(x) y).  Internally it runs the constraint as a
 * scalar one in the variables (x, y_1..y_r) -- basis y_i x^a, rows
 * y_i y_j x^alpha -- so the Gram entries of Y keep the orthogonal rows of
 * Prop. 2 and share the scalar index map. */

/* min w^T u subject to the constraints (eq. (7), eq. (15)). */
typedef struct {
  int32_t n_vars;
  int32_t t;
  const double* w;                   /* [t] */
  int32_t n_constraints;
  const sos_constraint* constraints; /* [n_constraints] */
} sos_program;

/* solve_mode: how iterations are launched.
 *   0 auto: the persistent launch for a batch (n_progs > 1) whose Gram
 *     blocks are all small (N <= 96 FP64 projections, <= 112 mixed, <= 128 FP32), else
 *     one CUDA graph of per-phase kernels per iteration;
 *   1 one CUDA graph of per-phase kernels per iteration (any block size);
 *   2 the persistent launch (error SOS_ERR_UNSUPPORTED with a large block).
 * The persistent launch runs all iterations of a solve in one cooperative
 * kernel; residual checks and termination happen on the device.  At setup an
 * autotuner times a few iterations of every candidate -- persistent grids of
 * 1..4 CTAs per SM with a round-robin or a work-queue block schedule and, in
 * auto mode, the per-phase graph -- keeps the fastest, and resets the iterate
 * to the cold start. */
typedef struct {
  int32_t precision;      /* SOS_PREC_* */
  int32_t k_check;        /* residual check period in iterations (>= 1) */
  void* cuda_stream;      /* cudaStream_t to issue work on, or NULL */
  int32_t solve_mode;     /* 0, 1 or 2 as above */
  int32_t large_method;   /* projection of blocks too large for one CTA:
                             0 auto = Newton-Schulz on the tensor cores for
                             FP32 projections, grid Jacobi for FP64;
                             1 grid Jacobi; 2 Newton-Schulz (FP32 forms) */
  int32_t warm_restart;   /* the Jacobi projections start from the previous
                             iteration's eigenvectors and restart from the
                             identity after this many warm iterations;
                             0 = 1024, 1 = every iteration cold */
  int32_t weighted_form;  /* weighted blocks (eq. (37)): 0 auto, per program by
                             eq. (42) -- directly while the Woodbury core
                             t + sum N_i (N_i + 1) / 2 over weighted blocks is
                             smaller than m, else with extra polynomials;
                             1 always directly; 2 always with extra
                             polynomials: p s becomes p r with r free (its
                             coefficients r_beta, one per monomial of v v^T
                             in the order of eq. (4), follow the t variables)
                             and a new identity r = v^T X v (after the
                             program's constraints) holds X as a plain block.
                             sos_dims, the iterate and the solution then
                             describe that program. */
  double infeas_tol;      /* tolerance of the infeasibility certificates of
                             sos_solve, independent of its tol; 0 = 1e-7 */
  int32_t wait_limit_us;  /* bound of every grid-wide wait of the cooperative
                             kernels, in microseconds; 0 = about 2 s.  A wait
                             that runs out makes the kernel return early and
                             the next synchronising call report
                             SOS_ERR_TIMEOUT; the context stays usable */
  int32_t reserved;       /* must be zero */
} sos_options;

/* Per-instance solve report.  x, y, s are optional caller-allocated HOST
 * buffers (NULL to skip) receiving the normalised solution
 * xi = u_xi / tau (n_x), y = u_y / tau (m) and the dual slack z = v_z / tau
 * of eq. (17) (n_x).  Residuals follow the definitions documented with
 * sos_solve. */
typedef struct {
  double* x;
  double* y;
  double* s;
  double res_primal;
  double res_dual;
  double gap;
  double obj_primal;   /* c^T xi */
  double obj_dual;     /* b^T y */
  double tau;
  double kappa;
  int32_t iters;
  int32_t status;      /* SOS_* status */
} sos_result;

/* Builds the conic data of every program (coefficient matching eq. (11),
 * index map of the indicator matrices eq. (8) and eq. (38)), splits the
 * columns into the orthogonal part (plain Gram blocks, Prop. 1) and the
 * low-rank part (free variables and weighted blocks), factors the FP64
 * Woodbury core I + A_L^T P^-1 A_L (eq. (28)) once, precomputes M^-1 zeta
 * (eq. (25)), copies everything to the device and sets the iterate to the
 * cold start u = v = (0, 0, 1).  n_progs >= 1 instances are solved together
 * (batched); each keeps its own data and status.
 * Errors: SOS_ERR_INVALID_ARG (a monomial of g_i, of a block product or of a
 * weight product that is not among the rows; non-positive sizes),
 * SOS_ERR_FACTOR, SOS_ERR_CUDA, SOS_ERR_UNSUPPORTED. */
int sos_setup(const sos_program* progs, int32_t n_progs, const sos_options* opts, sos_handle** out);

/* Releases all device and host memory of the handle (NULL is a no-op). */
void sos_destroy(sos_handle* h);

/* Message of the last error on h (or of the last failed sos_setup when h is
 * NULL).  The string stays valid until the next call on the same handle. */
const char* sos_last_error(const sos_handle* h);

/* Sizes of instance inst: dims = {n_x, m, t, t_eff, n_blocks, total Gram
 * entries}, where t_eff = t + sum of packed sizes of weighted blocks is the
 * order of the Woodbury core. */
int sos_dims(const sos_handle* h, int32_t inst, int64_t dims[6]);

/* Runs ADMM (eq. (20)) from the current iterate until every instance has
 * terminated or max_iter iterations have run.  Every k_check iterations each
 * running instance is checked (tau > 1e-12 (kappa + 1)):
 *   res_primal = |A xi - b| / (1 + |b|),  res_dual = |A^T y + z - c| / (1 + |c|),
 *   gap = |c^T xi - b^T y| / (1 + |c^T xi| + |b^T y|),
 * SOLVED when all three are <= tol; while kappa > tau (the embedding's
 * infeasibility branch, eq. (18)-(19)) PRIMAL_INFEASIBLE when b^T u_y > 0 and
 * |A^T u_y + v_z| / b^T u_y <= infeas_tol, DUAL_INFEASIBLE when c^T u_xi < 0
 * and |A u_xi| / -c^T u_xi <= infeas_tol (sos_options.infeas_tol, default
 * 1e-7: with the residual tolerance, a feasible program whose optimal value
 * exceeds |c| / tol passes the primal test during the iteration);
 * NUMERICAL on a non-finite iterate.  A
 * terminated instance is frozen (its iterate no longer changes).
 * results: array of n_progs reports (may be NULL).  Returns SOS_OK or an
 * error code (SOS_ERR_TIMEOUT if a bounded device wait expired). */
int sos_solve(sos_handle* h, double tol, int32_t max_iter, sos_result* results);

/* Runs exactly iters ADMM iterations on every running instance with no
 * residual checks (the timing and parity entry point).  Asynchronous: returns
 * after enqueueing the work on the handle's stream. */
int sos_iterate(sos_handle* h, int32_t iters);

/* Waits for the handle's stream and reports a device-side error flag
 * (SOS_ERR_TIMEOUT) raised by any kernel since the last call. */
int sos_sync(sos_handle* h);

/* Copies the HSDE iterates of all instances (concatenated in instance order,
 * each [n_x + m + 1]) to / from HOST buffers.  set_iterate also marks every
 * instance as running (warm start, resume from a checkpoint).  Both calls
 * synchronise the handle's stream before returning.  One contiguous copy
 * each way goes through a device staging buffer (2 x the concatenated length
 * in doubles, allocated by the first call and owned by the handle); pinned
 * host buffers copy at full link speed, pageable ones through the CUDA driver's
 * staging.  Errors: SOS_ERR_INVALID_ARG (NULL), SOS_ERR_CUDA. */
int sos_get_iterate(sos_handle* h, double* u, double* v);
int sos_set_iterate(sos_handle* h, const double* u, const double* v);

/* The same exchange with DEVICE buffers of sum_i (n_x + m + 1) doubles each
 * (same layout and row order as above), for callers whose data already
 * lives on the GPU (a warm-start predictor, a pipeline of solves).  The copy
 * runs on the handle's stream and the call returns without waiting: the
 * caller orders its own producers and consumers of u, v with that stream
 * (sos_stream).  The first call builds a position map on the device
 * (8 bytes per element).  set marks every instance as running. */
int sos_get_iterate_device(sos_handle* h, double* u, double* v);
int sos_set_iterate_device(sos_handle* h, const double* u, const double* v);

/* Exponents of all monomials of degree <= degree in n_vars variables in the
 * graded order of eq. (4) (x1 > x2 > ... within a degree).  Writes at most
 * capacity rows to out (may be NULL) and the total count to *count. */
int sos_monomials(int32_t n_vars, int32_t degree, int32_t* out, int64_t capacity, int64_t* count);

/* Host-only view of the index map of ONE program (no GPU needed), for
 * checking the setup: dims as in sos_dims; if the arrays are non-NULL,
 * ent_row[n_x] receives for each packed entry the row of its single nonzero
 * for a plain Gram entry (eq. (8)) or -1 for a low-rank entry (free variable
 * or weighted block), p_diag[m] the diagonal of P = I + A_D A_D^T (Prop. 1),
 * b[m] the coefficients of g_0, and *zeta_h the scalar zeta^T M^{-1} zeta of
 * eq. (25); weighted_form as in sos_options.  Errors as sos_setup. */
int sos_host_plan(const sos_program* prog, int32_t weighted_form, int64_t dims[6], int32_t* ent_row, double* p_diag,
                  double* b, double* zeta_h);

/* Projection onto the PSD cone of ONE symmetric N x N matrix (the Gram-block
 * part of the cone projection of eq. (20b)): out = svec(P_S+(smat(in))),
 * P_S+(X) = V max(Lambda, 0) V^T.  in, out: DEVICE pointers to N(N+1)/2
 * doubles in the packed order above (they must not overlap).  The work runs
 * on stream (a cudaStream_t; NULL = legacy default stream) and the call
 * returns when it has finished.  The call allocates its scratch (about
 * 5 N^2 doubles for N > 96, less below) with cudaMalloc and frees it before
 * returning.  Errors: SOS_ERR_INVALID_ARG (N < 1 or NULL pointers),
 * SOS_ERR_CUDA, SOS_ERR_TIMEOUT; the message is in sos_last_error(NULL). */
int sos_psd_project(const double* in, double* out, int32_t N, void* stream);

/* The projection of the mixed-precision form (SOS_PREC_MIXED), for one block.
 * N <= 112: cyclic Jacobi in FP32, then one refinement with FP64 sums -- the
 * eigenvector matrix V is re-orthonormalised with F = V^T V - I, the Ritz
 * matrix B = V^T W V is formed, and its off-diagonal part enters to first
 * order (the derivative of the eigenvalue map max(., 0) at diag(B)); the
 * result is accurate to about 1e-7 |W|_F, where the FP32 Jacobi alone gives
 * about 1e-5 |W|_F.  N > 112: P(W) = (W + W sign(W)) / 2 with sign(W) by the
 * Newton-Schulz iteration on the tensor cores (BF16 three-part operands,
 * FP32 accumulation), as the large blocks of that form; accurate to about
 * 1e-5 |W|_F, less for eigenvalues closer to zero than the iteration's
 * stopping tolerance resolves.  Same contract as sos_psd_project (device
 * pointers to N(N+1)/2 packed doubles; off-diagonal entries scaled by
 * sqrt 2); an N whose Newton-Schulz grid needs more CTAs than the GPU has
 * SMs returns SOS_ERR_UNSUPPORTED.
 * Errors: SOS_ERR_INVALID_ARG, SOS_ERR_UNSUPPORTED, SOS_ERR_CUDA,
 * SOS_ERR_TIMEOUT. */
int sos_psd_project_mixed(const double* in, double* out, int32_t N, void* stream);

/* Allocation-free variant of sos_psd_project, for callers that cannot call
 * cudaMalloc: code whose device memory is owned by a pool or allocator it
 * may not bypass, latency-critical loops that must not block on the CUDA
 * allocator, or plugins whose host forbids device allocations after start-up.
 * The paper has no counterpart: this is a deployment convenience.
 *
 * Same contract as sos_psd_project (in, out: DEVICE pointers to N(N+1)/2
 * packed doubles, not overlapping; work on stream; the call synchronises
 * that stream and returns when the projection has finished),
 * except that the call allocates nothing: its scratch is one fixed array of
 * about 3 MB compiled into the library, resident on every GPU that loads the
 * library until the process exits.
 * - N must satisfy 1 <= N <= SOS_NOALLOC_MAX_N; larger N is rejected with
 *   SOS_ERR_INVALID_ARG and a message in sos_last_error(NULL).
 * - The first call on each device (with that device current) looks up the
 *   device address of the scratch array once; make that first call before
 *   any stream capture begins.
 * - Every call uses the same scratch array, which keeps the previous call's
 *   contents (the call clears what must start at zero).  Calls whose work
 *   overlaps on the GPU -- from several host threads, or on several streams --
 *   race on that array and corrupt each other's results: serialise them.
 * Errors: SOS_ERR_INVALID_ARG, SOS_ERR_CUDA, SOS_ERR_TIMEOUT. */
#define SOS_NOALLOC_MAX_N 256
int sos_psd_project_noalloc(const double* in, double* out, int32_t N, void* stream);

/* ---- learned warm start: the network ----
 * A multilayer perceptron theta -> predicted iterate used to warm-start the
 * solver on a parametric family of SOS programs (the paper has no learned
 * component; this is the warm-start form built around its solver):
 *   h1 = relu(X W1^T + b1), h2 = relu(h1 W2^T + b2), y = h2 W3^T + b3,
 * trained with Adam (beta1 0.9, beta2 0.999, eps 1e-8) on the mean squared
 * error of targets standardised per output column (mean/std set by
 * sos_mlp_fit_scaling; identity until then).  All products run on the tensor
 * cores (tcgen05) with BF16 operands and FP32 accumulation; weights, moments
 * and activations are FP32.  Flat parameter order: W1 [n_hidden x n_in], b1,
 * W2 [n_hidden x n_hidden], b2, W3 [n_out x n_hidden], b3.
 * Data pointers X [batch x n_in] and Y [batch x n_out] are row-major DEVICE
 * pointers owned by the caller; params/grads are HOST arrays of
 * sos_mlp_param_count floats.  Work runs on the stream given at creation and
 * every call returns after it has finished.  Errors: SOS_ERR_INVALID_ARG,
 * SOS_ERR_CUDA, SOS_ERR_TIMEOUT (message in sos_last_error(NULL)). */
typedef struct sos_mlp sos_mlp;
int sos_mlp_create(int32_t n_in, int32_t n_hidden, int32_t n_out, uint64_t seed, void* cuda_stream, sos_mlp** out);
void sos_mlp_destroy(sos_mlp* net);
int64_t sos_mlp_param_count(const sos_mlp* net);
int sos_mlp_set_params(sos_mlp* net, const float* params);  /* also resets the Adam moments */
int sos_mlp_get_params(const sos_mlp* net, float* params);
/* per-column mean and standard deviation of the training targets Y [rows x n_out] */
int sos_mlp_fit_scaling(sos_mlp* net, const float* Y, int32_t rows);
/* loss (standardised targets) and, if grads != NULL, its gradient */
int sos_mlp_gradients(sos_mlp* net, const float* X, const float* Y, int32_t batch, double* loss, float* grads);
/* one Adam step on a batch; *loss (may be NULL) is the loss before the step */
int sos_mlp_train_step(sos_mlp* net, const float* X, const float* Y, int32_t batch, float lr, double* loss);
/* Y = de-standardised prediction for X */
int sos_mlp_predict(sos_mlp* net, const float* X, float* Y, int32_t batch);

/* Diagnostics (synchronises the handle's stream): out[0] = iterations run
 * since setup, out[1] = number of Gram blocks, out[2] = largest number of
 * Jacobi sweeps (or Newton-Schulz iterations) any block needed in the last
 * projection, out[3] = their total over all blocks. */
int sos_stats(sos_handle* h, int64_t out[4]);

/* Launch configuration chosen for the handle: out[0] = 1 for the persistent
 * launch (0: per-phase kernels), out[1] = its grid size (CTAs) -- or, for the
 * per-phase path with a large block projected by the grid Jacobi kernel, the
 * grid size the autotuner chose for that kernel (a quarter, half or all of
 * the SMs) --, out[2] = 1
 * for the work-queue block schedule (0: round-robin, largest block first),
 * out[3] = candidates timed by the autotuner, out[4] = microseconds per
 * iteration of the chosen candidate during tuning. */
int sos_tuning(const sos_handle* h, int32_t out[5]);

/* Sets the bound of the grid-wide waits (as sos_options.wait_limit_us; 0 =
 * about 2 s) for the iterations issued from now on.  Errors:
 * SOS_ERR_INVALID_ARG (us < 0), SOS_ERR_CUDA. */
int sos_set_wait_limit(sos_handle* h, int32_t us);

/* Number of CUDA kernels one ADMM iteration launches for this handle. */
int sos_launches_per_iteration(const sos_handle* h);

/* Profiling hooks (used by the benchmark to time single stages with events
 * on the handle's stream).  sos_stream returns the cudaStream_t in use.
 * sos_run_stage enqueues one stage of one iteration: 0 = affine step (all
 * kernels up to the cone projection), 1 = PSD projection of small blocks,
 * 2 = PSD projection of large blocks, 3 = one full iteration, and single
 * kernels of the affine step: 4 = row gather r = w2_hat - A w1_hat,
 * x = P^-1 r (eq. (27b)), 5 = y = A_L^T x, 6 = Woodbury solve
 * z = L^-T L^-1 y (eq. (28)), 7 = sigma_2 = x - P^-1 A_L z, 8 = per-instance
 * scalars (eq. (24b), (25)) and free variables, 9 = u_y, v_y and u_hat_2
 * rows; and single kernels of the large-block projection (stage 2 is
 * 15, 10..14 in that order): 15 = warm attempt, the FP64 refinement and
 * reconstruction started from the previous iteration's eigenvectors (it
 * does nothing unless the last iteration left them and no cool-down after
 * a failed attempt is running; when it succeeds, 10..14 do nothing),
 * 10 = gather of W into a dense FP32 copy, 11 = Householder reduction to
 * tridiagonal form, 12 = eigenvectors of the tridiagonal matrix mapped
 * back, 13 = FP64 refinement and reconstruction (10..13 and 15 do nothing
 * for blocks that the FP64 tridiagonal path does not take), 14 = grid
 * Jacobi kernel (the whole projection of those blocks; after a successful
 * tridiagonal path it does nothing).  Stages 4..15 run out of order leave
 * the iterate meaningless; they exist to time one kernel.
 * sos_stage_bytes gives the algorithmic bytes of one launch of a stage:
 * every array element the stage has to read or write, counted once (the
 * numerator of an HBM roofline fraction).  Errors: SOS_ERR_INVALID_ARG. */
void* sos_stream(sos_handle* h);
int sos_run_stage(sos_handle* h, int32_t stage);
int sos_stage_bytes(const sos_handle* h, int32_t stage, int64_t* bytes);

#ifdef __cplusplus
}
#endif
#endif /* LIBSOS_SOS_H */
