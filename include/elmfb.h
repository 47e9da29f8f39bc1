/*
 * elmfb.h -- C ABI of the GB300 multilevel ELM-FBPINN solver (arxiv 2409.01949).
 *
 * The method (paper §3): a linear PDE  N[u] = f  on interior collocation
 * points and linear boundary conditions  B_b[u] = g_b  on boundary point sets
 * are fitted by the multilevel random-feature model
 *
 *     u_hat(x) = (1/L) sum_l sum_j w_j^(l)(x) sum_k a_ljk phi_ljk(x)
 *
 * (Eq. multilevel_solution), whose hidden parameters are fixed, so the
 * physics-informed loss (Eq. multilevel_loss) is the linear least-squares
 * problem  min_a ||M a - h||  (Eq. multilevel_ls) with a block-sparse M
 * (Eq. multilevel_domain_decomp).  This library creates the decomposition and
 * random features, assembles M and h on the GPU, solves for a, and evaluates
 * u_hat.
 *
 * Conventions shared by every entry point:
 *   - Every function returns an int status, ELMFB_OK (0) on success.  On an
 *     error the handle keeps a message readable through elmfb_last_error().
 *   - Pointer arguments may be host or device memory (CUDA unified
 *     addressing decides); they are borrowed for the duration of the call
 *     and copied.  Outputs are caller-allocated.
 *   - One handle is bound to one CUDA stream and one device; handles are not
 *     thread-safe.  The handle owns all device memory it allocates and frees
 *     it in elmfb_destroy().
 *   - Indices are 0-based.  Column q of M is (level l, subdomain j, feature k)
 *     with q = sum_{m<l} J_m K + j K + k (paper §3 "Indexing conventions");
 *     2-D subdomains are numbered j = j_y n_l + j_x.  Rows of M are the
 *     interior points in the order given, then each boundary set in order
 *     (paper §3, rows of Eq. multilevel_ls).
 */
#ifndef ELMFB_H
#define ELMFB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes --------------------------------------------------------- */
enum {
  ELMFB_OK = 0,
  ELMFB_ERR_INVALID_ARG = 1,  /* bad size, pointer, or option                   */
  ELMFB_ERR_OOM = 2,          /* allocation failed (device, or the host handle)  */
  ELMFB_ERR_CUDA = 3,         /* a CUDA runtime call failed (message has details) */
  ELMFB_ERR_STATE = 4,        /* call out of order (e.g. solve before assemble)   */
  ELMFB_ERR_NOT_CONVERGED = 5,/* iteration cap reached; coefficients still valid  */
  ELMFB_ERR_BREAKDOWN = 6,    /* factorisation pivot or Krylov scalar <= 0         */
  ELMFB_ERR_NONFINITE = 7,    /* NaN/Inf produced (flag raised by a kernel)       */
  ELMFB_ERR_TIMEOUT = 8,      /* a bounded device-side wait gave up               */
  ELMFB_ERR_UNSUPPORTED = 9   /* size or feature outside the documented limits     */
};

/* ---- precision of the stored system (paper §4.1 states none) --------------- */
enum {
  ELMFB_FP64 = 0,   /* panels, Gram and solver vectors in FP64                  */
  ELMFB_FP32 = 1,   /* panels FP32, FP64 solver vectors and reductions          */
  ELMFB_MIXED = 2,  /* FP32 panels + BF16 copy for tensor-core Gram blocks       */
  ELMFB_DF32 = 3,   /* panels as FP32 pairs (hi + lo, ~48-bit significand, same
                       8 bytes as FP64), products and sums in float-float
                       arithmetic on the FP32 pipes; entries evaluated in FP64.
                       The solvers need K a multiple of 4, K <= 128, at most 30
                       covering panels per cell and (covering panels per
                       cell) x K <= 1696 (else UNSUPPORTED)                   */
  ELMFB_FP32_DF32 = 4 /* mixed precision with refinement: FP32 panels for the
                       iterations plus FP32-pair (ELMFB_DF32) panels of the
                       same entries (12 bytes per entry) for FP64-accurate
                       residuals; elmfb_solve's `refine` outer steps of LSQR
                       each solve min ||M_fp32 d - r|| for r = h - M a formed
                       from the pair panels, then a += d.  Same limits as
                       ELMFB_DF32                                             */
};

/* ---- subdomain centre placement (paper §4.1 "Domain decomposition") -------- */
enum {
  ELMFB_PLACE_CELL = 0,     /* mu_j = lo + (j + 1/2) (hi - lo) / n              */
  ELMFB_PLACE_ENDPOINT = 1  /* mu_j = lo + j (hi - lo) / (n - 1); n = 1: midpoint */
};

/* ---- solvers ---------------------------------------------------------------- */
enum {
  ELMFB_SOLVE_LSQR = 0,     /* right-preconditioned LSQR on M (paper §3, §4.1)   */
  ELMFB_SOLVE_PCG = 1,      /* preconditioned CG on the Gram normal equations    */
  ELMFB_SOLVE_FCG_GNN = 2,  /* flexible CG with the learned preconditioner       */
  ELMFB_SOLVE_QR = 3        /* dense Householder QR with column pivoting: the
                               basic least-squares solution with the rank cut
                               |R_kk| <= rcond |R_11|; needs the dense M (rows x
                               (columns + 1) FP64) to fit in device memory     */
};

/* ---- preconditioners --------------------------------------------------------- */
enum {
  ELMFB_PREC_NONE = 0,      /* plain LSQR, the paper's protocol                  */
  ELMFB_PREC_BLOCK_JACOBI = 1,/* per-subdomain Cholesky of the shifted diagonal
                               Gram block (not in the paper)                      */
  ELMFB_PREC_BJ_GNN = 2,    /* FCG only: block-Jacobi plus the learned correction */
  ELMFB_PREC_BJ_COARSE = 3  /* FCG only: block-Jacobi on the subdomains of the finer
                               levels and, on all columns of levels 1..coarse_levels
                               together, the inverse of their shifted joint Gram
                               block (a coarse-level correction; not in the paper) */
};

typedef struct elmfb_ctx* elmfb_t;

/* Decomposition and random features (paper §3 "Problem and model definition",
 * §4.1 "Domain decomposition" and "weight initialisation").
 *   dim          1 or 2
 *   lo, hi       domain box [lo_i, hi_i] per dimension (entries >= dim ignored)
 *   n_levels     L >= 1, at most ELMFB_MAX_LEVELS
 *   levels       [n_levels] subdomains per dimension at each level (J_l = n^dim)
 *   delta        width ratio delta > 1; half-width sigma = delta * spacing / 2
 *   placement    ELMFB_PLACE_*
 *   features     K >= 1 random features per subdomain, at most ELMFB_MAX_FEATURES
 *   seed         SplitMix64 seed of the parameter stream
 *   weight_scale a: every hidden weight and bias is drawn from U(-a, a)
 *   precision    ELMFB_FP64 / ELMFB_FP32 / ELMFB_MIXED / ELMFB_DF32 /
 *                ELMFB_FP32_DF32
 *   n_holes, holes  0 .. ELMFB_MAX_HOLES boxes (lo_x, lo_y, hi_x, hi_y; 1-D:
 *                lo, -, hi, -) cut out of the domain: every subdomain whose
 *                centre lies inside a hole is discarded -- strictly between
 *                its faces, a face on the domain box's boundary counting as
 *                part of the hole (paper §4.1:
 *                on the L-shaped domain of §4.4 the subdomains outside the
 *                domain are discarded).  The remaining subdomains keep their
 *                order and are renumbered consecutively, so N_Phi = K x (kept
 *                subdomains); windows are normalised over the kept subdomains
 *                of a level, and a point no kept subdomain of level l covers
 *                gets no term from that level.
 *   ansatz_omega w > 0: hard-constraint ansatz of paper §4.3, the model is
 *                u~(x) = A(x) u_hat(x), A = prod_i tanh(w (x_i - lo_i))
 *                tanh(w (hi_i - x_i)), which vanishes on the box boundary; the
 *                columns of M become Op[A w_j phi_jk] and elmfb_eval returns
 *                u~.  0: no ansatz.
 * Parameter stream: output i of SplitMix64(seed) is
 * mix(seed + (i+1) * 0x9E3779B97F4A7C15); column q of the full grid (before
 * any discarding) draws outputs q*(dim+1)+p (p < dim: weight p, p = dim:
 * bias); u = (z >> 40) * 2^-24, value = a (2u - 1).  The feature input is
 * (x - mu_j) / sigma_j. */
#define ELMFB_MAX_LEVELS 12
#define ELMFB_MAX_FEATURES 256
#define ELMFB_MAX_ROWSETS 16
#define ELMFB_MAX_HOLES 4
typedef struct {
  int dim;
  double lo[2];
  double hi[2];
  int n_levels;
  int levels[ELMFB_MAX_LEVELS];
  double delta;
  int placement;
  int features;
  uint64_t seed;
  double weight_scale;
  int precision;
  int n_holes;
  double holes[ELMFB_MAX_HOLES][4];
  double ansatz_omega;
} elmfb_config;

/* Create a handle on the current CUDA device, bound to `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  Draws the random
 * parameters (host, SplitMix64) and uploads the geometry tables.
 * Errors: INVALID_ARG for an out-of-range field, OOM, CUDA. */
int elmfb_create(elmfb_t* out, const elmfb_config* cfg, void* cuda_stream);

/* Release every device buffer of the handle.  NULL is accepted. */
void elmfb_destroy(elmfb_t h);

/* Message of the last error on this handle ("" if none).  The string is owned
 * by the handle and valid until the next call on it. */
const char* elmfb_last_error(elmfb_t h);

/* One block of rows of Eq. multilevel_ls.  The operator applied to the model
 * is the constant-coefficient operator
 *     Op[v] = c0 v + sum_i c1[i] d_i v + sum_i c2[i] d_ii v
 * (paper §3: N and B_b linear).  The first row set of elmfb_assemble is the
 * interior set N[u] = f, row scale 1/sqrt(N_I) ("Definition of vectors");
 * every later set is a boundary set B_b[u] = g_b with penalty weight
 * lambda_b > 0, row scale sqrt(lambda_b / N_B^(b)).
 *   points  [n * dim] row-major FP64 coordinates, inside the domain box
 *   rhs     [n] FP64 values of f or g_b at the points (unscaled)          */
typedef struct {
  int64_t n;
  const double* points;
  const double* rhs;
  double c0;
  double c1[2];
  double c2[2];
  double weight;      /* lambda_b; ignored for the interior set */
} elmfb_rowset;

/* Assemble M and h on the device (paper §3 "Definition of the system
 * matrices": N_{n,q} = N[w_j phi_jk](x_n) / (sqrt(N_I) L), B_{p,q} =
 * sqrt(lambda_b/N_B^(b)) B_b[w_j phi_jk](x_p) / L), applying the operator to
 * w_j phi_jk analytically by the product rule.  Sorts rows by the cells of
 * the common refinement of all subdomain supports and stores M as dense
 * per-subdomain panels M_j = M restricted to I_j x K_j (Eq.
 * multilevel_domain_decomp).  Replaces any previous system of the handle.
 *   n_sets  1 .. ELMFB_MAX_ROWSETS; sets[0] is the interior set
 * Errors: INVALID_ARG (empty interior set, points outside the box, bad sizes),
 * UNSUPPORTED (2^31 or more rows or padded panel rows), OOM, CUDA.  Blocks until the assembly has finished on the handle's stream. */
int elmfb_assemble(elmfb_t h, int n_sets, const elmfb_rowset* sets);

/* Sizes of the handle's problem. */
typedef struct {
  int64_t n_columns;       /* N_Phi = K sum_l J_l                          */
  int64_t n_rows;          /* N_I + N_B (0 before elmfb_assemble)           */
  int64_t n_subdomains;    /* sum_l J_l                                     */
  int64_t nnz;             /* stored panel entries, padding rows excluded   */
  int64_t panel_rows;      /* stored panel rows including padding           */
  int64_t n_cells;         /* cells of the common refinement of supports     */
  int64_t n_gram_pairs;    /* subdomain pairs (i <= j) sharing a cell        */
  double gram_flops;       /* 2 K^2 x shared rows, summed over those pairs  */
  int features;
  int n_levels;
  int dim;
  int precision;
} elmfb_sizes;
int elmfb_get_sizes(elmfb_t h, elmfb_sizes* out);

/* Fixed random parameters of every column (paper §3 Eq. shallow networks):
 * W [N_Phi * dim] row-major, b [N_Phi].  Either pointer may be NULL. */
int elmfb_get_params(elmfb_t h, double* W, double* b);

/* Dense copy of selected rows of the assembled M and of h, for checking.
 *   rows [n] row indices (paper order); out [n * N_Phi] row-major FP64;
 *   h_out [n] or NULL.   Errors: STATE before assemble, INVALID_ARG. */
int elmfb_get_rows(elmfb_t h, const int64_t* rows, int64_t n, double* out, double* h_out);

/* Gram blocks G_ij = M_i^T M_j of every subdomain pair (i <= j) whose
 * supports share collocation points -- the normal-equations matrix of Eq.
 * multilevel_ls with the block structure of Eq. multilevel_domain_decomp --
 * computed on the tcgen05 tensor cores from BF16 copies of the panels with
 * FP32 accumulation.  Needs ELMFB_MIXED precision and K <= 128 (UNSUPPORTED
 * otherwise); STATE before assemble; TIMEOUT if a pipeline wait gave up.
 * The blocks stay on the device (n_gram_pairs x K x K FP32). */
int elmfb_compute_gram(elmfb_t h);

/* Copy Gram blocks out: ij [2n] pairs (i, j) of subdomain indices (either
 * order), out [n * K * K] FP64 row-major (row = feature of i, column =
 * feature of j).  Blocks of pairs that share no rows are zero. */
int elmfb_get_gram(elmfb_t h, int64_t n, const int* ij, double* out);

/* Solver options and report. */
typedef struct {
  int method;          /* ELMFB_SOLVE_*                                       */
  int preconditioner;  /* ELMFB_PREC_*                                        */
  int max_iter;        /* iteration cap (the paper uses 15000)                */
  double atol;         /* stop when ||M^T r|| <= atol ||M|| ||r|| (estimates) */
  double btol;         /* stop when ||r|| <= btol ||h||; 0 disables both tests */
  double shift;        /* Cholesky shift eps: G_jj + eps tr(G_jj)/K I          */
  int check_every;     /* host checks convergence every this many iterations;
                          with FP32 and FP32-pair panels the stopping tests
                          also run on the device after every iteration, so
                          the iteration count does not depend on it       */
  int warm_start;      /* nonzero: start from the handle's current coefficients */
  int refine;          /* outer refinement steps (>= 1).  PCG: each recomputes
                          g = M^T (h - M a) from the panels and runs max_iter
                          PCG iterations on the tensor-core Gram for the
                          update.  LSQR with ELMFB_FP32_DF32 panels: each
                          forms r = h - M a from the pair panels and runs
                          LSQR (max_iter, atol/btol/ntol) on the FP32 panels
                          for the update d of min ||M d - r||            */
  double gram_shift;   /* PCG: Tikhonov shift mu, as a fraction of the mean
                          Gram diagonal, added to the Gram operator          */
  double rcond;        /* QR: rank cut, a column is dropped once the largest
                          remaining column norm is <= rcond |R_11|           */
  double ntol;         /* LSQR: also stop when ||(M P)^T r|| <= ntol ||(M P)^T h||
                          (the preconditioned normal-equations residual
                          relative to its start, LSQR's estimate); 0 disables */
  int coarse_levels;   /* ELMFB_PREC_BJ_COARSE: the coarse block holds the columns
                          of levels 1..coarse_levels (at most 4096 of them);
                          its shift is `shift` x tr / (its columns)          */
  int autotune;        /* LSQR: nonzero picks the fused pass's work-unit size by
                          timing (elmfb_tuning_table); the choice is kept per
                          shape class for the life of the process.  In
                          elmfb_batch_solve with more than one worker it only
                          uses classes tuned before (a timing beside other
                          instances would measure them too): tune a batch's
                          classes with one worker first                   */
  int graph;           /* LSQR: nonzero captures the kernels of one check
                          interval as a CUDA graph and replays it (one launch
                          per check_every iterations); needs a handle stream
                          other than the legacy default stream and profiling
                          off, else the kernels are launched one by one.
                          Instances of elmfb_batch_solve that share launches
                          (batch_shared) run in the batch's rounds instead  */
  int batch_shared;    /* elmfb_batch_solve, LSQR on FP32 panels with
                          block-Jacobi: nonzero (the default) runs the
                          instances' iterations in shared multi-instance
                          launches; 0 launches each instance's kernels alone.
                          Results are the same either way               */
  double drop_tol;     /* block-Jacobi: 0 (the default) keeps every column;
                          > 0 drops a column of a block whose Cholesky pivot
                          (its Schur complement) is at most drop_tol times its
                          shifted diagonal, i.e. one numerically dependent on
                          the block's earlier columns; its coefficient stays 0
                          (info->precond_dropped counts them).  For FP32
                          panels on under-resolved subdomains (fewer
                          collocation points than features), whose Gram
                          blocks are singular up to FP32 rounding        */
} elmfb_solve_opts;

typedef struct {
  int status;                 /* ELMFB_OK or NOT_CONVERGED                     */
  int iterations;
  double residual_norm;       /* ||M a - h|| (LSQR estimate)                   */
  double normal_residual_norm;/* ||M^T (M a - h)|| (estimate, preconditioned) */
  double setup_ms;            /* preconditioner set-up time                    */
  double solve_ms;            /* iteration time                                */
  int precond_retries;        /* block-Jacobi: factorisations that met a
                                 non-positive pivot and were redone with the
                                 shift raised 100-fold (once per retry)        */
  int rank;                   /* QR: numerical rank (pivots kept); else 0     */
  double sigma_max;           /* extreme singular-value estimates of the
                                 solved operator: LSQR, those of the Golub-
                                 Kahan bidiagonal B_k of M P (sigma_max from
                                 below, sigma_min from above: kappa(B_k) <=
                                 kappa(M P)); QR, |R_11| and |R_rr|; else 0  */
  double sigma_min;
  int precond_dropped;        /* block-Jacobi with drop_tol: columns dropped  */
} elmfb_solve_info;

/* Fill opts with the defaults: LSQR, block-Jacobi, max_iter 15000,
 * atol = btol = 1e-10, shift 1e-12, check_every 50, cold start, refine 1,
 * gram_shift 0, rcond 1e-13, ntol 0, coarse_levels 2, autotune 0, graph 0,
 * batch_shared 1, drop_tol 0. */
void elmfb_default_solve_opts(elmfb_solve_opts* opts);

/* Solve min ||M a - h|| for the coefficients a (paper Eq. multilevel_ls; the
 * paper uses LSQR, §3 and §4.1).  The result stays in the handle.
 * ELMFB_SOLVE_PCG (not in the paper) solves the normal equations instead:
 * `refine` outer steps a += PCG(G_bf16 + mu I, M^T (h - M a)), each with
 * max_iter PCG iterations preconditioned by the block-Jacobi factors; it
 * needs ELMFB_MIXED precision (tensor-core Gram).
 * ELMFB_SOLVE_QR (a direct solve; the paper's LSQR resolves the small
 * singular directions only slowly) factors the dense M with column pivoting
 * in FP64 and returns the basic solution of rank `rank`; info->iterations =
 * rank, residual_norm = ||M a - h|| exactly.  UNSUPPORTED when the dense M
 * does not fit in device memory.
 * Errors: STATE before assemble, BREAKDOWN, NONFINITE, INVALID_ARG; TIMEOUT
 * when an on-device wait for a bulk copy ran out.
 * Returns NOT_CONVERGED (with valid coefficients) at the iteration cap. */
int elmfb_solve(elmfb_t h, const elmfb_solve_opts* opts, elmfb_solve_info* info);

/* The Golub-Kahan bidiagonal of the last LSQR solve (Paige & Saunders 1982,
 * their §3; M P with the solve's preconditioner P): alpha [k + 1] and
 * beta [k + 1] with beta_1 = ||h||, B_k lower bidiagonal with alpha_1..alpha_k
 * on its diagonal and beta_2..beta_{k+1} below it; k = the solve's
 * iterations, recorded up to max_iter + 1 entries.  *k_out receives k; either
 * array may be NULL; at most `max` entries of each are written. */
int elmfb_get_bidiagonal(elmfb_t h, int64_t max, double* alpha, double* beta, int64_t* k_out);

/* ---- learned preconditioner (not in the paper) ------------------------------
 * A message-passing network on the subdomain graph (nodes = subdomains, edges
 * = pairs sharing collocation points): input layer K -> 64, three layers
 * A_l[s] = relu(W_self A_{l-1}[s] + W_nb mean_{t in N(s)} A_{l-1}[t] + b),
 * output layer 64 -> K.  ELMFB_SOLVE_FCG_GNN runs flexible CG on M^T M a =
 * M^T h (operator applied through the panels) with z = B r + s N(B r / s),
 * s = ||B r||, B the block-Jacobi factor, when preconditioner ==
 * ELMFB_PREC_BJ_GNN (block-Jacobi alone otherwise).
 * Weight layout: W_in (64 x K), b_in (64), then per layer W_self (64 x 64),
 * W_nb (64 x 64), b (64), then W_out (K x 64), b_out (K); FP32 row-major. */
int64_t elmfb_gnn_num_weights(elmfb_t h);
/* neighbour lists: off [n_subdomains + 1], nb [n_edges] (either may be NULL) */
int elmfb_gnn_graph(elmfb_t h, int* off, int* nb, int64_t* n_edges);
int elmfb_gnn_set_weights(elmfb_t h, const float* w);
int elmfb_gnn_get_weights(elmfb_t h, float* w);
/* Forward pass on `batch` samples x [batch][n_subdomains][K]; with targets t
 * and per-sample weights wb also the loss (1/batch) sum_b wb_b ||y_b - t_b||^2
 * and, if grad != NULL, its gradient w.r.t. the weights (for checking). */
int elmfb_gnn_eval(elmfb_t h, int batch, const float* x, const float* t, const float* wb,
                   float* y, float* grad, double* loss);
/* The forward pass as FCG's learned preconditioner applies it: every layer's
 * operands (weights, input, activations, neighbour means formed in FP32) are
 * rounded to bfloat16 (to nearest, ties to even) and multiplied on the tensor
 * cores with FP32 accumulation; bias and ReLU in FP32.  x, y [batch][n_subdomains][K]
 * (host or device).  Needs K a multiple of 16 up to 128 (else
 * ELMFB_ERR_UNSUPPORTED; FCG then applies elmfb_gnn_eval's FP32 forward), and
 * weights (ELMFB_ERR_STATE before elmfb_gnn_set_weights / elmfb_gnn_train). */
int elmfb_gnn_infer(elmfb_t h, int batch, const float* x, float* y);
/* Train on pairs from block-Jacobi FCG solves of this system with n_rhs other
 * right-hand sides rhs [n_rhs][n_rows] (unscaled, row order of assemble):
 * solve_iters recorded iterations per solve (errors against the iterate
 * after 2 solve_iters), `epochs` passes of Adam (learning rate lr) over
 * mini-batches of 8; weights initialised from SplitMix64(seed) with a zero
 * output layer.  loss2 [2] receives the first and last epoch losses. */
int elmfb_gnn_train(elmfb_t h, int n_rhs, const double* rhs, int solve_iters, int epochs,
                    double lr, uint64_t seed, double* loss2);

/* ---- batched solves (not in the paper) ---------------------------------------
 * Solve many independent instances: each item is a full problem (create
 * config + row sets), optionally with evaluation points, an output buffer
 * for u_hat and reference values for the error norms.  n_workers (1..256)
 * host threads, each with its own non-blocking stream, take the instances in
 * decreasing order of estimated work; each uses its item's solver options,
 * else the batch's (opts->batch_shared is taken from the batch's).  With
 * opts->batch_shared, the LSQR iterations of the instances that are
 * iterating at the same time (FP32 panels, block-Jacobi) run as shared
 * launches: one fused pass, one slice-sum and one tail launch per iteration
 * and launch shape over all of them, every check_every iterations a check of
 * each instance's own stopping tests.  Results are identical to solving the
 * instances one by one.  Returns the first non-OK instance status
 * (NOT_CONVERGED counts as OK), else ELMFB_OK; ELMFB_ERR_CUDA without
 * touching `results` if the batch's own stream, event or buffers cannot be
 * made.  An instance that no worker took (none could create its stream)
 * reports ELMFB_ERR_CUDA in its result.  Pointers may be host or device
 * memory, as elsewhere. */
typedef struct {
  elmfb_config cfg;
  int n_sets;
  const elmfb_rowset* sets;
  int64_t n_eval;             /* 0: no evaluation                        */
  const double* eval_points;  /* [n_eval * dim]                          */
  double* eval_out;           /* [n_eval] u_hat                          */
  const double* eval_ref;     /* [n_eval] reference values, or NULL      */
  double* coeffs_out;         /* [N_Phi] coefficients, or NULL           */
  const elmfb_solve_opts* opts;  /* this instance's solver options, or NULL
                                    for the batch's                      */
} elmfb_batch_item;
typedef struct {
  int status;
  int iterations;
  double rel_l2, e_l1, max_abs;   /* NaN without eval_ref                */
  double total_ms;                /* host wall time of the instance      */
  int64_t launches;               /* kernels launched for the instance   */
  char message[160];              /* the instance's last error text, or "" */
} elmfb_batch_result;
int elmfb_batch_solve(int n, const elmfb_batch_item* items, const elmfb_solve_opts* opts,
                      int n_workers, elmfb_batch_result* results);

/* The autotuner's record (not in the paper).  A shape class is (panel
 * precision, K, most covering panels of a cell, floor(log2 padded rows)); for
 * each class seen by a solve with `autotune`, the fused LSQR pass was timed at
 * three work-unit sizes (the heuristic size, half and twice it) and the
 * fastest is used from then on.  Writes up to `max` entries and returns the
 * number of classes (negative status on a bad argument). */
typedef struct {
  int precision, features, covering_panels, rows_log2;
  int unit_rows;        /* the choice                          */
  int candidates[3];    /* the unit sizes timed                */
  double ms[3];         /* their average pass time (CUDA events) */
} elmfb_tuning_entry;
int elmfb_tuning_table(int max, elmfb_tuning_entry* out);

/* Copy the coefficients a [N_Phi] out of / into the handle. */
int elmfb_get_coeffs(elmfb_t h, double* a);
int elmfb_set_coeffs(elmfb_t h, const double* a);

/* Evaluate u_hat (paper Eq. multilevel_solution) at n points.
 *   xs [n * dim] row-major FP64 inside the domain box; out [n] FP64. */
int elmfb_eval(elmfb_t h, const double* xs, int64_t n, double* out);

/* Error norms of u_hat against reference values, reduced on the device in
 * FP64: out[0] = ||u_hat - u||_2 / ||u||_2, out[1] = e_L1 of paper Eq.
 * l1_error (population standard deviation of u), out[2] = max |u_hat - u|. */
int elmfb_error_norms(elmfb_t h, const double* u_hat, const double* u_ref, int64_t n,
                      double* out3);

/* Per-stage device times (ms) of the last calls, by CUDA events:
 * [0] create upload, [1] cell sort, [2] panel assembly, [3] Gram,
 * [4] preconditioner set-up, [5] iterations, [6] eval, [7] total assemble.  */
#define ELMFB_N_STAGES 8
int elmfb_stage_times(elmfb_t h, double* ms);

/* Number of this library's kernels launched since the handle was created. */
int64_t elmfb_kernel_launches(elmfb_t h);

/* Per-kernel device timing.  With profiling on, the main kernels are
 * bracketed by CUDA events on the handle's stream; elmfb_kernel_stats()
 * synchronises the stream and returns, for up to `max` kernels, the name
 * (static string), the summed device time (ms), the number of timed launches
 * and the algorithmic bytes one launch must move (inputs read once, outputs
 * written once; the roofline numerator).  Returns the number of kernels
 * reported (>= 0) or a negative status.  elmfb_set_profiling(h, 1) clears the
 * totals. */
int elmfb_set_profiling(elmfb_t h, int on);
/* Profiling restricted to one kernel, named as elmfb_kernel_stats() names it
 * (e.g. "fused_Mt_MTu"): the other kernels run without events around them.
 * Clears the totals.  INVALID_ARG for an unknown name. */
int elmfb_set_profiling_only(elmfb_t h, const char* kernel);
/* Time only every stride-th launch of each profiled kernel (stride >= 1; 1,
 * the default, times every launch), so that a long run carries few events.
 * INVALID_ARG for stride < 1. */
int elmfb_set_profiling_stride(elmfb_t h, int stride);

/* Device memory of destroyed handles stays cached in the library's
 * stream-ordered pool on each device, so that the next handle reuses it
 * without returning memory to the system at every synchronisation.  This call
 * synchronises the device (-1: the current one) and releases that cache. */
int elmfb_trim_memory(int device);
int elmfb_kernel_stats(elmfb_t h, int max, const char** names, double* total_ms,
                       int64_t* launches, double* bytes_per_launch);

/* Error norms that allocate nothing.  The paper has no counterpart: this entry
 * exists for callers that cannot allocate device memory when they need the
 * result -- for example because their framework's memory pool already holds
 * the device, or because they run where calling an allocator is not allowed.
 * It computes the same three numbers as elmfb_error_norms() (relative L2,
 * e_L1 with the population standard deviation, max |u_hat - u_ref|) but needs
 * no handle, makes no staging copies and calls no allocating routine.
 *   u_hat, u_ref  [n] FP64 in the current device's memory (or managed
 *                 memory), read in place; host pointers and memory of another
 *                 device are rejected with ELMFB_ERR_INVALID_ARG
 *   n             1 .. ELMFB_NOALLOC_MAX_POINTS; larger n returns
 *                 ELMFB_ERR_UNSUPPORTED before anything runs
 *   out3          [3] host memory
 *   cuda_stream   stream to run on (cudaStream_t, NULL = default stream);
 *                 the call synchronises it before returning
 * Scratch: a fixed 12 KB array in the library's device globals, one per
 * device, held until the process exits.  The first call on a device looks up
 * that array's device address (one-time set-up with the device current) and
 * caches it; after a cudaDeviceReset() of that device the cached address is
 * stale, so do not call this entry point again in that process.  Every call
 * shares the array: calls that overlap on the GPU race and must be ordered by
 * the caller.  Each call copies the partial sums to host memory and
 * synchronises the stream, so it cannot be called while that stream is being
 * captured.  An error already pending from earlier CUDA runtime calls is
 * reported as ELMFB_ERR_CUDA and left pending for its owner.  Returns
 * ELMFB_OK, INVALID_ARG, UNSUPPORTED or CUDA; there is no handle, so no
 * message is kept. */
#define ELMFB_NOALLOC_MAX_POINTS ((int64_t)1 << 24)
int elmfb_error_norms_noalloc(const double* u_hat, const double* u_ref, int64_t n, double* out3,
                              void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* ELMFB_H */
