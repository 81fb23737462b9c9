/*
 * scsf.h - C ABI of the GB300 (sm_103a) SCSF library: sorting Chebyshev
 * subspace filter for sequences of discretised symmetric eigenvalue problems.
 *
 * Problem statement (paper Sec. 2.1, Eq. (eq:eq_basic)): for a sequence of
 * symmetric matrices A^(i), i = 1..n_ops, find the k algebraically smallest
 * eigenpairs A^(i) v_j = lambda_j v_j. The library
 *   - orders the problems by the truncated-FFT greedy sort (Alg. 2), and
 *   - solves them in that order by Chebyshev filtered subspace iteration
 *     (Alg. 1, Alg. 3), each warm-started from the previous problem's block.
 *
 * Conventions for every entry point:
 *   - Array arguments are DEVICE pointers on the context's device unless a
 *     comment says "host". The caller owns every buffer; the library never
 *     frees or retains caller memory beyond the call.
 *   - Work is enqueued on the context's stream in stream order. Outputs are
 *     valid once that stream has been synchronised. Entry points that need a
 *     host decision (the solver's lock/stop test) synchronise the stream
 *     internally and return after their last kernel has finished.
 *   - Dense blocks are row-major with the column index fastest:
 *     element (row r, column c) of an R x C block with leading dimension ld is
 *     at p[r*ld + c]. Grid nodes are numbered I = i*n + j (Sec. 2.1, row-major).
 *   - Errors are returned as scsf_status; scsf_last_error() gives a message.
 *     No exceptions cross the ABI and there is no CPU fallback: a missing or
 *     unusable GPU is an error (SCSF_ERR_CUDA).
 *   - Contexts are not thread-safe; use one context per host thread.
 */
#ifndef SCSF_H
#define SCSF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SCSF_OK = 0,
  SCSF_ERR_INVALID_ARG = 1,   /* a size, pointer or parameter is out of range        */
  SCSF_ERR_CUDA = 2,          /* a CUDA runtime call or kernel launch failed         */
  SCSF_ERR_NOT_CONVERGED = 3, /* max_iter reached before k pairs met the tolerance   */
  SCSF_ERR_BREAKDOWN = 4,     /* Cholesky QR met a non-positive pivot twice          */
  SCSF_ERR_TIMEOUT = 5,       /* a bounded device-side wait gave up                  */
  SCSF_ERR_NO_MEMORY = 6      /* the caller's workspace is smaller than required     */
} scsf_status;

typedef struct scsf_ctx scsf_ctx;

/* Create a context on CUDA device `device` that enqueues on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream). *out receives the
 * handle. The context owns only small pinned host staging buffers. */
scsf_status scsf_create(scsf_ctx** out, int device, void* cuda_stream);
void scsf_destroy(scsf_ctx* ctx);
/* Message for the last failing call on this context; valid until the next call. */
const char* scsf_last_error(const scsf_ctx* ctx);
/* Library version as major*10000 + minor*100 + patch. */
int scsf_version(void);

/* ---------------------------------------------------------------------------
 * Truncated-FFT greedy sort (Alg. 2, Sec. 3.1).
 *
 * fields   : [n_ops][p][p] FP64, the parameter matrix P^(i) of each problem.
 * p0       : kept low-frequency block, 1 <= p0 <= p. Features are the DFT
 *            coefficients F[k1][k2] = (1/p) sum_{x,y} P[x][y]
 *            exp(-2 pi i (k1 x + k2 y)/p) for 0 <= k1, k2 < p0 (unshifted
 *            indices, unitary scaling; App. F).
 * start    : index of the first problem of the chain (Alg. 2 uses problem 1;
 *            indices here are 0-based).
 * workspace: device scratch of at least scsf_sort_workspace_size(n_ops, p0)
 *            bytes, 256-byte aligned.
 * perm_out : [n_ops] int32, the visiting order. Each step appends the
 *            remaining problem with the smallest squared Frobenius distance
 *            between feature blocks (FP64, fixed summation order); equal
 *            distances go to the smaller index.
 * Limits: 1 <= n_ops <= 65536, 1 <= p0 <= min(p, 64), p <= 1024 and
 * (2 p + 2 p p0) * 8 bytes <= 220 KiB (one CTA per problem holds a p x p0 block). */
size_t scsf_sort_workspace_size(int64_t n_ops, int p0);
scsf_status scsf_sort(scsf_ctx* ctx, const double* fields, int64_t n_ops, int p, int p0,
                      int start, void* workspace, size_t workspace_bytes, int32_t* perm_out);
/* scsf_sort that also writes dist_out [n_ops] (FP64, device): the squared feature distance
 * from each visited problem to its predecessor in the chain (0 for the first); the
 * learned proposal uses it to find far steps. Same arguments and limits otherwise. */
scsf_status scsf_sort_dist(scsf_ctx* ctx, const double* fields, int64_t n_ops, int p, int p0,
                           int start, void* workspace, size_t workspace_bytes, int32_t* perm_out,
                           double* dist_out);

/* scsf_sort without a caller workspace, for callers that cannot allocate device
 * memory where they sort (a host framework that owns all device memory through
 * its own fixed pool, or a latency-critical loop that must not enter the
 * allocator). The paper has no counterpart: this is a deployment convenience.
 * Same arguments, results and validation as scsf_sort (invalid arguments return
 * SCSF_ERR_INVALID_ARG first); the scratch lives in a static device array of
 * scsf_sort_noalloc_capacity() bytes (8 MiB). scsf_create reserves it on its device
 * (it looks up the array's device address, cudaGetSymbolAddress, which loads the
 * module holding it), so create the context before a memory pool takes the rest of
 * the device; if that failed, the first call on the device does the lookup again
 * (make it before any stream capture). The array stays until the process exits.
 * Valid sizes with scsf_sort_workspace_size(n_ops, p0) above the capacity
 * (n_ops > 8184 at p0 = 8) return SCSF_ERR_NO_MEMORY. The call allocates nothing
 * (no cudaMalloc/cudaFree, no allocating library routine). All calls on a
 * device share the one array and each call rewrites what it reads, so calls
 * that overlap on the GPU (other streams, other threads) race: serialise them. */
size_t scsf_sort_noalloc_capacity(void);
scsf_status scsf_sort_noalloc(scsf_ctx* ctx, const double* fields, int64_t n_ops, int p, int p0,
                              int start, int32_t* perm_out);

/* ---------------------------------------------------------------------------
 * Operators (App. D.2), Dirichlet boundary, n x n interior grid, h = 1/(n+1).
 *
 * SCSF_OP_DIV_A_GRAD: -div(a grad u), conservative 5-point form
 *   (A u)_ij = [a_{i+1/2,j}(u_ij-u_{i+1,j}) + a_{i-1/2,j}(u_ij-u_{i-1,j})
 *             + a_{i,j+1/2}(u_ij-u_{i,j+1}) + a_{i,j-1/2}(u_ij-u_{i,j-1})]/h^2
 *   ax: [n+1][n] FP64, ax[f][j] = a on the x-face between nodes (f-1, j), (f, j)
 *   ay: [n][n+1] FP64, ay[i][g] = a on the y-face between nodes (i, g-1), (i, g)
 * SCSF_OP_LAP_PLUS_V: -Lap u + V u (same stencil with a == 1, plus diag V)
 *   v : [n][n] FP64
 * SCSF_OP_CSR: any real symmetric matrix of `rows` rows in CSR form (device arrays):
 *   row_ptr [rows + 1] int32 (row_ptr[0] = 0, nondecreasing), col [nnz] int32 in
 *   [0, rows), val [nnz] FP64, nnz = row_ptr[rows] < 2^31; duplicate (row, col)
 *   entries add. Symmetry is not checked: a nonsymmetric matrix gives meaningless
 *   output, not an error. n is ignored. Only SCSF_FP64 solves take it (the mixed
 *   form's FP32 and defect-corrected filters are stencil kernels), on chains made
 *   by scsf_chain_create_rows; scsf_cheb_filter and scsf_assemble_bounds take it,
 *   scsf_cheb_filter_f32 / _dc return SCSF_ERR_INVALID_ARG.
 * SCSF_OP_PLATE: thin-plate vibration div(grad(D lap u)) = lambda rho u (App. D.2 item 4)
 *   on the n x n grid, simply supported (u = 0 and D lap u = 0 on the boundary):
 *   K = L diag(D) L with L = -Lap_h (the 5-point Dirichlet Laplacian), M = diag(rho).
 *   plate_d, plate_rho: [n][n] FP64 at the nodes, rho > 0; 2 <= n <= 12851 (13 n^2 CSR
 *   slots indexed in int32). The solver works on the
 *   symmetric standard form C = M^{-1/2} K M^{-1/2} (13-point, assembled on the device into
 *   the chain's workspace): evals are the generalized eigenvalues, resid the relative
 *   residuals of C, and evecs the M-orthonormal modes u = M^{-1/2} v (u^T M u = 1), signed
 *   as below. SCSF_FP64 only (stencil chains of side n); scsf_cheb_filter and
 *   scsf_assemble_bounds apply / bound C.
 * Unused pointers may be NULL; rows / row_ptr / col / val are read only for SCSF_OP_CSR,
 * plate_d / plate_rho only for SCSF_OP_PLATE. */
typedef enum {
  SCSF_OP_DIV_A_GRAD = 0,
  SCSF_OP_LAP_PLUS_V = 1,
  SCSF_OP_CSR = 2,
  SCSF_OP_PLATE = 3
} scsf_op_kind;

typedef struct {
  int kind;          /* scsf_op_kind                           */
  int n;             /* interior grid side, N = n*n (stencils), 2 <= n <= 46340 */
  const double* ax;
  const double* ay;
  const double* v;
  int64_t rows;            /* SCSF_OP_CSR: N = rows, 1 <= rows < 2^31 */
  const int32_t* row_ptr;  /* SCSF_OP_CSR                              */
  const int32_t* col;      /* SCSF_OP_CSR                              */
  const double* val;       /* SCSF_OP_CSR                              */
  const double* plate_d;   /* SCSF_OP_PLATE: D   [n][n]                */
  const double* plate_rho; /* SCSF_OP_PLATE: rho [n][n]                */
  const double* field;     /* the problem's parameter field P [n][n] at the nodes (the sort
                              input: a for SCSF_OP_DIV_A_GRAD, V for SCSF_OP_LAP_PLUS_V); read
                              only by chain heads when params.use_proposal, NULL otherwise */
} scsf_operator;

/* SCSF_FP64: Alg. 3 as written, every step in FP64.
 * SCSF_MIXED (not in the paper; its filter runs in one precision): an FP32 phase (filter,
 *   Cholesky QR2, Rayleigh-Ritz, rotation in FP32, no locking) until the wanted residuals
 *   reach the FP32 floor or stall, then FP64 iterations with locking whose filter is
 *   defect-corrected (the recurrence on Z = Y - X diag(y(theta)) runs in FP32, driven by the
 *   FP64 residual block) and whose orthonormalisation and Rayleigh-Ritz are FP64. Every
 *   returned pair meets tol in FP64 exactly as in SCSF_FP64. Needs k_b % 4 == 0.
 * Both forms: 1 <= k_b = k + nex <= scsf_max_block_width() (512) and k_b <= N. */
typedef enum { SCSF_FP64 = 0, SCSF_MIXED = 1 } scsf_precision;

/* How the tall block products of Alg. 3 are computed: the Gram matrices X^T X of the
 * Cholesky QR (orthonormalisation step), the Rayleigh-Ritz matrix Q^T (A Q), the rotation
 * X = Q Z and the triangular solve X R^{-1}, plus the deflation products against locked
 * columns. The paper forms them in FP64 on CPU cores.
 * SCSF_PRODUCT_TENSOR (default): on the tcgen05 tensor cores from BF16 digit planes with
 *   exact FP32 accumulation (the error-free splitting of Ozaki, Ogita and Oishi; 8 base-128
 *   digits per operand for FP64-phase products, an error of about 2^-55 of |a_i| |b_j| per
 *   term, on a par with FP64 arithmetic; 4 digits for the mixed form's FP32 phase).
 *   Results do not depend on the summation order (integer sums, one final rounding).
 * SCSF_PRODUCT_FP64: FP64 (and, in the FP32 phase, FP32) fused multiply-adds on the CUDA
 *   cores. */
typedef enum { SCSF_PRODUCT_TENSOR = 0, SCSF_PRODUCT_FP64 = 1 } scsf_product_method;

typedef struct {
  int k;             /* wanted eigenpairs (L in the paper), >= 1                          */
  int nex;           /* extra block columns; < 0 selects ceil(0.2 k) (App. D.4)            */
  int degree;        /* Chebyshev degree m >= 1 (Alg. 1)                                  */
  double tol;        /* relative residual ||A v - lambda v|| / ||A v|| to lock (App. D.5) */
  int max_iter;      /* outer iterations per problem (Alg. 3 repeat loop), >= 1           */
  int precision;     /* scsf_precision                                                    */
  uint64_t seed;     /* Philox seed of the random head block (Sec. 3.2, first problem)    */
  int degree_fp32;   /* SCSF_MIXED: Chebyshev degree of the FP32 phase (<= 0: degree)     */
  double switch_tol; /* SCSF_MIXED: leave the FP32 phase once every wanted residual is at
                        or below this (> 0), besides the FP32-floor and stall rules       */
  int products;      /* scsf_product_method of the block products                         */
  int use_proposal;  /* 1: chain heads start from the learned proposal (see scsf_proposal_*):
                        64 block columns from the network's coarse subspace prolonged to the
                        grid, the rest from the seeded Philox block, and filter bounds from
                        its predicted log(lambda_1), log(lambda_64) with lambda_kb taken as
                        lambda_64 k_b / 64 (2-D Weyl law). Needs stencil operators with
                        n a multiple of 32, k_b >= 64 and op->field set at heads           */
  const float* proposal; /* use_proposal: the network's FP32 parameters (device,
                        scsf_proposal_param_count() floats), read at every head           */
  int bound;         /* scsf_bound: the upper end beta of the filter's damped interval      */
  int column_degree; /* SCSF_MIXED, FP64 phase: 1 gives each group of 4 active columns its
                        own degree m_g <= degree from its previous residual r_j and Ritz
                        value theta_j, m_j = ceil(ln(8 r_j / tol) / ln rho_j) + 2 with
                        rho_j = |t_j| + sqrt(t_j^2 - 1), t_j = (theta_j - c) / e, clamped to
                        [8, degree], m_g the largest m_j of the group (the per-vector degree
                        of Winkelmann et al., ChASE, 2019); 0: every column takes degree    */
} scsf_params;

/* beta, the upper end of the damped interval [alpha, beta] (Sec. 2.2), must lie above the
 * spectrum. SCSF_BOUND_GERSHGORIN: the Gershgorin bound of the assembled operator (rigorous).
 * SCSF_BOUND_LANCZOS: 16 FP32 Lanczos steps from a seeded start per problem; beta = the largest
 * Ritz value of the Lanczos tridiagonal plus the norm of the last Lanczos residual, widened by
 * 0.2 % and never above the Gershgorin bound (the estimate of Sec. 3.2; Zhou and Li 2011).
 * A tighter beta widens the filter's amplification of the wanted end. */
typedef enum { SCSF_BOUND_GERSHGORIN = 0, SCSF_BOUND_LANCZOS = 1 } scsf_bound;

typedef struct {
  int iters;             /* outer iterations (Alg. 3 repeat loop)            */
  int converged;         /* 1 if k pairs met tol                             */
  int filter_steps;      /* stencil SpMM steps applied in the filter         */
  int locked;            /* pairs locked at exit                             */
  double flops_fp64;     /* algorithmic FP64 flops issued                    */
  double filter_bytes;   /* algorithmic filter bytes (3 blocks per step)     */
  double filter_elems;   /* sum over filter steps of N * active columns      */
  double rot_flops;      /* algorithmic flops of the block rotations X = Q Z */
  int rot_launches;      /* block-rotation GEMM launches                     */
  int launches;          /* kernels launched by this call                    */
  /* Per-phase device time in ms (CUDA events on the context stream), filled
   * only after scsf_set_timing(ctx, 1); zero otherwise. */
  double t_filter_ms;    /* Chebyshev filter                          */
  double t_orth_ms;      /* deflation + Cholesky QR                  */
  double t_rr_ms;        /* A Q and Q^T A Q                          */
  double t_eig_ms;       /* reduced eigensolve                       */
  double t_rot_ms;       /* rotation X = Q Z (one GEMM launch)       */
  double t_resid_ms;     /* residual norms                           */
  /* SCSF_MIXED only: the FP32 phase (counted in iters; t_filter_ms is FP64 only). */
  int iters_fp32;        /* outer iterations run in FP32                     */
  int filter32_steps;    /* FP32 stencil steps                               */
  double filter32_elems; /* sum over FP32 filter steps of N * columns        */
  double t_filter32_ms;  /* FP32 filter time                                 */
  /* SCSF_MIXED only: FP64-phase iterations filter through the defect-corrected form
   * (FP32 recurrence on Z = Y - X diag(y(theta)) driven by the FP64 residual block;
   * these steps are not in filter_steps / filter_elems / t_filter_ms). */
  int filter_dc_steps;   /* defect-corrected filter steps                    */
  double filter_dc_elems;/* sum over those steps of N * active columns       */
  double t_filter_dc_ms; /* defect-corrected filter time                     */
  /* Optional convergence history (input): when history is a host array of at
   * least 3 * max_iter doubles, iteration i writes {max, median residual of the
   * wanted unlocked pairs, pairs locked so far} to history[3 i .. 3 i + 2]. */
  double* history;
  double beta;           /* upper end of the damped interval used (scsf_params.bound)   */
  double beta_gershgorin;/* the Gershgorin bound of the operator                         */
  int chol_shifts;       /* shifted Cholesky QR restarts (S + s I) in FP64-phase iterations */
  int chol_shifts_fp32;  /* the same in the mixed form's FP32 phase                       */
} scsf_stats;

/* Enables (1) or disables (0) per-phase CUDA-event timing in scsf_stats. */
scsf_status scsf_set_timing(scsf_ctx* ctx, int enable);
/* Number of kernels this library has launched in this process so far. */
long long scsf_launch_count(void);

/* Largest block width (k + nex) the solver accepts. */
int scsf_max_block_width(void);

/* Device workspace (bytes) for problems with grid side <= n_max under params. */
size_t scsf_solve_workspace_size(const scsf_params* params, int n_max);
/* Device workspace (bytes) for SCSF_OP_CSR problems of <= rows rows (SCSF_FP64 only;
 * 0 for SCSF_MIXED or rows out of range). */
size_t scsf_solve_workspace_size_rows(const scsf_params* params, int64_t rows);

/* ---------------------------------------------------------------------------
 * Chain solve (Alg. 3 applied along a sorted sequence, Sec. 3.2).
 *
 * A chain keeps the previous problem's final block (N x k_b, k_b = k + nex)
 * and its Ritz values in the workspace as the warm start of the next problem.
 * The first problem of a chain starts from a Philox-normal block (seeded by
 * params->seed) with filter bounds lambda = Gershgorin lower bound,
 * alpha = lo + 2 (k_b/N)(hi - lo), beta = Gershgorin upper bound.
 *
 * scsf_chain_create: allocates only a small host-side handle; `workspace`
 *   (device, >= scsf_solve_workspace_size(params, n) bytes, 256-byte aligned)
 *   must stay alive and untouched by the caller until scsf_chain_destroy.
 * scsf_chain_create_rows: the same for SCSF_OP_CSR operators of `rows` rows
 *   (workspace >= scsf_solve_workspace_size_rows(params, rows)); SCSF_FP64 only,
 *   SCSF_ERR_INVALID_ARG otherwise. A chain takes only the operator kind it was made
 *   for (stencil chains: stencils of side n; row chains: CSR of `rows` rows).
 * scsf_chain_seed: replaces the warm start by a caller block (device
 *   [N][k_b] FP64, row-major) and its Ritz values (host [k_b] FP64); both are
 *   copied. Used to resume a chain or to inject a proposed subspace.
 * scsf_chain_step: solves one problem whose grid side equals the chain's n (CSR: whose
 *   row count equals the chain's rows).
 *   evals  : [k] FP64 ascending eigenvalues
 *   resid  : [k] FP64 relative residuals (App. D.5)
 *   evecs  : [N][k] FP64 row-major (column j is eigenvector j, unit 2-norm, signed so that
 *            its largest-magnitude entry, lowest row on ties, is positive) or NULL
 *   stats  : host pointer or NULL
 *   On SCSF_ERR_NOT_CONVERGED the locked pairs come first, the other
 *   eigenvalue slots hold NaN, and the warm start is kept for the next step.
 *   An operator with a NaN or Inf coefficient (SCSF_OP_PLATE: also rho <= 0) is rejected
 *   with SCSF_ERR_INVALID_ARG before any iteration (its Gershgorin bounds are not finite). */
typedef struct scsf_chain scsf_chain;
scsf_status scsf_chain_create(scsf_ctx* ctx, const scsf_params* params, int n,
                              void* workspace, size_t workspace_bytes, scsf_chain** out);
scsf_status scsf_chain_create_rows(scsf_ctx* ctx, const scsf_params* params, int64_t rows,
                                   void* workspace, size_t workspace_bytes, scsf_chain** out);
scsf_status scsf_chain_seed(scsf_chain* chain, const double* block, const double* ritz_host);
scsf_status scsf_chain_step(scsf_chain* chain, const scsf_operator* op, double* evals,
                            double* resid, double* evecs, scsf_stats* stats);
/* The next scsf_chain_step starts as a chain head (Gaussian block, or the learned proposal
 * with params.use_proposal) instead of from the previous problem's block: for a step whose
 * sorted predecessor is far away (scsf_far_steps). */
scsf_status scsf_chain_restart(scsf_chain* chain);
/* Far steps of a sorted chain (host arrays): dist[n_ops] = the squared feature distances
 * from scsf_sort_dist (dist[0] = 0 for the head); far[0] = 1, and far[i] = 1 for i >= 1 when
 * dist[i] is above the `quantile` (0..1) of dist[1..n_ops-1] (linear interpolation between
 * order statistics), else 0. Those steps are restarted from the learned proposal. */
scsf_status scsf_far_steps(const double* dist, int64_t n_ops, double quantile, int32_t* far);
void scsf_chain_destroy(scsf_chain* chain);

/* Solve n_ops problems (same n; or all SCSF_OP_CSR with the same rows) in the given
 * order as one chain.
 * ops    : host array of n_ops operator descriptors (device pointers inside)
 * evals  : [n_ops][k], resid: [n_ops][k], evecs: [n_ops][N][k] or NULL,
 * stats  : host [n_ops] or NULL. Returns the first non-OK status, after
 *          finishing the remaining problems. */
scsf_status scsf_solve(scsf_ctx* ctx, const scsf_operator* ops, int64_t n_ops,
                       const scsf_params* params, void* workspace, size_t workspace_bytes,
                       double* evals, double* resid, double* evecs, scsf_stats* stats);

/* ---------------------------------------------------------------------------
 * Batched solve: many independent chains in flight on one GPU (App. D.6 splits
 * the dataset into chunks, each solved by its own SCSF instance).
 *
 * Each chain is solved exactly as scsf_solve would (same kernels, same results);
 * chains differ freely in grid side, k and parameters. Up to `concurrency`
 * chains run at once, each on its own stream driven by its own host thread, so
 * the latency-bound phases of one chain overlap with the others. The call
 * returns when every chain is done; chains[i].status holds each chain's status.
 * workspace: device, >= scsf_batch_workspace_size(chains, n_chains,
 * concurrency) bytes, 256-byte aligned; it is split into one slot per worker.
 * Inputs must be ready on the context's stream when the call is made. */
typedef struct {
  const scsf_operator* ops;  /* host array of n_ops descriptors in solve order (same n,
                                or all CSR with the same rows)                          */
  int64_t n_ops;
  scsf_params params;
  double* evals;             /* [n_ops][k]                                             */
  double* resid;             /* [n_ops][k]                                             */
  double* evecs;             /* [n_ops][N][k] or NULL                                  */
  scsf_stats* stats;         /* host [n_ops] or NULL                                   */
  int status;                /* out                                                    */
} scsf_batch_chain;

size_t scsf_batch_workspace_size(const scsf_batch_chain* chains, int n_chains, int concurrency);
scsf_status scsf_solve_batched(scsf_ctx* ctx, scsf_batch_chain* chains, int n_chains,
                               int concurrency, void* workspace, size_t workspace_bytes);

/* ---------------------------------------------------------------------------
 * Learned proposal for chain heads (Sec. 3.2 starts a chain from a random
 * block; this network proposes a better start). A Fourier neural operator maps
 * the coefficient field P (the sort's parameter matrix, s x s nodes, s a
 * multiple of 32, entries > 0) to log(lambda_1), log(lambda_kb) and a 32 x 32 x 64
 * coarse block whose span should approximate the lowest eigenvectors. The
 * filter and the FP64 residual test still decide every result.
 *
 * params: FP32 [scsf_proposal_param_count()] (master copy; matrices are used
 * in BF16, accumulation is FP32). workspace: scsf_proposal_workspace_size(batch).
 * fields: FP64 [batch][s][s]. bounds_out: FP32 [batch][2]; block_out: FP32
 * [batch][1024][64] (row = coarse node I*32 + J). Either output may be NULL.
 * train_step: forward + loss + backward (+ Adam when adam_m/adam_v non-NULL,
 * step >= 1 and lr > 0); targets_bounds FP32 [batch][2] (log-bounds),
 * targets_Q FP32 [batch][1024][64] orthonormal; loss_host (host, 3 doubles):
 * batch means of sub = 64 - tr((G + 1e-3 I)^-1 C^T C) (G = Y^T Y, C = Q^T Y: the
 * squared sines of the principal angles between the block and the targets),
 * orth = |G - I|_F^2 and bounds = |s - t|^2; the objective whose gradient is taken
 * is sub + 0.01 orth + bounds. grad_out FP32 [param_count] or NULL.
 * targets: pools fine eigenvectors (FP64 [batch][n*n][lde], first 64 columns)
 * over 4x4 (n/32 x n/32) blocks and orthonormalises them (Cholesky QR2, FP64).
 * prolong: bilinear interpolation of coarse blocks to the n x n grid (zero
 * Dirichlet boundary) into fine (FP64 [batch][n*n][ld_fine], columns 0..63). */
size_t scsf_proposal_param_count(void);
size_t scsf_proposal_workspace_size(int batch);
scsf_status scsf_proposal_init(scsf_ctx* ctx, float* params, uint64_t seed);
scsf_status scsf_proposal_forward(scsf_ctx* ctx, const float* params, const double* fields,
                                  int batch, int s, float* bounds_out, float* block_out,
                                  void* workspace, size_t workspace_bytes);
scsf_status scsf_proposal_train_step(scsf_ctx* ctx, float* params, float* adam_m, float* adam_v,
                                     int step, float lr, const double* fields, int batch, int s,
                                     const float* targets_bounds, const float* targets_Q,
                                     double* loss_host, float* grad_out, void* workspace,
                                     size_t workspace_bytes);
size_t scsf_proposal_target_scratch(void);
scsf_status scsf_proposal_targets(scsf_ctx* ctx, const double* evecs, int batch, int n, int lde,
                                  float* Q_out, void* scratch, size_t scratch_bytes);
scsf_status scsf_proposal_prolong(scsf_ctx* ctx, const float* block, int batch, int n,
                                  double* fine, int ld_fine);

/* ---------------------------------------------------------------------------
 * Building blocks exported for kernel-level parity tests. Same conventions.
 *
 * scsf_cheb_filter: Y = C_m(Abar) X / C_m(t_lambda) by the scaled recurrence of
 *   Alg. 1 (Abar = (A - cI)/e, t_lambda = (lambda - c)/e) for the operator `op`.
 *   X, Y: [N][ncols] FP64 with leading dimensions ldx, ldy (>= ncols);
 *   scratch: device, >= 8 (2 N ncols + 3 N + 4096) + 8192 bytes, plus 4 (14 N + 1) + 104 N
 *   for SCSF_OP_PLATE. X and Y must not overlap.
 * scsf_assemble_bounds: Gershgorin bounds of A (host out[2] = {lo, hi}; NaN or Inf when a
 *   coefficient is not finite); scratch as for scsf_cheb_filter with ncols = 0.
 * scsf_cholqr2: Q = X R^{-1} with X = Q R (Alg. 3, orthonormalisation) by Cholesky QR2:
 *   G = X^T X, R1 from the Cholesky factor of D^-1 G D^-1 (D = diag(G)^(1/2)) taken in
 *   FP32, Q1 = X R1^{-1}; then the same in FP64 on Q1. Shifted restarts on a failed pivot;
 *   shifts_host[2] (host, or NULL) receives the restarts per pass. X [rows][ncols] FP64
 *   (ldx), Q [rows][ncols] (ldq), 1 <= ncols <= min(rows, 512); X and Q must not overlap;
 *   scratch >= scsf_cholqr2_scratch(rows, ncols). SCSF_ERR_BREAKDOWN if a pass still fails.
 * scsf_small_eigh: all eigenpairs of a symmetric k x k FP64 matrix S
 *   (row-major, k <= scsf_max_block_width()): evals [k] ascending, Z [k][k]
 *   with eigenvector j in column j. scratch >= scsf_small_eigh_scratch(k). */
scsf_status scsf_cheb_filter(scsf_ctx* ctx, const scsf_operator* op, const double* X, int ldx,
                             int ncols, int degree, double lambda, double c, double e,
                             double* Y, int ldy, void* scratch, size_t scratch_bytes);
scsf_status scsf_assemble_bounds(scsf_ctx* ctx, const scsf_operator* op, double* bounds_host,
                                 void* scratch, size_t scratch_bytes);
size_t scsf_cholqr2_scratch(int rows, int ncols);
scsf_status scsf_cholqr2(scsf_ctx* ctx, const double* X, int ldx, int rows, int ncols, double* Q,
                         int ldq, int* shifts_host, void* scratch, size_t scratch_bytes);
/* scsf_cheb_filter on FP32 blocks (the mixed form's filter): X, Y [N][ncols]
 * FP32 with ncols and ldx multiples of 4 and ldy == ncols; the operator is assembled in FP64
 * and rounded to FP32; scratch >= 2 N ncols 4 + 6 N 8 + 64 KiB bytes. */
scsf_status scsf_cheb_filter_f32(scsf_ctx* ctx, const scsf_operator* op, const float* X, int ldx,
                                 int ncols, int degree, double lambda, double c, double e,
                                 float* Y, int ldy, void* scratch, size_t scratch_bytes);
/* Defect-corrected filter (the mixed form's FP64-phase filter): the same Y as
 * scsf_cheb_filter, computed as Y = X diag(y_m(theta)) + Z_m, where y_i(theta_j) runs
 * the filter's scalar recurrence at theta_j and Z_i the block recurrence driven by
 * s1 R diag(y_i), R = A X - X diag(theta) formed in FP64 and stored in FP32, Z in FP32.
 * Any theta gives the same Y up to rounding; Ritz values (small R) make the FP32
 * rounding negligible. The paper has no counterpart (its filter runs in one precision).
 * X, Y: FP64 [N][ncols] (ldx, ldy >= ncols), theta: device FP64 [ncols],
 * 1 <= ncols <= scsf_max_block_width(); scratch >= scsf_cheb_filter_dc_scratch(). */
size_t scsf_cheb_filter_dc_scratch(int n, int ncols, int degree);
scsf_status scsf_cheb_filter_dc(scsf_ctx* ctx, const scsf_operator* op, const double* X, int ldx,
                                const double* theta, int ncols, int degree, double lambda,
                                double c, double e, double* Y, int ldy, void* scratch,
                                size_t scratch_bytes);
/* scsf_cheb_filter_dc with a degree per group of 4 columns: columns [4 g, 4 g + 4) are
 * filtered to degree group_degrees[g] (host array of ceil(ncols / 4) ints, each in
 * [1, degree]), Y_j = X_j y_{m_g}(theta_j) + Z_{m_g, j}, exactly the degree-m_g filter of
 * those columns. Needs the cluster-resident filter (the operator's bands and the degree's
 * step table in one cluster's shared memory): SCSF_ERR_INVALID_ARG otherwise. Same scratch as
 * scsf_cheb_filter_dc. */
scsf_status scsf_cheb_filter_dc_grouped(scsf_ctx* ctx, const scsf_operator* op, const double* X,
                                        int ldx, const double* theta, int ncols, int degree,
                                        const int* group_degrees, double lambda, double c,
                                        double e, double* Y, int ldy, void* scratch,
                                        size_t scratch_bytes);
/* Rotation of a block by a small matrix, Y = X M (Alg. 3, rotation X = Q Z; also the
 * triangular solve X R^{-1} of Cholesky QR): X FP64 [rows][k] (ldx), M FP64 [k][n] (ldm),
 * Y FP64 [rows][n] (ldy), all device, Y must not overlap X or M; 1 <= k, n <= 512. */
scsf_status scsf_block_rotate(scsf_ctx* ctx, const double* X, int ldx, int rows, int k,
                              const double* M, int ldm, int n, double* Y, int ldy);
/* Block products with a selectable method (scsf_product_method; see scsf_params.products).
 * scsf_block_gram: C = A^T B (Alg. 3: the Gram matrix X^T X of Cholesky QR, the
 *   Rayleigh-Ritz matrix Q^T (A Q), the coefficients of deflation against locked columns).
 *   A [rows][m] (lda), B [rows][n] (ldb), C [m][n] (ldc), FP64, device; symmetric != 0
 *   promises that C is symmetric (m == n; A == B, or B = S A for a symmetric S): only
 *   the upper half is formed and mirrored.
 * scsf_block_rotate_ex: Y = alpha X M + beta Y (Alg. 3: the rotation X = Q Z, the
 *   triangular solve X R^{-1} of Cholesky QR, the deflation update Y - V C).
 *   X [rows][k] (ldx), M [k][n] (ldm), Y [rows][n] (ldy), FP64, device; Y must not
 *   overlap X or M.
 * Both: 1 <= m, n, k <= 512, 1 <= rows < 2^31; slices: digits per operand of the tensor
 * method (4, 7 or 8; ignored by SCSF_PRODUCT_FP64); scratch: device, 256-byte aligned,
 * >= scsf_block_product_scratch(rows, max width, slices) bytes. The call synchronises the
 * context's stream and returns SCSF_ERR_TIMEOUT if a bounded wait inside the tensor-core
 * kernel gave up (Y or C undefined then). */
size_t scsf_block_product_scratch(int64_t rows, int kmax, int slices);
scsf_status scsf_block_gram(scsf_ctx* ctx, const double* A, int lda, const double* B, int ldb,
                            int rows, int m, int n, int symmetric, int method, int slices,
                            double* C, int ldc, void* scratch, size_t scratch_bytes);
scsf_status scsf_block_rotate_ex(scsf_ctx* ctx, const double* X, int ldx, int rows, int k,
                                 const double* M, int ldm, int n, double alpha, double beta,
                                 int method, int slices, double* Y, int ldy, void* scratch,
                                 size_t scratch_bytes);
/* Profiling: average device time (ms, host out) of the tensor-core kernel of the symmetric Gram
 * product X^T X with 8 digits (X [rows][m], ldx), the digit planes prepared once and `reps`
 * launches of the kernel alone bracketed by CUDA events on the context's stream. Same
 * scratch as scsf_block_product_scratch(rows, m, 8); the Gram matrix itself is not returned. */
scsf_status scsf_block_gram_kernel_time(scsf_ctx* ctx, const double* X, int ldx, int rows, int m,
                                        int reps, void* scratch, size_t scratch_bytes,
                                        float* ms_host);
size_t scsf_small_eigh_scratch(int k);
scsf_status scsf_small_eigh(scsf_ctx* ctx, const double* S, int k, double* evals, double* Z,
                            void* scratch, size_t scratch_bytes);

#ifdef __cplusplus
}
#endif
#endif /* SCSF_H */
