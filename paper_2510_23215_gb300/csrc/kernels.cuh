// Host-side launchers of the SCSF kernels (all enqueue on `st`, return the
// launch error). Layouts: row-major blocks, column index fastest.
#pragma once

#include <string>

#include "../../include/scsf.h"
#include "common.cuh"

namespace scsf {

// Context accessors for entry points defined outside api.cu.
int ctx_device(const scsf_ctx* ctx);
cudaStream_t ctx_stream(const scsf_ctx* ctx);
bool ctx_timing(const scsf_ctx* ctx);
// Raises (never lowers) a kernel's dynamic shared-memory limit on the current
// device. The attribute is per function, so concurrent chains with different
// block widths must not shrink it under each other's launches.
cudaError_t ensure_dynamic_smem(const void* fn, size_t bytes);

// Stores `msg` as the context's last error and returns `status`.
scsf_status set_error(scsf_ctx* ctx, scsf_status status, const std::string& msg);
// Range and pointer checks of the sort entry points (SCSF_OK or SCSF_ERR_INVALID_ARG).
scsf_status validate_sort_args(scsf_ctx* ctx, const double* fields, int64_t n_ops, int p, int p0,
                               int start, const int32_t* perm_out);
// Looks up (and so reserves) the allocation-free sort's static scratch on `device` (current).
cudaError_t noalloc_prepare(int device);

// ---- operator assembly (stencil.cu) -------------------------------------
// Builds d/we/wn for -div(a grad u) (ax, ay) or -Lap u + V u (v), and writes
// the Gershgorin bounds {lo, hi} to bounds[0..1] (device). `partials` holds
// 2 * assemble_blocks(n) doubles.
int assemble_blocks(int n);
cudaError_t launch_assemble(int kind, int n, const double* ax, const double* ay, const double* v,
                            double* d, double* we, double* wn, double* partials, double* bounds,
                            cudaStream_t st);

// One scaled three-term step on an N x ncols block (Alg. 1 recurrence):
//   out = s1 * (A cur) + s2 * cur + s3 * prev       (prev may be null when s3 == 0)
cudaError_t launch_cheb_step_f64(const Stencil& A, const double* cur, int ldc, const double* prev,
                                 int ldp, double* out, int ldo, int ncols, double s1, double s2,
                                 double s3, cudaStream_t st);

// Column sums of r_j = ||(A X)_j - theta_j X_j||^2 and ||(A X)_j||^2 without
// storing A X. partials: [resid_blocks(n)][2][ncols]; out2: [2][ncols]. With R32
// non-null the residual block A X - X diag(theta) is also stored there in FP32 (ld ldr).
int resid_blocks(int n);
int resid_blocks_rows(long long N);
int assemble_blocks_rows(long long N);
// The thin-plate operator's standard form as a 13-slot-per-row CSR matrix (rp [n^2 + 1],
// ci / val [13 n^2]); D and rho at the n x n nodes.
cudaError_t launch_plate_csr(int n, const double* D, const double* rho, int* rp, int* ci,
                             double* val, cudaStream_t st);
// V[r][c] /= sqrt(w[r]) for r < rows, c < ncols.
cudaError_t launch_scale_rows_rsqrt(int rows, int ncols, double* V, int ldv, const double* w,
                                    cudaStream_t st);
// Gershgorin bounds {lo, hi} of a symmetric CSR matrix (partials: assemble_blocks_rows(rows) x 2).
cudaError_t launch_csr_bounds(int rows, const int* rp, const int* ci, const double* val,
                              double* partials, double* bounds, cudaStream_t st);
cudaError_t launch_residual_norms(const Stencil& A, const double* X, int ldx, int ncols,
                                  const double* theta, double* partials, double* out2,
                                  cudaStream_t st, float* R32 = nullptr, int ldr = 0);

// ---- FP64 block BLAS (blas64.cu) ----------------------------------------
// C[m x n] = A^T B over `rows` rows, A: rows x m (lda), B: rows x n (ldb).
// symmetric: C is known to be symmetric (A == B, or A^T B with B = S A for a symmetric S):
// only the upper tiles are computed, then mirrored.
size_t gemm_tn_partials(int rows, int m, int n, bool symmetric);
cudaError_t launch_gemm_tn(int rows, int m, int n, const double* A, int lda, const double* B,
                           int ldb, double* C, int ldc, bool symmetric, double* partials,
                           cudaStream_t st);
// C[rows x n] = alpha * A[rows x k] M[k x n] + beta * C; upper: M upper triangular.
// C may alias nothing but itself (in-place update is safe).
cudaError_t launch_gemm_nn(int rows, int k, int n, double alpha, const double* A, int lda,
                           const double* M, int ldm, double beta, double* C, int ldc, bool upper,
                           cudaStream_t st);
// Cholesky QR factor (chol.cu): G = L L^T (FP32 or FP64, shifted restarts on
// breakdown) and Rinv = (L^T)^{-1} (upper, ld k, one warp per column).
// L: k x k scratch (the FP32 path up to kSmallBlockWidth leaves it untouched).
// status[0]: shifted restarts used, 1000 = failed. Up to
// kSmallBlockWidth the factor runs in one CTA's shared memory; wider matrices take a
// blocked factorisation in wide_scratch (chol_wide_scratch_bytes(k)) and synchronise
// the stream once per attempt.
size_t chol_wide_scratch_bytes(int k);
cudaError_t launch_chol_rinv(int k, const double* G, int ldg, bool fp32, double* L, double* Rinv,
                             int* status, cudaStream_t st, void* wide_scratch = nullptr);
// out[i*ld_out + j] = in[i*ld_in + j], i < rows, j < cols.
cudaError_t launch_copy2d(int rows, int cols, const double* in, int ld_in, double* out, int ld_out,
                          cudaStream_t st);
// Gathers columns: out[r][j] = in[r][cols[j]] (cols: device int32 [ncols]).
cudaError_t launch_gather_cols(int rows, int ncols, const double* in, int ld_in, const int* cols,
                               double* out, int ld_out, cudaStream_t st);
// Flip each column of V [rows][ncols] so that its largest-magnitude entry (lowest row on
// ties) is positive.
cudaError_t launch_normalize_signs(int rows, int ncols, double* V, int ldv, cudaStream_t st);

// ---- reduced eigensolve (eig.cu) ----------------------------------------
// All eigenpairs of the symmetric k x k S (ascending, FP64 accuracy): probe of the diagonal
// trailing block, FP32 tridiagonal start (Householder, multisection, inverse iteration),
// Ogita-Aishima FP64 refinement, cluster-local FP64 Jacobi, sort.
size_t small_eigh_scratch_bytes(int k);
cudaError_t launch_small_eigh(int k, const double* S, int lds, double* evals, double* Z, int ldz,
                              void* scratch, cudaStream_t st);

// The FP32 phase's variant: the same start with one refinement step and no round-robin
// fallback; eigenvector accuracy ~1e-7 relative, enough while residuals are far above the
// FP64 target.
cudaError_t launch_small_eigh_f32(int k, const double* S, int lds, double* evals, double* Z,
                                  int ldz, void* scratch, cudaStream_t st);

// ---- FP32 kernels of the mixed-precision path (mixed.cu) ----------------
// Stencil kernels need ncols % 4 == 0 and leading dimensions % 4 == 0.
cudaError_t launch_to_f32(const double* in, float* out, long long count, cudaStream_t st);
cudaError_t launch_block_f32_to_f64(int rows, int cols, const float* in, int ld_in, double* out,
                                    int ld_out, cudaStream_t st);
cudaError_t launch_block_f64_to_f32(int rows, int cols, const double* in, int ld_in, float* out,
                                    int ld_out, cudaStream_t st);
cudaError_t launch_cheb_step_f32(const Stencil32& A, const float* cur, int ldc, const float* prev,
                                 int ldp, float* out, int ldo, int ncols, float s1, float s2,
                                 float s3, cudaStream_t st, int threads = 256);
// The whole m-step FP32 filter in one launch, each 4-column group held in the shared memory
// of a thread-block cluster (coef: device [m][3] step scalars; Y_m written to out).
// Returns cudaErrorNotSupported when the grid is too large for the cluster's shared memory
// or the widths are not multiples of 4 (the caller then uses per-step launches).
cudaError_t launch_cheb_filter_f32_resident(const Stencil32& A, const float* Y0, int ld0, float* out,
                                            int ldo, int ncols, int m, const float* coef,
                                            cudaStream_t st);
// The whole defect-corrected remainder recurrence (Z_m, FP32, into out with ld ldo) in one
// launch, resident in cluster shared memory like the FP32 filter. coef: device [m][3] step
// scalars; ytab: device [m][ncols]. cudaErrorNotSupported: use the per-step kernels.
// gdeg (device, optional): per 4-column group its own degree (<= m): the group's Z stops
// after that many steps (per-column degrees, the column split of Alg. 1).
cudaError_t launch_dc_filter_resident(const Stencil32& A, const float* R, int ldr, int ncols,
                                      const float* ytab, const float* coef, int m, float* out,
                                      int ldo, cudaStream_t st, const int* gdeg = nullptr);
// The step with {s1, s2, s3} read from device memory at coef (for captured graphs; the
// caller counts the launch). prev is read whenever non-null.
cudaError_t launch_cheb_step_f32_tab(const Stencil32& A, const float* cur, int ldc,
                                     const float* prev, int ldp, float* out, int ldo, int ncols,
                                     const float* coef, int threads, cudaStream_t st);
cudaError_t launch_residual_norms_f32(const Stencil32& A, const float* X, int ldx, int ncols,
                                      const double* theta, double* partials, double* out2,
                                      cudaStream_t st);
// Defect-corrected filter (any ncols and leading dimensions): with R = A X - X diag(theta),
// the filtered block is Y_m = X diag(y_m(theta)) + Z_m, where y_i are the scalar
// recurrences of the filter at the Ritz values and Z_i obeys the same recurrence with
// the extra term s1 R diag(y_i) (Z_0 = 0). Z is small when R is, so FP32 suffices.
//   ytab: per column y_0 .. y_{degree-1} (FP32, [degree][ncols]), computed in chunks of
//   kDcChunk steps whose coefficients travel by value; state [2][ncols] (FP64) carries
//   (y_{i-1}, y_i) between chunks and ends with y_degree in state[1].
constexpr int kDcChunk = 128;
struct DcSteps {
  int i0, count;
  double s1[kDcChunk], s2[kDcChunk], s3[kDcChunk];
};
// gdeg (optional, per 4-column group its degree d): ysel[c] = y_d(theta_c) in FP64.
cudaError_t launch_dc_ytab(const double* theta, int ncols, const DcSteps& P, float* ytab,
                           double* state, cudaStream_t st, const int* gdeg = nullptr,
                           double* ysel = nullptr);
// out = s1 (A cur) + s2 cur + s3 prev + s1 R diag(ycol); cur == nullptr means Z_0 = 0.
cudaError_t launch_cheb_step_dc(const Stencil32& A, const float* cur, const float* prev, int ld,
                                const float* R, int ldr, const float* ycol, float* out,
                                int ncols, float s1, float s2, float s3, cudaStream_t st);
// Y = X diag(ym) + Z in FP64.
cudaError_t launch_dc_combine(int rows, int ncols, const double* X, int ldx, const double* ym,
                              const float* Z, int ldz, double* Y, int ldy, cudaStream_t st);
size_t gemm_tn_f32_partials(int rows, int m, int n, bool symmetric);
cudaError_t launch_gemm_tn_f32(int rows, int m, int n, const float* A, int lda, const float* B,
                               int ldb, double* C, int ldc, bool symmetric, float* partials,
                               cudaStream_t st);
cudaError_t launch_gemm_nn_f32(int rows, int k, int n, float alpha, const float* A, int lda,
                               const double* M, int ldm, float beta, float* C, int ldc, bool upper,
                               cudaStream_t st);

// ---- tensor-core split products (ozaki.cu) ----------------------------------
// FP64-accurate A^T B and A M on tcgen05 tensor cores: operands cut into `slices` base-128
// digit planes (BF16), exact FP32 accumulation per 64-row chunk, integer level sums, one
// rounding to FP64 at the end. slices 8 for FP64-class products (7: ~10x the error), kOzSlicesF32 for
// the FP32 phase. scratch: device, >= oz_scratch_bytes(rows, kmax, slices) for products
// with rows rows and m, n, k <= kmax; 256-byte aligned. err: device int set to 1 when a
// bounded wait inside the kernel gave up (results then undefined).
constexpr int kOzSlicesF64 = 8;
constexpr int kOzSlicesF32 = 4;
size_t oz_scratch_bytes(int rows, int kmax, int slices);
// C[m x n] = A^T B over rows rows (symmetric: A == B, only the upper tiles, mirrored)
cudaError_t launch_gemm_tn_oz(int rows, int m, int n, const double* A, int lda, const double* B,
                              int ldb, double* C, int ldc, bool symmetric, int slices,
                              void* scratch, size_t scratch_bytes, int* err, cudaStream_t st);
// Times the tensor-core kernel of the symmetric Gram product A^T A (8 digits) alone: the digit
// planes are prepared once, then `reps` launches are bracketed by CUDA events on `st`.
cudaError_t time_gemm_tn_oz(int rows, int m, const double* A, int lda, int slices, void* scratch,
                            size_t scratch_bytes, int* err, int reps, cudaStream_t st,
                            float* ms_out);
cudaError_t launch_gemm_tn_oz_f32(int rows, int m, int n, const float* A, int lda, const float* B,
                                  int ldb, double* C, int ldc, bool symmetric, void* scratch,
                                  size_t scratch_bytes, int* err, cudaStream_t st);
// C[rows x n] = alpha A[rows x k] M[k x n] + beta C (C must not overlap A or M)
cudaError_t launch_gemm_nn_oz(int rows, int k, int n, double alpha, const double* A, int lda,
                              const double* M, int ldm, double beta, double* C, int ldc,
                              int slices, void* scratch, size_t scratch_bytes, int* err,
                              cudaStream_t st);
cudaError_t launch_gemm_nn_oz_f32(int rows, int k, int n, float alpha, const float* A, int lda,
                                  const double* M, int ldm, float beta, float* C, int ldc,
                                  void* scratch, size_t scratch_bytes, int* err, cudaStream_t st);

// ---- spectrum upper bound by Lanczos (bound.cu) ---------------------------
// K (<= 32) FP32 Lanczos steps in one CTA; out[0] = min(theta_max(T_K) + |beta_K| with a small
// relative margin, cap). vecs: lanczos_scratch_bytes(N) of device scratch.
size_t lanczos_scratch_bytes(long long N);
cudaError_t launch_lanczos_bound(const Stencil& A, int steps, unsigned long long seed, float* vecs,
                                 double cap, double* out, cudaStream_t st);

// ---- random head block (rng.cu) -----------------------------------------
cudaError_t launch_philox_normal(double* out, int rows, int cols, int ld, uint64_t seed,
                                 cudaStream_t st);

// ---- sort (sort.cu) ------------------------------------------------------
size_t sort_workspace_bytes(int64_t n_ops, int p0);
// dist (optional, n_ops): squared feature distance from each sorted problem to its
// predecessor (0 for the first).
cudaError_t launch_sort(const double* fields, int64_t n_ops, int p, int p0, int start,
                        void* workspace, int32_t* perm, cudaStream_t st, double* dist = nullptr);

}  // namespace scsf
