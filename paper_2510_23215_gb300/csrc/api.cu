// C ABI of the SCSF library: contexts, the sort entry point, and the chain
// loop that runs Chebyshev filtered subspace iteration (Alg. 3) on each
// problem of a sorted sequence, warm-started from the previous problem.
//
// The loop is host code issuing stream-ordered kernels; the only device ->
// host traffic per outer iteration is the Ritz values and residual norms of
// the active block (2-3 k_b doubles), which decide locking and termination.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/scsf.h"
#include "kernels.cuh"

using namespace scsf;

struct scsf_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  std::string err;
  double* pinned = nullptr;  // host staging
  size_t pinned_count = 0;
  bool timing = false;
  cudaEvent_t ev[7] = {};
};

namespace scsf {
static std::atomic<long long> g_launches{0};
static thread_local long long t_launches = 0;  // this thread's launches (graph captures)
void note_launch() {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  ++t_launches;
}
}  // namespace scsf

namespace {

// FP32-phase filters of up to this degree replay a captured graph (scalars in a device table)
constexpr int kMaxGraphSteps = 1024;
constexpr size_t kPinnedCoefOffset = 4 * kMaxBlockWidth + 64;  // doubles before the float table
constexpr size_t kPinnedGdegOffset = kPinnedCoefOffset + (3 * kMaxGraphSteps + 1) / 2;
constexpr size_t kPinnedDoubles = kPinnedGdegOffset + kMaxBlockWidth / 8 + 1;  // + group degrees

scsf_status fail(scsf_ctx* ctx, scsf_status s, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return s;
}

#define SCSF_CUDA(ctx, expr)                                                              \
  do {                                                                                    \
    cudaError_t _e = (expr);                                                              \
    if (_e != cudaSuccess)                                                                \
      return fail((ctx), SCSF_ERR_CUDA,                                                   \
                  std::string(#expr) + ": " + cudaGetErrorString(_e));                    \
  } while (0)

}  // namespace

namespace scsf {
cudaError_t ensure_dynamic_smem(const void* fn, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, size_t> granted;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  size_t& cur = granted[{fn, dev}];
  if (bytes <= cur) return cudaSuccess;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) cur = bytes;
  return e;
}
int ctx_device(const scsf_ctx* ctx) { return ctx->device; }
cudaStream_t ctx_stream(const scsf_ctx* ctx) { return ctx->stream; }
bool ctx_timing(const scsf_ctx* ctx) { return ctx->timing; }
scsf_status set_error(scsf_ctx* ctx, scsf_status status, const std::string& msg) {
  return fail(ctx, status, msg);
}
}  // namespace scsf

namespace {

int block_width(const scsf_params* p) {
  const int nex = (p->nex >= 0) ? p->nex : (int)std::ceil(0.2 * p->k);
  return p->k + nex;
}

constexpr int64_t kMaxCsrRows = 0x7fffffff - 1;

bool op_ok(const scsf_operator* op) {
  if (!op) return false;
  if (op->kind == SCSF_OP_CSR)
    return op->rows >= 1 && op->rows <= kMaxCsrRows && op->row_ptr && op->col && op->val;
  if (op->n < 2 || op->n > 46340) return false;  // N = n^2 is indexed in int32
  if (op->kind == SCSF_OP_PLATE)  // 13 CSR slots a row, indexed in int32
    return op->plate_d && op->plate_rho && 13LL * op->n * op->n < 0x7fffffffLL;
  if (op->kind == SCSF_OP_DIV_A_GRAD) return op->ax && op->ay;
  if (op->kind == SCSF_OP_LAP_PLUS_V) return op->v != nullptr;
  return false;
}

// Rows of the operator's matrix (N = n^2 for the stencils).
size_t op_rows(const scsf_operator& op) {
  return op.kind == SCSF_OP_CSR ? (size_t)op.rows : (size_t)op.n * op.n;
}

// The CSR arrays of a SCSF_OP_CSR operator attached to a stencil descriptor.
Stencil with_csr(Stencil A, const scsf_operator& op) {
  A.rp = op.row_ptr;
  A.ci = op.col;
  A.val = op.val;
  A.rows = (int)op.rows;
  return A;
}

// Device buffers of one chain, carved from the caller's workspace.
struct ChainBufs {
  double *V, *B0, *B1, *B2;        // N x kb blocks (row-major, ld = kb)
  double *d, *we, *wn;             // stencil coefficients
  double *asm_partials, *bounds;   // Gershgorin reduction (+ the Lanczos estimate in bounds[2])
  float* lanczos;                  // Lanczos vectors (3 N)
  double *G, *Rinv, *H, *Z, *C;    // kb x kb small matrices
  double *theta, *res2;            // kb, 2*kb
  double *gemm_partials, *res_partials;
  void* eigh_scratch;
  void* chol_wide;  // k_b > kSmallBlockWidth: blocked Cholesky working copy
  int* status;
  int* cols;
  // FP32 phase of the mixed form (null otherwise); in the FP64 phase V32 holds the
  // FP32 residual block of the defect-corrected filter, B32 its remainder blocks
  float *V32, *B32[3], *d32, *we32, *wn32, *partials32;
  float* coef32;  // [kMaxGraphSteps][3] scalars of the captured FP32 filter
  float* ytab;  // [degree][kb] scalar filter values at the Ritz values
  double* ym;   // [3][kb] recurrence state (y_{m-1}, y_m), then y at each column's own degree
  int* gdeg;    // per group of 4 active columns its degree (column_degree)
  // FP64 stencil chains: the thin-plate operator assembled as CSR (13 slots a row)
  int *prp, *pci;
  double* pval;
  // tensor-core block products: digit planes, exponents and exact split partials
  void* oz;
  size_t oz_bytes;
  // learned proposal at chain heads: network workspace, predicted log-bounds, coarse block
  void* prop_ws;
  size_t prop_ws_bytes;
  float *prop_bounds, *prop_block;
};

template <typename Cv>
void carve_chain(Cv& c, size_t N, int kb, bool mixed, int degree, bool plate, bool tensor,
                 bool proposal, ChainBufs& b) {
  const size_t blk = N * kb;
  const size_t kk = (size_t)kb * kb;
  const int T = (kb + kGemmTile - 1) / kGemmTile;
  b.V = c.template take<double>(blk);
  b.B0 = c.template take<double>(blk);
  b.B1 = c.template take<double>(blk);
  b.B2 = c.template take<double>(blk);
  b.d = c.template take<double>(N);
  b.we = c.template take<double>(N);
  b.wn = c.template take<double>(N);
  b.asm_partials = c.template take<double>(2 * (size_t)assemble_blocks_rows((long long)N));
  b.bounds = c.template take<double>(4);  // {lo, hi (Gershgorin), Lanczos estimate}
  b.lanczos = c.template take<float>(lanczos_scratch_bytes((long long)N) / sizeof(float));
  b.G = c.template take<double>(kk);
  b.Rinv = c.template take<double>(kk);
  b.H = c.template take<double>(kk);
  b.Z = c.template take<double>(kk);
  b.C = c.template take<double>(kk);
  b.theta = c.template take<double>(kb);
  b.res2 = c.template take<double>(2 * (size_t)kb);
  b.gemm_partials = c.template take<double>((size_t)(kSplitTarget + T * T) * kGemmTile * kGemmTile);
  b.res_partials = c.template take<double>((size_t)resid_blocks_rows((long long)N) * 2 * kb);
  b.eigh_scratch = c.template take<char>(small_eigh_scratch_bytes(kb));
  b.chol_wide = (kb > kSmallBlockWidth) ? c.template take<char>(chol_wide_scratch_bytes(kb)) : nullptr;
  b.status = c.template take<int>(4);
  b.cols = c.template take<int>(kb);
  b.oz = nullptr;
  b.oz_bytes = 0;
  if (tensor) {
    b.oz_bytes = oz_scratch_bytes((int)N, kb, kOzSlicesF64);
    b.oz = c.template take<char>(b.oz_bytes);
  }
  b.prop_ws = nullptr;
  b.prop_ws_bytes = 0;
  b.prop_bounds = b.prop_block = nullptr;
  if (proposal) {
    b.prop_ws_bytes = scsf_proposal_workspace_size(1);
    b.prop_ws = c.template take<char>(b.prop_ws_bytes);
    b.prop_bounds = c.template take<float>(2);
    b.prop_block = c.template take<float>(1024 * 64);
  }
  b.prp = b.pci = nullptr;
  b.pval = nullptr;
  if (plate) {
    b.prp = c.template take<int>(N + 1);
    b.pci = c.template take<int>(13 * N);
    b.pval = c.template take<double>(13 * N);
  }
  b.V32 = b.d32 = b.we32 = b.wn32 = b.partials32 = nullptr;
  b.B32[0] = b.B32[1] = b.B32[2] = nullptr;
  b.ytab = nullptr;
  b.ym = nullptr;
  b.gdeg = nullptr;
  b.coef32 = nullptr;
  if (mixed) {
    b.coef32 = c.template take<float>(3 * (size_t)kMaxGraphSteps);
    b.ytab = c.template take<float>((size_t)std::max(degree, 1) * kb);
    b.ym = c.template take<double>(3 * (size_t)kb);
    b.gdeg = c.template take<int>((size_t)(kb + 3) / 4);
    b.V32 = c.template take<float>(blk);
    for (auto& p : b.B32) p = c.template take<float>(blk);
    b.d32 = c.template take<float>(N);
    b.we32 = c.template take<float>(N);
    b.wn32 = c.template take<float>(N);
    b.partials32 = c.template take<float>(std::max(gemm_tn_f32_partials((int)N, kb, kb, true),
                                                   gemm_tn_f32_partials((int)N, kb, kb, false)));
  }
}

struct SizeCarve {
  size_t used = 0;
  template <typename T>
  T* take(size_t count) {
    used += align256(count * sizeof(T));
    return nullptr;
  }
};

Stencil stencil_of(const ChainBufs& b, int n) { return Stencil{b.d, b.we, b.wn, n}; }

// Alg. 1 on an N x ncols block: Y_m = C_m(Abar) Y_0 / C_m(t_lambda).
// Y_i is written to bufs[(i - 1) % 3]; returns the buffer that holds Y_m.
cudaError_t run_filter(const Stencil& A, const double* Y0, int ld0, int ncols, int degree,
                       double lam, double c, double e, double* const bufs[3], const int lds[3],
                       int* which, cudaStream_t st) {
  const double sigma1 = e / (lam - c);
  // Y_1 = sigma_1 Abar Y_0 = (sigma_1/e) A Y_0 - (sigma_1 c/e) Y_0
  cudaError_t err = launch_cheb_step_f64(A, Y0, ld0, nullptr, 0, bufs[0], lds[0], ncols,
                                         sigma1 / e, -sigma1 * c / e, 0.0, st);
  if (err != cudaSuccess) return err;
  double sigma = sigma1;
  const double* prev = Y0;
  int ldp = ld0;
  int cur = 0;
  for (int i = 1; i < degree; ++i) {
    const double sigma_next = 1.0 / (2.0 / sigma1 - sigma);
    const int nxt = i % 3;
    // Y_{i+1} = 2 sigma_{i+1} Abar Y_i - sigma_{i+1} sigma_i Y_{i-1}
    err = launch_cheb_step_f64(A, bufs[cur], lds[cur], prev, ldp, bufs[nxt], lds[nxt], ncols,
                               2.0 * sigma_next / e, -2.0 * sigma_next * c / e,
                               -sigma_next * sigma, st);
    if (err != cudaSuccess) return err;
    prev = bufs[cur];
    ldp = lds[cur];
    cur = nxt;
    sigma = sigma_next;
  }
  *which = cur;
  return cudaSuccess;
}

// The same recurrence on FP32 blocks (scalars computed in FP64, applied in FP32).
// The m step scalars {s1, s2, s3} of the scaled recurrence (Alg. 1), as FP32, into the host
// staging array h and then into the device table dev.
cudaError_t upload_filter_coefs(int m, double lam, double c, double e, float* h, float* dev,
                                cudaStream_t st) {
  const double sigma1 = e / (lam - c);
  double sigma = sigma1;
  h[0] = (float)(sigma1 / e);
  h[1] = (float)(-sigma1 * c / e);
  h[2] = 0.f;
  for (int i = 1; i < m; ++i) {
    const double sigma_next = 1.0 / (2.0 / sigma1 - sigma);
    h[3 * i] = (float)(2.0 * sigma_next / e);
    h[3 * i + 1] = (float)(-2.0 * sigma_next * c / e);
    h[3 * i + 2] = (float)(-sigma_next * sigma);
    sigma = sigma_next;
  }
  return cudaMemcpyAsync(dev, h, 3 * (size_t)m * sizeof(float), cudaMemcpyHostToDevice, st);
}

cudaError_t run_filter_f32(const Stencil32& A, const float* Y0, int ld0, int ncols, int degree,
                           double lam, double c, double e, float* const bufs[3], int ld,
                           int* which, cudaStream_t st) {
  const double sigma1 = e / (lam - c);
  cudaError_t err = launch_cheb_step_f32(A, Y0, ld0, nullptr, 0, bufs[0], ld, ncols,
                                         (float)(sigma1 / e), (float)(-sigma1 * c / e), 0.f, st);
  if (err != cudaSuccess) return err;
  double sigma = sigma1;
  const float* prev = Y0;
  int ldp = ld0;
  int cur = 0;
  for (int i = 1; i < degree; ++i) {
    const double sigma_next = 1.0 / (2.0 / sigma1 - sigma);
    const int nxt = i % 3;
    err = launch_cheb_step_f32(A, bufs[cur], ld, prev, ldp, bufs[nxt], ld, ncols,
                               (float)(2.0 * sigma_next / e), (float)(-2.0 * sigma_next * c / e),
                               (float)(-sigma_next * sigma), st);
    if (err != cudaSuccess) return err;
    prev = bufs[cur];
    ldp = ld;
    cur = nxt;
    sigma = sigma_next;
  }
  *which = cur;
  return cudaSuccess;
}

template <typename Cv>
void carve_filter_dc(Cv& cv, int n, int ncols, int degree, float** R, float* z[3], double** d,
                     double** we, double** wn, float** d32, float** we32, float** wn32,
                     double** part, double** bnd, double** rpart, double** res2, float** ytab,
                     double** ym, float** coef, int** gdeg) {
  const size_t N = (size_t)n * n;
  *R = cv.template take<float>(N * ncols);
  for (int i = 0; i < 3; ++i) z[i] = cv.template take<float>(N * ncols);
  *d = cv.template take<double>(N);
  *we = cv.template take<double>(N);
  *wn = cv.template take<double>(N);
  *d32 = cv.template take<float>(N);
  *we32 = cv.template take<float>(N);
  *wn32 = cv.template take<float>(N);
  *part = cv.template take<double>(2 * (size_t)assemble_blocks(n));
  *bnd = cv.template take<double>(2);
  *rpart = cv.template take<double>((size_t)resid_blocks(n) * 2 * ncols);
  *res2 = cv.template take<double>(2 * (size_t)ncols);
  *ytab = cv.template take<float>((size_t)std::max(degree, 1) * ncols);
  *ym = cv.template take<double>(3 * (size_t)ncols);
  *coef = cv.template take<float>(3 * (size_t)std::max(degree, 1));
  *gdeg = cv.template take<int>((size_t)(ncols + 3) / 4);
}

// Defect-corrected filter of the FP64 phase (mixed form): X (FP64, ncols active
// columns) with its residual block R = A X - X diag(theta) (FP32) and Ritz values theta
// (device). The remainder Z runs through zb; Y = X diag(y_m) + Z_m lands in Y (FP64).
// Optional deflation of the remainder against locked columns before the combine: the
// active X is already orthogonal to them, so only Z carries locked components; removing
// them here with FP32 products (one classical Gram-Schmidt pass) leaves one FP64 pass for
// the caller instead of two.
struct DcDeflate {
  const float* V32 = nullptr;  // FP32 copies of the locked columns (ld ldv)
  int ldv = 0, nl = 0;
  double* C = nullptr;         // nl x ncols
  float* partials = nullptr;   // gemm_tn_f32 partial sums
};

// Degree of one column under the per-column rule (Winkelmann et al., ChASE, 2019): the
// scaled filter of degree d leaves column j's error components from [alpha, beta] at most
// 1 / |C_d(t_j)| <= 2 rho_j^-d of their size relative to the column, t_j = (theta_j - c) / e,
// rho_j = |t_j| + sqrt(t_j^2 - 1), so d = ln(8 r_j / tol) / ln rho_j steps bring a residual
// r_j to tol / 4; two steps of margin, clamped to [8, m]. Columns inside the damped interval
// (the guard columns near alpha) and columns without a finite residual take m.
int column_degree(double theta, double r, double c, double e, double tol, int m) {
  constexpr int kMinDegree = 8;
  const int lo = std::min(kMinDegree, m);
  const double t = (theta - c) / e;
  if (!(t < -1.0) || !std::isfinite(r)) return m;
  if (!(r > 0.125 * tol)) return lo;
  const double rho = -t + std::sqrt(t * t - 1.0);
  if (!(rho > 1.0 + 1e-12)) return m;
  const double d = std::ceil(std::log(8.0 * r / tol) / std::log(rho)) + 2.0;
  if (!(d < (double)m)) return m;
  return std::max(lo, (int)d);
}

cudaError_t run_filter_dc(const Stencil32& A, const double* X, int ldx, const float* R, int ldr,
                          const double* theta, int ncols, int degree, double lam, double c,
                          double e, float* const zb[3], int ldz, float* ytab, double* ystate,
                          double* Y, int ldy, cudaStream_t st, const DcDeflate* defl = nullptr,
                          float* coef_dev = nullptr, float* coef_host = nullptr,
                          const int* gdeg = nullptr, bool* grouped = nullptr) {
  // gdeg (device): per group of 4 columns its degree <= degree, honoured by the resident
  // filter only (the per-step fallback runs every column to degree); *grouped says which ran.
  // coefficients of step i (Y_i -> Y_{i+1}): s1 A Y_i + s2 Y_i + s3 Y_{i-1}
  std::vector<double> s1(degree), s2(degree), s3(degree);
  const double sigma1 = e / (lam - c);
  double sigma = sigma1;
  s1[0] = sigma1 / e;
  s2[0] = -sigma1 * c / e;
  s3[0] = 0.0;
  for (int i = 1; i < degree; ++i) {
    const double sigma_next = 1.0 / (2.0 / sigma1 - sigma);
    s1[i] = 2.0 * sigma_next / e;
    s2[i] = -2.0 * sigma_next * c / e;
    s3[i] = -sigma_next * sigma;
    sigma = sigma_next;
  }
  cudaError_t err = cudaSuccess;
  DcSteps P;
  for (int i0 = 0; i0 < degree; i0 += kDcChunk) {
    P.i0 = i0;
    P.count = std::min(kDcChunk, degree - i0);
    for (int q = 0; q < P.count; ++q) {
      P.s1[q] = s1[i0 + q];
      P.s2[q] = s2[i0 + q];
      P.s3[q] = s3[i0 + q];
    }
    if ((err = launch_dc_ytab(theta, ncols, P, ytab, ystate, st, gdeg,
                              gdeg ? ystate + 2 * ncols : nullptr)) != cudaSuccess)
      return err;
  }
  int cur = 0;
  bool resident = false;
  if (coef_dev && coef_host) {  // the whole recurrence in one cluster-resident launch
    for (int i = 0; i < degree; ++i) {
      coef_host[3 * i] = (float)s1[i];
      coef_host[3 * i + 1] = (float)s2[i];
      coef_host[3 * i + 2] = (float)s3[i];
    }
    err = cudaMemcpyAsync(coef_dev, coef_host, 3 * (size_t)degree * sizeof(float),
                          cudaMemcpyHostToDevice, st);
    if (err != cudaSuccess) return err;
    err = launch_dc_filter_resident(A, R, ldr, ncols, ytab, coef_dev, degree, zb[0], ldz, st,
                                    gdeg);
    if (err == cudaSuccess) resident = true;
    else if (err != cudaErrorNotSupported) return err;
    else cudaGetLastError();
  }
  if (!resident) {
  // Z_1 = s1 R diag(y_0), y_0 = 1; Z_0 = 0
  err = launch_cheb_step_dc(A, nullptr, nullptr, ldz, R, ldr, ytab, zb[0], ncols, (float)s1[0],
                            0.f, 0.f, st);
  if (err != cudaSuccess) return err;
  const float* prev = nullptr;
  for (int i = 1; i < degree; ++i) {
    const int nxt = i % 3;
    err = launch_cheb_step_dc(A, zb[cur], prev, ldz, R, ldr, ytab + (size_t)i * ncols, zb[nxt],
                              ncols, (float)s1[i], (float)s2[i], (float)s3[i], st);
    if (err != cudaSuccess) return err;
    prev = zb[cur];
    cur = nxt;
  }
  }
  if (defl && defl->nl > 0) {
    const int N = A.n * A.n;
    err = launch_gemm_tn_f32(N, defl->nl, ncols, defl->V32, defl->ldv, zb[cur], ldz, defl->C, ncols,
                             false, defl->partials, st);
    if (err != cudaSuccess) return err;
    err = launch_gemm_nn_f32(N, defl->nl, ncols, -1.f, defl->V32, defl->ldv, defl->C, ncols, 1.f,
                             zb[cur], ldz, false, st);
    if (err != cudaSuccess) return err;
  }
  // y at each column's own degree (computed with the table) where the groups stopped early
  const double* ym = (resident && gdeg) ? ystate + 2 * ncols : ystate + ncols;
  if (grouped) *grouped = resident && gdeg;
  return launch_dc_combine(A.n * A.n, ncols, X, ldx, ym, zb[cur], ldz, Y, ldy, st);
}

// Launch width of the FP32 filter step per (n, k_b): the first chain of a shape times
// 128 / 256 / 512 / 1024 threads per CTA over 16 steps each on its own buffers (CUDA events
// on its stream) and keeps the fastest for the process.
int tuned_f32_threads(const Stencil32& A, const float* X, int kb, float* out, cudaStream_t st) {
  static std::mutex mu;
  static std::map<std::pair<int, int>, int> best;
  const std::pair<int, int> key(A.n, kb);
  {
    std::lock_guard<std::mutex> g(mu);
    auto it = best.find(key);
    if (it != best.end()) return it->second;
  }
  int pick = 256;
  float pick_ms = INFINITY;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) {
    for (int threads : {128, 256, 512, 1024}) {
      launch_cheb_step_f32(A, X, kb, nullptr, 0, out, kb, kb, 1.f, 0.f, 0.f, st, threads);
      cudaEventRecord(e0, st);
      for (int r = 0; r < 16; ++r)
        launch_cheb_step_f32(A, X, kb, nullptr, 0, out, kb, kb, 1.f, 0.f, 0.f, st, threads);
      cudaEventRecord(e1, st);
      float ms = INFINITY;
      if (cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess &&
          ms < pick_ms) {
        pick_ms = ms;
        pick = threads;
      }
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaGetLastError();
  std::lock_guard<std::mutex> g(mu);
  best.emplace(key, pick);
  return pick;
}

}  // namespace

struct scsf_chain {
  scsf_ctx* ctx = nullptr;
  scsf_params p{};
  int n = 0, N = 0, kb = 0;
  ChainBufs b{};
  bool has_block = false;
  std::vector<double> ritz;  // Ritz values of the kept block (warm start)
  // captured FP32-phase filter (a11): m table-driven steps on fixed buffers
  cudaGraphExec_t g32 = nullptr;
  int g32_m = 0, g32_threads = 0;
  // captured reduced eigensolves, keyed by (width, FP32-phase form): {key, graph, launches}
  struct EighGraph {
    int key;
    cudaGraphExec_t exec;
    int launches;
  };
  std::vector<EighGraph> eigh_graphs;
  std::vector<int> eigh_seen;
  ~scsf_chain() {
    if (g32) cudaGraphExecDestroy(g32);
    for (auto& g : eigh_graphs) cudaGraphExecDestroy(g.exec);
  }
};

namespace {

// The FP32 filter of the mixed form's FP32 phase as a replay of a captured graph: the m
// steps' scalars go to the device table b.coef32 (one small copy), the graph (captured
// once per chain and degree, on the chain's fixed buffers) runs the m table-driven steps.
// Y_i lands in B32[(i - 1) % 3] exactly as in run_filter_f32.
cudaError_t run_filter_f32_graph(scsf_chain* ch, const Stencil32& A, int m, double lam, double c,
                                 double e, int* which, cudaStream_t st) {
  ChainBufs& b = ch->b;
  const int kb = ch->kb;
  // preferred: the whole filter in one launch, resident in cluster shared memory
  if (m <= kMaxGraphSteps) {
    float* h = reinterpret_cast<float*>(ch->ctx->pinned + kPinnedCoefOffset);
    cudaError_t err = upload_filter_coefs(m, lam, c, e, h, b.coef32, st);
    if (err != cudaSuccess) return err;
    const int w = (m - 1) % 3;
    err = launch_cheb_filter_f32_resident(A, b.V32, kb, b.B32[w], kb, kb, m, b.coef32, st);
    if (err == cudaSuccess) {
      *which = w;
      return cudaSuccess;
    }
    if (err != cudaErrorNotSupported) return err;
    cudaGetLastError();
  }
  // the legacy default stream cannot be captured: plain launches there
  if (m > kMaxGraphSteps || st == nullptr || st == cudaStreamLegacy || st == cudaStreamPerThread)
    return run_filter_f32(A, b.V32, kb, kb, m, lam, c, e, b.B32, kb, which, st);
  cudaError_t err;
  if (!ch->g32 || ch->g32_m != m) {
    if (ch->g32) {
      cudaGraphExecDestroy(ch->g32);
      ch->g32 = nullptr;
    }
    const int threads = tuned_f32_threads(A, b.V32, kb, b.B32[0], st);
    if ((err = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) return err;
    const float* prev = nullptr;
    const float* cur = b.V32;
    for (int i = 0; i < m; ++i) {
      float* out = b.B32[i % 3];
      err = launch_cheb_step_f32_tab(A, cur, kb, prev, kb, out, kb, kb, b.coef32 + 3 * i, threads, st);
      if (err != cudaSuccess) break;
      prev = cur;
      cur = out;
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t end = cudaStreamEndCapture(st, &graph);
    if (err == cudaSuccess) err = end;
    if (err == cudaSuccess) err = cudaGraphInstantiate(&ch->g32, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (err != cudaSuccess) return err;
    ch->g32_m = m;
    ch->g32_threads = threads;
  }
  float* h = reinterpret_cast<float*>(ch->ctx->pinned + kPinnedCoefOffset);
  if ((err = upload_filter_coefs(m, lam, c, e, h, b.coef32, st)) != cudaSuccess) return err;
  if ((err = cudaGraphLaunch(ch->g32, st)) != cudaSuccess) return err;
  for (int i = 0; i < m; ++i) note_launch();
  *which = (m - 1) % 3;
  return cudaSuccess;
}

// The reduced eigensolve of width ka (FP32-phase form or FP64 accuracy) on the chain's fixed
// buffers (H in, theta and Z out). About 30 launches with arguments that only depend on the
// width, so a chain captures them as a CUDA graph the second time a width occurs and replays
// the graph afterwards (the first call runs plainly: it also sets function attributes, which
// must not happen inside a capture). At most kMaxEighGraphs widths are kept per chain.
constexpr size_t kMaxEighGraphs = 8;

cudaError_t run_small_eigh(scsf_chain* ch, bool f32, int ka, cudaStream_t st) {
  ChainBufs& b = ch->b;
  auto direct = [&]() {
    return f32 ? launch_small_eigh_f32(ka, b.H, ka, b.theta, b.Z, ka, b.eigh_scratch, st)
               : launch_small_eigh(ka, b.H, ka, b.theta, b.Z, ka, b.eigh_scratch, st);
  };
  if (st == nullptr || st == cudaStreamLegacy || st == cudaStreamPerThread) return direct();
  const int key = 2 * ka + (f32 ? 1 : 0);
  for (auto& g : ch->eigh_graphs)
    if (g.key == key) {
      for (int i = 0; i < g.launches; ++i) note_launch();
      return cudaGraphLaunch(g.exec, st);
    }
  if (std::find(ch->eigh_seen.begin(), ch->eigh_seen.end(), key) == ch->eigh_seen.end()) {
    ch->eigh_seen.push_back(key);
    return direct();
  }
  cudaError_t err = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
  if (err != cudaSuccess) return err;
  const long long l0 = scsf::t_launches;
  err = direct();
  const int nl = (int)(scsf::t_launches - l0);
  cudaGraph_t graph = nullptr;
  const cudaError_t end = cudaStreamEndCapture(st, &graph);
  if (err == cudaSuccess) err = end;
  cudaGraphExec_t exec = nullptr;
  if (err == cudaSuccess) err = cudaGraphInstantiate(&exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (err != cudaSuccess) return err;
  if (ch->eigh_graphs.size() >= kMaxEighGraphs) {
    cudaGraphExecDestroy(ch->eigh_graphs.front().exec);
    ch->eigh_graphs.erase(ch->eigh_graphs.begin());
  }
  ch->eigh_graphs.push_back({key, exec, nl});
  return cudaGraphLaunch(exec, st);
}

}  // namespace

// ---------------------------------------------------------------------------
extern "C" {

int scsf_version(void) { return 100; }
long long scsf_launch_count(void) { return scsf::g_launches.load(); }

scsf_status scsf_set_timing(scsf_ctx* ctx, int enable) {
  if (!ctx) return SCSF_ERR_INVALID_ARG;
  SCSF_CUDA(ctx, cudaSetDevice(ctx->device));
  if (enable && !ctx->ev[0])
    for (auto& e : ctx->ev) SCSF_CUDA(ctx, cudaEventCreate(&e));
  ctx->timing = enable != 0;
  return SCSF_OK;
}
int scsf_max_block_width(void) { return kMaxBlockWidth; }

scsf_status scsf_create(scsf_ctx** out, int device, void* cuda_stream) {
  if (!out) return SCSF_ERR_INVALID_ARG;
  *out = nullptr;
  scsf_ctx* ctx = new (std::nothrow) scsf_ctx();
  if (!ctx) return SCSF_ERR_NO_MEMORY;
  int count = 0;
  cudaError_t e = cudaGetDeviceCount(&count);
  if (e != cudaSuccess || device < 0 || device >= count) {
    delete ctx;
    return SCSF_ERR_CUDA;
  }
  ctx->device = device;
  ctx->stream = static_cast<cudaStream_t>(cuda_stream);
  if (cudaSetDevice(device) != cudaSuccess ||
      cudaMallocHost(&ctx->pinned, kPinnedDoubles * sizeof(double)) != cudaSuccess) {
    delete ctx;
    return SCSF_ERR_CUDA;
  }
  // reserve the allocation-free sort's static scratch on this device now, while the caller
  // is still setting up (a failure here is retried, and reported, by scsf_sort_noalloc)
  noalloc_prepare(device);
  ctx->pinned_count = kPinnedDoubles;
  *out = ctx;
  return SCSF_OK;
}

void scsf_destroy(scsf_ctx* ctx) {
  if (!ctx) return;
  if (ctx->pinned) cudaFreeHost(ctx->pinned);
  for (auto& e : ctx->ev)
    if (e) cudaEventDestroy(e);
  delete ctx;
}

const char* scsf_last_error(const scsf_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

size_t scsf_sort_workspace_size(int64_t n_ops, int p0) {
  if (n_ops <= 0 || p0 <= 0) return 0;
  return sort_workspace_bytes(n_ops, p0);
}

}  // extern "C"

namespace scsf {
scsf_status validate_sort_args(scsf_ctx* ctx, const double* fields, int64_t n_ops, int p, int p0,
                               int start, const int32_t* perm_out) {
  if (!fields || !perm_out) return fail(ctx, SCSF_ERR_INVALID_ARG, "null pointer");
  if (n_ops < 1 || n_ops > 65536) return fail(ctx, SCSF_ERR_INVALID_ARG, "n_ops out of [1, 65536]");
  if (p < 1 || p > 1024 || p0 < 1 || p0 > p)
    return fail(ctx, SCSF_ERR_INVALID_ARG, "need 1 <= p0 <= p <= 1024");
  if ((size_t)(2 * p + 2 * p * p0) * sizeof(double) > 220 * 1024)
    return fail(ctx, SCSF_ERR_INVALID_ARG, "p * p0 too large for one CTA's shared memory");
  if (p0 > 64) return fail(ctx, SCSF_ERR_INVALID_ARG, "p0 > 64 is not supported");
  if (start < 0 || start >= n_ops) return fail(ctx, SCSF_ERR_INVALID_ARG, "start out of range");
  return SCSF_OK;
}
}  // namespace scsf

extern "C" {

scsf_status scsf_sort_dist(scsf_ctx* ctx, const double* fields, int64_t n_ops, int p, int p0,
                           int start, void* workspace, size_t workspace_bytes, int32_t* perm_out,
                           double* dist_out) {
  if (!ctx) return SCSF_ERR_INVALID_ARG;
  const scsf_status v = validate_sort_args(ctx, fields, n_ops, p, p0, start, perm_out);
  if (v != SCSF_OK) return v;
  if (!workspace) return fail(ctx, SCSF_ERR_INVALID_ARG, "null pointer");
  if (workspace_bytes < sort_workspace_bytes(n_ops, p0))
    return fail(ctx, SCSF_ERR_NO_MEMORY, "sort workspace too small");
  SCSF_CUDA(ctx, cudaSetDevice(ctx->device));
  SCSF_CUDA(ctx, launch_sort(fields, n_ops, p, p0, start, workspace, perm_out, ctx->stream,
                             dist_out));
  return SCSF_OK;
}

scsf_status scsf_sort(scsf_ctx* ctx, const double* fields, int64_t n_ops, int p, int p0, int start,
                      void* workspace, size_t workspace_bytes, int32_t* perm_out) {
  return scsf_sort_dist(ctx, fields, n_ops, p, p0, start, workspace, workspace_bytes, perm_out,
                        nullptr);
}

size_t scsf_solve_workspace_size(const scsf_params* params, int n_max) {
  if (!params || n_max < 2) return 0;
  const int kb = block_width(params);
  if (kb < 1 || kb > kMaxBlockWidth) return 0;
  SizeCarve c;
  ChainBufs b;
  const bool mixed = params->precision == SCSF_MIXED;
  carve_chain(c, (size_t)n_max * n_max, kb, mixed, params->degree, !mixed,
              params->products == SCSF_PRODUCT_TENSOR, params->use_proposal != 0, b);
  return c.used;
}

size_t scsf_solve_workspace_size_rows(const scsf_params* params, int64_t rows) {
  if (!params || rows < 1 || rows > kMaxCsrRows || params->precision != SCSF_FP64) return 0;
  const int kb = block_width(params);
  if (kb < 1 || kb > kMaxBlockWidth) return 0;
  SizeCarve c;
  ChainBufs b;
  carve_chain(c, (size_t)rows, kb, false, params->degree, false,
              params->products == SCSF_PRODUCT_TENSOR, false, b);
  return c.used;
}

}  // extern "C"

namespace {

// n >= 2: a chain of n x n stencil operators; n == 0: a chain of CSR operators of N rows.
scsf_status chain_create(scsf_ctx* ctx, const scsf_params* params, int n, long long N,
                         void* workspace, size_t workspace_bytes, scsf_chain** out) {
  if (!ctx) return SCSF_ERR_INVALID_ARG;
  if (!params || !out || !workspace) return fail(ctx, SCSF_ERR_INVALID_ARG, "null pointer");
  *out = nullptr;
  const int kb = block_width(params);
  if (params->k < 1 || kb > kMaxBlockWidth)
    return fail(ctx, SCSF_ERR_INVALID_ARG,
                "need 1 <= k and k + nex <= " + std::to_string(kMaxBlockWidth));
  if (N < kb) return fail(ctx, SCSF_ERR_INVALID_ARG, "operator too small for the block width");
  if (N > 0x7fffffffLL) return fail(ctx, SCSF_ERR_INVALID_ARG, "N = n^2 must stay below 2^31");
  if (params->degree < 1 || !(params->tol > 0.0) || params->max_iter < 1)
    return fail(ctx, SCSF_ERR_INVALID_ARG, "need degree >= 1, tol > 0, max_iter >= 1");
  if (params->precision != SCSF_FP64 && params->precision != SCSF_MIXED)
    return fail(ctx, SCSF_ERR_INVALID_ARG, "precision must be SCSF_FP64 or SCSF_MIXED");
  if (params->products != SCSF_PRODUCT_TENSOR && params->products != SCSF_PRODUCT_FP64)
    return fail(ctx, SCSF_ERR_INVALID_ARG,
                "products must be SCSF_PRODUCT_TENSOR or SCSF_PRODUCT_FP64");
  if (params->bound != SCSF_BOUND_GERSHGORIN && params->bound != SCSF_BOUND_LANCZOS)
    return fail(ctx, SCSF_ERR_INVALID_ARG, "bound must be SCSF_BOUND_GERSHGORIN or _LANCZOS");
  if (params->use_proposal &&
      (!params->proposal || n < 32 || n % 32 != 0 || kb < 64))
    return fail(ctx, SCSF_ERR_INVALID_ARG,
                "use_proposal needs the network parameters, a stencil chain with n a multiple "
                "of 32 and k + nex >= 64");
  if (params->precision == SCSF_MIXED && n == 0)
    return fail(ctx, SCSF_ERR_INVALID_ARG,
                "SCSF_MIXED needs a stencil operator (its FP32 filters are stencil kernels)");
  if (params->precision == SCSF_MIXED && kb % 4 != 0)
    return fail(ctx, SCSF_ERR_INVALID_ARG,
                "SCSF_MIXED needs k + nex divisible by 4 (float4 block rows)");
  if (reinterpret_cast<uintptr_t>(workspace) % 256 != 0)
    return fail(ctx, SCSF_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
  scsf_chain* ch = new (std::nothrow) scsf_chain();
  if (!ch) return fail(ctx, SCSF_ERR_NO_MEMORY, "host allocation failed");
  ch->ctx = ctx;
  ch->p = *params;
  ch->n = n;
  ch->N = (int)N;
  ch->kb = kb;
  Carve c(workspace, workspace_bytes);
  const bool mixed = params->precision == SCSF_MIXED;
  carve_chain(c, (size_t)N, kb, mixed, params->degree, n > 0 && !mixed,
              params->products == SCSF_PRODUCT_TENSOR, params->use_proposal != 0, ch->b);
  if (!c.ok) {
    delete ch;
    return fail(ctx, SCSF_ERR_NO_MEMORY, "solve workspace too small");
  }
  ch->ritz.assign(kb, 0.0);
  *out = ch;
  return SCSF_OK;
}

}  // namespace

extern "C" {

scsf_status scsf_chain_create(scsf_ctx* ctx, const scsf_params* params, int n, void* workspace,
                              size_t workspace_bytes, scsf_chain** out) {
  if (!ctx) return SCSF_ERR_INVALID_ARG;
  if (n < 2) return fail(ctx, SCSF_ERR_INVALID_ARG, "grid too small for the block width");
  return chain_create(ctx, params, n, (long long)n * n, workspace, workspace_bytes, out);
}

scsf_status scsf_chain_create_rows(scsf_ctx* ctx, const scsf_params* params, int64_t rows,
                                   void* workspace, size_t workspace_bytes, scsf_chain** out) {
  if (!ctx) return SCSF_ERR_INVALID_ARG;
  if (rows < 1 || rows > kMaxCsrRows)
    return fail(ctx, SCSF_ERR_INVALID_ARG, "rows must be in [1, 2^31 - 2]");
  return chain_create(ctx, params, 0, rows, workspace, workspace_bytes, out);
}

void scsf_chain_destroy(scsf_chain* chain) { delete chain; }

scsf_status scsf_chain_restart(scsf_chain* ch) {
  if (!ch) return SCSF_ERR_INVALID_ARG;
  ch->has_block = false;
  return SCSF_OK;
}

scsf_status scsf_far_steps(const double* dist, int64_t n_ops, double quantile, int32_t* far) {
  if (!dist || !far || n_ops < 1 || !(quantile >= 0.0 && quantile <= 1.0))
    return SCSF_ERR_INVALID_ARG;
  far[0] = 1;
  if (n_ops == 1) return SCSF_OK;
  std::vector<double> v(dist + 1, dist + n_ops);
  std::sort(v.begin(), v.end());
  const double pos = quantile * (double)(v.size() - 1);
  const size_t lo = (size_t)std::floor(pos);
  const size_t hi = std::min(lo + 1, v.size() - 1);
  const double thr = v[lo] + (pos - (double)lo) * (v[hi] - v[lo]);
  for (int64_t i = 1; i < n_ops; ++i) far[i] = dist[i] > thr ? 1 : 0;
  return SCSF_OK;
}

scsf_status scsf_chain_seed(scsf_chain* ch, const double* block, const double* ritz_host) {
  if (!ch) return SCSF_ERR_INVALID_ARG;
  scsf_ctx* ctx = ch->ctx;
  if (!block || !ritz_host) return fail(ctx, SCSF_ERR_INVALID_ARG, "null pointer");
  SCSF_CUDA(ctx, cudaSetDevice(ctx->device));
  SCSF_CUDA(ctx, cudaMemcpyAsync(ch->b.V, block, (size_t)ch->N * ch->kb * sizeof(double),
                                 cudaMemcpyDeviceToDevice, ctx->stream));
  ch->ritz.assign(ritz_host, ritz_host + ch->kb);
  ch->has_block = true;
  return SCSF_OK;
}

scsf_status scsf_chain_step(scsf_chain* ch, const scsf_operator* op, double* evals, double* resid,
                            double* evecs, scsf_stats* stats) {
  if (!ch) return SCSF_ERR_INVALID_ARG;
  scsf_ctx* ctx = ch->ctx;
  cudaStream_t st = ctx->stream;
  if (!op_ok(op)) return fail(ctx, SCSF_ERR_INVALID_ARG, "bad operator descriptor");
  const bool csr = op->kind == SCSF_OP_CSR;
  if (csr != (ch->n == 0))
    return fail(ctx, SCSF_ERR_INVALID_ARG,
                csr ? "CSR operator on a stencil chain" : "stencil operator on a CSR chain");
  if (csr ? op->rows != ch->N : op->n != ch->n)
    return fail(ctx, SCSF_ERR_INVALID_ARG, "operator size differs from the chain's");
  const bool plate = op->kind == SCSF_OP_PLATE;
  if (plate && ch->p.precision != SCSF_FP64)
    return fail(ctx, SCSF_ERR_INVALID_ARG,
                "the thin-plate operator takes SCSF_FP64 only (the mixed form's filters are 5-point)");
  if (!evals || !resid) return fail(ctx, SCSF_ERR_INVALID_ARG, "null output pointer");
  SCSF_CUDA(ctx, cudaSetDevice(ctx->device));
  const int n = ch->n, N = ch->N, kb = ch->kb, k = ch->p.k, m = ch->p.degree;
  ChainBufs& b = ch->b;
  Stencil A = csr ? with_csr(stencil_of(b, n), *op) : stencil_of(b, n);
  if (plate) {
    A.rp = b.prp;
    A.ci = b.pci;
    A.val = b.pval;
    A.rows = N;
  }
  double* h = ctx->pinned;

  // operator coefficients and Gershgorin bounds
  if (csr) {
    SCSF_CUDA(ctx, launch_csr_bounds(N, op->row_ptr, op->col, op->val, b.asm_partials, b.bounds, st));
  } else if (plate) {
    SCSF_CUDA(ctx, launch_plate_csr(n, op->plate_d, op->plate_rho, b.prp, b.pci, b.pval, st));
    SCSF_CUDA(ctx, launch_csr_bounds(N, b.prp, b.pci, b.pval, b.asm_partials, b.bounds, st));
  } else
    SCSF_CUDA(ctx, launch_assemble(op->kind, n, op->ax, op->ay, op->v, b.d, b.we, b.wn,
                                   b.asm_partials, b.bounds, st));
  const bool lanczos = ch->p.bound == SCSF_BOUND_LANCZOS;
  if (lanczos)  // capped at the Gershgorin bound on the device
    SCSF_CUDA(ctx, launch_lanczos_bound(A, 16, ch->p.seed ^ 0x5bd1e995ull, b.lanczos, INFINITY,
                                        b.bounds + 2, st));
  SCSF_CUDA(ctx, cudaMemcpyAsync(h, b.bounds, (lanczos ? 3 : 2) * sizeof(double),
                                 cudaMemcpyDeviceToHost, st));
  SCSF_CUDA(ctx, cudaStreamSynchronize(st));
  const double lo = h[0], hi_g = h[1];
  const double hi = (lanczos && std::isfinite(h[2]) && h[2] < hi_g) ? h[2] : hi_g;
  // the bounds kernels keep a NaN, and an infinite coefficient makes hi infinite
  if (!std::isfinite(lo) || !std::isfinite(hi))
    return fail(ctx, SCSF_ERR_INVALID_ARG,
                "operator has non-finite coefficients (NaN or Inf; for the plate, rho <= 0)");
  const double beta = hi;
  double lam, alpha;
  if (!ch->has_block && ch->p.use_proposal) {
    // head from the learned proposal: the network's coarse subspace prolonged to the grid
    // in columns 0..63, the seeded Gaussian block in the rest; filter bounds from its
    // predicted log(lambda_1), log(lambda_64), lambda_kb ~ lambda_64 k_b / 64 (2-D Weyl law)
    if (!op->field)
      return fail(ctx, SCSF_ERR_INVALID_ARG, "use_proposal: the head operator has no field");
    scsf_status ps = scsf_proposal_forward(ctx, ch->p.proposal, op->field, 1, n, b.prop_bounds,
                                           b.prop_block, b.prop_ws, b.prop_ws_bytes);
    if (ps != SCSF_OK) return ps;
    if ((ps = scsf_proposal_prolong(ctx, b.prop_block, 1, n, b.V, kb)) != SCSF_OK) return ps;
    if (kb > 64) SCSF_CUDA(ctx, launch_philox_normal(b.V + 64, N, kb - 64, kb, ch->p.seed, st));
    float* hb = reinterpret_cast<float*>(h + 8);
    SCSF_CUDA(ctx, cudaMemcpyAsync(hb, b.prop_bounds, 2 * sizeof(float), cudaMemcpyDeviceToHost, st));
    SCSF_CUDA(ctx, cudaStreamSynchronize(st));
    const double l1 = std::exp((double)hb[0]), l64 = std::exp((double)hb[1]);
    lam = std::isfinite(l1) ? std::max(l1, lo) : lo;
    alpha = std::isfinite(l64) ? std::max(l64 * kb / 64.0, l64) : lo + 2.0 * ((double)kb / N) * (hi - lo);
  } else if (!ch->has_block) {  // head of the chain: random block (Sec. 3.2)
    SCSF_CUDA(ctx, launch_philox_normal(b.V, N, kb, kb, ch->p.seed, st));
    lam = lo;
    alpha = lo + 2.0 * ((double)kb / N) * (hi - lo);
  } else {               // warm start: previous block and Ritz values (Alg. 3, warm start)
    lam = *std::min_element(ch->ritz.begin(), ch->ritz.end());
    alpha = *std::max_element(ch->ritz.begin(), ch->ritz.end());
  }

  std::vector<double> locked_val, locked_res;
  std::vector<double> theta_h(kb), r_h(kb);
  int nl = 0, it = 0, filter_steps = 0, rot_launches = 0;
  double flops = 0.0, fbytes = 0.0, felems = 0.0, rot_flops = 0.0;
  double tms[6] = {0, 0, 0, 0, 0, 0};
  const long long launches0 = scsf_launch_count();
  // optional convergence history: {max, median residual of wanted unlocked pairs, locked}
  double* hist = stats ? stats->history : nullptr;
  auto record = [&](int iter, int count, int locked) {
    if (!hist || iter < 1 || iter > ch->p.max_iter) return;
    std::vector<double> v(r_h.begin(), r_h.begin() + std::max(0, std::min(count, (int)r_h.size())));
    double mx = 0.0, med = 0.0;
    if (!v.empty()) {
      mx = *std::max_element(v.begin(), v.end());
      std::nth_element(v.begin(), v.begin() + v.size() / 2, v.end());
      med = v[v.size() / 2];
    }
    hist[3 * (iter - 1)] = mx;
    hist[3 * (iter - 1) + 1] = med;
    hist[3 * (iter - 1) + 2] = locked;
  };
  const bool timing = ctx->timing;
  auto mark = [&](int i) -> cudaError_t {
    return timing ? cudaEventRecord(ctx->ev[i], st) : cudaSuccess;
  };
  bool converged = false;
  bool fp32_first = true;  // first Cholesky QR factor in FP32
  int chol_shifts32 = 0, chol_shifts64 = 0;  // shifted Cholesky restarts per phase
  int it32 = 0, filter32_steps = 0;
  double felems32 = 0.0, t_filter32 = 0.0;
  // defect-corrected filter of the mixed form's FP64 phase: residual block in b.V32
  // (columns aligned with b.V), Ritz values of the active columns at dc_theta
  const bool mixed = ch->p.precision == SCSF_MIXED;
  const Stencil32 A32{b.d32, b.we32, b.wn32, n};
  bool have_R = false;
  const double* dc_theta = nullptr;
  int dc_steps = 0;
  double dc_elems = 0.0, t_filter_dc = 0.0;
  // per-column degrees of the defect-corrected filter: the previous residual and Ritz value
  // of active column j are r_h[prev_off + j], theta_h[prev_off + j] once have_prev is set
  const bool coldeg = mixed && ch->p.column_degree != 0;
  bool have_prev = false;
  int prev_off = 0;

  // the tall block products (rows = N): tensor-core digit-split products or CUDA-core FMAs
  const bool tc = ch->p.products == SCSF_PRODUCT_TENSOR;
  int* oz_err = b.status + 2;  // set by a tensor-core product whose bounded wait gave up
  if (tc) SCSF_CUDA(ctx, cudaMemsetAsync(oz_err, 0, sizeof(int), st));
  auto tn64 = [&](int m_, int n_, const double* A_, int lda_, const double* B_, int ldb_,
                  double* C_, int ldc_, bool sym_) -> cudaError_t {
    return tc ? launch_gemm_tn_oz(N, m_, n_, A_, lda_, B_, ldb_, C_, ldc_, sym_, kOzSlicesF64,
                                  b.oz, b.oz_bytes, oz_err, st)
              : launch_gemm_tn(N, m_, n_, A_, lda_, B_, ldb_, C_, ldc_, sym_, b.gemm_partials, st);
  };
  auto nn64 = [&](int k_, int n_, double al, const double* A_, int lda_, const double* M_,
                  int ldm_, double be, double* C_, int ldc_, bool upper_) -> cudaError_t {
    return tc ? launch_gemm_nn_oz(N, k_, n_, al, A_, lda_, M_, ldm_, be, C_, ldc_, kOzSlicesF64,
                                  b.oz, b.oz_bytes, oz_err, st)
              : launch_gemm_nn(N, k_, n_, al, A_, lda_, M_, ldm_, be, C_, ldc_, upper_, st);
  };
  auto tn32 = [&](int m_, int n_, const float* A_, int lda_, const float* B_, int ldb_,
                  double* C_, int ldc_, bool sym_) -> cudaError_t {
    return tc ? launch_gemm_tn_oz_f32(N, m_, n_, A_, lda_, B_, ldb_, C_, ldc_, sym_, b.oz,
                                      b.oz_bytes, oz_err, st)
              : launch_gemm_tn_f32(N, m_, n_, A_, lda_, B_, ldb_, C_, ldc_, sym_, b.partials32, st);
  };
  auto nn32 = [&](int k_, int n_, float al, const float* A_, int lda_, const double* M_, int ldm_,
                  float be, float* C_, int ldc_, bool upper_) -> cudaError_t {
    return tc ? launch_gemm_nn_oz_f32(N, k_, n_, al, A_, lda_, M_, ldm_, be, C_, ldc_, b.oz,
                                      b.oz_bytes, oz_err, st)
              : launch_gemm_nn_f32(N, k_, n_, al, A_, lda_, M_, ldm_, be, C_, ldc_, upper_, st);
  };

  // FP32 phase of the mixed form: the whole block iterates in FP32 (filter, Cholesky
  // QR, Rayleigh-Ritz, rotation) without locking, until the wanted residuals stop
  // improving, i.e. the subspace has converged to FP32 accuracy. FP32 storage floors
  // the relative residual near eps32 ||A|| / lambda, so locking at the tolerance is
  // left to the FP64 phase, which starts from this block.
  if (mixed) {
    SCSF_CUDA(ctx, launch_to_f32(b.d, b.d32, N, st));
    SCSF_CUDA(ctx, launch_to_f32(b.we, b.we32, N, st));
    SCSF_CUDA(ctx, launch_to_f32(b.wn, b.wn32, N, st));
    SCSF_CUDA(ctx, launch_block_f64_to_f32(N, kb, b.V, kb, b.V32, kb, st));
    double prev_score = INFINITY;
    const int max32 = std::max(0, ch->p.max_iter - 10);
    const int m32 = (ch->p.degree_fp32 > 0) ? ch->p.degree_fp32 : m;
    while (it32 < max32) {
      ++it32;
      if (!(alpha < beta)) alpha = lam + 0.5 * (beta - lam);
      if (!(lam < alpha)) lam = alpha - 1e-3 * (beta - alpha);
      const double c = 0.5 * (alpha + beta), e = 0.5 * (beta - alpha);
      int which = 0;
      SCSF_CUDA(ctx, mark(0));
      SCSF_CUDA(ctx, run_filter_f32_graph(ch, A32, m32, lam, c, e, &which, st));
      SCSF_CUDA(ctx, mark(1));
      filter32_steps += m32;
      felems32 += (double)m32 * N * kb;
      float* Y = b.B32[which];
      float* F1 = b.B32[(which + 1) % 3];
      float* F2 = b.B32[(which + 2) % 3];
      // Cholesky QR2 with the second factor folded into the small matrices, as in the FP64
      // phase: Q1 = Y R1^{-1}; Q1^T Q1 = R2^T R2; H = R2^{-T} (Q1^T A Q1) R2^{-1};
      // X = Q1 (R2^{-1} Z) -- the same H and X as with Q = Q1 R2^{-1}, one tall product fewer.
      SCSF_CUDA(ctx, tn32(kb, kb, Y, kb, Y, kb, b.G, kb, true));
      SCSF_CUDA(ctx, launch_chol_rinv(kb, b.G, kb, true, b.C, b.Rinv, b.status, st, b.chol_wide));
      SCSF_CUDA(ctx, nn32(kb, kb, 1.f, Y, kb, b.Rinv, kb, 0.f, F1, kb, true));
      std::swap(Y, F1);  // Y = Q1
      SCSF_CUDA(ctx, tn32(kb, kb, Y, kb, Y, kb, b.G, kb, true));
      SCSF_CUDA(ctx, launch_chol_rinv(kb, b.G, kb, true, b.C, b.Rinv, b.status + 1, st,
                                      b.chol_wide));
      SCSF_CUDA(ctx, mark(2));
      SCSF_CUDA(ctx, launch_cheb_step_f32(A32, Y, kb, nullptr, 0, F2, kb, kb, 1.f, 0.f, 0.f, st));
      // Q1^T (A Q1) is symmetric (A is): only its upper tiles are formed, then mirrored
      SCSF_CUDA(ctx, tn32(kb, kb, Y, kb, F2, kb, b.H, kb, true));
      // H = R2^{-T} (H1 R2^{-1}) with T = H1 R2^{-1} in b.G
      SCSF_CUDA(ctx, launch_gemm_nn(kb, kb, kb, 1.0, b.H, kb, b.Rinv, kb, 0.0, b.G, kb, true, st));
      SCSF_CUDA(ctx, launch_gemm_tn(kb, kb, kb, b.Rinv, kb, b.G, kb, b.H, kb, false, b.gemm_partials,
                                    st));
      SCSF_CUDA(ctx, mark(3));
      SCSF_CUDA(ctx, run_small_eigh(ch, true, kb, st));
      SCSF_CUDA(ctx, mark(4));
      // X = Q1 M, M = R2^{-1} Z in b.C
      SCSF_CUDA(ctx, launch_gemm_nn(kb, kb, kb, 1.0, b.Rinv, kb, b.Z, kb, 0.0, b.C, kb, false, st));
      SCSF_CUDA(ctx, nn32(kb, kb, 1.f, Y, kb, b.C, kb, 0.f, b.V32, kb, false));
      SCSF_CUDA(ctx, mark(5));
      SCSF_CUDA(ctx, launch_residual_norms_f32(A32, b.V32, kb, kb, b.theta, b.res_partials, b.res2, st));
      SCSF_CUDA(ctx, mark(6));
      SCSF_CUDA(ctx, cudaMemcpyAsync(h, b.theta, kb * sizeof(double), cudaMemcpyDeviceToHost, st));
      SCSF_CUDA(ctx, cudaMemcpyAsync(h + kMaxBlockWidth, b.res2, 2 * kb * sizeof(double),
                                     cudaMemcpyDeviceToHost, st));
      SCSF_CUDA(ctx, cudaMemcpyAsync(h + 3 * kMaxBlockWidth, b.status, 3 * sizeof(int),
                                     cudaMemcpyDeviceToHost, st));
      SCSF_CUDA(ctx, cudaStreamSynchronize(st));
      {
        int st3[3];
        std::memcpy(st3, h + 3 * kMaxBlockWidth, sizeof(st3));
        if (tc && st3[2] != 0)
          return fail(ctx, SCSF_ERR_TIMEOUT, "a tensor-core block product gave up waiting");
        chol_shifts32 += (st3[0] % 1000) + (st3[1] % 1000);
      }
      if (timing) {
        float ms = 0.f;
        SCSF_CUDA(ctx, cudaEventElapsedTime(&ms, ctx->ev[0], ctx->ev[1]));
        t_filter32 += ms;
        for (int i = 1; i < 6; ++i) {
          SCSF_CUDA(ctx, cudaEventElapsedTime(&ms, ctx->ev[i], ctx->ev[i + 1]));
          tms[i] += ms;
        }
      }
      // A vector stored in FP32 carries rounding noise of relative size ~eps32 in every
      // eigendirection, which puts a floor of about c eps32 ||A|| / |theta_j| under its
      // relative residual (||A|| <= beta). Once every wanted vector is at its floor the
      // subspace has converged to FP32 accuracy and the FP64 phase takes over.
      double score = 0.0, max_r = 0.0;
      int at_floor = 0;
      for (int j = 0; j < kb; ++j) {
        theta_h[j] = h[j];
        const double rr = h[kMaxBlockWidth + j], aa = h[kMaxBlockWidth + kb + j];
        r_h[j] = (aa > 0.0) ? std::sqrt(rr / aa) : 1.0;
        if (j < k) {
          const double floor_j = 16.0 * 5.96e-8 * beta / std::max(std::fabs(theta_h[j]), 1e-300);
          at_floor += (r_h[j] <= std::max(floor_j, ch->p.tol)) ? 1 : 0;
          score += std::log(std::max(r_h[j], 1e-300));
          max_r = std::max(max_r, r_h[j]);
        }
      }
      for (int j = 0; j < kb; ++j) ch->ritz[j] = theta_h[j];
      lam = theta_h[0];
      alpha = theta_h[kb - 1];
      record(it32, k, 0);
      if (at_floor == k) break;
      if (ch->p.switch_tol > 0.0 && max_r <= ch->p.switch_tol) break;
      // safety: stop when the wanted residuals improve by less than 1.05x on average
      if (score > prev_score - k * std::log(1.05)) break;
      prev_score = score;
    }
    SCSF_CUDA(ctx, launch_block_f32_to_f64(N, kb, b.V32, kb, b.V, kb, st));
    if (it32 > 0) {  // FP64 residual block of the FP32 phase's Ritz pairs
      SCSF_CUDA(ctx, launch_residual_norms(A, b.V, kb, kb, b.theta, b.res_partials, b.res2, st,
                                           b.V32, kb));
      have_R = true;
      dc_theta = b.theta;
      if (coldeg) {  // the FP64 residuals of the FP32 phase's pairs seed the degree rule
        SCSF_CUDA(ctx, cudaMemcpyAsync(h + kMaxBlockWidth, b.res2, 2 * kb * sizeof(double),
                                       cudaMemcpyDeviceToHost, st));
        SCSF_CUDA(ctx, cudaStreamSynchronize(st));
        for (int j = 0; j < kb; ++j) {
          const double rr = h[kMaxBlockWidth + j], aa = h[kMaxBlockWidth + kb + j];
          r_h[j] = (aa > 0.0) ? std::sqrt(rr / aa) : INFINITY;
        }
        have_prev = true;
        prev_off = 0;
      }
    }
  }

  for (it = it32 + 1; it <= ch->p.max_iter; ++it) {
    const int ka = kb - nl;
    if (!(alpha < beta)) alpha = lam + 0.5 * (beta - lam);
    if (!(lam < alpha)) lam = alpha - 1e-3 * (beta - alpha);
    const double c = 0.5 * (alpha + beta), e = 0.5 * (beta - alpha);
    // filter step: Chebyshev filter on the active columns
    double* bufs[3] = {b.B0, b.B1, b.B2};
    const int lds[3] = {kb, kb, kb};
    int which = 0;
    const bool dc = mixed && have_R;
    SCSF_CUDA(ctx, mark(0));
    if (dc) {
      // locked columns [0, nl) of b.V32 hold FP32 copies of the locked vectors
      DcDeflate defl;
      defl.V32 = b.V32;
      defl.ldv = kb;
      defl.nl = nl;
      defl.C = b.C;
      defl.partials = b.partials32;
      const bool per_col = coldeg && have_prev && m <= kMaxGraphSteps;
      double col_elems = 0.0;
      if (per_col) {
        int* hg = reinterpret_cast<int*>(ctx->pinned + kPinnedGdegOffset);
        for (int g = 0; 4 * g < ka; ++g) {
          int dg = 1;
          const int j1 = std::min(4 * g + 4, ka);
          for (int j = 4 * g; j < j1; ++j)
            dg = std::max(dg, column_degree(theta_h[prev_off + j], r_h[prev_off + j], c, e,
                                            ch->p.tol, m));
          hg[g] = dg;
          col_elems += (double)dg * N * (j1 - 4 * g);
        }
        SCSF_CUDA(ctx, cudaMemcpyAsync(b.gdeg, hg, ((ka + 3) / 4) * sizeof(int),
                                       cudaMemcpyHostToDevice, st));
      }
      bool grouped = false;
      SCSF_CUDA(ctx, run_filter_dc(A32, b.V + nl, kb, b.V32 + nl, kb, dc_theta, ka, m, lam, c, e,
                                   b.B32, kb, b.ytab, b.ym, bufs[0], kb, st, &defl,
                                   (m <= kMaxGraphSteps) ? b.coef32 : nullptr,
                                   reinterpret_cast<float*>(ctx->pinned + kPinnedCoefOffset),
                                   per_col ? b.gdeg : nullptr, &grouped));
      dc_steps += m;
      dc_elems += grouped ? col_elems : (double)m * N * ka;
    } else {
      SCSF_CUDA(ctx, run_filter(A, b.V + nl, kb, ka, m, lam, c, e, bufs, lds, &which, st));
      filter_steps += m;
      felems += (double)m * N * ka;
      fbytes += (double)m * N * ka * 24.0;
      flops += (double)m * N * ka * 14.0;
    }
    SCSF_CUDA(ctx, mark(1));
    double* Y = bufs[which];
    double* F1 = bufs[(which + 1) % 3];
    double* F2 = bufs[(which + 2) % 3];
    // orthonormalise [locked | active]: CGS2 against the locked block, then CholQR2
    if (nl > 0) {
      // the defect-corrected filter already took the first pass (in FP32, on Z)
      const int passes = dc ? 1 : 2;
      for (int pass = 0; pass < passes; ++pass) {
        SCSF_CUDA(ctx, tn64(nl, ka, b.V, kb, Y, kb, b.C, ka, false));
        SCSF_CUDA(ctx, nn64(nl, ka, -1.0, b.V, kb, b.C, ka, 1.0, Y, kb, false));
      }
      flops += 4.0 * passes * N * nl * ka;
    }
    if (!mixed) {
      for (int pass = 0; pass < 2; ++pass) {
        SCSF_CUDA(ctx, tn64(ka, ka, Y, kb, Y, kb, b.G, ka, true));
        // the first factor only has to precondition, so it is taken in FP32
        SCSF_CUDA(ctx, launch_chol_rinv(ka, b.G, ka, pass == 0 && fp32_first, b.C, b.Rinv,
                                        b.status + pass, st, b.chol_wide));
        SCSF_CUDA(ctx, nn64(ka, ka, 1.0, Y, kb, b.Rinv, ka, 0.0, F1, kb, true));
        std::swap(Y, F1);
        flops += 2.0 * N * ka * ka;
      }
      SCSF_CUDA(ctx, mark(2));
      // Rayleigh quotient G = Q^T A Q on the active columns
      SCSF_CUDA(ctx, launch_cheb_step_f64(A, Y, kb, nullptr, 0, F2, kb, ka, 1.0, 0.0, 0.0, st));
      SCSF_CUDA(ctx, tn64(ka, ka, Y, kb, F2, kb, b.H, ka, true));
      SCSF_CUDA(ctx, mark(3));
      // reduced eigenproblem and rotation back
      SCSF_CUDA(ctx, run_small_eigh(ch, false, ka, st));
      SCSF_CUDA(ctx, mark(4));
      SCSF_CUDA(ctx, nn64(ka, ka, 1.0, Y, kb, b.Z, ka, 0.0, b.V + nl, kb, false));
      SCSF_CUDA(ctx, mark(5));
    } else {
      // Mixed form: the same Cholesky QR2, Rayleigh-Ritz and rotation with two FP64 block
      // products fewer. Pass 1's Gram matrix is taken in FP32 when its factor is (both only
      // precondition); pass 2 only factors Q1^T Q1 = R2^T R2, and R2^{-1} is folded into the
      // small matrices: H = R2^{-T} (Q1^T A Q1) R2^{-1}, X = Q1 (R2^{-1} Z), the same H and X
      // as with Q = Q1 R2^{-1}.
      if (fp32_first) {
        SCSF_CUDA(ctx, launch_block_f64_to_f32(N, ka, Y, kb, b.B32[0], kb, st));
        SCSF_CUDA(ctx, tn32(ka, ka, b.B32[0], kb, b.B32[0], kb, b.G, ka, true));
      } else {
        SCSF_CUDA(ctx, tn64(ka, ka, Y, kb, Y, kb, b.G, ka, true));
      }
      SCSF_CUDA(ctx, launch_chol_rinv(ka, b.G, ka, fp32_first, b.C, b.Rinv, b.status, st,
                                      b.chol_wide));
      SCSF_CUDA(ctx, nn64(ka, ka, 1.0, Y, kb, b.Rinv, ka, 0.0, F1, kb, true));
      std::swap(Y, F1);  // Y = Q1
      SCSF_CUDA(ctx, tn64(ka, ka, Y, kb, Y, kb, b.G, ka, true));
      SCSF_CUDA(ctx, launch_chol_rinv(ka, b.G, ka, false, b.C, b.Rinv, b.status + 1, st,
                                      b.chol_wide));
      flops += 1.5 * N * ka * ka;
      SCSF_CUDA(ctx, mark(2));
      SCSF_CUDA(ctx, launch_cheb_step_f64(A, Y, kb, nullptr, 0, F2, kb, ka, 1.0, 0.0, 0.0, st));
      SCSF_CUDA(ctx, tn64(ka, ka, Y, kb, F2, kb, b.H, ka, true));
      // H = R2^{-T} (H1 R2^{-1}) with T = H1 R2^{-1} in b.G
      SCSF_CUDA(ctx, launch_gemm_nn(ka, ka, ka, 1.0, b.H, ka, b.Rinv, ka, 0.0, b.G, ka, true, st));
      SCSF_CUDA(ctx, launch_gemm_tn(ka, ka, ka, b.Rinv, ka, b.G, ka, b.H, ka, false, b.gemm_partials,
                                    st));
      SCSF_CUDA(ctx, mark(3));
      SCSF_CUDA(ctx, run_small_eigh(ch, false, ka, st));
      SCSF_CUDA(ctx, mark(4));
      // X = Q1 M, M = R2^{-1} Z in b.C
      SCSF_CUDA(ctx, launch_gemm_nn(ka, ka, ka, 1.0, b.Rinv, ka, b.Z, ka, 0.0, b.C, ka, false, st));
      SCSF_CUDA(ctx, nn64(ka, ka, 1.0, Y, kb, b.C, ka, 0.0, b.V + nl, kb, false));
      SCSF_CUDA(ctx, mark(5));
    }
    rot_launches += 1;
    rot_flops += 2.0 * N * ka * ka;
    // residuals of the new Ritz pairs (App. D.5), then lock a converged prefix
    SCSF_CUDA(ctx, launch_residual_norms(A, b.V + nl, kb, ka, b.theta, b.res_partials, b.res2, st,
                                         mixed ? b.V32 + nl : nullptr, kb));
    SCSF_CUDA(ctx, mark(6));
    flops += (double)N * ka * (2.0 * ka * 2 + 12.0) + 2.0 * N * ka * ka;
    SCSF_CUDA(ctx, cudaMemcpyAsync(h, b.theta, ka * sizeof(double), cudaMemcpyDeviceToHost, st));
    SCSF_CUDA(ctx, cudaMemcpyAsync(h + kMaxBlockWidth, b.res2, 2 * ka * sizeof(double),
                                   cudaMemcpyDeviceToHost, st));
    SCSF_CUDA(ctx, cudaMemcpyAsync(h + 3 * kMaxBlockWidth, b.status, 3 * sizeof(int),
                                   cudaMemcpyDeviceToHost, st));
    SCSF_CUDA(ctx, cudaStreamSynchronize(st));
    if (timing) {
      for (int i = 0; i < 6; ++i) {
        float ms = 0.f;
        SCSF_CUDA(ctx, cudaEventElapsedTime(&ms, ctx->ev[i], ctx->ev[i + 1]));
        if (i == 0 && dc) t_filter_dc += ms;
        else tms[i] += ms;
      }
    }
    int chol_status[3];
    std::memcpy(chol_status, h + 3 * kMaxBlockWidth, sizeof(chol_status));
    if (tc && chol_status[2] != 0)
      return fail(ctx, SCSF_ERR_TIMEOUT, "a tensor-core block product gave up waiting");
    // an FP32 first factor that needed a shift preconditions too weakly for one FP64 pass
    // to reach FP64 orthogonality: take the first factor in FP64 for the rest of this problem
    chol_shifts64 += (chol_status[0] % 1000) + (chol_status[1] % 1000);
    if (fp32_first && chol_status[0] > 0) fp32_first = false;
    if (chol_status[0] >= 1000 || chol_status[1] >= 1000)
      return fail(ctx, SCSF_ERR_BREAKDOWN, "Cholesky QR broke down even with a shift");
    for (int j = 0; j < ka; ++j) {
      theta_h[j] = h[j];
      const double rr = h[kMaxBlockWidth + j], aa = h[kMaxBlockWidth + ka + j];
      r_h[j] = (aa > 0.0) ? std::sqrt(rr / aa) : (rr > 0.0 ? INFINITY : 0.0);
    }
    record(it, std::max(0, k - nl), nl);
    int nconv = 0;
    while (nconv < ka && r_h[nconv] <= ch->p.tol) ++nconv;
    for (int j = 0; j < nconv; ++j) {
      locked_val.push_back(theta_h[j]);
      locked_res.push_back(r_h[j]);
    }
    for (int j = 0; j < ka; ++j) ch->ritz[nl + j] = theta_h[j];
    if (mixed && nconv > 0)  // FP32 copies of the newly locked vectors (deflation of Z)
      SCSF_CUDA(ctx, launch_block_f64_to_f32(N, nconv, b.V + nl, kb, b.V32 + nl, kb, st));
    nl += nconv;
    have_R = mixed;
    dc_theta = b.theta + nconv;
    have_prev = coldeg;
    prev_off = nconv;
    if (nl >= k) {
      converged = true;
      break;
    }
    if (nl >= kb) break;
    lam = theta_h[nconv];
    alpha = theta_h[ka - 1];
  }
  if (it > ch->p.max_iter) it = ch->p.max_iter;
  ch->has_block = true;

  // outputs: the k smallest locked pairs in ascending order
  std::vector<int> order(locked_val.size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int c2) { return locked_val[a] < locked_val[c2]; });
  const int nout = std::min<int>(k, (int)order.size());
  std::vector<double> ev(k, NAN), rs(k, NAN);
  std::vector<int> cols(k, 0);
  for (int j = 0; j < nout; ++j) {
    ev[j] = locked_val[order[j]];
    rs[j] = locked_res[order[j]];
    cols[j] = order[j];
  }
  if (!converged) {  // report the best active pairs after the locked ones
    for (int j = nout; j < k; ++j) {
      const int a = j - nout;
      if (a < kb - nl) rs[j] = r_h[a];
      cols[j] = std::min(nl + a, kb - 1);
    }
  }
  std::memcpy(h, ev.data(), k * sizeof(double));
  std::memcpy(h + kMaxBlockWidth, rs.data(), k * sizeof(double));
  std::memcpy(h + 2 * kMaxBlockWidth, cols.data(), k * sizeof(int));
  SCSF_CUDA(ctx, cudaMemcpyAsync(evals, h, k * sizeof(double), cudaMemcpyHostToDevice, st));
  SCSF_CUDA(ctx, cudaMemcpyAsync(resid, h + kMaxBlockWidth, k * sizeof(double),
                                 cudaMemcpyHostToDevice, st));
  if (evecs) {
    SCSF_CUDA(ctx, cudaMemcpyAsync(b.cols, h + 2 * kMaxBlockWidth, k * sizeof(int),
                                   cudaMemcpyHostToDevice, st));
    SCSF_CUDA(ctx, launch_gather_cols(N, k, b.V, kb, b.cols, evecs, k, st));
    if (plate)  // modes of K u = lambda M u: u = M^{-1/2} v
      SCSF_CUDA(ctx, launch_scale_rows_rsqrt(N, k, evecs, k, op->plate_rho, st));
    SCSF_CUDA(ctx, launch_normalize_signs(N, k, evecs, k, st));
  }
  SCSF_CUDA(ctx, cudaStreamSynchronize(st));  // staging buffer is reused by the next call
  if (stats) {
    stats->iters = it;
    stats->converged = converged ? 1 : 0;
    stats->filter_steps = filter_steps;
    stats->locked = nl;
    stats->flops_fp64 = flops;
    stats->filter_bytes = fbytes;
    stats->filter_elems = felems;
    stats->rot_flops = rot_flops;
    stats->rot_launches = rot_launches;
    stats->launches = (int)(scsf_launch_count() - launches0);
    stats->t_filter_ms = tms[0];
    stats->t_orth_ms = tms[1];
    stats->t_rr_ms = tms[2];
    stats->t_eig_ms = tms[3];
    stats->t_rot_ms = tms[4];
    stats->t_resid_ms = tms[5];
    stats->iters_fp32 = it32;
    stats->filter32_steps = filter32_steps;
    stats->filter32_elems = felems32;
    stats->t_filter32_ms = t_filter32;
    stats->filter_dc_steps = dc_steps;
    stats->filter_dc_elems = dc_elems;
    stats->t_filter_dc_ms = t_filter_dc;
    stats->beta = beta;
    stats->beta_gershgorin = hi_g;
    stats->chol_shifts_fp32 = chol_shifts32;
    stats->chol_shifts = chol_shifts64;
  }
  if (!converged) return fail(ctx, SCSF_ERR_NOT_CONVERGED, "max_iter reached before convergence");
  return SCSF_OK;
}

scsf_status scsf_solve(scsf_ctx* ctx, const scsf_operator* ops, int64_t n_ops,
                       const scsf_params* params, void* workspace, size_t workspace_bytes,
                       double* evals, double* resid, double* evecs, scsf_stats* stats) {
  if (!ctx) return SCSF_ERR_INVALID_ARG;
  if (!ops || n_ops < 1) return fail(ctx, SCSF_ERR_INVALID_ARG, "no operators");
  scsf_chain* ch = nullptr;
  scsf_status s =
      ops[0].kind == SCSF_OP_CSR
          ? scsf_chain_create_rows(ctx, params, ops[0].rows, workspace, workspace_bytes, &ch)
          : scsf_chain_create(ctx, params, ops[0].n, workspace, workspace_bytes, &ch);
  if (s != SCSF_OK) return s;
  const int k = params->k;
  const size_t N = op_rows(ops[0]);
  scsf_status first = SCSF_OK;
  std::string first_msg;
  for (int64_t i = 0; i < n_ops; ++i) {
    s = scsf_chain_step(ch, &ops[i], evals + i * k, resid + i * k, evecs ? evecs + i * N * k : nullptr,
                        stats ? stats + i : nullptr);
    if (s != SCSF_OK && first == SCSF_OK) {
      first = s;
      first_msg = "problem " + std::to_string(i) + ": " + ctx->err;
      if (s != SCSF_ERR_NOT_CONVERGED) break;
    }
  }
  scsf_chain_destroy(ch);
  if (first != SCSF_OK) ctx->err = first_msg;
  return first;
}

// ---- building blocks ------------------------------------------------------
scsf_status scsf_assemble_bounds(scsf_ctx* ctx, const scsf_operator* op, double* bounds_host,
                                 void* scratch, size_t scratch_bytes) {
  if (!ctx) return SCSF_ERR_INVALID_ARG;
  if (!op_ok(op) || !bounds_host || !scratch) return fail(ctx, SCSF_ERR_INVALID_ARG, "bad argument");
  const bool csr = op->kind == SCSF_OP_CSR, plate = op->kind == SCSF_OP_PLATE;
  const size_t N = op_rows(*op);
  Carve c(scratch, scratch_bytes);
  double* d = csr ? nullptr : c.take<double>(N);
  double* we = csr ? nullptr : c.take<double>(N);
  double* wn = csr ? nullptr : c.take<double>(N);
  double* part = c.take<double>(2 * (size_t)assemble_blocks_rows((long long)N));
  double* bnd = c.take<double>(2);
  int* prp = plate ? c.take<int>(N + 1) : nullptr;
  int* pci = plate ? c.take<int>(13 * N) : nullptr;
  double* pval = plate ? c.take<double>(13 * N) : nullptr;
  if (!c.ok) return fail(ctx, SCSF_ERR_NO_MEMORY, "scratch too small");
  SCSF_CUDA(ctx, cudaSetDevice(ctx->device));
  if (csr) {
    SCSF_CUDA(ctx, launch_csr_bounds((int)N, op->row_ptr, op->col, op->val, part, bnd, ctx->stream));
  } else if (plate) {
    SCSF_CUDA(ctx, launch_plate_csr(op->n, op->plate_d, op->plate_rho, prp, pci, pval, ctx->stream));
    SCSF_CUDA(ctx, launch_csr_bounds((int)N, prp, pci, pval, part, bnd, ctx->stream));
  } else
    SCSF_CUDA(ctx, launch_assemble(op->kind, op->n, op->ax, op->ay, op->v, d, we, wn, part, bnd,
                                   ctx->stream));
  SCSF_CUDA(ctx, cudaMemcpyAsync(ctx->pinned, bnd, 2 * sizeof(double), cudaMemcpyDeviceToHost,
                                 ctx->stream));
  SCSF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  bounds_host[0] = ctx->pinned[0];
  bounds_host[1] = ctx->pinned[1];
  return SCSF_OK;
}

scsf_status scsf_cheb_filter(scsf_ctx* ctx, const scsf_operator* op, const double* X, int ldx,
                             int ncols, int degree, double lambda, double c, double e, double* Y,
                             int ldy, void* scratch, size_t scratch_bytes) {
  if (!ctx) return SCSF_ERR_INVALID_ARG;
  if (!op_ok(op) || !X || !Y || !scratch) return fail(ctx, SCSF_ERR_INVALID_ARG, "bad argument");
  if (ncols < 1 || ldx < ncols || ldy < ncols || degree < 1 || !(e > 0.0) || lambda == c)
    return fail(ctx, SCSF_ERR_INVALID_ARG, "bad sizes or filter parameters");
  const bool csr = op->kind == SCSF_OP_CSR, plate = op->kind == SCSF_OP_PLATE;
  const bool stencil = !csr && !plate;
  const int n = op->n;
  const size_t N = op_rows(*op);
  Carve cv(scratch, scratch_bytes);
  double* s0 = cv.take<double>(N * ncols);
  double* s1 = cv.take<double>(N * ncols);
  double* d = stencil ? cv.take<double>(N) : nullptr;
  double* we = stencil ? cv.take<double>(N) : nullptr;
  double* wn = stencil ? cv.take<double>(N) : nullptr;
  double* part = stencil ? cv.take<double>(2 * (size_t)assemble_blocks(n)) : nullptr;
  double* bnd = stencil ? cv.take<double>(2) : nullptr;
  int* prp = plate ? cv.take<int>(N + 1) : nullptr;
  int* pci = plate ? cv.take<int>(13 * N) : nullptr;
  double* pval = plate ? cv.take<double>(13 * N) : nullptr;
  if (!cv.ok) return fail(ctx, SCSF_ERR_NO_MEMORY, "scratch too small");
  SCSF_CUDA(ctx, cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  if (stencil)
    SCSF_CUDA(ctx, launch_assemble(op->kind, n, op->ax, op->ay, op->v, d, we, wn, part, bnd, st));
  if (plate) SCSF_CUDA(ctx, launch_plate_csr(n, op->plate_d, op->plate_rho, prp, pci, pval, st));
  Stencil A = csr ? with_csr(Stencil{nullptr, nullptr, nullptr, 0}, *op) : Stencil{d, we, wn, n};
  if (plate) {
    A.rp = prp;
    A.ci = pci;
    A.val = pval;
    A.rows = (int)N;
  }
  double* bufs[3] = {s0, s1, Y};
  const int lds[3] = {ncols, ncols, ldy};
  int which = 0;
  SCSF_CUDA(ctx, run_filter(A, X, ldx, ncols, degree, lambda, c, e, bufs, lds, &which, st));
  if (bufs[which] != Y)
    SCSF_CUDA(ctx, launch_copy2d((int)N, ncols, bufs[which], lds[which], Y, ldy, st));
  return SCSF_OK;
}

scsf_status scsf_cheb_filter_f32(scsf_ctx* ctx, const scsf_operator* op, const float* X, int ldx,
                                 int ncols, int degree, double lambda, double c, double e,
                                 float* Y, int ldy, void* scratch, size_t scratch_bytes) {
  if (!ctx) return SCSF_ERR_INVALID_ARG;
  if (!op_ok(op) || !X || !Y || !scratch) return fail(ctx, SCSF_ERR_INVALID_ARG, "bad argument");
  if (op->kind == SCSF_OP_CSR || op->kind == SCSF_OP_PLATE)
    return fail(ctx, SCSF_ERR_INVALID_ARG, "the FP32 filter takes 5-point stencil operators only");
  if (ncols < 4 || ncols % 4 || ldx % 4 || ldx < ncols || ldy != ncols || degree < 1 ||
      !(e > 0.0) || lambda == c)
    return fail(ctx, SCSF_ERR_INVALID_ARG,
                "need ncols and ldx multiples of 4, ldy == ncols, valid filter parameters");
  const int n = op->n;
  const size_t N = (size_t)n * n;
  Carve cv(scratch, scratch_bytes);
  float* s0 = cv.take<float>(N * ncols);
  float* s1 = cv.take<float>(N * ncols);
  double* d = cv.take<double>(N);
  double* we = cv.take<double>(N);
  double* wn = cv.take<double>(N);
  float* d32 = cv.take<float>(N);
  float* we32 = cv.take<float>(N);
  float* wn32 = cv.take<float>(N);
  double* part = cv.take<double>(2 * (size_t)assemble_blocks(n));
  double* bnd = cv.take<double>(2);
  float* coefd = cv.take<float>(3 * (size_t)degree);
  if (!cv.ok) return fail(ctx, SCSF_ERR_NO_MEMORY, "scratch too small");
  SCSF_CUDA(ctx, cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  SCSF_CUDA(ctx, launch_assemble(op->kind, n, op->ax, op->ay, op->v, d, we, wn, part, bnd, st));
  SCSF_CUDA(ctx, launch_to_f32(d, d32, N, st));
  SCSF_CUDA(ctx, launch_to_f32(we, we32, N, st));
  SCSF_CUDA(ctx, launch_to_f32(wn, wn32, N, st));
  const Stencil32 A{d32, we32, wn32, n};
  // the cluster-resident filter where the grid fits, else one launch per step
  {
    std::vector<float> hc(3 * (size_t)degree);
    SCSF_CUDA(ctx, upload_filter_coefs(degree, lambda, c, e, hc.data(), coefd, st));
    const cudaError_t er = launch_cheb_filter_f32_resident(A, X, ldx, Y, ncols, ncols, degree, coefd, st);
    if (er == cudaSuccess) return SCSF_OK;
    if (er != cudaErrorNotSupported) SCSF_CUDA(ctx, er);
    cudaGetLastError();
  }
  // Y_i goes to rot[(i-1) % 3]; copy at the end if Y_m did not land in Y
  float* rot[3] = {s0, s1, Y};
  int which = 0;
  SCSF_CUDA(ctx, run_filter_f32(A, X, ldx, ncols, degree, lambda, c, e, rot, ncols, &which, st));
  if (rot[which] != Y)
    SCSF_CUDA(ctx, cudaMemcpyAsync(Y, rot[which], N * ncols * sizeof(float),
                                   cudaMemcpyDeviceToDevice, st));
  return SCSF_OK;
}

size_t scsf_cheb_filter_dc_scratch(int n, int ncols, int degree) {
  if (n < 1 || ncols < 1 || ncols > kMaxBlockWidth || degree < 1) return 0;
  SizeCarve sc;
  float *R, *z[3], *d32, *we32, *wn32, *ytab, *coef;
  double *d, *we, *wn, *part, *bnd, *rpart, *res2, *ym;
  int* gdeg;
  carve_filter_dc(sc, n, ncols, degree, &R, z, &d, &we, &wn, &d32, &we32, &wn32, &part, &bnd,
                  &rpart, &res2, &ytab, &ym, &coef, &gdeg);
  return sc.used + 256;
}

namespace {

// scsf_cheb_filter_dc, and with group_degrees (host) its per-column-group form.
scsf_status cheb_filter_dc(scsf_ctx* ctx, const scsf_operator* op, const double* X, int ldx,
                           const double* theta, int ncols, int degree, const int* group_degrees,
                           double lambda, double c, double e, double* Y, int ldy, void* scratch,
                           size_t scratch_bytes) {
  if (!ctx) return SCSF_ERR_INVALID_ARG;
  if (!op_ok(op) || !X || !Y || !theta || !scratch)
    return fail(ctx, SCSF_ERR_INVALID_ARG, "bad argument");
  if (op->kind == SCSF_OP_CSR || op->kind == SCSF_OP_PLATE)
    return fail(ctx, SCSF_ERR_INVALID_ARG,
                "the defect-corrected filter takes 5-point stencil operators only");
  if (ncols < 1 || ncols > kMaxBlockWidth || ldx < ncols || ldy < ncols || degree < 1 ||
      !(e > 0.0) || lambda == c)
    return fail(ctx, SCSF_ERR_INVALID_ARG, "need 1 <= ncols <= 512, ld >= ncols, valid filter parameters");
  const int groups = (ncols + 3) / 4;
  if (group_degrees) {
    for (int g = 0; g < groups; ++g)
      if (group_degrees[g] < 1 || group_degrees[g] > degree)
        return fail(ctx, SCSF_ERR_INVALID_ARG, "group degrees must lie in [1, degree]");
  }
  const int n = op->n;
  Carve cv(scratch, scratch_bytes);
  float *R, *z[3], *d32, *we32, *wn32, *ytab, *coef;
  double *d, *we, *wn, *part, *bnd, *rpart, *res2, *ym;
  int* gdeg;
  carve_filter_dc(cv, n, ncols, degree, &R, z, &d, &we, &wn, &d32, &we32, &wn32, &part, &bnd,
                  &rpart, &res2, &ytab, &ym, &coef, &gdeg);
  if (!cv.ok) return fail(ctx, SCSF_ERR_NO_MEMORY, "scratch too small");
  SCSF_CUDA(ctx, cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  const size_t N = (size_t)n * n;
  if (group_degrees)
    SCSF_CUDA(ctx, cudaMemcpyAsync(gdeg, group_degrees, groups * sizeof(int), cudaMemcpyHostToDevice, st));
  SCSF_CUDA(ctx, launch_assemble(op->kind, n, op->ax, op->ay, op->v, d, we, wn, part, bnd, st));
  SCSF_CUDA(ctx, launch_to_f32(d, d32, N, st));
  SCSF_CUDA(ctx, launch_to_f32(we, we32, N, st));
  SCSF_CUDA(ctx, launch_to_f32(wn, wn32, N, st));
  const Stencil A{d, we, wn, n};
  const Stencil32 A32{d32, we32, wn32, n};
  SCSF_CUDA(ctx, launch_residual_norms(A, X, ldx, ncols, theta, rpart, res2, st, R, ncols));
  std::vector<float> hcoef(3 * (size_t)degree);
  bool grouped = false;
  SCSF_CUDA(ctx, run_filter_dc(A32, X, ldx, R, ncols, theta, ncols, degree, lambda, c, e, z, ncols,
                               ytab, ym, Y, ldy, st, nullptr,
                               coef, hcoef.data(), group_degrees ? gdeg : nullptr, &grouped));
  SCSF_CUDA(ctx, cudaStreamSynchronize(st));  // hcoef is the source of an asynchronous copy
  if (group_degrees && !grouped)
    return fail(ctx, SCSF_ERR_INVALID_ARG,
                "per-group degrees need the cluster-resident filter (grid too large for shared memory)");
  return SCSF_OK;
}

}  // namespace

scsf_status scsf_cheb_filter_dc(scsf_ctx* ctx, const scsf_operator* op, const double* X, int ldx,
                                const double* theta, int ncols, int degree, double lambda,
                                double c, double e, double* Y, int ldy, void* scratch,
                                size_t scratch_bytes) {
  return cheb_filter_dc(ctx, op, X, ldx, theta, ncols, degree, nullptr, lambda, c, e, Y, ldy,
                        scratch, scratch_bytes);
}

scsf_status scsf_cheb_filter_dc_grouped(scsf_ctx* ctx, const scsf_operator* op, const double* X,
                                        int ldx, const double* theta, int ncols, int degree,
                                        const int* group_degrees, double lambda, double c,
                                        double e, double* Y, int ldy, void* scratch,
                                        size_t scratch_bytes) {
  if (!group_degrees) return ctx ? fail(ctx, SCSF_ERR_INVALID_ARG, "null group_degrees") : SCSF_ERR_INVALID_ARG;
  return cheb_filter_dc(ctx, op, X, ldx, theta, ncols, degree, group_degrees, lambda, c, e, Y, ldy,
                        scratch, scratch_bytes);
}

scsf_status scsf_block_rotate(scsf_ctx* ctx, const double* X, int ldx, int rows, int k,
                              const double* M, int ldm, int n, double* Y, int ldy) {
  if (!ctx) return SCSF_ERR_INVALID_ARG;
  if (!X || !M || !Y) return fail(ctx, SCSF_ERR_INVALID_ARG, "null pointer");
  if (rows < 1 || k < 1 || n < 1 || k > kMaxBlockWidth || n > kMaxBlockWidth || ldx < k ||
      ldm < n || ldy < n)
    return fail(ctx, SCSF_ERR_INVALID_ARG, "need 1 <= k, n <= 512 and leading dimensions >= widths");
  SCSF_CUDA(ctx, cudaSetDevice(ctx->device));
  SCSF_CUDA(ctx, launch_gemm_nn(rows, k, n, 1.0, X, ldx, M, ldm, 0.0, Y, ldy, false, ctx->stream));
  return SCSF_OK;
}

size_t scsf_block_product_scratch(int64_t rows, int kmax, int slices) {
  if (rows < 1 || rows > 0x7fffffffLL || kmax < 1 || kmax > kMaxBlockWidth) return 0;
  if (slices != 4 && slices != 7 && slices != 8) return 0;
  const size_t fp64 = gemm_tn_partials((int)rows, kmax, kmax, false) * sizeof(double);
  return 256 + std::max(fp64, oz_scratch_bytes((int)rows, kmax, slices));
}

}  // extern "C"

namespace {

// Validates a product call and carves its error flag; returns SCSF_OK or the failure.
scsf_status product_setup(scsf_ctx* ctx, int64_t rows, int w1, int w2, int method, int slices,
                          void* scratch, size_t scratch_bytes, int** err, void** rest,
                          size_t* rest_bytes) {
  if (rows < 1 || rows > 0x7fffffffLL || w1 < 1 || w2 < 1 || w1 > kMaxBlockWidth ||
      w2 > kMaxBlockWidth)
    return fail(ctx, SCSF_ERR_INVALID_ARG, "need 1 <= rows < 2^31 and widths in [1, 512]");
  if (method != SCSF_PRODUCT_TENSOR && method != SCSF_PRODUCT_FP64)
    return fail(ctx, SCSF_ERR_INVALID_ARG, "method must be SCSF_PRODUCT_TENSOR or SCSF_PRODUCT_FP64");
  if (method == SCSF_PRODUCT_TENSOR && slices != 4 && slices != 7 && slices != 8)
    return fail(ctx, SCSF_ERR_INVALID_ARG, "slices must be 4, 7 or 8");
  if (!scratch || reinterpret_cast<uintptr_t>(scratch) % 256 != 0)
    return fail(ctx, SCSF_ERR_INVALID_ARG, "scratch must be a 256-byte aligned device buffer");
  if (scratch_bytes < scsf_block_product_scratch(rows, std::max(w1, w2),
                                                 method == SCSF_PRODUCT_TENSOR ? slices : 7))
    return fail(ctx, SCSF_ERR_NO_MEMORY, "scratch smaller than scsf_block_product_scratch()");
  *err = static_cast<int*>(scratch);
  *rest = static_cast<char*>(scratch) + 256;
  *rest_bytes = scratch_bytes - 256;
  return SCSF_OK;
}

scsf_status product_finish(scsf_ctx* ctx, int* err) {
  int* h = reinterpret_cast<int*>(ctx->pinned);
  SCSF_CUDA(ctx, cudaMemcpyAsync(h, err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  SCSF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (h[0] != 0) return fail(ctx, SCSF_ERR_TIMEOUT, "a tensor-core product gave up waiting");
  return SCSF_OK;
}

}  // namespace

extern "C" {

scsf_status scsf_block_gram(scsf_ctx* ctx, const double* A, int lda, const double* B, int ldb,
                            int rows, int m, int n, int symmetric, int method, int slices,
                            double* C, int ldc, void* scratch, size_t scratch_bytes) {
  if (!ctx) return SCSF_ERR_INVALID_ARG;
  if (!A || !B || !C) return fail(ctx, SCSF_ERR_INVALID_ARG, "null pointer");
  int* err;
  void* rest;
  size_t rest_bytes;
  scsf_status s = product_setup(ctx, rows, m, n, method, slices, scratch, scratch_bytes, &err,
                                &rest, &rest_bytes);
  if (s != SCSF_OK) return s;
  if (lda < m || ldb < n || ldc < n || (symmetric && m != n))
    return fail(ctx, SCSF_ERR_INVALID_ARG, "need lda >= m, ldb >= n, ldc >= n (symmetric: m == n)");
  SCSF_CUDA(ctx, cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  SCSF_CUDA(ctx, cudaMemsetAsync(err, 0, sizeof(int), st));
  if (method == SCSF_PRODUCT_TENSOR)
    SCSF_CUDA(ctx, launch_gemm_tn_oz(rows, m, n, A, lda, B, ldb, C, ldc, symmetric != 0, slices,
                                     rest, rest_bytes, err, st));
  else
    SCSF_CUDA(ctx, launch_gemm_tn(rows, m, n, A, lda, B, ldb, C, ldc, symmetric != 0,
                                  static_cast<double*>(rest), st));
  return product_finish(ctx, err);
}

scsf_status scsf_block_gram_kernel_time(scsf_ctx* ctx, const double* X, int ldx, int rows, int m,
                                        int reps, void* scratch, size_t scratch_bytes,
                                        float* ms_host) {
  if (!ctx) return SCSF_ERR_INVALID_ARG;
  if (!X || !ms_host) return fail(ctx, SCSF_ERR_INVALID_ARG, "null pointer");
  int* err;
  void* rest;
  size_t rest_bytes;
  scsf_status s = product_setup(ctx, rows, m, m, SCSF_PRODUCT_TENSOR, 8, scratch, scratch_bytes,
                                &err, &rest, &rest_bytes);
  if (s != SCSF_OK) return s;
  if (ldx < m || reps < 1) return fail(ctx, SCSF_ERR_INVALID_ARG, "need ldx >= m and reps >= 1");
  SCSF_CUDA(ctx, cudaSetDevice(ctx->device));
  SCSF_CUDA(ctx, cudaMemsetAsync(err, 0, sizeof(int), ctx->stream));
  SCSF_CUDA(ctx, time_gemm_tn_oz(rows, m, X, ldx, 8, rest, rest_bytes, err, reps, ctx->stream,
                                 ms_host));
  return product_finish(ctx, err);
}

scsf_status scsf_block_rotate_ex(scsf_ctx* ctx, const double* X, int ldx, int rows, int k,
                                 const double* M, int ldm, int n, double alpha, double beta,
                                 int method, int slices, double* Y, int ldy, void* scratch,
                                 size_t scratch_bytes) {
  if (!ctx) return SCSF_ERR_INVALID_ARG;
  if (!X || !M || !Y) return fail(ctx, SCSF_ERR_INVALID_ARG, "null pointer");
  int* err;
  void* rest;
  size_t rest_bytes;
  scsf_status s = product_setup(ctx, rows, k, n, method, slices, scratch, scratch_bytes, &err,
                                &rest, &rest_bytes);
  if (s != SCSF_OK) return s;
  if (ldx < k || ldm < n || ldy < n)
    return fail(ctx, SCSF_ERR_INVALID_ARG, "need ldx >= k, ldm >= n, ldy >= n");
  SCSF_CUDA(ctx, cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  SCSF_CUDA(ctx, cudaMemsetAsync(err, 0, sizeof(int), st));
  if (method == SCSF_PRODUCT_TENSOR)
    SCSF_CUDA(ctx, launch_gemm_nn_oz(rows, k, n, alpha, X, ldx, M, ldm, beta, Y, ldy, slices, rest,
                                     rest_bytes, err, st));
  else
    SCSF_CUDA(ctx, launch_gemm_nn(rows, k, n, alpha, X, ldx, M, ldm, beta, Y, ldy, false, st));
  return product_finish(ctx, err);
}

}  // extern "C"

namespace {

template <typename Cv>
void carve_cholqr2(Cv& cv, int rows, int ncols, double** G, double** L, double** Rinv,
                   double** partials, double** F, void** wide, int** status) {
  const size_t kk = (size_t)ncols * ncols;
  *G = cv.template take<double>(kk);
  *L = cv.template take<double>(kk);
  *Rinv = cv.template take<double>(kk);
  *partials = cv.template take<double>(gemm_tn_partials(rows, ncols, ncols, true));
  *F = cv.template take<double>((size_t)rows * ncols);
  *wide = (ncols > kSmallBlockWidth) ? (void*)cv.template take<char>(chol_wide_scratch_bytes(ncols))
                                     : nullptr;
  *status = cv.template take<int>(2);
}

}  // namespace

extern "C" {

size_t scsf_cholqr2_scratch(int rows, int ncols) {
  if (rows < 1 || ncols < 1 || ncols > kMaxBlockWidth || ncols > rows) return 0;
  SizeCarve sc;
  double *G, *L, *Rinv, *partials, *F;
  void* wide;
  int* status;
  carve_cholqr2(sc, rows, ncols, &G, &L, &Rinv, &partials, &F, &wide, &status);
  return sc.used;
}

scsf_status scsf_cholqr2(scsf_ctx* ctx, const double* X, int ldx, int rows, int ncols, double* Q,
                         int ldq, int* shifts_host, void* scratch, size_t scratch_bytes) {
  if (!ctx) return SCSF_ERR_INVALID_ARG;
  if (!X || !Q || !scratch) return fail(ctx, SCSF_ERR_INVALID_ARG, "null pointer");
  if (rows < 1 || ncols < 1 || ncols > kMaxBlockWidth || ncols > rows || ldx < ncols || ldq < ncols)
    return fail(ctx, SCSF_ERR_INVALID_ARG, "need 1 <= ncols <= min(rows, 512), ld >= ncols");
  Carve cv(scratch, scratch_bytes);
  double *G, *L, *Rinv, *partials, *F;
  void* wide;
  int* status;
  carve_cholqr2(cv, rows, ncols, &G, &L, &Rinv, &partials, &F, &wide, &status);
  if (!cv.ok) return fail(ctx, SCSF_ERR_NO_MEMORY, "scratch too small");
  SCSF_CUDA(ctx, cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  // pass 1 (FP32 factor of the FP64 Gram matrix) into F, pass 2 (FP64) into Q
  SCSF_CUDA(ctx, launch_gemm_tn(rows, ncols, ncols, X, ldx, X, ldx, G, ncols, true, partials, st));
  SCSF_CUDA(ctx, launch_chol_rinv(ncols, G, ncols, true, L, Rinv, status, st, wide));
  SCSF_CUDA(ctx, launch_gemm_nn(rows, ncols, ncols, 1.0, X, ldx, Rinv, ncols, 0.0, F, ncols, true, st));
  SCSF_CUDA(ctx, launch_gemm_tn(rows, ncols, ncols, F, ncols, F, ncols, G, ncols, true, partials, st));
  SCSF_CUDA(ctx, launch_chol_rinv(ncols, G, ncols, false, L, Rinv, status + 1, st, wide));
  SCSF_CUDA(ctx, launch_gemm_nn(rows, ncols, ncols, 1.0, F, ncols, Rinv, ncols, 0.0, Q, ldq, true, st));
  int* h = reinterpret_cast<int*>(ctx->pinned);
  SCSF_CUDA(ctx, cudaMemcpyAsync(h, status, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
  SCSF_CUDA(ctx, cudaStreamSynchronize(st));
  if (shifts_host) {
    shifts_host[0] = h[0];
    shifts_host[1] = h[1];
  }
  if (h[0] >= 1000 || h[1] >= 1000)
    return fail(ctx, SCSF_ERR_BREAKDOWN, "Cholesky QR broke down even with a shift");
  return SCSF_OK;
}

size_t scsf_small_eigh_scratch(int k) {
  if (k < 1 || k > kMaxBlockWidth) return 0;
  return small_eigh_scratch_bytes(k);
}

scsf_status scsf_small_eigh(scsf_ctx* ctx, const double* S, int k, double* evals, double* Z,
                            void* scratch, size_t scratch_bytes) {
  if (!ctx) return SCSF_ERR_INVALID_ARG;
  if (!S || !evals || !Z || !scratch) return fail(ctx, SCSF_ERR_INVALID_ARG, "null pointer");
  if (k < 1 || k > kMaxBlockWidth) return fail(ctx, SCSF_ERR_INVALID_ARG, "k out of range");
  if (scratch_bytes < small_eigh_scratch_bytes(k))
    return fail(ctx, SCSF_ERR_NO_MEMORY, "scratch too small");
  SCSF_CUDA(ctx, cudaSetDevice(ctx->device));
  SCSF_CUDA(ctx, launch_small_eigh(k, S, k, evals, Z, k, scratch, ctx->stream));
  return SCSF_OK;
}

}  // extern "C"
