// Operator assembly and the fused 5-point stencil kernels (FP64 path).
//
// Sec. 2.1 / App. D.2: the operator is the conservative central-difference
// discretisation of -div(a grad u) (or -Lap u + V u) on the n x n interior grid
// with Dirichlet boundaries; it is never formed as a sparse matrix. Each kernel
// reads the three coefficient arrays d/we/wn and the block rows it needs.
#include "kernels.cuh"

namespace scsf {
namespace {

// min / max that keep a NaN (fmin / fmax drop one), so a non-finite operator coefficient
// reaches the Gershgorin bounds, where the chain rejects the operator.
__device__ __forceinline__ double nan_min(double a, double b) {
  return (isnan(a) || isnan(b)) ? a + b : fmin(a, b);
}
__device__ __forceinline__ double nan_max(double a, double b) {
  return (isnan(a) || isnan(b)) ? a + b : fmax(a, b);
}


constexpr int kAsmThreads = 256;
constexpr int kRowsPerBlock = 8;   // nodes per CTA in the stencil kernels (blockDim.y)
constexpr int kMaxColChunks = kSmallBlockWidth / 32;  // per column slice (blockIdx.y)

__global__ void assemble_kernel(int kind, int n, const double* __restrict__ ax,
                                const double* __restrict__ ay, const double* __restrict__ v,
                                double* __restrict__ d, double* __restrict__ we,
                                double* __restrict__ wn, double* __restrict__ partials) {
  const int N = n * n;
  const double h = 1.0 / (n + 1);
  const double inv_h2 = 1.0 / (h * h);
  double lo = INFINITY, hi = -INFINITY;
  for (int I = blockIdx.x * blockDim.x + threadIdx.x; I < N; I += gridDim.x * blockDim.x) {
    const int i = I / n, j = I - (I / n) * n;
    double a_w, a_e, a_s, a_n, extra;
    if (kind == 0) {
      a_w = ax[(size_t)i * n + j];            // face between (i-1, j) and (i, j)
      a_e = ax[(size_t)(i + 1) * n + j];      // face between (i, j) and (i+1, j)
      a_s = ay[(size_t)i * (n + 1) + j];      // face between (i, j-1) and (i, j)
      a_n = ay[(size_t)i * (n + 1) + j + 1];  // face between (i, j) and (i, j+1)
      extra = 0.0;
    } else {
      a_w = a_e = a_s = a_n = 1.0;
      extra = v[I];
    }
    const double dI = (a_w + a_e + a_s + a_n) * inv_h2 + extra;
    const double cE = (i < n - 1) ? a_e * inv_h2 : 0.0;
    const double cW = (i > 0) ? a_w * inv_h2 : 0.0;
    const double cN = (j < n - 1) ? a_n * inv_h2 : 0.0;
    const double cS = (j > 0) ? a_s * inv_h2 : 0.0;
    d[I] = dI;
    we[I] = cE;
    wn[I] = cN;
    const double radius = cE + cW + cN + cS;
    lo = nan_min(lo, dI - radius);
    hi = nan_max(hi, dI + radius);
  }
  __shared__ double slo[kAsmThreads], shi[kAsmThreads];
  slo[threadIdx.x] = lo;
  shi[threadIdx.x] = hi;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      slo[threadIdx.x] = nan_min(slo[threadIdx.x], slo[threadIdx.x + s]);
      shi[threadIdx.x] = nan_max(shi[threadIdx.x], shi[threadIdx.x + s]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = slo[0];
    partials[gridDim.x + blockIdx.x] = shi[0];
  }
}

__global__ void bounds_reduce_kernel(const double* __restrict__ partials, int nb,
                                     double* __restrict__ bounds) {
  __shared__ double slo[256], shi[256];
  double lo = INFINITY, hi = -INFINITY;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    lo = nan_min(lo, partials[b]);
    hi = nan_max(hi, partials[nb + b]);
  }
  slo[threadIdx.x] = lo;
  shi[threadIdx.x] = hi;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      slo[threadIdx.x] = nan_min(slo[threadIdx.x], slo[threadIdx.x + s]);
      shi[threadIdx.x] = nan_max(shi[threadIdx.x], shi[threadIdx.x + s]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    bounds[0] = slo[0];
    bounds[1] = shi[0];
  }
}

// Gershgorin bounds of a CSR matrix: per row the diagonal entry -/+ the sum of the
// off-diagonal magnitudes, reduced per CTA into partials [gridDim][2].
__global__ void csr_bounds_kernel(int rows, const int* __restrict__ rp, const int* __restrict__ ci,
                                  const double* __restrict__ val, double* __restrict__ partials) {
  double lo = INFINITY, hi = -INFINITY;
  for (int I = blockIdx.x * blockDim.x + threadIdx.x; I < rows; I += gridDim.x * blockDim.x) {
    double dI = 0.0, radius = 0.0;
    for (int p = rp[I]; p < rp[I + 1]; ++p) {
      if (ci[p] == I) dI += val[p];
      else radius += fabs(val[p]);
    }
    lo = nan_min(lo, dI - radius);
    hi = nan_max(hi, dI + radius);
  }
  __shared__ double slo[kAsmThreads], shi[kAsmThreads];
  slo[threadIdx.x] = lo;
  shi[threadIdx.x] = hi;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      slo[threadIdx.x] = nan_min(slo[threadIdx.x], slo[threadIdx.x + s]);
      shi[threadIdx.x] = nan_max(shi[threadIdx.x], shi[threadIdx.x + s]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = slo[0];
    partials[gridDim.x + blockIdx.x] = shi[0];
  }
}

// Thin-plate operator (App. D.2 item 4) in symmetric standard form C = S K S, K = L diag(D) L,
// S = diag(rho)^(-1/2), L = -Lap_h with Dirichlet rows (u = 0 and D lap u = 0 on the boundary:
// the simply supported plate). Row I = (i, j) couples the 13 nodes with |di| + |dj| <= 2:
//   C_IK = s_I s_K / h^4 sum_J l_IJ D_J l_JK,  l = h^2 L (4 on the diagonal, -1 to each
// interior neighbour), J over I and its interior neighbours. Fixed 13 slots per row
// (row_ptr[I] = 13 I) in ascending column order; slots outside the grid hold (col I, 0).
__device__ __forceinline__ double plate_l(int pi, int pj, int qi, int qj) {
  const int d = abs(pi - qi) + abs(pj - qj);
  return d == 0 ? 4.0 : (d == 1 ? -1.0 : 0.0);
}

__global__ void plate_csr_kernel(int n, const double* __restrict__ D, const double* __restrict__ rho,
                                 int* __restrict__ rp, int* __restrict__ ci,
                                 double* __restrict__ val) {
  const int N = n * n;
  const double h2 = 1.0 / ((double)(n + 1) * (n + 1));
  const double inv_h4 = 1.0 / (h2 * h2);
  constexpr int kOff[13][2] = {{-2, 0}, {-1, -1}, {-1, 0}, {-1, 1}, {0, -2}, {0, -1}, {0, 0},
                               {0, 1},  {0, 2},   {1, -1}, {1, 0},  {1, 1},  {2, 0}};
  constexpr int kNb[5][2] = {{0, 0}, {-1, 0}, {0, -1}, {0, 1}, {1, 0}};
  for (int I = blockIdx.x * blockDim.x + threadIdx.x; I < N; I += gridDim.x * blockDim.x) {
    const int i = I / n, j = I - i * n;
    const double sI = 1.0 / sqrt(rho[I]);
    rp[I] = 13 * I;
    if (I == N - 1) rp[N] = 13 * N;
    for (int q = 0; q < 13; ++q) {
      const int ki = i + kOff[q][0], kj = j + kOff[q][1];
      double v = 0.0;
      int col = I;
      if (ki >= 0 && ki < n && kj >= 0 && kj < n) {
        col = ki * n + kj;
        double acc = 0.0;
        for (int t = 0; t < 5; ++t) {
          const int ji = i + kNb[t][0], jj = j + kNb[t][1];
          if (ji < 0 || ji >= n || jj < 0 || jj >= n) continue;
          const double lk = plate_l(ji, jj, ki, kj);
          if (lk != 0.0) acc += plate_l(i, j, ji, jj) * D[ji * n + jj] * lk;
        }
        v = sI * (1.0 / sqrt(rho[col])) * acc * inv_h4;
      }
      ci[13 * I + q] = col;
      val[13 * I + q] = v;
    }
  }
}

// (A y)_I for one column: y points at row I of the block (element c).
struct NodeCoeffs {
  double d, wE, wW, wN, wS;
  int i, j;
};

__device__ __forceinline__ NodeCoeffs load_coeffs(const Stencil& A, int I) {
  NodeCoeffs k;
  const int n = A.n;
  k.i = I / n;
  k.j = I - k.i * n;
  k.d = A.d[I];
  k.wE = A.we[I];
  k.wW = (k.i > 0) ? A.we[I - n] : 0.0;
  k.wN = A.wn[I];
  k.wS = (k.j > 0) ? A.wn[I - 1] : 0.0;
  return k;
}

// Off-diagonal part sum_nb w_nb y_nb for column c of the row at `row` (ld elements per row).
__device__ __forceinline__ double offdiag_sum(const NodeCoeffs& k, int n, const double* row,
                                              size_t ld, int c) {
  double acc = 0.0;
  if (k.i < n - 1) acc = fma(k.wE, row[(size_t)n * ld + c], acc);
  if (k.i > 0) acc = fma(k.wW, row[-(ptrdiff_t)((size_t)n * ld) + c], acc);
  if (k.j < n - 1) acc = fma(k.wN, row[ld + c], acc);
  if (k.j > 0) acc = fma(k.wS, row[-(ptrdiff_t)ld + c], acc);
  return acc;
}

__global__ void __launch_bounds__(32 * kRowsPerBlock)
cheb_step_f64_kernel(Stencil A, const double* __restrict__ cur, int ldc,
                     const double* __restrict__ prev, int ldp, double* __restrict__ out, int ldo,
                     int ncols, double s1, double s2, double s3) {
  const int N = stencil_rows(A);
  const int I = blockIdx.x * kRowsPerBlock + threadIdx.y;
  if (I >= N) return;
  if (A.rp) {  // CSR: out = s1 (A cur) + s2 cur + s3 prev, A cur = sum over the row's entries
    const int p0 = A.rp[I], p1 = A.rp[I + 1];
    const double* row = cur + (size_t)I * ldc;
    const double* prow = prev ? prev + (size_t)I * ldp : nullptr;
    double* orow = out + (size_t)I * ldo;
    for (int c = threadIdx.x; c < ncols; c += 32) {
      double acc = 0.0;
      for (int p = p0; p < p1; ++p) acc = fma(A.val[p], cur[(size_t)A.ci[p] * ldc + c], acc);
      double r = fma(s1, acc, s2 * row[c]);
      if (prow) r = fma(s3, prow[c], r);
      orow[c] = r;
    }
    return;
  }
  const NodeCoeffs k = load_coeffs(A, I);
  const double diag = fma(s1, k.d, s2);
  const double* row = cur + (size_t)I * ldc;
  const double* prow = prev ? prev + (size_t)I * ldp : nullptr;
  double* orow = out + (size_t)I * ldo;
  for (int c = threadIdx.x; c < ncols; c += 32) {
    const double acc = offdiag_sum(k, A.n, row, (size_t)ldc, c);
    double r = fma(-s1, acc, diag * row[c]);
    if (prow) r = fma(s3, prow[c], r);
    orow[c] = r;
  }
}

__global__ void __launch_bounds__(32 * kRowsPerBlock)
residual_norms_kernel(Stencil A, const double* __restrict__ X, int ldx, int ncols,
                      const double* __restrict__ theta, double* __restrict__ partials,
                      float* __restrict__ R32, int ldr) {
  const int N = stencil_rows(A);
  const int c0 = blockIdx.y * kSmallBlockWidth;  // this CTA's column slice
  double rr[kMaxColChunks], aa[kMaxColChunks];
#pragma unroll
  for (int q = 0; q < kMaxColChunks; ++q) rr[q] = aa[q] = 0.0;
  for (int I = blockIdx.x * kRowsPerBlock + threadIdx.y; I < N; I += gridDim.x * kRowsPerBlock) {
    const NodeCoeffs k = A.rp ? NodeCoeffs{} : load_coeffs(A, I);
    const double* row = X + (size_t)I * ldx;
#pragma unroll
    for (int q = 0; q < kMaxColChunks; ++q) {
      const int c = c0 + threadIdx.x + 32 * q;
      if (c < ncols) {
        const double x = row[c];
        double ax;
        if (A.rp) {
          ax = 0.0;
          for (int p = A.rp[I]; p < A.rp[I + 1]; ++p)
            ax = fma(A.val[p], X[(size_t)A.ci[p] * ldx + c], ax);
        } else {
          ax = fma(k.d, x, -offdiag_sum(k, A.n, row, (size_t)ldx, c));
        }
        const double r = fma(-theta[c], x, ax);
        if (R32) R32[(size_t)I * ldr + c] = (float)r;
        rr[q] = fma(r, r, rr[q]);
        aa[q] = fma(ax, ax, aa[q]);
      }
    }
  }
  __shared__ double s_r[kRowsPerBlock][kSmallBlockWidth];
  __shared__ double s_a[kRowsPerBlock][kSmallBlockWidth];
#pragma unroll
  for (int q = 0; q < kMaxColChunks; ++q) {
    const int lc = threadIdx.x + 32 * q;
    s_r[threadIdx.y][lc] = rr[q];
    s_a[threadIdx.y][lc] = aa[q];
  }
  __syncthreads();
  if (threadIdx.y == 0) {
    for (int lc = threadIdx.x; lc < kSmallBlockWidth && c0 + lc < ncols; lc += 32) {
      double sr = 0.0, sa = 0.0;
      for (int y = 0; y < kRowsPerBlock; ++y) {
        sr += s_r[y][lc];
        sa += s_a[y][lc];
      }
      partials[((size_t)blockIdx.x * 2 + 0) * ncols + c0 + lc] = sr;
      partials[((size_t)blockIdx.x * 2 + 1) * ncols + c0 + lc] = sa;
    }
  }
}

// out2[t] = sum over the nb per-block partials, t < 2 ncols: one warp per output, the lanes
// striding over the blocks (many loads in flight), then a fixed-order shuffle tree.
__global__ void column_partials_reduce_kernel(const double* __restrict__ partials, int nb,
                                              int ncols, double* __restrict__ out2) {
  const int t = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (t >= 2 * ncols) return;
  const int which = t / ncols, c = t - which * ncols;
  double s = 0.0;
  for (int b = lane; b < nb; b += 32) s += partials[((size_t)b * 2 + which) * ncols + c];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) out2[t] = s;
}

}  // namespace

int assemble_blocks_rows(long long N) {
  long long b = (N + kAsmThreads - 1) / kAsmThreads;
  return (int)(b < 304 ? b : 304);
}

int assemble_blocks(int n) { return assemble_blocks_rows((long long)n * n); }

cudaError_t launch_plate_csr(int n, const double* D, const double* rho, int* rp, int* ci,
                             double* val, cudaStream_t st) {
  plate_csr_kernel<<<assemble_blocks(n), kAsmThreads, 0, st>>>(n, D, rho, rp, ci, val);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_csr_bounds(int rows, const int* rp, const int* ci, const double* val,
                              double* partials, double* bounds, cudaStream_t st) {
  const int nb = assemble_blocks_rows(rows);
  csr_bounds_kernel<<<nb, kAsmThreads, 0, st>>>(rows, rp, ci, val, partials);
  note_launch();
  bounds_reduce_kernel<<<1, 256, 0, st>>>(partials, nb, bounds);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_assemble(int kind, int n, const double* ax, const double* ay, const double* v,
                            double* d, double* we, double* wn, double* partials, double* bounds,
                            cudaStream_t st) {
  const int nb = assemble_blocks(n);
  assemble_kernel<<<nb, kAsmThreads, 0, st>>>(kind, n, ax, ay, v, d, we, wn, partials);
  note_launch();
  bounds_reduce_kernel<<<1, 256, 0, st>>>(partials, nb, bounds);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_cheb_step_f64(const Stencil& A, const double* cur, int ldc, const double* prev,
                                 int ldp, double* out, int ldo, int ncols, double s1, double s2,
                                 double s3, cudaStream_t st) {
  const int N = stencil_rows(A);
  dim3 block(32, kRowsPerBlock);
  dim3 grid((N + kRowsPerBlock - 1) / kRowsPerBlock);
  cheb_step_f64_kernel<<<grid, block, 0, st>>>(A, cur, ldc, (s3 != 0.0) ? prev : nullptr, ldp, out,
                                               ldo, ncols, s1, s2, s3);
  note_launch();
  return cudaGetLastError();
}

int resid_blocks_rows(long long N) {
  long long b = (N + kRowsPerBlock - 1) / kRowsPerBlock;
  return (int)(b < 304 ? b : 304);
}

int resid_blocks(int n) { return resid_blocks_rows((long long)n * n); }

cudaError_t launch_residual_norms(const Stencil& A, const double* X, int ldx, int ncols,
                                  const double* theta, double* partials, double* out2,
                                  cudaStream_t st, float* R32, int ldr) {
  if (ncols > kMaxBlockWidth || (R32 && ldr < ncols)) return cudaErrorInvalidValue;
  const int nb = resid_blocks_rows(stencil_rows(A));
  const dim3 grid(nb, (ncols + kSmallBlockWidth - 1) / kSmallBlockWidth);
  residual_norms_kernel<<<grid, dim3(32, kRowsPerBlock), 0, st>>>(A, X, ldx, ncols, theta,
                                                                  partials, R32, ldr);
  note_launch();
  column_partials_reduce_kernel<<<(2 * ncols + 3) / 4, 128, 0, st>>>(partials, nb, ncols, out2);
  note_launch();
  return cudaGetLastError();
}

}  // namespace scsf
