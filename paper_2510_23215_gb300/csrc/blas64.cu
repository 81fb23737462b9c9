// FP64 block kernels for the plain path: tall-skinny Gram / projection
// products (Alg. 3, orthonormalisation to eigensolve), block rotation, Cholesky + triangular inverse.
//
// GB300 executes FP64 at about 2 FMA/clk/SM, so these kernels are bound by
// the FP64 pipe, not by memory: they spread the work over all SMs (split-K
// for the N-long reductions) and skip the zero half of triangular operands.
#include <algorithm>

#include "kernels.cuh"

namespace scsf {
namespace {

constexpr int TS = kGemmTile;  // 32

// ---- C = A^T B, split over rows into chunks --------------------------------
__device__ __forceinline__ void sym_tile_from_index(int t, int T, int& ti, int& tj) {
  ti = 0;
  while (t >= T - ti) {
    t -= T - ti;
    ++ti;
  }
  tj = ti + t;
}

__global__ void __launch_bounds__(256)
gemm_tn_partial_kernel(int rows, int m, int n, const double* __restrict__ A, int lda,
                       const double* __restrict__ B, int ldb, bool symmetric, int chunk_rows,
                       double* __restrict__ partials) {
  __shared__ double As[TS][TS + 1];
  __shared__ double Bs[TS][TS + 1];
  int ti, tj;
  if (symmetric) {
    sym_tile_from_index(blockIdx.x, (m + TS - 1) / TS, ti, tj);
  } else {
    const int tn = (n + TS - 1) / TS;
    ti = blockIdx.x / tn;
    tj = blockIdx.x - ti * tn;
  }
  const int i0 = ti * TS, j0 = tj * TS;
  const int r_begin = blockIdx.y * chunk_rows;
  const int r_end = min(rows, r_begin + chunk_rows);
  const int t = threadIdx.x;
  const int ty = t >> 4, tx = t & 15;
  double acc[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
  for (int r0 = r_begin; r0 < r_end; r0 += TS) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = t + 256 * q;       // 0..1023
      const int rr = e >> 5, cc = e & 31;
      const int r = r0 + rr;
      const bool rin = r < r_end;
      As[rr][cc] = (rin && i0 + cc < m) ? A[(size_t)r * lda + i0 + cc] : 0.0;
      Bs[rr][cc] = (rin && j0 + cc < n) ? B[(size_t)r * ldb + j0 + cc] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int rr = 0; rr < TS; ++rr) {
      const double a0 = As[rr][2 * ty], a1 = As[rr][2 * ty + 1];
      const double b0 = Bs[rr][2 * tx], b1 = Bs[rr][2 * tx + 1];
      acc[0][0] = fma(a0, b0, acc[0][0]);
      acc[0][1] = fma(a0, b1, acc[0][1]);
      acc[1][0] = fma(a1, b0, acc[1][0]);
      acc[1][1] = fma(a1, b1, acc[1][1]);
    }
    __syncthreads();
  }
  double* P = partials + (size_t)blockIdx.y * m * n;
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const int i = i0 + 2 * ty + a, j = j0 + 2 * tx + b;
      if (i < m && j < n) P[(size_t)i * n + j] = acc[a][b];
    }
}

__global__ void gemm_tn_reduce_kernel(int m, int n, int nchunk, bool symmetric,
                                      const double* __restrict__ partials, double* __restrict__ C,
                                      int ldc) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m * n) return;
  int i = e / n, j = e - (e / n) * n;
  int si = i, sj = j;
  if (symmetric && i > j) { si = j; sj = i; }
  double s = 0.0;
  for (int c = 0; c < nchunk; ++c) s += partials[(size_t)c * m * n + (size_t)si * n + sj];
  C[(size_t)i * ldc + j] = s;
}

struct TnPlan {
  int ntiles, nchunk, chunk_rows;
};

TnPlan plan_tn(int rows, int m, int n, bool symmetric) {
  TnPlan p;
  const int tm = (m + TS - 1) / TS, tn = (n + TS - 1) / TS;
  p.ntiles = symmetric ? tm * (tm + 1) / 2 : tm * tn;
  const int max_chunks = std::max(1, (rows + TS - 1) / TS);
  int want = (kSplitTarget + p.ntiles - 1) / p.ntiles;
  want = std::max(1, std::min(want, max_chunks));
  int cr = (rows + want - 1) / want;
  cr = ((cr + TS - 1) / TS) * TS;
  p.chunk_rows = std::max(cr, TS);
  p.nchunk = (rows + p.chunk_rows - 1) / p.chunk_rows;
  if (p.nchunk < 1) p.nchunk = 1;
  return p;
}

// ---- C = alpha A M + beta C -------------------------------------------------
template <int BM, int BN>
__global__ void __launch_bounds__(256)
gemm_nn_kernel(int rows, int K, int n, double alpha, const double* __restrict__ A, int lda,
               const double* __restrict__ M, int ldm, double beta, double* C, int ldc,
               bool upper) {
  constexpr int BK = 32;
  constexpr int RM = BM / 16, RN = BN / 16;  // outputs per thread
  __shared__ double As[BM][BK + 1];
  __shared__ double Ms[BK][BN + 1];
  const int r0 = blockIdx.y * BM, j0 = blockIdx.x * BN;
  const int t = threadIdx.x, ty = t >> 4, tx = t & 15;
  double acc[RM][RN];
#pragma unroll
  for (int a = 0; a < RM; ++a)
#pragma unroll
    for (int b = 0; b < RN; ++b) acc[a][b] = 0.0;
  const int k_end = upper ? min(K, j0 + BN) : K;
  for (int k0 = 0; k0 < k_end; k0 += BK) {
    for (int e = t; e < BM * BK; e += 256) {
      const int rr = e / BK, kk = e - (e / BK) * BK;
      const int r = r0 + rr, kc = k0 + kk;
      As[rr][kk] = (r < rows && kc < K) ? A[(size_t)r * lda + kc] : 0.0;
    }
    for (int e = t; e < BK * BN; e += 256) {
      const int kk = e / BN, jj = e - (e / BN) * BN;
      const int kc = k0 + kk, j = j0 + jj;
      Ms[kk][jj] = (kc < K && j < n) ? M[(size_t)kc * ldm + j] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < BK; ++kk) {
      double av[RM], mv[RN];
#pragma unroll
      for (int a = 0; a < RM; ++a) av[a] = As[ty + 16 * a][kk];
#pragma unroll
      for (int b = 0; b < RN; ++b) mv[b] = Ms[kk][tx + 16 * b];
#pragma unroll
      for (int a = 0; a < RM; ++a)
#pragma unroll
        for (int b = 0; b < RN; ++b) acc[a][b] = fma(av[a], mv[b], acc[a][b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < RM; ++a)
#pragma unroll
    for (int b = 0; b < RN; ++b) {
      const int r = r0 + ty + 16 * a, j = j0 + tx + 16 * b;
      if (r < rows && j < n) {
        double* c = C + (size_t)r * ldc + j;
        *c = (beta == 0.0) ? alpha * acc[a][b] : fma(alpha, acc[a][b], beta * (*c));
      }
    }
}

// Small outputs (the k_b x k_b products of the eigensolve's refinement): 8 x 8 tiles of 64
// threads, one output each, so a 120 x 120 result spreads over 225 CTAs instead of 64 (the
// FP64 pipe, 2 FMA per clock per SM, is the bound, and it is per SM).
__global__ void __launch_bounds__(64)
gemm_nn_small_kernel(int rows, int K, int n, double alpha, const double* __restrict__ A, int lda,
                     const double* __restrict__ M, int ldm, double beta, double* C, int ldc,
                     bool upper) {
  constexpr int T = 8, BK = 32;
  __shared__ double As[T][BK + 1];
  __shared__ double Ms[BK][T + 1];
  const int r0 = blockIdx.y * T, j0 = blockIdx.x * T;
  const int t = threadIdx.x, ty = t >> 3, tx = t & 7;
  double acc = 0.0;
  const int k_end = upper ? min(K, j0 + T) : K;
  for (int k0 = 0; k0 < k_end; k0 += BK) {
    for (int e = t; e < T * BK; e += 64) {
      const int rr = e / BK, kk = e - rr * BK;
      const int r = r0 + rr, kc = k0 + kk;
      As[rr][kk] = (r < rows && kc < K) ? A[(size_t)r * lda + kc] : 0.0;
      const int k2 = e / T, jj = e - k2 * T;
      const int kc2 = k0 + k2, j = j0 + jj;
      Ms[k2][jj] = (kc2 < K && j < n) ? M[(size_t)kc2 * ldm + j] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < BK; ++kk) acc = fma(As[ty][kk], Ms[kk][tx], acc);
    __syncthreads();
  }
  const int r = r0 + ty, j = j0 + tx;
  if (r < rows && j < n) {
    double* c = C + (size_t)r * ldc + j;
    *c = (beta == 0.0) ? alpha * acc : fma(alpha, acc, beta * (*c));
  }
}

__global__ void copy2d_kernel(int rows, int cols, const double* __restrict__ in, int ld_in,
                              double* __restrict__ out, int ld_out) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)rows * cols) return;
  const int r = (int)(e / cols), c = (int)(e - (e / cols) * cols);
  out[(size_t)r * ld_out + c] = in[(size_t)r * ld_in + c];
}

__global__ void gather_cols_kernel(int rows, int ncols, const double* __restrict__ in, int ld_in,
                                   const int* __restrict__ cols, double* __restrict__ out,
                                   int ld_out) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)rows * ncols) return;
  const int r = (int)(e / ncols), c = (int)(e - (e / ncols) * ncols);
  out[(size_t)r * ld_out + c] = in[(size_t)r * ld_in + cols[c]];
}

}  // namespace

size_t gemm_tn_partials(int rows, int m, int n, bool symmetric) {
  TnPlan p = plan_tn(rows, m, n, symmetric);
  return (size_t)p.nchunk * m * n;
}

cudaError_t launch_gemm_tn(int rows, int m, int n, const double* A, int lda, const double* B,
                           int ldb, double* C, int ldc, bool symmetric, double* partials,
                           cudaStream_t st) {
  if (m <= 0 || n <= 0) return cudaSuccess;
  if (symmetric && m != n) return cudaErrorInvalidValue;
  TnPlan p = plan_tn(rows, m, n, symmetric);
  dim3 grid(p.ntiles, p.nchunk);
  gemm_tn_partial_kernel<<<grid, 256, 0, st>>>(rows, m, n, A, lda, B, ldb, symmetric,
                                               p.chunk_rows, partials);
  note_launch();
  const int tot = m * n;
  gemm_tn_reduce_kernel<<<(tot + 255) / 256, 256, 0, st>>>(m, n, p.nchunk, symmetric, partials,
                                                           C, ldc);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_gemm_nn(int rows, int k, int n, double alpha, const double* A, int lda,
                           const double* M, int ldm, double beta, double* C, int ldc, bool upper,
                           cudaStream_t st) {
  if (rows <= 0 || n <= 0) return cudaSuccess;
  const long long big_tiles = (long long)((rows + 31) / 32) * ((n + 31) / 32);
  if (big_tiles >= 152) {
    dim3 grid((n + 31) / 32, (rows + 31) / 32);
    gemm_nn_kernel<32, 32><<<grid, 256, 0, st>>>(rows, k, n, alpha, A, lda, M, ldm, beta, C, ldc,
                                                 upper);
  note_launch();
  } else if ((long long)((rows + 15) / 16) * ((n + 15) / 16) >= 152) {
    dim3 grid((n + 15) / 16, (rows + 15) / 16);
    gemm_nn_kernel<16, 16><<<grid, 256, 0, st>>>(rows, k, n, alpha, A, lda, M, ldm, beta, C, ldc,
                                                 upper);
  note_launch();
  } else {
    dim3 grid((n + 7) / 8, (rows + 7) / 8);
    gemm_nn_small_kernel<<<grid, 64, 0, st>>>(rows, k, n, alpha, A, lda, M, ldm, beta, C, ldc, upper);
    note_launch();
  }
  return cudaGetLastError();
}

cudaError_t launch_copy2d(int rows, int cols, const double* in, int ld_in, double* out, int ld_out,
                          cudaStream_t st) {
  const long long tot = (long long)rows * cols;
  if (tot <= 0) return cudaSuccess;
  copy2d_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(rows, cols, in, ld_in, out, ld_out);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_gather_cols(int rows, int ncols, const double* in, int ld_in, const int* cols,
                               double* out, int ld_out, cudaStream_t st) {
  const long long tot = (long long)rows * ncols;
  if (tot <= 0) return cudaSuccess;
  gather_cols_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(rows, ncols, in, ld_in, cols,
                                                                     out, ld_out);
  note_launch();
  return cudaGetLastError();
}

namespace {
// Sign convention of the returned eigenvectors: each column is flipped so that its entry of
// largest magnitude (the lowest row index among equal magnitudes) is positive. One CTA per
// column: a (magnitude, index) reduction, then the flip.
__global__ void __launch_bounds__(256)
normalize_signs_kernel(int rows, double* __restrict__ V, int ldv) {
  __shared__ double s_m[256];
  __shared__ int s_i[256];
  const int c = blockIdx.x, t = threadIdx.x;
  double m = -1.0;
  int mi = 0x7fffffff;
  for (int r = t; r < rows; r += blockDim.x) {
    const double a = fabs(V[(size_t)r * ldv + c]);
    if (a > m || (a == m && r < mi)) {
      m = a;
      mi = r;
    }
  }
  s_m[t] = m;
  s_i[t] = mi;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (t < o) {
      const double om = s_m[t + o];
      const int oi = s_i[t + o];
      if (om > s_m[t] || (om == s_m[t] && oi < s_i[t])) {
        s_m[t] = om;
        s_i[t] = oi;
      }
    }
    __syncthreads();
  }
  const bool flip = V[(size_t)s_i[0] * ldv + c] < 0.0;
  if (flip)
    for (int r = t; r < rows; r += blockDim.x) V[(size_t)r * ldv + c] = -V[(size_t)r * ldv + c];
}
}  // namespace

// V[r][c] /= sqrt(w[r]): maps standard-form eigenvectors v of M^{-1/2} K M^{-1/2} to the
// M-orthonormal solutions u = M^{-1/2} v of K u = lambda M u (M = diag(w)).
__global__ void scale_rows_rsqrt_kernel(int rows, int ncols, double* __restrict__ V, int ldv,
                                        const double* __restrict__ w) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < (size_t)rows * ncols;
       e += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / ncols), c = (int)(e - (size_t)r * ncols);
    V[(size_t)r * ldv + c] /= sqrt(w[r]);
  }
}

cudaError_t launch_scale_rows_rsqrt(int rows, int ncols, double* V, int ldv, const double* w,
                                    cudaStream_t st) {
  if (rows <= 0 || ncols <= 0) return cudaSuccess;
  const size_t total = (size_t)rows * ncols;
  const int blocks = (int)std::min<size_t>((total + 255) / 256, 152 * 8);
  scale_rows_rsqrt_kernel<<<blocks, 256, 0, st>>>(rows, ncols, V, ldv, w);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_normalize_signs(int rows, int ncols, double* V, int ldv, cudaStream_t st) {
  if (rows <= 0 || ncols <= 0) return cudaSuccess;
  normalize_signs_kernel<<<ncols, 256, 0, st>>>(rows, V, ldv);
  note_launch();
  return cudaGetLastError();
}

}  // namespace scsf
