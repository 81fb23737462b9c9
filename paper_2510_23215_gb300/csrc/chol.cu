// Cholesky factor and triangular inverse for Cholesky QR (Alg. 3, orthonormalisation).
//
// CholQR2 factors two Gram matrices per outer iteration. The first factor only
// has to make X R^{-1} well conditioned, so it is computed in FP32 (60x the FP64
// rate on GB300); the second, which fixes the final orthonormality, in FP64.
// Both factorisations run in one CTA with the matrix in shared memory
// (right-looking, one column per step, the trailing update on a 32 x 32 thread
// grid without index division). The inverse R^{-1} = (L^{-1})^T is spread over
// k single-warp CTAs: one warp forward-substitutes one column of L^{-1}, in FP32 for
// the first pass and FP64 for the second.
#include <algorithm>

#include "kernels.cuh"

namespace scsf {
namespace {

__host__ __device__ __forceinline__ int odd_stride(int k) { return (k % 2 == 0) ? k + 1 : k; }

// G = L L^T for k x k symmetric positive definite G (lower triangle read).
// On a non-positive pivot the factorisation restarts on G + s I (shifted
// Cholesky QR) with s growing 100x per retry, starting at c_eps k trace(G).
// Writes L (lower, FP64, ld k, zeros above) and status = number of shifted
// restarts, or 1000 if the last attempt still failed. blockDim = (32, 32).
template <typename T>
__global__ void __launch_bounds__(1024)
chol_kernel(int k, const double* __restrict__ G, int ldg, double* __restrict__ L,
            int* __restrict__ status, double shift_eps) {
  extern __shared__ unsigned char smraw[];
  T* S = reinterpret_cast<T*>(smraw);  // k x ks
  const int ks = odd_stride(k);
  __shared__ T dinv_s;
  __shared__ int bad;
  __shared__ double trace;
  const int tx = threadIdx.x, ty = threadIdx.y, t = ty * 32 + tx;
  if (t == 0) {
    double tr = 0.0;
    for (int i = 0; i < k; ++i) tr += fabs(G[(size_t)i * ldg + i]);
    trace = tr;
  }
  __syncthreads();
  int attempt = 0;
  for (; attempt < 4; ++attempt) {
    const double shift = (attempt == 0) ? 0.0 : shift_eps * k * trace * pow(100.0, attempt - 1);
    for (int i = ty; i < k; i += 32)
      for (int j = tx; j <= i; j += 32)
        S[i * ks + j] = (T)(G[(size_t)i * ldg + j] + ((i == j) ? shift : 0.0));
    if (t == 0) bad = 0;
    __syncthreads();
    for (int j = 0; j < k; ++j) {
      if (t == 0) {
        const T p = S[j * ks + j];
        if (!(p > T(0))) {
          if (bad == 0) bad = j + 1;
          S[j * ks + j] = T(1);
          dinv_s = T(1);
        } else {
          const T l = sqrt(p);
          S[j * ks + j] = l;
          dinv_s = T(1) / l;
        }
      }
      __syncthreads();
      const T inv = dinv_s;
      for (int i = j + 1 + t; i < k; i += 1024) S[i * ks + j] *= inv;
      __syncthreads();
      // trailing lower triangle: S[i][c] -= L[i][j] L[c][j], j < c <= i
      for (int i = j + 1 + ty; i < k; i += 32) {
        const T lij = S[i * ks + j];
        for (int c = j + 1 + tx; c <= i; c += 32) S[i * ks + c] -= lij * S[c * ks + j];
      }
      __syncthreads();
    }
    if (bad == 0) break;
    __syncthreads();
  }
  for (int i = ty; i < k; i += 32)
    for (int j = tx; j < k; j += 32) L[(size_t)i * k + j] = (j <= i) ? (double)S[i * ks + j] : 0.0;
  if (t == 0) status[0] = (bad != 0) ? 1000 : attempt;
}

// Rinv = (L^{-1})^T (upper, ld k): one warp per column j of L^{-1}, one warp per CTA so
// that the columns spread over the SMs (the FP64 pipe of one SM is narrow). Column-
// oriented forward substitution: lane l keeps the running sums s_r of the rows
// r = l + 32 q in registers; at step i the owner lane of row i forms
// x_i = -s_i / L_ii (x_j = 1 / L_jj), broadcasts it, and every lane adds L_ri x_i to
// its rows r > i. L is staged 32 columns at a time ([k][33] tile, conflict-free).
// T = float serves the first (preconditioning) Cholesky QR pass, T = double the second.
constexpr int kTrinvRowsPerLane = (kMaxBlockWidth + 31) / 32;

template <typename T>
__global__ void __launch_bounds__(32)
trinv_kernel(int k, const double* __restrict__ L, double* __restrict__ Rinv) {
  extern __shared__ unsigned char tile_raw[];
  T* tile = reinterpret_cast<T*>(tile_raw);  // [k][33]
  const int lane = threadIdx.x, j = blockIdx.x;
  T s[kTrinvRowsPerLane], dinv[kTrinvRowsPerLane], x[kTrinvRowsPerLane];
#pragma unroll
  for (int q = 0; q < kTrinvRowsPerLane; ++q) {
    const int r = lane + 32 * q;
    s[q] = T(0);
    x[q] = T(0);
    dinv[q] = (r >= j && r < k) ? T(1) / (T)L[(size_t)r * k + r] : T(0);
  }
#pragma unroll
  for (int cq = 0; cq < kTrinvRowsPerLane; ++cq) {
    const int c0 = 32 * cq;
    if (c0 < k && c0 + 31 >= j) {
      // stage L[r][c0 + t] for rows r >= max(j, c0), t < 32
      __syncwarp();
      const int rfirst = max(j, c0);
      const int c = c0 + lane;
      for (int r = rfirst; r < k; ++r)
        tile[r * 33 + lane] = (c < k && c <= r) ? (T)L[(size_t)r * k + c] : T(0);
      __syncwarp();
      for (int t = 0; t < 32; ++t) {
        const int i = c0 + t;
        if (i >= k) break;
        if (i < j) continue;
        T xi = (i == j) ? dinv[cq] : -s[cq] * dinv[cq];
        xi = __shfl_sync(0xffffffffu, xi, t);
        if (lane == t) x[cq] = xi;
#pragma unroll
        for (int q = cq; q < kTrinvRowsPerLane; ++q) {
          const int r = lane + 32 * q;
          if (r > i && r < k) s[q] = fma(tile[r * 33 + t], xi, s[q]);
        }
      }
    }
  }
  double* row = Rinv + (size_t)j * k;
#pragma unroll
  for (int q = 0; q < kTrinvRowsPerLane; ++q) {
    const int r = lane + 32 * q;
    if (r < k) row[r] = (r >= j) ? (double)x[q] : 0.0;
  }
}

template <typename T>
cudaError_t launch_chol_t(int k, const double* G, int ldg, double* L, int* status, double eps,
                          cudaStream_t st) {
  const size_t smem = (size_t)k * odd_stride(k) * sizeof(T);
  cudaError_t e = ensure_dynamic_smem((const void*)chol_kernel<T>, smem);
  if (e != cudaSuccess) return e;
  chol_kernel<T><<<1, dim3(32, 32), smem, st>>>(k, G, ldg, L, status, eps);
  note_launch();
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_chol_rinv(int k, const double* G, int ldg, bool fp32, double* L, double* Rinv,
                             int* status, cudaStream_t st) {
  if (k <= 0 || k > kMaxBlockWidth) return cudaErrorInvalidValue;
  cudaError_t e = fp32 ? launch_chol_t<float>(k, G, ldg, L, status, 1e-6, st)
                       : launch_chol_t<double>(k, G, ldg, L, status, 1e-14, st);
  if (e != cudaSuccess) return e;
  if (fp32) {
    const size_t smem = (size_t)k * 33 * sizeof(float);
    if ((e = ensure_dynamic_smem((const void*)trinv_kernel<float>, smem)) != cudaSuccess) return e;
    trinv_kernel<float><<<k, 32, smem, st>>>(k, L, Rinv);
  } else {
    const size_t smem = (size_t)k * 33 * sizeof(double);
    if ((e = ensure_dynamic_smem((const void*)trinv_kernel<double>, smem)) != cudaSuccess) return e;
    trinv_kernel<double><<<k, 32, smem, st>>>(k, L, Rinv);
  }
  note_launch();
  return cudaGetLastError();
}

}  // namespace scsf
