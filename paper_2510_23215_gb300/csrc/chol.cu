// Cholesky factor and triangular inverse for Cholesky QR (Alg. 3, orthonormalisation).
//
// CholQR2 factors two Gram matrices per outer iteration. The first factor only
// has to make X R^{-1} well conditioned, so it is computed in FP32 (60x the FP64
// rate on GB300); the second, which fixes the final orthonormality, in FP64.
// When a diagonal entry of G lies outside [2^-100, 2^100] -- columns of X far outside FP32's
// range, as after a high-degree filter that scales them by 1 / C_m(t_lambda) -- both factor
// the diagonally scaled Gram matrix S = D^-1 G D^-1 instead and return L = D L_S (G = L L^T),
// D_ii the power of two just below sqrt(G_ii) (S_ii in [1, 4)): exact, and within a factor
// of 4 of the optimal diagonal preconditioner (van der Sluis). Otherwise D = I and the factor
// is the plain one.
// Both factorisations run in one CTA with the matrix in shared memory (right-looking,
// blocked in 32-column panels: the diagonal block by one warp, the rows below it one
// thread each, the rank-32 trailing update on a 32 x 32 thread grid). The inverse R^{-1} = (L^{-1})^T is spread over
// k single-warp CTAs: one warp forward-substitutes one column of L^{-1}, in FP32 for
// the first pass and FP64 for the second.
#include <algorithm>

#include "kernels.cuh"

namespace scsf {
namespace {

__host__ __device__ __forceinline__ int odd_stride(int k) { return (k % 2 == 0) ? k + 1 : k; }

// A positive finite diagonal entry outside [2^-100, 2^100] switches the scaling on.
__device__ __forceinline__ bool chol_out_of_range(double g) {
  return g > 0.0 && g < INFINITY && (g < 0x1p-100 || g > 0x1p100);
}

// Scale of row / column i: 2^floor(e / 2) for G_ii = m 2^e (m in [1, 2)), or 1 for a
// diagonal that is not positive and finite (the pivot then fails and the shifted restart
// takes over).
__device__ __forceinline__ double chol_scale(double g) {
  if (!(g > 0.0 && g < INFINITY)) return 1.0;
  const int e = ilogb(g);
  return ldexp(1.0, (e >= 0) ? e / 2 : -((1 - e) / 2));
}

// G = L L^T for k x k symmetric positive definite G (lower triangle read), k <= 160,
// through S = D^-1 G D^-1 (D from chol_scale). On a non-positive pivot the factorisation
// restarts on S + s I (shifted Cholesky QR) with s growing 100x per retry, starting at
// c_eps k trace(S). Writes L (lower, FP64, ld k, zeros above) and status = number of
// shifted restarts, or 1000 if the last attempt still failed.
// Blocked in 32-column panels with the matrix in shared memory, three barriers a panel:
// warp 0 factors the panel's diagonal block (warp-synchronous, one column a step), one
// thread per row below it solves its panel row against the diagonal block, and all
// threads apply the panel's rank-32 update to the trailing lower triangle.
// blockDim = (32, 32) for FP32, (32, 16) for FP64.
template <typename T>
__global__ void __launch_bounds__(sizeof(T) == 8 ? 512 : 1024)
chol_blocked_kernel(int k, const double* __restrict__ G, int ldg, double* __restrict__ L,
                    int* __restrict__ status, double shift_eps) {
  extern __shared__ unsigned char smraw[];
  T* S = reinterpret_cast<T*>(smraw);  // k x ks
  const int ks = odd_stride(k);
  constexpr int PW = 32;
  __shared__ T dinv[PW];
  __shared__ int bad;
  __shared__ double trace;
  __shared__ double sc[kSmallBlockWidth], isc[kSmallBlockWidth];
  __shared__ double red[32];
  __shared__ int scaled;
  const int tx = threadIdx.x, ty = threadIdx.y, t = ty * 32 + tx;
  const int ny = blockDim.y, nthr = 32 * blockDim.y;  // blockDim = (32, ny)
  if (t == 0) scaled = 0;
  __syncthreads();
  for (int i = t; i < k; i += nthr)
    if (chol_out_of_range(G[(size_t)i * ldg + i])) scaled = 1;
  __syncthreads();
  // scales are powers of two: their reciprocals are exact, so S = G isc_i isc_j is exact
  double part = 0.0;
  for (int i = t; i < k; i += nthr) {
    const double g = G[(size_t)i * ldg + i];
    const double d = scaled ? chol_scale(g) : 1.0;
    sc[i] = d;
    isc[i] = 1.0 / d;
    part += fabs(g) * isc[i] * isc[i];
  }
  for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  if (tx == 0) red[ty] = part;
  __syncthreads();
  if (t == 0) {
    double tr = 0.0;
    for (int w = 0; w < ny; ++w) tr += red[w];
    trace = tr;
  }
  __syncthreads();
  int attempt = 0;
  for (; attempt < 4; ++attempt) {
    const double shift = (attempt == 0) ? 0.0 : shift_eps * k * trace * pow(100.0, attempt - 1);
    for (int i = ty; i < k; i += ny)
      for (int j = tx; j <= i; j += 32) {
        const double g = G[(size_t)i * ldg + j];
        S[i * ks + j] = (T)((scaled ? g * isc[i] * isc[j] : g) + ((i == j) ? shift : 0.0));
      }
    if (t == 0) bad = 0;
    __syncthreads();
    for (int p = 0; p < k; p += PW) {
      const int w = min(PW, k - p);
      if (ty == 0) {  // diagonal block: lane = row within the panel, its row in registers
        const int lane = tx;
        T row[PW];
#pragma unroll
        for (int c = 0; c < PW; ++c)
          row[c] = (lane < w && c <= lane) ? S[(p + lane) * ks + p + c] : T(0);
#pragma unroll
        for (int j = 0; j < PW; ++j) {
          if (j < w) {
            T piv = __shfl_sync(0xffffffffu, row[j], j);
            if (!(piv > T(0))) {
              if (lane == 0 && bad == 0) bad = p + j + 1;
              piv = T(1);
            }
            const T l = sqrt(piv), inv = T(1) / l;
            if (lane == j) {
              row[j] = l;
              dinv[j] = inv;
            }
            if (lane > j) row[j] *= inv;  // L[r][j]
            // row[c] -= L[r][j] L[c][j] for j < c <= r
#pragma unroll
            for (int c = j + 1; c < PW; ++c) {
              const T lcj = __shfl_sync(0xffffffffu, row[j], c);
              if (lane >= c) row[c] = fma(-row[j], lcj, row[c]);
            }
          }
        }
        if (lane < w)
#pragma unroll
          for (int c = 0; c < PW; ++c)
            if (c <= lane) S[(p + lane) * ks + p + c] = row[c];
      }
      __syncthreads();
      // rows below the panel: L21 = A21 L11^{-T}, forward substitution along each row (the
      // row in registers, the diagonal block read as broadcasts)
      for (int r = p + w + t; r < k; r += nthr) {
        T x[PW];
#pragma unroll
        for (int c = 0; c < PW; ++c) x[c] = (c < w) ? S[r * ks + p + c] : T(0);
#pragma unroll
        for (int j = 0; j < PW; ++j) {
          if (j < w) {
            const T* lj = S + (p + j) * ks + p;
            T v = x[j];
#pragma unroll
            for (int c = 0; c < j; ++c) v = fma(-x[c], lj[c], v);
            x[j] = v * dinv[j];
          }
        }
#pragma unroll
        for (int c = 0; c < PW; ++c)
          if (c < w) S[r * ks + p + c] = x[c];
      }
      __syncthreads();
      // trailing lower triangle: S[r][c] -= sum_q L[r][p + q] L[c][p + q]
      const int q0 = p + w;
      for (int r = q0 + ty; r < k; r += ny) {
        const T* lr = S + r * ks + p;
        for (int c = q0 + tx; c <= r; c += 32) {
          const T* lc = S + c * ks + p;
          T acc = T(0);
          for (int q = 0; q < w; ++q) acc = fma(lr[q], lc[q], acc);
          S[r * ks + c] -= acc;
        }
      }
      __syncthreads();
    }
    if (bad == 0) break;
    __syncthreads();
  }
  for (int i = ty; i < k; i += ny)
    for (int j = tx; j < k; j += 32)
      L[(size_t)i * k + j] = (j <= i) ? (double)S[i * ks + j] * sc[i] : 0.0;
  if (t == 0) status[0] = (bad != 0) ? 1000 : attempt;
}

// Rinv = (L^{-1})^T (upper, ld k): one warp per column j of L^{-1}, one warp per CTA so
// that the columns spread over the SMs (the FP64 pipe of one SM is narrow). Column-
// oriented forward substitution: lane l keeps the running sums s_r of the rows
// r = l + 32 q in registers; at step i the owner lane of row i forms
// x_i = -s_i / L_ii (x_j = 1 / L_jj), broadcasts it, and every lane adds L_ri x_i to
// its rows r > i. L is staged 32 columns at a time ([k][33] tile, conflict-free).
// T = float serves the first (preconditioning) Cholesky QR pass, T = double the second.
template <typename T, int kTrinvRowsPerLane>
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

// ---- wide blocks (k > kSmallBlockWidth): blocked right-looking Cholesky in global memory.
// The working copy M (T, k x k, lower triangle) lives in the scratch; per 32-column panel one
// CTA factors the panel (diagonal block and the rows below it, staged in shared memory), then
// a tiled kernel applies the panel's rank-32 update to the trailing lower triangle.
constexpr int kPanel = 32;

template <typename T>
__global__ void chol_load_kernel(int k, const double* __restrict__ G, int ldg,
                                 const double* __restrict__ sc, double shift, T* __restrict__ M) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)k * k) return;
  const int i = (int)(e / k), j = (int)(e - (long long)i * k);
  if (j <= i) M[e] = (T)(G[(size_t)i * ldg + j] / (sc[i] * sc[j]) + ((i == j) ? shift : 0.0));
}

template <typename T>
__global__ void __launch_bounds__(1024)
chol_panel_kernel(int k, T* __restrict__ M, int p, int* __restrict__ bad) {
  extern __shared__ unsigned char praw[];
  T* P = reinterpret_cast<T*>(praw);  // rows p..k-1, 33 columns (32 used)
  __shared__ T dinv_s;
  const int t = threadIdx.x, nt = blockDim.x;
  const int rows = k - p, w = min(kPanel, k - p);
  for (int e = t; e < rows * kPanel; e += nt) {
    const int r = e / kPanel, c = e - r * kPanel;
    P[r * 33 + c] = (c < w && c <= r) ? M[(size_t)(p + r) * k + p + c] : T(0);
  }
  __syncthreads();
  for (int j = 0; j < w; ++j) {
    if (t == 0) {
      T piv = P[j * 33 + j];
      if (!(piv > T(0))) {
        atomicMax(bad, 1);
        piv = T(1);
      }
      const T l = sqrt(piv);
      P[j * 33 + j] = l;
      dinv_s = T(1) / l;
    }
    __syncthreads();
    const T inv = dinv_s;
    for (int r = j + 1 + t; r < rows; r += nt) P[r * 33 + j] *= inv;
    __syncthreads();
    // rank-1 update of the panel columns c in (j, w), rows r >= c
    const int nc = w - j - 1;
    if (nc > 0)
      for (int e = t; e < (rows - j - 1) * nc; e += nt) {
        const int r = j + 1 + e / nc, c = j + 1 + e % nc;
        if (c <= r) P[r * 33 + c] -= P[r * 33 + j] * P[c * 33 + j];
      }
    __syncthreads();
  }
  for (int e = t; e < rows * kPanel; e += nt) {
    const int r = e / kPanel, c = e - r * kPanel;
    if (c < w && c <= r) M[(size_t)(p + r) * k + p + c] = P[r * 33 + c];
  }
}

// M[r][c] -= sum_{q < 32} M[r][p + q] M[c][p + q] for p + 32 <= c <= r < k, one 32 x 32 tile
// (tile row >= tile column) per CTA.
template <typename T>
__global__ void __launch_bounds__(1024)
chol_trailing_kernel(int k, T* __restrict__ M, int p) {
  __shared__ T Lr[32][33], Lc[32][33];
  const int q0 = p + kPanel;
  const int nt = (k - q0 + 31) / 32;
  // blockIdx.x enumerates the lower-triangular tiles (ti >= tj)
  int ti = 0, rem = blockIdx.x;
  while (rem > ti) {
    rem -= ti + 1;
    ++ti;
  }
  const int tj = rem;
  if (ti >= nt) return;
  const int r0 = q0 + 32 * ti, c0 = q0 + 32 * tj;
  const int tx = threadIdx.x, ty = threadIdx.y;
  Lr[ty][tx] = (r0 + ty < k) ? M[(size_t)(r0 + ty) * k + p + tx] : T(0);
  Lc[ty][tx] = (c0 + ty < k) ? M[(size_t)(c0 + ty) * k + p + tx] : T(0);
  __syncthreads();
  const int r = r0 + ty, c = c0 + tx;
  if (r < k && c < k && c <= r) {
    T acc = T(0);
#pragma unroll 8
    for (int q = 0; q < 32; ++q) acc = fma(Lr[ty][q], Lc[tx][q], acc);
    M[(size_t)r * k + c] -= acc;
  }
}

template <typename T>
__global__ void chol_store_kernel(int k, const T* __restrict__ M, const double* __restrict__ sc,
                                  double* __restrict__ L) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)k * k) return;
  const int i = (int)(e / k), j = (int)(e - (long long)i * k);
  L[e] = (j <= i) ? (double)M[e] * sc[i] : 0.0;
}

// Row scales sc[i] (chol_scale of G_ii when any diagonal entry is out of range, else 1) and
// trace(D^-1 G D^-1) into *out. One CTA.
__global__ void chol_trace_kernel(int k, const double* __restrict__ G, int ldg,
                                  double* __restrict__ sc, double* out) {
  __shared__ double red[256];
  __shared__ int scaled;
  if (threadIdx.x == 0) scaled = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < k; i += blockDim.x)
    if (chol_out_of_range(G[(size_t)i * ldg + i])) scaled = 1;
  __syncthreads();
  double s = 0.0;
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    const double g = G[(size_t)i * ldg + i], d = scaled ? chol_scale(g) : 1.0;
    sc[i] = d;
    s += fabs(g) / (d * d);
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

// Factor with the scaling and restart rule of chol_blocked_kernel (shift c_eps k trace(S)
// 100^(attempt-1)); the host reads the failure flag after each attempt (wide blocks only).
template <typename T>
cudaError_t launch_chol_wide(int k, const double* G, int ldg, double* L, int* status, double eps,
                             void* scratch, cudaStream_t st) {
  Carve cv(scratch, chol_wide_scratch_bytes(k));
  T* M = cv.take<T>((size_t)k * k);
  int* bad = cv.take<int>(4);
  double* tr = cv.take<double>(1);
  double* sc = cv.take<double>(k);
  if (!cv.ok) return cudaErrorInvalidValue;
  const size_t psmem = (size_t)k * 33 * sizeof(T);
  cudaError_t e = ensure_dynamic_smem((const void*)chol_panel_kernel<T>, psmem);
  if (e != cudaSuccess) return e;
  chol_trace_kernel<<<1, 256, 0, st>>>(k, G, ldg, sc, tr);
  note_launch();
  double trace = 0.0;
  if ((e = cudaMemcpyAsync(&trace, tr, sizeof(double), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return e;
  const long long kk = (long long)k * k;
  const int eb = (int)((kk + 255) / 256);
  int attempt = 0, h_bad = 0;
  for (; attempt < 4; ++attempt) {
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
    const double shift = (attempt == 0) ? 0.0 : eps * k * trace * pow(100.0, attempt - 1);
    if ((e = cudaMemsetAsync(bad, 0, sizeof(int), st)) != cudaSuccess) return e;
    chol_load_kernel<T><<<eb, 256, 0, st>>>(k, G, ldg, sc, shift, M);
    note_launch();
    for (int p = 0; p < k; p += kPanel) {
      chol_panel_kernel<T><<<1, 1024, psmem, st>>>(k, M, p, bad);
      note_launch();
      const int nt = (k - p - kPanel + 31) / 32;
      if (nt > 0) {
        chol_trailing_kernel<T><<<nt * (nt + 1) / 2, dim3(32, 32), 0, st>>>(k, M, p);
        note_launch();
      }
    }
    if ((e = cudaMemcpyAsync(&h_bad, bad, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
      return e;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
    if (h_bad == 0) break;
  }
  chol_store_kernel<T><<<eb, 256, 0, st>>>(k, M, sc, L);
  note_launch();
  const int code = (h_bad != 0) ? 1000 : attempt;
  if ((e = cudaMemcpyAsync(status, &code, sizeof(int), cudaMemcpyHostToDevice, st)) != cudaSuccess)
    return e;
  // `code` lives on this stack frame: the copy must finish before it is popped
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_chol_t(int k, const double* G, int ldg, double* L, int* status, double eps,
                          cudaStream_t st) {
  const size_t smem = (size_t)k * odd_stride(k) * sizeof(T);
  cudaError_t e = ensure_dynamic_smem((const void*)chol_blocked_kernel<T>, smem);
  if (e != cudaSuccess) return e;
  // FP64 rows of the diagonal block need 64 registers each: half the threads, twice the registers
  chol_blocked_kernel<T><<<1, dim3(32, sizeof(T) == 8 ? 16 : 32), smem, st>>>(k, G, ldg, L, status, eps);
  note_launch();
  return cudaGetLastError();
}

}  // namespace

size_t chol_wide_scratch_bytes(int k) {
  return align256((size_t)k * k * sizeof(double)) + align256((size_t)k * sizeof(double)) + 512;
}

cudaError_t launch_chol_rinv(int k, const double* G, int ldg, bool fp32, double* L, double* Rinv,
                             int* status, cudaStream_t st, void* wide_scratch) {
  if (k <= 0 || k > kMaxBlockWidth) return cudaErrorInvalidValue;
  cudaError_t e;
  if (k <= kSmallBlockWidth) {
    e = fp32 ? launch_chol_t<float>(k, G, ldg, L, status, 1e-6, st)
             : launch_chol_t<double>(k, G, ldg, L, status, 1e-14, st);
  } else {
    if (!wide_scratch) return cudaErrorInvalidValue;
    e = fp32 ? launch_chol_wide<float>(k, G, ldg, L, status, 1e-6, wide_scratch, st)
             : launch_chol_wide<double>(k, G, ldg, L, status, 1e-14, wide_scratch, st);
  }
  if (e != cudaSuccess) return e;
  const size_t smem = (size_t)k * 33 * (fp32 ? sizeof(float) : sizeof(double));
  if (k <= kSmallBlockWidth) {
    constexpr int R = (kSmallBlockWidth + 31) / 32;
    if (fp32) {
      if ((e = ensure_dynamic_smem((const void*)trinv_kernel<float, R>, smem)) != cudaSuccess) return e;
      trinv_kernel<float, R><<<k, 32, smem, st>>>(k, L, Rinv);
    } else {
      if ((e = ensure_dynamic_smem((const void*)trinv_kernel<double, R>, smem)) != cudaSuccess) return e;
      trinv_kernel<double, R><<<k, 32, smem, st>>>(k, L, Rinv);
    }
  } else {
    constexpr int R = (kMaxBlockWidth + 31) / 32;
    if (fp32) {
      if ((e = ensure_dynamic_smem((const void*)trinv_kernel<float, R>, smem)) != cudaSuccess) return e;
      trinv_kernel<float, R><<<k, 32, smem, st>>>(k, L, Rinv);
    } else {
      if ((e = ensure_dynamic_smem((const void*)trinv_kernel<double, R>, smem)) != cudaSuccess) return e;
      trinv_kernel<double, R><<<k, 32, smem, st>>>(k, L, Rinv);
    }
  }
  note_launch();
  return cudaGetLastError();
}

}  // namespace scsf
