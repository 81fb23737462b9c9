// Learned proposal: a small Fourier neural operator that maps a coefficient
// field to (i) the log of the spectrum bounds lambda_1, lambda_kb and (ii) a
// coarse-grid block of 64 vectors whose span approximates the lowest
// eigenvectors. It seeds chain heads (Sec. 3.2 starts them from random blocks);
// the Chebyshev filter and the FP64 residual check still decide every result.
//
// Network (all kernels here; weights stored in BF16, FP32 master copy for Adam, every
// matrix product on the tensor cores with FP32 accumulation, FP32 activations split into two
// BF16 parts):
//   pool   : mean of log a over 4x4 node blocks of the s x s field -> S x S, S = 32
//   lift   : in = (pooled, x, y) -> v0 = in Wl + bl                    (3 -> W)
//   layer l: a_l = Re(G (R_l (F v_{l-1}))) + v_{l-1} Wp_l + bp_l,
//            v_l = gelu(a_l) (l < L), v_L = a_L
//            F: truncated DFT to M = 2*12 x 12 modes (+-k1, k2 >= 0), R_l: one
//            complex W x W matrix per mode, G: Hermitian-completed inverse DFT
//   heads  : Y = gelu(v_L Wh + bh) Wy (S*S x 64 block, a pointwise 32 -> 128 -> 64 MLP so
//            the block can have full rank); s = mean_p(v_L) Wb + bb (2 log-bounds)
// Objective per sample: sub + mu orth + |s - t|^2 with Q an orthonormal basis of the
// pooled true eigenvectors, G = Y^T Y, C = Q^T Y and
//   sub  = 64 - tr((G + delta I)^-1 C^T C)   (sum of squared sines of the principal
//          angles between span(Y) and span(Q) as delta -> 0; invariant to Y -> Y S),
//   orth = |G - I|_F^2 (keeps the columns well conditioned), delta = 1e-3, mu = 0.01.
// Gradient: d sub / dY = 2 (Y T - Q C M), M = (G + delta I)^-1, T = M C^T C M.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include <cuda_bf16.h>

#include "../../include/scsf.h"
#include "kernels.cuh"

namespace scsf {
namespace {

constexpr int S = 32;            // coarse grid side
constexpr int P = S * S;         // coarse points
constexpr int W = 32;            // width
constexpr int MODES = 12;        // kept modes per axis (k1 uses +- MODES)
constexpr int M1 = 2 * MODES;    // k1 in {0..11} U {S-12..S-1}
constexpr int M = M1 * MODES;    // kept complex modes
constexpr int L = 4;             // Fourier layers
constexpr int KY = 64;           // coarse block columns
constexpr int H = 128;           // hidden width of the block head (full-rank 64-column output)
constexpr int CIN = 3;           // pooled log a, x, y
constexpr double kRidge = 1e-3;  // delta in the subspace loss (G + delta I)^-1
constexpr float kOrthWeight = 0.01f;  // mu: weight of |Y^T Y - I|^2 in the objective

// flat FP32 parameter layout
struct Layout {
  size_t Wl, bl, Rr[L], Ri[L], Wp[L], bp[L], Wh, bh, Wy, Wb, bb, total;
  Layout() {
    size_t o = 0;
    auto take = [&](size_t n) { size_t r = o; o += (n + 63) & ~size_t(63); return r; };
    Wl = take(CIN * W);
    bl = take(W);
    for (int l = 0; l < L; ++l) {
      Rr[l] = take((size_t)M * W * W);
      Ri[l] = take((size_t)M * W * W);
      Wp[l] = take(W * W);
      bp[l] = take(W);
    }
    Wh = take(W * H);
    bh = take(H);
    Wy = take(H * KY);
    Wb = take(W * 2);
    bb = take(2);
    total = o;
  }
};
const Layout kLay;

// ---- strided-batched GEMM ------------------------------------------------
// C[z] = alpha * op(A[z]) op(B[z]) + beta * C[z]; op(X) = X or X^T (ta/tb).
// A: element (r, c) of op(A) (rows x K) is A[r*lda + c] (ta = 0) or A[c*lda + r].
// On the tensor cores: mma.sync m16n8k16, BF16 operands, FP32 accumulation. An FP32 operand
// x enters as hi + lo with hi = bf16(x), lo = bf16(x - hi) (16 significant bits) and each
// product takes hi*hi + hi*lo + lo*hi (the dropped lo*lo term is 2^-16 of the kept ones); a
// BF16 operand (the weights) has lo = 0 and costs no extra product. Tile 64 x 64 x 32 per
// CTA of four warps, each warp a 32 x 32 block of 2 x 4 MMA tiles.
constexpr int kTcBM = 64, kTcBN = 64, kTcBK = 32;

__device__ __forceinline__ void bf16_split(float x, float& hi, float& lo) {
  hi = __bfloat162float(__float2bfloat16_rn(x));
  lo = x - hi;
}
__device__ __forceinline__ uint32_t bf16_pack(float e0, float e1) {  // e0 in the low half
  return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(e0)) |
         ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(e1)) << 16);
}
__device__ __forceinline__ void mma_16816(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

template <typename TA, typename TB>
__global__ void __launch_bounds__(128)
bgemm_tc_kernel(int rows, int cols, int K, float alpha, const TA* __restrict__ A, int lda,
                long long sA, bool ta, const TB* __restrict__ B, int ldb, long long sB, bool tb,
                float beta, float* __restrict__ C, int ldc, long long sC) {
  constexpr bool kSplitA = sizeof(TA) == 4, kSplitB = sizeof(TB) == 4;
  __shared__ float As[kTcBM][kTcBK + 4];  // op(A) tile [m][k]
  __shared__ float Bs[kTcBN][kTcBK + 4];  // op(B) tile, transposed: [n][k]
  const int z = blockIdx.z;
  A += z * sA;
  B += z * sB;
  C += z * sC;
  const int r0 = blockIdx.y * kTcBM, c0 = blockIdx.x * kTcBN;
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  const int g = lane >> 2, q = lane & 3;
  float acc[2][4][4];
#pragma unroll
  for (int mi = 0; mi < 2; ++mi)
#pragma unroll
    for (int ni = 0; ni < 4; ++ni)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[mi][ni][c] = 0.f;
  for (int k0 = 0; k0 < K; k0 += kTcBK) {
    for (int e = t; e < kTcBM * kTcBK; e += 128) {
      const int i = e >> 5, j = e & 31;
      const int r = r0 + i, kk = k0 + j;
      As[i][j] = (r < rows && kk < K)
                     ? (float)(ta ? A[(size_t)kk * lda + r] : A[(size_t)r * lda + kk]) : 0.f;
      const int cc = c0 + i;
      Bs[i][j] = (kk < K && cc < cols)
                     ? (float)(tb ? B[(size_t)cc * ldb + kk] : B[(size_t)kk * ldb + cc]) : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int ks = 0; ks < kTcBK; ks += 16) {
      uint32_t ah[2][4], al[2][4];
#pragma unroll
      for (int mi = 0; mi < 2; ++mi) {
        const float* r_lo = &As[wm + 16 * mi + g][ks + 2 * q];
        const float* r_hi = &As[wm + 16 * mi + g + 8][ks + 2 * q];
        const float x[8] = {r_lo[0], r_lo[1], r_hi[0], r_hi[1], r_lo[8], r_lo[9], r_hi[8], r_hi[9]};
        float h[8], l[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) bf16_split(x[u], h[u], l[u]);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          ah[mi][u] = bf16_pack(h[2 * u], h[2 * u + 1]);
          al[mi][u] = kSplitA ? bf16_pack(l[2 * u], l[2 * u + 1]) : 0u;
        }
      }
      uint32_t bh[4][2], bl[4][2];
#pragma unroll
      for (int ni = 0; ni < 4; ++ni) {
        const float* col = &Bs[wn + 8 * ni + g][ks + 2 * q];
        const float y[4] = {col[0], col[1], col[8], col[9]};
        float h[4], l[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) bf16_split(y[u], h[u], l[u]);
        bh[ni][0] = bf16_pack(h[0], h[1]);
        bh[ni][1] = bf16_pack(h[2], h[3]);
        bl[ni][0] = kSplitB ? bf16_pack(l[0], l[1]) : 0u;
        bl[ni][1] = kSplitB ? bf16_pack(l[2], l[3]) : 0u;
      }
#pragma unroll
      for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni) {
          mma_16816(acc[mi][ni], ah[mi], bh[ni]);
          if (kSplitA) mma_16816(acc[mi][ni], al[mi], bh[ni]);
          if (kSplitB) mma_16816(acc[mi][ni], ah[mi], bl[ni]);
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int mi = 0; mi < 2; ++mi)
#pragma unroll
    for (int ni = 0; ni < 4; ++ni)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int r = r0 + wm + 16 * mi + g + ((c & 2) ? 8 : 0);
        const int cc = c0 + wn + 8 * ni + 2 * q + (c & 1);
        if (r < rows && cc < cols) {
          float* p = C + (size_t)r * ldc + cc;
          *p = (beta == 0.f) ? alpha * acc[mi][ni][c] : fmaf(alpha, acc[mi][ni][c], beta * (*p));
        }
      }
}

template <typename TA, typename TB>
cudaError_t bgemm(int batch, int rows, int cols, int K, float alpha, const TA* A, int lda,
                  long long sA, bool ta, const TB* B, int ldb, long long sB, bool tb, float beta,
                  float* C, int ldc, long long sC, cudaStream_t st) {
  if (batch <= 0 || rows <= 0 || cols <= 0) return cudaSuccess;
  dim3 grid((cols + kTcBN - 1) / kTcBN, (rows + kTcBM - 1) / kTcBM, batch);
  bgemm_tc_kernel<TA, TB><<<grid, 128, 0, st>>>(rows, cols, K, alpha, A, lda, sA, ta, B, ldb, sB,
                                                tb, beta, C, ldc, sC);
  note_launch();
  return cudaGetLastError();
}

// ---- elementwise kernels --------------------------------------------------
__device__ __forceinline__ float gelu_f(float x) {
  const float k0 = 0.7978845608028654f, k1 = 0.044715f;  // sqrt(2/pi); tanh approximation
  return 0.5f * x * (1.f + tanhf(k0 * (x + k1 * x * x * x)));
}
__device__ __forceinline__ float gelu_grad(float x) {
  const float k0 = 0.7978845608028654f, k1 = 0.044715f;
  const float u = k0 * (x + k1 * x * x * x);
  const float th = tanhf(u);
  return 0.5f * (1.f + th) + 0.5f * x * (1.f - th * th) * k0 * (1.f + 3.f * k1 * x * x);
}

__global__ void bias_act_kernel(long long rows, int w, const float* __restrict__ bias,
                                float* __restrict__ a, float* __restrict__ v, bool act) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= rows * w) return;
  const float x = a[e] + bias[e % w];
  a[e] = x;
  v[e] = act ? gelu_f(x) : x;
}

__global__ void gelu_back_kernel(long long count, const float* __restrict__ a,
                                 const float* __restrict__ dv, float* __restrict__ da) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < count) da[e] = dv[e] * gelu_grad(a[e]);
}

// in[b][p][3] from fields a (s x s, pooled 4x4 in log space) and coordinates
__global__ void pool_input_kernel(int batch, int s, const double* __restrict__ fields,
                                  float* __restrict__ in) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= batch * P) return;
  const int b = e / P, p = e - b * P, I = p / S, J = p - I * S;
  const int f = s / S;
  const double* F = fields + (size_t)b * s * s;
  double acc = 0.0;
  for (int di = 0; di < f; ++di)
    for (int dj = 0; dj < f; ++dj) acc += log(F[(size_t)(I * f + di) * s + J * f + dj]);
  float* o = in + (size_t)e * CIN;
  o[0] = (float)(acc / (f * f));
  o[1] = (I + 0.5f) / S;
  o[2] = (J + 0.5f) / S;
}

// DFT matrices: Fr/Fi [M][P] (forward, e^{-i theta}); Gr/Gs [P][M] (inverse real part:
// u = Gr Ur - Gs Ui with the Hermitian weight 2 on k2 > 0 columns and 1/P scaling)
__global__ void dft_tables_kernel(float* Fr, float* Fi, float* Gr, float* Gs) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= M * P) return;
  const int m = e / P, p = e - m * P;
  const int a = m / MODES, k2 = m - a * MODES;
  const int k1 = (a < MODES) ? a : S - M1 + a;  // 0..11, then 20..31
  const int x = p / S, y = p - x * S;
  const int ph = (k1 * x + k2 * y) % S;
  double sn, cs;
  sincospi(2.0 * ph / S, &sn, &cs);
  Fr[e] = (float)cs;
  Fi[e] = (float)(-sn);
  const double w = (k2 == 0 ? 1.0 : 2.0) / P;
  Gr[(size_t)p * M + m] = (float)(w * cs);
  Gs[(size_t)p * M + m] = (float)(w * sn);
}

__global__ void mean_rows_kernel(int batch, int rows, int w, const float* __restrict__ x,
                                 float* __restrict__ out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= batch * w) return;
  const int b = e / w, c = e - b * w;
  float s = 0.f;
  for (int r = 0; r < rows; ++r) s += x[((size_t)b * rows + r) * w + c];
  out[e] = s / rows;
}

// out[b][j] = sum_w g[b][w] Wb[w][j] + bb[j], j < 2
__global__ void bounds_head_kernel(int batch, const float* __restrict__ g,
                                   const __nv_bfloat16* __restrict__ Wb, const float* __restrict__ bb,
                                   float* __restrict__ out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= batch * 2) return;
  const int b = e / 2, j = e - b * 2;
  float s = bb[j];
  for (int w = 0; w < W; ++w) s += g[b * W + w] * __bfloat162float(Wb[w * 2 + j]);
  out[e] = s;
}

__global__ void to_bf16_kernel(long long count, const float* __restrict__ in,
                               __nv_bfloat16* __restrict__ out) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < count) out[e] = __float2bfloat16_rn(in[e]);
}

// column sums of x [rows][w] in two deterministic stages: kColsumChunks row chunks of
// partial sums (32 columns x 8 row lanes per block), then one sum per column
constexpr int kColsumChunks = 64;

__global__ void colsum_partial_kernel(long long rows, int w, const float* __restrict__ x,
                                      float* __restrict__ part) {
  __shared__ float red[8][33];
  const int c = blockIdx.x * 32 + threadIdx.x;
  const long long chunk = (rows + kColsumChunks - 1) / kColsumChunks;
  const long long r0 = blockIdx.y * chunk;
  const long long r1 = r0 + chunk < rows ? r0 + chunk : rows;
  float s = 0.f;
  if (c < w)
    for (long long r = r0 + threadIdx.y; r < r1; r += 8) s += x[r * w + c];
  red[threadIdx.y][threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.y == 0 && c < w) {
    float t = 0.f;
    for (int i = 0; i < 8; ++i) t += red[i][threadIdx.x];
    part[(size_t)blockIdx.y * w + c] = t;
  }
}

__global__ void colsum_final_kernel(int w, const float* __restrict__ part, float* __restrict__ out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= w) return;
  float s = 0.f;
  for (int i = 0; i < kColsumChunks; ++i) s += part[(size_t)i * w + c];
  out[c] = s;
}

void colsum(long long rows, int w, const float* x, float* out, float* part, cudaStream_t st) {
  colsum_partial_kernel<<<dim3((w + 31) / 32, kColsumChunks), dim3(32, 8), 0, st>>>(rows, w, x, part);
  note_launch();
  colsum_final_kernel<<<(w + 127) / 128, 128, 0, st>>>(w, part, out);
  note_launch();
}

// M = (G + delta I)^-1 per sample (G = Y^T Y, K x K SPD): in-place Gauss-Jordan in FP64
// shared memory, no pivoting (the ridge keeps every pivot positive), one CTA per sample.
__global__ void __launch_bounds__(256) ridge_inverse_kernel(const float* __restrict__ G,
                                                            float* __restrict__ Minv) {
  __shared__ double a[KY][KY + 1];
  __shared__ double colp[KY], rowp[KY];
  const int b = blockIdx.x, tid = threadIdx.x;
  const float* g = G + (size_t)b * KY * KY;
  for (int e = tid; e < KY * KY; e += blockDim.x) {
    const int i = e / KY, j = e - i * KY;
    a[i][j] = 0.5 * ((double)g[i * KY + j] + (double)g[j * KY + i]) + (i == j ? kRidge : 0.0);
  }
  for (int p = 0; p < KY; ++p) {
    __syncthreads();
    if (tid < KY) colp[tid] = a[tid][p];
    __syncthreads();
    const double piv = 1.0 / colp[p];
    if (tid < KY) rowp[tid] = (tid == p ? 1.0 : a[p][tid]) * piv;
    __syncthreads();
    for (int e = tid; e < KY * KY; e += blockDim.x) {
      const int i = e / KY, j = e - i * KY;
      if (i == p) a[i][j] = rowp[j];
      else a[i][j] = (j == p ? 0.0 : a[i][j]) - colp[i] * rowp[j];
    }
  }
  __syncthreads();
  float* m = Minv + (size_t)b * KY * KY;
  for (int e = tid; e < KY * KY; e += blockDim.x) {
    const int i = e / KY, j = e - i * KY;
    m[e] = (float)(0.5 * (a[i][j] + a[j][i]));
  }
}

// S = (2 T + 4 mu (G - I)) / B, the right factor of the Y-part of dY
__global__ void block_grad_factor_kernel(int batch, const float* __restrict__ T,
                                         const float* __restrict__ G, float* __restrict__ S) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)batch * KY * KY) return;
  const int ij = (int)(e % (KY * KY)), i = ij / KY, j = ij - i * KY;
  S[e] = (2.f * T[e] + 4.f * kOrthWeight * (G[e] - (i == j ? 1.f : 0.f))) / batch;
}

// batch means of: K - sum(M o C^T C) (subspace), |G - I|^2 (orthonormality), |s - t|^2
// (bounds); ds = 2 (s - t) / B
__global__ void loss_reduce_kernel(int batch, const float* __restrict__ Minv,
                                   const float* __restrict__ CtC, const float* __restrict__ G,
                                   const float* __restrict__ s, const float* __restrict__ t,
                                   float* __restrict__ ds, double* __restrict__ loss3) {
  __shared__ double red[3][256];
  double l1 = 0, l2 = 0, l3 = 0;
  const long long n2 = (long long)batch * KY * KY;
  for (long long e = threadIdx.x; e < n2; e += blockDim.x) {
    const int ij = (int)(e % (KY * KY)), i = ij / KY, j = ij - i * KY;
    l1 -= (double)Minv[e] * CtC[e];
    const double d = G[e] - (i == j ? 1.0 : 0.0);
    l2 += d * d;
  }
  for (int e = threadIdx.x; e < batch * 2; e += blockDim.x) {
    const double d = (double)s[e] - t[e];
    l3 += d * d;
    ds[e] = (float)(2.0 * d / batch);
  }
  red[0][threadIdx.x] = l1;
  red[1][threadIdx.x] = l2;
  red[2][threadIdx.x] = l3;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o)
      for (int q = 0; q < 3; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    loss3[0] = (double)KY + red[0][0] / batch;
    loss3[1] = red[1][0] / batch;
    loss3[2] = red[2][0] / batch;
  }
}

// dWb[w][j] = sum_b g[b][w] ds[b][j]; dbb[j] = sum_b ds[b][j]; dv4 += (ds Wb^T)/P broadcast
__global__ void bounds_back_kernel(int batch, const float* __restrict__ g, const float* __restrict__ ds,
                                   const __nv_bfloat16* __restrict__ Wb, float* __restrict__ dWb,
                                   float* __restrict__ dbb, float* __restrict__ dv4) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < W * 2) {
    const int w = t / 2, j = t - w * 2;
    float s = 0.f;
    for (int b = 0; b < batch; ++b) s += g[b * W + w] * ds[b * 2 + j];
    dWb[t] = s;
  }
  if (t < 2) {
    float s = 0.f;
    for (int b = 0; b < batch; ++b) s += ds[b * 2 + t];
    dbb[t] = s;
  }
  const long long n = (long long)batch * P * W;
  for (long long e = t; e < n; e += (long long)gridDim.x * blockDim.x) {
    const int w = (int)(e % W);
    const int b = (int)(e / ((long long)P * W));
    const float dg = ds[b * 2] * __bfloat162float(Wb[w * 2]) + ds[b * 2 + 1] * __bfloat162float(Wb[w * 2 + 1]);
    dv4[e] += dg / P;
  }
}

__global__ void adam_kernel(long long count, float* __restrict__ p, const float* __restrict__ g,
                            float* __restrict__ m, float* __restrict__ v, float lr, float b1,
                            float b2, float eps, float c1, float c2, __nv_bfloat16* __restrict__ pb) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= count) return;
  const float gi = g[e];
  const float mi = b1 * m[e] + (1.f - b1) * gi;
  const float vi = b2 * v[e] + (1.f - b2) * gi * gi;
  m[e] = mi;
  v[e] = vi;
  const float pi = p[e] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  p[e] = pi;
  pb[e] = __float2bfloat16_rn(pi);
}

// fine[b][i*n + j][c] (FP64, ld ldf) = bilinear interpolation of coarse[b][p][c], coarse
// node (I, J) sits at fine index position f*I + (f-1)/2; zero outside (Dirichlet)
__global__ void prolong_kernel(int batch, int n, int f, const float* __restrict__ Y,
                               double* __restrict__ fine, int ldf, long long sfine) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long per = (long long)n * n * KY;
  if (e >= batch * per) return;
  const int b = (int)(e / per);
  const long long r = e - b * per;
  const int node = (int)(r / KY), c = (int)(r - (long long)node * KY);
  const int i = node / n, j = node - i * n;
  const double ci = (i - 0.5 * (f - 1)) / f, cj = (j - 0.5 * (f - 1)) / f;
  const int i0 = (int)floor(ci), j0 = (int)floor(cj);
  const double wi = ci - i0, wj = cj - j0;
  const float* Yb = Y + (size_t)b * P * KY;
  auto at = [&](int I, int J) -> double {
    if (I < 0 || J < 0 || I >= S || J >= S) return 0.0;
    return (double)Yb[(size_t)(I * S + J) * KY + c];
  };
  const double v = (1 - wi) * (1 - wj) * at(i0, j0) + wi * (1 - wj) * at(i0 + 1, j0) +
                   (1 - wi) * wj * at(i0, j0 + 1) + wi * wj * at(i0 + 1, j0 + 1);
  fine[b * sfine + (size_t)node * ldf + c] = v;
}

// coarse target: pooled (mean over f x f blocks) fine eigenvectors, FP64 [P][KY]
__global__ void pool_vectors_kernel(int n, int f, const double* __restrict__ evecs, int lde,
                                    double* __restrict__ out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= P * KY) return;
  const int p = e / KY, c = e - p * KY, I = p / S, J = p - I * S;
  double s = 0.0;
  for (int di = 0; di < f; ++di)
    for (int dj = 0; dj < f; ++dj) s += evecs[(size_t)((I * f + di) * n + J * f + dj) * lde + c];
  out[e] = s;
}

__global__ void f64_to_f32_kernel(long long count, const double* __restrict__ in,
                                  float* __restrict__ out) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < count) out[e] = (float)in[e];
}

unsigned nb(long long count, int t = 256) { return (unsigned)((count + t - 1) / t); }

// ---- workspace -------------------------------------------------------------
struct Acts {
  float *in, *v[L + 1], *a[L + 1], *Vr[L], *Vi[L], *Ur, *Ui, *hpre, *hid, *dhid, *Y, *g, *s;
  float *Fr, *Fi, *Gr, *Gs;
  // backward
  float *dv, *dvp, *da, *dUr, *dUi, *dVr, *dVi, *C1, *YtY, *CtC, *Mi, *Tt, *CM, *SmI, *dY, *ds, *part;
  float* grad;
  __nv_bfloat16* wb;  // bf16 copy of the parameters
  double* loss3;
};

template <typename Cv>
Acts carve_acts(Cv& c, int B) {
  Acts a{};
  const size_t bpw = (size_t)B * P * W, bmw = (size_t)B * M * W;
  a.in = c.template take<float>((size_t)B * P * CIN);
  for (int l = 0; l <= L; ++l) {
    a.v[l] = c.template take<float>(bpw);
    a.a[l] = c.template take<float>(bpw);
  }
  for (int l = 0; l < L; ++l) {
    a.Vr[l] = c.template take<float>(bmw);
    a.Vi[l] = c.template take<float>(bmw);
  }
  a.Ur = c.template take<float>(bmw);
  a.Ui = c.template take<float>(bmw);
  a.hpre = c.template take<float>((size_t)B * P * H);
  a.hid = c.template take<float>((size_t)B * P * H);
  a.dhid = c.template take<float>((size_t)B * P * H);
  a.Y = c.template take<float>((size_t)B * P * KY);
  a.g = c.template take<float>((size_t)B * W);
  a.s = c.template take<float>((size_t)B * 2);
  a.Fr = c.template take<float>((size_t)M * P);
  a.Fi = c.template take<float>((size_t)M * P);
  a.Gr = c.template take<float>((size_t)P * M);
  a.Gs = c.template take<float>((size_t)P * M);
  a.dv = c.template take<float>(bpw);
  a.dvp = c.template take<float>(bpw);
  a.da = c.template take<float>(bpw);
  a.dUr = c.template take<float>(bmw);
  a.dUi = c.template take<float>(bmw);
  a.dVr = c.template take<float>(bmw);
  a.dVi = c.template take<float>(bmw);
  a.C1 = c.template take<float>((size_t)B * KY * KY);
  a.YtY = c.template take<float>((size_t)B * KY * KY);
  a.SmI = c.template take<float>((size_t)B * KY * KY);
  a.CtC = c.template take<float>((size_t)B * KY * KY);
  a.Mi = c.template take<float>((size_t)B * KY * KY);
  a.Tt = c.template take<float>((size_t)B * KY * KY);
  a.CM = c.template take<float>((size_t)B * KY * KY);
  a.dY = c.template take<float>((size_t)B * P * KY);
  a.ds = c.template take<float>((size_t)B * 2);
  a.part = c.template take<float>((size_t)kColsumChunks * H);
  a.grad = c.template take<float>(kLay.total);
  a.wb = c.template take<__nv_bfloat16>(kLay.total);
  a.loss3 = c.template take<double>(4);
  return a;
}

struct SizeOnlyL {
  size_t used = 0;
  template <typename T>
  T* take(size_t count) {
    used += align256(count * sizeof(T));
    return nullptr;
  }
};

#define LTRY(x)                        \
  do {                                 \
    cudaError_t _e = (x);              \
    if (_e != cudaSuccess) return _e;  \
  } while (0)

// Forward pass: weights from the BF16 copy (matrices) and FP32 master (biases).
cudaError_t forward(const Acts& A, const float* prm, int B, int s, const double* fields,
                    cudaStream_t st) {
  const __nv_bfloat16* w = A.wb;
  const long long BP = (long long)B * P;
  pool_input_kernel<<<nb(BP), 256, 0, st>>>(B, s, fields, A.in);
  note_launch();
  dft_tables_kernel<<<nb((long long)M * P), 256, 0, st>>>(A.Fr, A.Fi, A.Gr, A.Gs);
  note_launch();
  // lift: v0 = in Wl + bl
  LTRY(bgemm(1, (int)BP, W, CIN, 1.f, A.in, CIN, 0, false, w + kLay.Wl, W, 0, false, 0.f, A.a[0], W,
             0, st));
  bias_act_kernel<<<nb(BP * W), 256, 0, st>>>(BP, W, prm + kLay.bl, A.a[0], A.v[0], false);
  note_launch();
  for (int l = 0; l < L; ++l) {
    const float* vin = A.v[l];
    float* al = A.a[l + 1];
    // Vhat = F v (per sample): [M x P] [P x W]
    LTRY(bgemm(B, M, W, P, 1.f, A.Fr, P, 0, false, vin, W, (long long)P * W, false, 0.f, A.Vr[l], W,
               (long long)M * W, st));
    LTRY(bgemm(B, M, W, P, 1.f, A.Fi, P, 0, false, vin, W, (long long)P * W, false, 0.f, A.Vi[l], W,
               (long long)M * W, st));
    // per mode m: Ur = Vr Rr - Vi Ri, Ui = Vr Ri + Vi Rr   ([B x W] [W x W], batch over m)
    const __nv_bfloat16* Rr = w + kLay.Rr[l];
    const __nv_bfloat16* Ri = w + kLay.Ri[l];
    const int ldv = M * W;
    LTRY(bgemm(M, B, W, W, 1.f, A.Vr[l], ldv, W, false, Rr, W, (long long)W * W, false, 0.f, A.Ur, ldv, W, st));
    LTRY(bgemm(M, B, W, W, -1.f, A.Vi[l], ldv, W, false, Ri, W, (long long)W * W, false, 1.f, A.Ur, ldv, W, st));
    LTRY(bgemm(M, B, W, W, 1.f, A.Vr[l], ldv, W, false, Ri, W, (long long)W * W, false, 0.f, A.Ui, ldv, W, st));
    LTRY(bgemm(M, B, W, W, 1.f, A.Vi[l], ldv, W, false, Rr, W, (long long)W * W, false, 1.f, A.Ui, ldv, W, st));
    // a = Gr Ur - Gs Ui (per sample) + v Wp + bp
    LTRY(bgemm(B, P, W, M, 1.f, A.Gr, M, 0, false, A.Ur, W, (long long)M * W, false, 0.f, al, W,
               (long long)P * W, st));
    LTRY(bgemm(B, P, W, M, -1.f, A.Gs, M, 0, false, A.Ui, W, (long long)M * W, false, 1.f, al, W,
               (long long)P * W, st));
    LTRY(bgemm(1, (int)BP, W, W, 1.f, vin, W, 0, false, w + kLay.Wp[l], W, 0, false, 1.f, al, W, 0, st));
    bias_act_kernel<<<nb(BP * W), 256, 0, st>>>(BP, W, prm + kLay.bp[l], al, A.v[l + 1], l + 1 < L);
    note_launch();
  }
  // heads: Y = gelu(v_L Wh + bh) Wy
  LTRY(bgemm(1, (int)BP, H, W, 1.f, A.v[L], W, 0, false, w + kLay.Wh, H, 0, false, 0.f, A.hpre, H, 0, st));
  bias_act_kernel<<<nb(BP * H), 256, 0, st>>>(BP, H, prm + kLay.bh, A.hpre, A.hid, true);
  note_launch();
  LTRY(bgemm(1, (int)BP, KY, H, 1.f, A.hid, H, 0, false, w + kLay.Wy, KY, 0, false, 0.f, A.Y, KY, 0, st));
  mean_rows_kernel<<<nb((long long)B * W), 256, 0, st>>>(B, P, W, A.v[L], A.g);
  note_launch();
  bounds_head_kernel<<<nb(B * 2), 256, 0, st>>>(B, A.g, w + kLay.Wb, prm + kLay.bb, A.s);
  note_launch();
  return cudaGetLastError();
}

// Loss and backward pass into A.grad (FP32, parameter layout). Q: [B][P][KY]
// orthonormal coarse targets, t: [B][2] log-bounds targets.
cudaError_t loss_backward(const Acts& A, int B, const float* Q, const float* t, cudaStream_t st) {
  const __nv_bfloat16* w = A.wb;
  const long long BP = (long long)B * P;
  const long long sPY = (long long)P * KY, sYY = (long long)KY * KY;
  // C = Q^T Y, G = Y^T Y, C^T C, M = (G + delta I)^-1
  LTRY(bgemm(B, KY, KY, P, 1.f, Q, KY, sPY, true, A.Y, KY, sPY, false, 0.f, A.C1, KY, sYY, st));
  LTRY(bgemm(B, KY, KY, P, 1.f, A.Y, KY, sPY, true, A.Y, KY, sPY, false, 0.f, A.YtY, KY, sYY, st));
  LTRY(bgemm(B, KY, KY, KY, 1.f, A.C1, KY, sYY, true, A.C1, KY, sYY, false, 0.f, A.CtC, KY, sYY, st));
  ridge_inverse_kernel<<<B, 256, 0, st>>>(A.YtY, A.Mi);
  note_launch();
  loss_reduce_kernel<<<1, 256, 0, st>>>(B, A.Mi, A.CtC, A.YtY, A.s, t, A.ds, A.loss3);
  note_launch();
  // dY = Y (2 T + 4 mu (G - I)) / B - (2 / B) Q (C M), T = M C^T C M
  // (CM holds T = M (C^T C M) until it is overwritten with C M)
  LTRY(bgemm(B, KY, KY, KY, 1.f, A.CtC, KY, sYY, false, A.Mi, KY, sYY, false, 0.f, A.Tt, KY, sYY, st));
  LTRY(bgemm(B, KY, KY, KY, 1.f, A.Mi, KY, sYY, false, A.Tt, KY, sYY, false, 0.f, A.CM, KY, sYY, st));
  block_grad_factor_kernel<<<nb((long long)B * sYY), 256, 0, st>>>(B, A.CM, A.YtY, A.SmI);
  note_launch();
  LTRY(bgemm(B, KY, KY, KY, 1.f, A.C1, KY, sYY, false, A.Mi, KY, sYY, false, 0.f, A.CM, KY, sYY, st));
  LTRY(bgemm(B, P, KY, KY, 1.f, A.Y, KY, sPY, false, A.SmI, KY, sYY, false, 0.f, A.dY, KY, sPY, st));
  LTRY(bgemm(B, P, KY, KY, -2.f / B, Q, KY, sPY, false, A.CM, KY, sYY, false, 1.f, A.dY, KY, sPY, st));
  float* g = A.grad;
  LTRY(cudaMemsetAsync(g, 0, sizeof(float) * kLay.total, st));
  // block head: dWy = hid^T dY, dhid = dY Wy^T, dhpre = dhid gelu'(hpre),
  // dWh = v4^T dhpre, dbh = colsum(dhpre), dv4 = dhpre Wh^T
  LTRY(bgemm(1, H, KY, (int)BP, 1.f, A.hid, H, 0, true, A.dY, KY, 0, false, 0.f, g + kLay.Wy, KY, 0, st));
  LTRY(bgemm(1, (int)BP, H, KY, 1.f, A.dY, KY, 0, false, w + kLay.Wy, KY, 0, true, 0.f, A.dhid, H, 0, st));
  gelu_back_kernel<<<nb(BP * H), 256, 0, st>>>(BP * H, A.hpre, A.dhid, A.dhid);
  note_launch();
  LTRY(bgemm(1, W, H, (int)BP, 1.f, A.v[L], W, 0, true, A.dhid, H, 0, false, 0.f, g + kLay.Wh, H, 0, st));
  colsum(BP, H, A.dhid, g + kLay.bh, A.part, st);
  LTRY(bgemm(1, (int)BP, W, H, 1.f, A.dhid, H, 0, false, w + kLay.Wh, H, 0, true, 0.f, A.dv, W, 0, st));
  // bounds head
  bounds_back_kernel<<<nb(BP * W), 256, 0, st>>>(B, A.g, A.ds, w + kLay.Wb, g + kLay.Wb, g + kLay.bb, A.dv);
  note_launch();
  const int ldv = M * W;
  for (int l = L - 1; l >= 0; --l) {
    // da = dv * gelu'(a) (no activation on the last layer)
    float* da = A.da;
    if (l + 1 < L) {
      gelu_back_kernel<<<nb(BP * W), 256, 0, st>>>(BP * W, A.a[l + 1], A.dv, da);
      note_launch();
    } else {
      LTRY(cudaMemcpyAsync(da, A.dv, sizeof(float) * BP * W, cudaMemcpyDeviceToDevice, st));
    }
    const float* vin = A.v[l];
    // pointwise: dWp = vin^T da, dbp = colsum(da), dvp = da Wp^T
    LTRY(bgemm(1, W, W, (int)BP, 1.f, vin, W, 0, true, da, W, 0, false, 0.f, g + kLay.Wp[l], W, 0, st));
    colsum(BP, W, da, g + kLay.bp[l], A.part, st);
    LTRY(bgemm(1, (int)BP, W, W, 1.f, da, W, 0, false, w + kLay.Wp[l], W, 0, true, 0.f, A.dvp, W, 0, st));
    // spectral: dUr = Gr^T da, dUi = -Gs^T da (per sample)
    LTRY(bgemm(B, M, W, P, 1.f, A.Gr, M, 0, true, da, W, (long long)P * W, false, 0.f, A.dUr, W,
               (long long)M * W, st));
    LTRY(bgemm(B, M, W, P, -1.f, A.Gs, M, 0, true, da, W, (long long)P * W, false, 0.f, A.dUi, W,
               (long long)M * W, st));
    // dRr = Vr^T dUr + Vi^T dUi ; dRi = Vr^T dUi - Vi^T dUr   ([W x B] [B x W], batch over m)
    float* dRr = g + kLay.Rr[l];
    float* dRi = g + kLay.Ri[l];
    const long long sWW = (long long)W * W;
    LTRY(bgemm(M, W, W, B, 1.f, A.Vr[l], ldv, W, true, A.dUr, ldv, W, false, 0.f, dRr, W, sWW, st));
    LTRY(bgemm(M, W, W, B, 1.f, A.Vi[l], ldv, W, true, A.dUi, ldv, W, false, 1.f, dRr, W, sWW, st));
    LTRY(bgemm(M, W, W, B, 1.f, A.Vr[l], ldv, W, true, A.dUi, ldv, W, false, 0.f, dRi, W, sWW, st));
    LTRY(bgemm(M, W, W, B, -1.f, A.Vi[l], ldv, W, true, A.dUr, ldv, W, false, 1.f, dRi, W, sWW, st));
    // dVr = dUr Rr^T + dUi Ri^T ; dVi = -dUr Ri^T + dUi Rr^T
    const __nv_bfloat16* Rr = w + kLay.Rr[l];
    const __nv_bfloat16* Ri = w + kLay.Ri[l];
    LTRY(bgemm(M, B, W, W, 1.f, A.dUr, ldv, W, false, Rr, W, sWW, true, 0.f, A.dVr, ldv, W, st));
    LTRY(bgemm(M, B, W, W, 1.f, A.dUi, ldv, W, false, Ri, W, sWW, true, 1.f, A.dVr, ldv, W, st));
    LTRY(bgemm(M, B, W, W, -1.f, A.dUr, ldv, W, false, Ri, W, sWW, true, 0.f, A.dVi, ldv, W, st));
    LTRY(bgemm(M, B, W, W, 1.f, A.dUi, ldv, W, false, Rr, W, sWW, true, 1.f, A.dVi, ldv, W, st));
    // dv_in = dvp + Fr^T dVr + Fi^T dVi (per sample); becomes dv of the layer below
    LTRY(bgemm(B, P, W, M, 1.f, A.Fr, P, 0, true, A.dVr, W, (long long)M * W, false, 1.f, A.dvp, W,
               (long long)P * W, st));
    LTRY(bgemm(B, P, W, M, 1.f, A.Fi, P, 0, true, A.dVi, W, (long long)M * W, false, 1.f, A.dvp, W,
               (long long)P * W, st));
    LTRY(cudaMemcpyAsync(A.dv, A.dvp, sizeof(float) * BP * W, cudaMemcpyDeviceToDevice, st));
  }
  // lift: dWl = in^T dv0, dbl = colsum(dv0)
  LTRY(bgemm(1, CIN, W, (int)BP, 1.f, A.in, CIN, 0, true, A.dv, W, 0, false, 0.f, g + kLay.Wl, W, 0, st));
  colsum(BP, W, A.dv, g + kLay.bl, A.part, st);
  return cudaGetLastError();
}

// Philox-free deterministic init (splitmix64 -> uniform), fan-in scaled.
__global__ void init_params_kernel(float* __restrict__ p, long long count, unsigned long long seed,
                                   Layout lay) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= count) return;
  unsigned long long z = seed + 0x9E3779B97F4A7C15ull * (unsigned long long)(e + 1);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  const float u = (float)((z >> 11) * (1.0 / 9007199254740992.0)) * 2.f - 1.f;  // [-1, 1)
  float scale = 0.f;
  auto in = [&](size_t off, size_t n) { return (size_t)e >= off && (size_t)e < off + n; };
  if (in(lay.Wl, CIN * W)) scale = 1.f / sqrtf((float)CIN);
  for (int l = 0; l < L; ++l) {
    if (in(lay.Rr[l], (size_t)M * W * W) || in(lay.Ri[l], (size_t)M * W * W)) scale = 1.f / W;
    if (in(lay.Wp[l], W * W)) scale = 1.f / sqrtf((float)W);
  }
  if (in(lay.Wh, W * H)) scale = 1.f / sqrtf((float)W);
  if (in(lay.Wy, H * KY)) scale = 1.f / sqrtf((float)H * P);  // unit-norm block columns
  if (in(lay.Wb, W * 2)) scale = 1.f / sqrtf((float)W);
  p[e] = scale * u;
}

}  // namespace
}  // namespace scsf

using namespace scsf;

extern "C" {

size_t scsf_proposal_param_count(void) { return kLay.total; }

size_t scsf_proposal_workspace_size(int batch) {
  if (batch < 1) return 0;
  SizeOnlyL s;
  carve_acts(s, batch);
  return s.used;
}

scsf_status scsf_proposal_init(scsf_ctx* ctx, float* params, uint64_t seed) {
  if (!ctx || !params) return SCSF_ERR_INVALID_ARG;
  if (cudaSetDevice(ctx_device(ctx)) != cudaSuccess) return set_error(ctx, SCSF_ERR_CUDA, "device");
  init_params_kernel<<<nb(kLay.total), 256, 0, ctx_stream(ctx)>>>(params, kLay.total, seed, kLay);
  note_launch();
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SCSF_OK : set_error(ctx, SCSF_ERR_CUDA, cudaGetErrorString(e));
}

static scsf_status prep(scsf_ctx* ctx, int batch, int s, void* ws, size_t ws_bytes, Acts* A) {
  if (batch < 1 || s < S || s % S != 0)
    return set_error(ctx, SCSF_ERR_INVALID_ARG, "need batch >= 1 and field side a multiple of 32");
  Carve c(ws, ws_bytes);
  *A = carve_acts(c, batch);
  if (!c.ok) return set_error(ctx, SCSF_ERR_NO_MEMORY, "proposal workspace too small");
  if (cudaSetDevice(ctx_device(ctx)) != cudaSuccess) return set_error(ctx, SCSF_ERR_CUDA, "device");
  return SCSF_OK;
}

scsf_status scsf_proposal_forward(scsf_ctx* ctx, const float* params, const double* fields, int batch,
                                  int s, float* bounds_out, float* block_out, void* workspace,
                                  size_t workspace_bytes) {
  if (!ctx || !params || !fields) return SCSF_ERR_INVALID_ARG;
  Acts A;
  scsf_status ss = prep(ctx, batch, s, workspace, workspace_bytes, &A);
  if (ss != SCSF_OK) return ss;
  cudaStream_t st = ctx_stream(ctx);
  to_bf16_kernel<<<nb(kLay.total), 256, 0, st>>>(kLay.total, params, A.wb);
  note_launch();
  cudaError_t e = forward(A, params, batch, s, fields, st);
  if (e == cudaSuccess && bounds_out)
    e = cudaMemcpyAsync(bounds_out, A.s, sizeof(float) * batch * 2, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess && block_out)
    e = cudaMemcpyAsync(block_out, A.Y, sizeof(float) * (size_t)batch * P * KY,
                        cudaMemcpyDeviceToDevice, st);
  return e == cudaSuccess ? SCSF_OK : set_error(ctx, SCSF_ERR_CUDA, cudaGetErrorString(e));
}

scsf_status scsf_proposal_train_step(scsf_ctx* ctx, float* params, float* adam_m, float* adam_v,
                                     int step, float lr, const double* fields, int batch, int s,
                                     const float* targets_bounds, const float* targets_Q,
                                     double* loss_host, float* grad_out, void* workspace,
                                     size_t workspace_bytes) {
  if (!ctx || !params || !fields || !targets_bounds || !targets_Q) return SCSF_ERR_INVALID_ARG;
  Acts A;
  scsf_status ss = prep(ctx, batch, s, workspace, workspace_bytes, &A);
  if (ss != SCSF_OK) return ss;
  cudaStream_t st = ctx_stream(ctx);
  to_bf16_kernel<<<nb(kLay.total), 256, 0, st>>>(kLay.total, params, A.wb);
  note_launch();
  cudaError_t e = forward(A, params, batch, s, fields, st);
  if (e == cudaSuccess) e = loss_backward(A, batch, targets_Q, targets_bounds, st);
  if (e == cudaSuccess && grad_out)
    e = cudaMemcpyAsync(grad_out, A.grad, sizeof(float) * kLay.total, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess && adam_m && adam_v && step >= 1 && lr > 0.f) {
    const float b1 = 0.9f, b2 = 0.999f;
    adam_kernel<<<nb(kLay.total), 256, 0, st>>>(kLay.total, params, A.grad, adam_m, adam_v, lr, b1, b2,
                                                1e-8f, 1.f - powf(b1, (float)step),
                                                1.f - powf(b2, (float)step), A.wb);
    note_launch();
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && loss_host) {
    double tmp[3];
    e = cudaMemcpyAsync(tmp, A.loss3, sizeof(tmp), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) std::memcpy(loss_host, tmp, sizeof(tmp));
  }
  return e == cudaSuccess ? SCSF_OK : set_error(ctx, SCSF_ERR_CUDA, cudaGetErrorString(e));
}

scsf_status scsf_proposal_prolong(scsf_ctx* ctx, const float* block, int batch, int n,
                                  double* fine, int ld_fine) {
  if (!ctx || !block || !fine) return SCSF_ERR_INVALID_ARG;
  if (n < S || n % S != 0 || ld_fine < KY)
    return set_error(ctx, SCSF_ERR_INVALID_ARG, "need n a multiple of 32 and ld_fine >= 64");
  if (cudaSetDevice(ctx_device(ctx)) != cudaSuccess) return set_error(ctx, SCSF_ERR_CUDA, "device");
  const long long tot = (long long)batch * n * n * KY;
  prolong_kernel<<<nb(tot), 256, 0, ctx_stream(ctx)>>>(batch, n, n / S, block, fine, ld_fine,
                                                       (long long)n * n * ld_fine);
  note_launch();
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SCSF_OK : set_error(ctx, SCSF_ERR_CUDA, cudaGetErrorString(e));
}

size_t scsf_proposal_target_scratch(void) {
  return align256(sizeof(double) * P * KY) * 3 + align256(sizeof(double) * KY * KY) * 3 +
         align256(sizeof(double) * (size_t)(kSplitTarget + 4) * 1024) + 256;
}

scsf_status scsf_proposal_targets(scsf_ctx* ctx, const double* evecs, int batch, int n, int lde,
                                  float* Q_out, void* scratch, size_t scratch_bytes) {
  if (!ctx || !evecs || !Q_out || !scratch) return SCSF_ERR_INVALID_ARG;
  if (n < S || n % S != 0 || lde < KY)
    return set_error(ctx, SCSF_ERR_INVALID_ARG, "need n a multiple of 32 and at least 64 vectors");
  if (scratch_bytes < scsf_proposal_target_scratch())
    return set_error(ctx, SCSF_ERR_NO_MEMORY, "scratch too small");
  if (cudaSetDevice(ctx_device(ctx)) != cudaSuccess) return set_error(ctx, SCSF_ERR_CUDA, "device");
  cudaStream_t st = ctx_stream(ctx);
  Carve c(scratch, scratch_bytes);
  double* Pc = c.take<double>((size_t)P * KY);
  double* T1 = c.take<double>((size_t)P * KY);
  double* T2 = c.take<double>((size_t)P * KY);
  double* G = c.take<double>(KY * KY);
  double* Lf = c.take<double>(KY * KY);
  double* Ri = c.take<double>(KY * KY);
  double* part = c.take<double>((size_t)(kSplitTarget + 4) * 1024);
  int* status = reinterpret_cast<int*>(c.take<double>(2));
  if (!c.ok) return set_error(ctx, SCSF_ERR_NO_MEMORY, "scratch too small");
  for (int b = 0; b < batch; ++b) {
    pool_vectors_kernel<<<nb(P * KY), 256, 0, st>>>(n, n / S, evecs + (size_t)b * n * n * lde, lde, Pc);
    note_launch();
    // CholQR2 in FP64 on the pooled block
    const double* X = Pc;
    double* outs[2] = {T1, T2};
    for (int pass = 0; pass < 2; ++pass) {
      cudaError_t e = launch_gemm_tn(P, KY, KY, X, KY, X, KY, G, KY, true, part, st);
      if (e == cudaSuccess) e = launch_chol_rinv(KY, G, KY, false, Lf, Ri, status, st);
      if (e == cudaSuccess) e = launch_gemm_nn(P, KY, KY, 1.0, X, KY, Ri, KY, 0.0, outs[pass], KY, true, st);
      if (e != cudaSuccess) return set_error(ctx, SCSF_ERR_CUDA, cudaGetErrorString(e));
      X = outs[pass];
    }
    f64_to_f32_kernel<<<nb(P * KY), 256, 0, st>>>((long long)P * KY, T2, Q_out + (size_t)b * P * KY);
    note_launch();
  }
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SCSF_OK : set_error(ctx, SCSF_ERR_CUDA, cudaGetErrorString(e));
}

}  // extern "C"
