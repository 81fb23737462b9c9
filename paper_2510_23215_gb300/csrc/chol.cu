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
// Up to kSmallBlockWidth both run in one CTA with the matrix in shared memory, right-looking
// in 32-column panels. The FP32 factor (chol_tile_kernel) forms the inverse in the same
// launch and keeps the serial part to the 32 pivots of each diagonal block: the rows below
// solve as a product with the block's inverse and the updates run on register tiles. The
// FP64 factor (chol_blocked_kernel) solves the rows below one thread each, and its inverse
// R^{-1} = (L^{-1})^T is spread over k single-warp CTAs, one column of L^{-1} each.
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

// Exact power-of-two scaling with the format change done on integer bits: the FP64 pipe of a
// GB300 SM is 1/64 of its FP32 rate, so the k^2 conversions of the Gram matrix and of the
// factors would otherwise cost more than the factorisation. Round-to-nearest-even, as the
// hardware conversion; values leaving the normal range take the FP64 path.
// The rare values outside the normal range: out of line, so that the common path is not
// if-converted into executing them (FP64 work for every element).
__device__ __noinline__ float f64_to_f32_pow2_slow(double g, int e) { return (float)ldexp(g, e); }
__device__ __noinline__ double f32_to_f64_pow2_slow(float x, int e) { return ldexp((double)x, e); }

__device__ __forceinline__ float f64_to_f32_pow2(double g, int e) {
  const unsigned hi = (unsigned)__double2hiint(g), lo = (unsigned)__double2loint(g);
  const unsigned sign = hi & 0x80000000u;
  const int ex = (int)((hi >> 20) & 0x7ff);
  if (ex == 0) return __uint_as_float(sign);  // zero or FP64-subnormal: below FP32's range
  int E = ex - 1023 + e;
  if (ex == 0x7ff || E < -126 || E > 127) return f64_to_f32_pow2_slow(g, e);
  // 24 significant bits: the implicit one, 20 bits of hi, the top 3 of lo; 29 bits remain
  unsigned r = 0x800000u | ((hi & 0xfffffu) << 3) | (lo >> 29);
  const unsigned rem = lo & 0x1fffffffu;
  if (rem > 0x10000000u || (rem == 0x10000000u && (r & 1u))) ++r;
  if (r == 0x1000000u) {
    r >>= 1;
    if (++E > 127) return __uint_as_float(sign | 0x7f800000u);
  }
  return __uint_as_float(sign | ((unsigned)(E + 127) << 23) | (r & 0x7fffffu));
}

__device__ __forceinline__ double f32_to_f64_pow2(float x, int e) {
  const unsigned b = __float_as_uint(x);
  const unsigned sign = b & 0x80000000u;
  if ((b & 0x7fffffffu) == 0u) return __hiloint2double((int)sign, 0);
  const int ex = (int)((b >> 23) & 0xff);
  const int E = ex - 127 + e;
  if (ex == 0 || ex == 255 || E < -1022 || E > 1023) return f32_to_f64_pow2_slow(x, e);
  const unsigned hi = sign | ((unsigned)(E + 1023) << 20) | ((b & 0x7fffffu) >> 3);
  return __hiloint2double((int)hi, (int)(b << 29));
}

// Exponent of chol_scale(g) (D_ii = 2^e), from the bits: g = m 2^x, m in [1, 2), e = floor(x / 2).
__device__ __forceinline__ int chol_scale_exp(double g) {
  if (!(g > 0.0 && g < INFINITY)) return 0;
  int x = (int)((__double_as_longlong(g) >> 52) & 0x7ff) - 1023;
  int bias = 0;
  if (x < -1022) {  // FP64-subnormal diagonal
    x = (int)((__double_as_longlong(g * 0x1p200) >> 52) & 0x7ff) - 1023;
    bias = 100;
  }
  return ((x >= 0) ? x / 2 : -((1 - x) / 2)) - bias;
}

// Blocked Cholesky with its inverse for the FP32 first factor (k <= kSmallBlockWidth), one CTA
// of 1024 threads, 32-column panels, the matrix in shared memory. Per panel: warp 0 factors
// the diagonal block with its rows in registers, each column broadcast through shared memory;
// 32 warps form the block's inverse L_pp^-1, one column each; the rows below then solve as a
// product with it, L_21 = A_21 L_pp^-T, and the trailing lower triangle takes the rank-32
// update (from a transposed copy of L_21), both on 2 x 2 register tiles, so that only the 32
// pivots of the diagonal block are serial. X = L^-1 is assembled by block rows alongside,
// block row i as soon as panel i has its diagonal inverse: X_ii = L_ii^-1 and
// X_ij = -L_ii^-1 sum_{j <= m < i} L_im X_mj (2 x 2 tiles), its off-diagonal blocks kept
// transposed in the upper triangle of the shared matrix. Scaling and
// shifted restarts as in chol_blocked_kernel. Output: Rinv = (L^-1)^T (upper, ld k) and
// status; L itself is not written (no caller reads the first factor).
constexpr int kTileThreads = 1024;
constexpr int kTileW = 32;
constexpr int kTilePLd = kSmallBlockWidth - kTileW + 4;  // rows of the transposed panel (even)

size_t chol_tile_smem(int k) {
  const int np = (k + kTileW - 1) / kTileW;
  const size_t sa = ((size_t)k * odd_stride(k) + 3) & ~(size_t)3;  // keeps the blocks aligned
  return (sa + (size_t)(2 * np) * kTileW * (kTileW + 1) + (size_t)kTileW * kTilePLd) * sizeof(float);
}

// One 4-column step of the diagonal-block factorisation (lane = row, column JB .. JB + 3): the
// rows of the step's 4 x 4 pivot block are broadcast and every lane factors it itself (four
// pivots, no exchange), solves its own row against it, and the 4 new entries of every row
// are broadcast for the rank-4 update of the rest. Two buffers each, alternating by step.
// Instantiated per step so that the row stays in registers.
template <int JB>
__device__ __forceinline__ void chol_tile_step4(float (&row)[kTileW], int lane, float* dblk_,
                                                float4* lblk_, float* dinv, int* bad) {
  constexpr int jb = JB;
  float* dsh = dblk_ + ((jb >> 2) & 1) * 16;
  float4* lsh = lblk_ + ((jb >> 2) & 1) * kTileW;
  if (lane >= jb && lane < jb + 4) {
#pragma unroll
    for (int q = 0; q < 4; ++q) dsh[(lane - jb) * 4 + q] = row[jb + q];
  }
  __syncwarp();
  const float4 v0 = reinterpret_cast<const float4*>(dsh)[0];
  const float4 v1 = reinterpret_cast<const float4*>(dsh)[1];
  const float4 v2 = reinterpret_cast<const float4*>(dsh)[2];
  const float4 v3 = reinterpret_cast<const float4*>(dsh)[3];
  bool ok = true;
  float d = v0.x;
  ok = ok && (d > 0.f);
  const float i0 = rsqrtf(ok ? d : 1.f), l00 = (ok ? d : 1.f) * i0;
  const float l10 = v1.x * i0, l20 = v2.x * i0, l30 = v3.x * i0;
  d = fmaf(-l10, l10, v1.y);
  const bool ok1 = d > 0.f;
  const float i1 = rsqrtf(ok1 ? d : 1.f), l11 = (ok1 ? d : 1.f) * i1;
  const float l21 = fmaf(-l20, l10, v2.y) * i1, l31 = fmaf(-l30, l10, v3.y) * i1;
  d = fmaf(-l21, l21, fmaf(-l20, l20, v2.z));
  const bool ok2 = d > 0.f;
  const float i2 = rsqrtf(ok2 ? d : 1.f), l22 = (ok2 ? d : 1.f) * i2;
  const float l32 = fmaf(-l31, l21, fmaf(-l30, l20, v3.z)) * i2;
  d = fmaf(-l32, l32, fmaf(-l31, l31, fmaf(-l30, l30, v3.w)));
  const bool ok3 = d > 0.f;
  const float i3 = rsqrtf(ok3 ? d : 1.f), l33 = (ok3 ? d : 1.f) * i3;
  if (!(ok && ok1 && ok2 && ok3) && lane == 0) *bad = 1;
  float x0 = row[jb], x1 = row[jb + 1], x2 = row[jb + 2], x3 = row[jb + 3];
  if (lane >= jb + 4) {
    x0 = x0 * i0;
    x1 = fmaf(-x0, l10, x1) * i1;
    x2 = fmaf(-x1, l21, fmaf(-x0, l20, x2)) * i2;
    x3 = fmaf(-x2, l32, fmaf(-x1, l31, fmaf(-x0, l30, x3))) * i3;
  } else if (lane >= jb) {  // rows of the pivot block: its factor
    const int q = lane - jb;
    x0 = (q == 0) ? l00 : (q == 1) ? l10 : (q == 2) ? l20 : l30;
    x1 = (q == 1) ? l11 : (q == 2) ? l21 : (q == 3) ? l31 : 0.f;
    x2 = (q == 2) ? l22 : (q == 3) ? l32 : 0.f;
    x3 = (q == 3) ? l33 : 0.f;
  }  // rows above the step: zeros in these columns
  row[jb] = x0;
  row[jb + 1] = x1;
  row[jb + 2] = x2;
  row[jb + 3] = x3;
  if (lane == 0) {
    dinv[jb] = i0;
    dinv[jb + 1] = i1;
    dinv[jb + 2] = i2;
    dinv[jb + 3] = i3;
  }
  lsh[lane] = make_float4(x0, x1, x2, x3);
  __syncwarp();
#pragma unroll
  for (int c = jb + 4; c < kTileW; ++c) {
    if (lane >= c) {
      const float4 v = lsh[c];
      row[c] = fmaf(-x0, v.x, fmaf(-x1, v.y, fmaf(-x2, v.z, fmaf(-x3, v.w, row[c]))));
    }
  }
}

template <int JB>
__device__ __forceinline__ void chol_tile_steps_from(float (&row)[kTileW], int lane, int w, float* d,
                                                     float4* l, float* dinv, int* bad) {
  if constexpr (JB < kTileW) {
    if (JB < w) {
      chol_tile_step4<JB>(row, lane, d, l, dinv, bad);
      chol_tile_steps_from<JB + 4>(row, lane, w, d, l, dinv, bad);
    }
  }
}
__device__ __forceinline__ void chol_tile_steps(float (&row)[kTileW], int lane, int w, float* d,
                                                float4* l, float* dinv, int* bad) {
  chol_tile_steps_from<0>(row, lane, w, d, l, dinv, bad);
}

__global__ void __launch_bounds__(kTileThreads)
chol_tile_kernel(int k, const double* __restrict__ G, int ldg, double* __restrict__ Rinv,
                 int* __restrict__ status, double shift_eps) {
  extern __shared__ __align__(16) float fsm[];
  constexpr int LS = kTileW + 1;  // stride of the 32 x 32 blocks
  const int ks = odd_stride(k);
  const int np = (k + kTileW - 1) / kTileW;
  float* S = fsm;                                        // k x ks: L below, X^T above the diagonal
  float* LI = S + (((size_t)k * ks + 3) & ~(size_t)3);  // per panel: L_pp^-1 [32][LS]
  float* TB = LI + (size_t)np * kTileW * LS;             // inverse assembly: [np][32][LS]
  float* P = TB + (size_t)np * kTileW * LS;              // the panel's L_21 transposed [32][kTilePLd]
  __shared__ int sexp[kSmallBlockWidth];                 // D_ii = 2^sexp[i]
  __shared__ float red[32], dinv[kTileW];
  __shared__ __align__(16) float dblk[2][16];
  __shared__ __align__(16) float4 lblk[2][kTileW];
  __shared__ float trace;
  __shared__ int bad;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  bool out = false;
  double gd = 0.0;
  if (t < k) {
    gd = G[(size_t)t * ldg + t];
    out = chol_out_of_range(gd);
  }
  const bool scaled = __syncthreads_or(out) != 0;
  {
    float part = 0.f;
    if (t < k) {
      const int e = scaled ? chol_scale_exp(gd) : 0;
      sexp[t] = e;
      part = fabsf(f64_to_f32_pow2(gd, -2 * e));
    }
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if (lane == 0) red[warp] = part;
  }
  __syncthreads();
  if (warp == 0) {
    float v = red[lane];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) trace = v;
  }
  int attempt = 0;
  for (; attempt < 4; ++attempt) {
    __syncthreads();
    const float shift = (attempt == 0) ? 0.f
                        : (float)(shift_eps * k * (double)trace * pow(100.0, attempt - 1));
    if (t == 0) bad = 0;
    // S = D^-1 G D^-1 + shift I (lower triangle): warp w takes rows w, w + 32, ..., the lanes
    // the columns; all of a thread's loads are issued before the first conversion
    {
      constexpr int R = kSmallBlockWidth / 32;
      double g[R][R];
#pragma unroll
      for (int a = 0; a < R; ++a)
#pragma unroll
        for (int b = 0; b < R; ++b) {
          const int i = warp + 32 * a, j = lane + 32 * b;
          g[a][b] = (i < k && j <= i) ? G[(size_t)i * ldg + j] : 0.0;
        }
#pragma unroll
      for (int a = 0; a < R; ++a)
#pragma unroll
        for (int b = 0; b < R; ++b) {
          const int i = warp + 32 * a, j = lane + 32 * b;
          if (i < k && j <= i)
            S[i * ks + j] = f64_to_f32_pow2(g[a][b], -(sexp[i] + sexp[j])) + ((i == j) ? shift : 0.f);
        }
    }
    __syncthreads();
    for (int p = 0; p < np; ++p) {
      const int c0 = p * kTileW, w = min(kTileW, k - c0);
      float* LIp = LI + (size_t)p * kTileW * LS;
      if (warp == 0) {
        // The diagonal block, lane = row, in 4-column steps (chol_tile_step4); rows and
        // columns past w are padded with the identity.
        float row[kTileW];
#pragma unroll
        for (int c = 0; c < kTileW; ++c)
          row[c] = (lane < w && c <= lane) ? S[(c0 + lane) * ks + c0 + c]
                                           : ((lane == c && lane >= w) ? 1.f : 0.f);
        chol_tile_steps(row, lane, w, &dblk[0][0], &lblk[0][0], dinv, &bad);
        if (lane < w)
#pragma unroll
          for (int c = 0; c < kTileW; ++c)
            if (c <= lane) S[(c0 + lane) * ks + c0 + c] = row[c];
      }
      __syncthreads();
      // column `warp` of L_pp^-1 by forward substitution, lane r holding x_r
      {
        const int c = warp;
        float x = 0.f;
        if (c < w) {
          float s = 0.f;
          for (int q = c; q < w; ++q) {
            float xq = ((q == c) ? 1.f : -s) * dinv[q];
            xq = __shfl_sync(0xffffffffu, xq, q);
            if (lane == q) x = xq;
            if (lane > q && lane < w) s = fmaf(S[(c0 + lane) * ks + c0 + q], xq, s);
          }
        }
        LIp[lane * LS + c] = (c < w && lane >= c && lane < w) ? x : 0.f;
      }
      __syncthreads();
      const int r0 = c0 + w, nr = k - r0;  // nr > 0 implies w == 32
      const int npr = (nr + 1) / 2;
      // L_21 = A_21 L_pp^-T on 2 x 2 tiles (rows tr, tr + 1, columns tc, tc + 1), and beside it
      // the first half of block row p of X = L^-1: T_j = sum_{j <= m < p} L_{p,m} X_{m,j}
      // (the rows of block p are final once its diagonal block is)
      float a00 = 0.f, a01 = 0.f, a10 = 0.f, a11 = 0.f;
      const bool mine = t < npr * (kTileW / 2);
      const int tr = r0 + 2 * (t / (kTileW / 2)), tc = 2 * (t % (kTileW / 2));
      if (mine) {
        const float* ra = S + (size_t)tr * ks + c0;
        const float* rb = S + (size_t)min(tr + 1, k - 1) * ks + c0;
        const float* l0 = LIp + tc * LS;
        const float* l1 = LIp + (tc + 1) * LS;
#pragma unroll 8
        for (int q = 0; q < kTileW; ++q) {  // L_pp^-1 is zero above its diagonal
          const float x0 = ra[q], x1 = rb[q], y0 = l0[q], y1 = l1[q];
          a00 = fmaf(x0, y0, a00);
          a01 = fmaf(x0, y1, a01);
          a10 = fmaf(x1, y0, a10);
          a11 = fmaf(x1, y1, a11);
        }
      }
      const int hw = (w + 1) / 2;
      const int ntl = p * hw * (kTileW / 2);  // 2 x 2 tiles of the T_j, j < p
      for (int e = t; e < ntl; e += kTileThreads) {
        const int bj = e / (hw * (kTileW / 2)), rem = e - bj * hw * (kTileW / 2);
        const int a = 2 * (rem / (kTileW / 2)), b = 2 * (rem % (kTileW / 2));
        const int ra = c0 + a, rb = min(ra + 1, k - 1);
        const int cb0 = bj * kTileW;
        const float* la = S + (size_t)ra * ks;
        const float* lb = S + (size_t)rb * ks;
        const float* xj = LI + (size_t)bj * kTileW * LS;
        float s00 = 0.f, s01 = 0.f, s10 = 0.f, s11 = 0.f;
#pragma unroll 8
        for (int q = 0; q < kTileW; ++q) {  // m = j: X_jj = L_jj^-1, zero above its diagonal
          const float x0 = la[cb0 + q], x1 = lb[cb0 + q];
          const float y0 = xj[q * LS + b], y1 = xj[q * LS + b + 1];
          s00 = fmaf(x0, y0, s00);
          s01 = fmaf(x0, y1, s01);
          s10 = fmaf(x1, y0, s10);
          s11 = fmaf(x1, y1, s11);
        }
        const float* xc0 = S + (size_t)(cb0 + b) * ks;
        const float* xc1 = S + (size_t)(cb0 + b + 1) * ks;
#pragma unroll 4
        for (int q = cb0 + kTileW; q < c0; ++q) {  // j < m < p: X_mj stored transposed
          const float x0 = la[q], x1 = lb[q], y0 = xc0[q], y1 = xc1[q];
          s00 = fmaf(x0, y0, s00);
          s01 = fmaf(x0, y1, s01);
          s10 = fmaf(x1, y0, s10);
          s11 = fmaf(x1, y1, s11);
        }
        float* tj = TB + (size_t)bj * kTileW * LS;
        tj[a * LS + b] = s00;
        tj[a * LS + b + 1] = s01;
        tj[(a + 1) * LS + b] = s10;  // row w of T_j (odd w) is padding: never read
        tj[(a + 1) * LS + b + 1] = s11;
      }
      __syncthreads();
      if (mine) {
        const int pr = tr - r0;
        S[tr * ks + c0 + tc] = a00;
        S[tr * ks + c0 + tc + 1] = a01;
        if (tr + 1 < k) {
          S[(tr + 1) * ks + c0 + tc] = a10;
          S[(tr + 1) * ks + c0 + tc + 1] = a11;
        }
        // transposed copy (row pr + 1 of an odd nr is padding: never stored back)
        *reinterpret_cast<float2*>(P + tc * kTilePLd + pr) = make_float2(a00, a10);
        *reinterpret_cast<float2*>(P + (tc + 1) * kTilePLd + pr) = make_float2(a01, a11);
      }
      // second half: X_{p,j} = -L_pp^-1 T_j, stored transposed in the upper triangle
      for (int e = t; e < ntl; e += kTileThreads) {
        const int bj = e / (hw * (kTileW / 2)), rem = e - bj * hw * (kTileW / 2);
        const int a = 2 * (rem / (kTileW / 2)), b = 2 * (rem % (kTileW / 2));
        const float* tj = TB + (size_t)bj * kTileW * LS;
        float s00 = 0.f, s01 = 0.f, s10 = 0.f, s11 = 0.f;
        const int qe = min(a + 1, w - 1);
        for (int q = 0; q <= qe; ++q) {  // L_pp^-1 is lower triangular
          const float x0 = LIp[a * LS + q], x1 = LIp[(a + 1) * LS + q];
          const float y0 = tj[q * LS + b], y1 = tj[q * LS + b + 1];
          s00 = fmaf(x0, y0, s00);
          s01 = fmaf(x0, y1, s01);
          s10 = fmaf(x1, y0, s10);
          s11 = fmaf(x1, y1, s11);
        }
        const int c = bj * kTileW + b;
        S[(size_t)c * ks + c0 + a] = -s00;
        S[(size_t)(c + 1) * ks + c0 + a] = -s01;
        if (a + 1 < w) {
          S[(size_t)c * ks + c0 + a + 1] = -s10;
          S[(size_t)(c + 1) * ks + c0 + a + 1] = -s11;
        }
      }
      __syncthreads();
      // trailing lower triangle: S[r][c] -= sum_q L21[r][q] L21[c][q], tiles (R, C), R >= C
      const int ntile = npr * (npr + 1) / 2;
      for (int e = t; e < ntile; e += kTileThreads) {
        int R = (int)((sqrtf(8.f * (float)e + 1.f) - 1.f) * 0.5f);
        while ((R + 1) * (R + 2) / 2 <= e) ++R;
        while (R * (R + 1) / 2 > e) --R;
        const int C = e - R * (R + 1) / 2;
        const int ra = r0 + 2 * R, ca = r0 + 2 * C;
        const float2* pr = reinterpret_cast<const float2*>(P + 2 * R);
        const float2* pc = reinterpret_cast<const float2*>(P + 2 * C);
        float s00 = 0.f, s01 = 0.f, s10 = 0.f, s11 = 0.f;
#pragma unroll 8
        for (int q = 0; q < kTileW; ++q) {
          const float2 x = pr[q * (kTilePLd / 2)], y = pc[q * (kTilePLd / 2)];
          s00 = fmaf(x.x, y.x, s00);
          s01 = fmaf(x.x, y.y, s01);
          s10 = fmaf(x.y, y.x, s10);
          s11 = fmaf(x.y, y.y, s11);
        }
        S[ra * ks + ca] -= s00;
        if (ca + 1 < k && ca + 1 <= ra) S[ra * ks + ca + 1] -= s01;
        if (ra + 1 < k) {
          S[(ra + 1) * ks + ca] -= s10;
          if (ca + 1 < k) S[(ra + 1) * ks + ca + 1] -= s11;
        }
      }
      __syncthreads();
    }
    if (bad == 0) break;
  }
  // Rinv[c][r] = X[r][c] / D_cc for r >= c: warp w takes rows c = w, w + 32, ...
  for (int c = warp; c < k; c += kTileThreads / 32) {
    const int bc = c / kTileW;
    for (int r = lane; r < k; r += 32) {
      float x = 0.f;
      if (r >= c)
        x = (r / kTileW == bc) ? LI[(size_t)bc * kTileW * LS + (r - bc * kTileW) * LS + (c - bc * kTileW)]
                               : S[(size_t)c * ks + r];
      Rinv[(size_t)c * k + r] = f32_to_f64_pow2(x, -sexp[c]);
    }
  }
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
    if (fp32) {  // factor and inverse in one launch
      const size_t smem = chol_tile_smem(k);
      if ((e = ensure_dynamic_smem((const void*)chol_tile_kernel, smem)) != cudaSuccess) return e;
      chol_tile_kernel<<<1, kTileThreads, smem, st>>>(k, G, ldg, Rinv, status, 1e-6);
      note_launch();
      return cudaGetLastError();
    }
    e = launch_chol_t<double>(k, G, ldg, L, status, 1e-14, st);
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
