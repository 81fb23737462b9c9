// FP32 kernels of the mixed-precision path: the FP32 phase of the solver runs
// the Chebyshev filter (Alg. 1), Cholesky QR, Rayleigh-Ritz and rotation on an
// FP32 copy of the block until its subspace stops improving at FP32 accuracy;
// the FP64 phase then finishes to the residual tolerance.
//
// Layout: row-major N x ld blocks with ld % 4 == 0 and the column count a
// multiple of 4 in the stencil kernels, so each thread moves one float4 of a
// node row (16-byte aligned, coalesced across the row). Small k x k matrices
// stay FP64 so the shared Cholesky and eigensolve kernels serve both phases.
#include <algorithm>
#include <condition_variable>
#include <map>
#include <mutex>
#include <set>

#include <cooperative_groups.h>

#include "kernels.cuh"

namespace scsf {
namespace {

constexpr int kThreads = 256;

__global__ void to_f32_kernel(const double* __restrict__ in, float* __restrict__ out, long long count) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) out[i] = (float)in[i];
}

__global__ void block_f32_to_f64_kernel(int rows, int cols, const float* __restrict__ in, int ld_in,
                                        double* __restrict__ out, int ld_out) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)rows * cols) return;
  const int r = (int)(e / cols), c = (int)(e - (long long)r * cols);
  out[(size_t)r * ld_out + c] = (double)in[(size_t)r * ld_in + c];
}

__global__ void block_f64_to_f32_kernel(int rows, int cols, const double* __restrict__ in, int ld_in,
                                        float* __restrict__ out, int ld_out) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)rows * cols) return;
  const int r = (int)(e / cols), c = (int)(e - (long long)r * cols);
  out[(size_t)r * ld_out + c] = (float)in[(size_t)r * ld_in + c];
}

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
__device__ __forceinline__ float4 fma4(float a, float4 x, float4 y) {
  return make_float4(fmaf(a, x.x, y.x), fmaf(a, x.y, y.y), fmaf(a, x.z, y.z), fmaf(a, x.w, y.w));
}

// out = s1 (A cur) + s2 cur + s3 prev, one float4 of one node row per thread.
__device__ __forceinline__ void cheb_step_f32_body(const Stencil32& A, const float* __restrict__ cur,
                                                   int ldc, const float* __restrict__ prev, int ldp,
                                                   float* __restrict__ out, int ldo, int quads,
                                                   float s1, float s2, float s3) {
  const int n = A.n;
  const long long N = (long long)n * n;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N * quads) return;
  const int I = (int)(t / quads);
  const int c = 4 * (int)(t - (long long)I * quads);
  const int i = I / n, j = I - i * n;
  const float* row = cur + (size_t)I * ldc + c;
  const float4 y = ld4(row);
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  if (i < n - 1) acc = fma4(A.we[I], ld4(row + (size_t)n * ldc), acc);
  if (i > 0) acc = fma4(A.we[I - n], ld4(row - (size_t)n * ldc), acc);
  if (j < n - 1) acc = fma4(A.wn[I], ld4(row + ldc), acc);
  if (j > 0) acc = fma4(A.wn[I - 1], ld4(row - ldc), acc);
  const float diag = fmaf(s1, A.d[I], s2);
  float4 r = make_float4(fmaf(-s1, acc.x, diag * y.x), fmaf(-s1, acc.y, diag * y.y),
                         fmaf(-s1, acc.z, diag * y.z), fmaf(-s1, acc.w, diag * y.w));
  if (prev) r = fma4(s3, ld4(prev + (size_t)I * ldp + c), r);
  st4(out + (size_t)I * ldo + c, r);
}

__global__ void __launch_bounds__(1024)
cheb_step_f32_kernel(Stencil32 A, const float* __restrict__ cur, int ldc,
                     const float* __restrict__ prev, int ldp, float* __restrict__ out, int ldo,
                     int quads, float s1, float s2, float s3) {
  cheb_step_f32_body(A, cur, ldc, prev, ldp, out, ldo, quads, s1, s2, s3);
}

// The same step with its scalars read from a device table (coef = {s1, s2, s3}), so that a
// captured graph of the whole filter can be replayed with new scalars every iteration.
__global__ void __launch_bounds__(1024)
cheb_step_f32_tab_kernel(Stencil32 A, const float* __restrict__ cur, int ldc,
                         const float* __restrict__ prev, int ldp, float* __restrict__ out, int ldo,
                         int quads, const float* __restrict__ coef) {
  cheb_step_f32_body(A, cur, ldc, prev, ldp, out, ldo, quads, coef[0], coef[1], coef[2]);
}

// ---- cluster-resident FP32 filter ----------------------------------------------
// The whole m-step recurrence for one group of 4 columns runs in one thread-block cluster:
// the kClu CTAs of the cluster split the n grid rows into bands, and each keeps its band of
// both recurrence levels (float4 per node, plus one halo row above and below) and its
// stencil coefficients in shared memory for all m steps. After every step the cluster
// synchronises and each CTA copies its neighbours' boundary rows of the new level into its
// halo rows through distributed shared memory. Global memory is touched only to load Y_0
// and the coefficients and to store Y_m; per step the traffic is the halo exchange.
namespace cg = cooperative_groups;

template <int kClu>
__device__ __forceinline__ int band_begin(int rank, int n) { return rank * n / kClu; }

template <int kClu>
__global__ void __launch_bounds__(1024)
cheb_filter_f32_cluster_kernel(Stencil32 A, const float* __restrict__ Y0, int ld0,
                               float* __restrict__ out, int ldo, int m,
                               const float* __restrict__ coef) {
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int n = A.n;
  const int r0 = band_begin<kClu>(rank, n), r1 = band_begin<kClu>(rank + 1, n);
  const int rows = r1 - r0;
  const int hrm = (n + kClu - 1) / kClu + 2;  // local rows incl. halos (same on every rank)
  const int cg4 = 4 * blockIdx.y;             // first column of this cluster's group
  const int t = threadIdx.x, nt = blockDim.x;
  extern __shared__ float4 sm4[];
  float4* L0 = sm4;
  float4* L1 = sm4 + (size_t)hrm * n;
  float* cd = reinterpret_cast<float*>(sm4 + 2 * (size_t)hrm * n);  // d, rows x n
  float* cwe = cd + (size_t)(hrm - 2) * n;  // we of global rows r0-1 .. r1-1, (rows+1) x n
  float* cwn = cwe + (size_t)(hrm - 1) * n; // wn, rows x n
  for (int e = t; e < rows * n; e += nt) {
    const int I = r0 * n + e;
    cd[e] = A.d[I];
    cwn[e] = A.wn[I];
  }
  for (int e = t; e < (rows + 1) * n; e += nt) {
    const int gi = r0 - 1 + e / n;
    cwe[e] = (gi >= 0) ? A.we[gi * n + (e - (e / n) * n)] : 0.f;
  }
  // Y_0: own rows and both halo rows (zero outside the grid); local row lr <-> global r0-1+lr
  for (int e = t; e < (rows + 2) * n; e += nt) {
    const int lr = e / n, j = e - lr * n, gi = r0 - 1 + lr;
    L0[e] = (gi >= 0 && gi < n) ? ld4(Y0 + (size_t)(gi * n + j) * ld0 + cg4)
                                : make_float4(0.f, 0.f, 0.f, 0.f);
  }
  __syncthreads();
  float4* C = L0;
  float4* P = L1;
  const int rows_above = (rank > 0) ? r0 - band_begin<kClu>(rank - 1, n) : 0;
  for (int s = 0; s < m; ++s) {
    const float s1 = coef[3 * s], s2 = coef[3 * s + 1], s3 = coef[3 * s + 2];
    for (int e = t; e < rows * n; e += nt) {
      const int q = e / n, j = e - q * n, lr = q + 1, gi = r0 + q;
      const float4* row = C + (size_t)lr * n + j;
      const float4 y = row[0];
      float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
      if (gi < n - 1) acc = fma4(cwe[(size_t)(q + 1) * n + j], row[n], acc);
      if (gi > 0) acc = fma4(cwe[(size_t)q * n + j], row[-n], acc);
      if (j < n - 1) acc = fma4(cwn[e], row[1], acc);
      if (j > 0) acc = fma4(cwn[e - 1], row[-1], acc);
      const float diag = fmaf(s1, cd[e], s2);
      float4 r = make_float4(fmaf(-s1, acc.x, diag * y.x), fmaf(-s1, acc.y, diag * y.y),
                             fmaf(-s1, acc.z, diag * y.z), fmaf(-s1, acc.w, diag * y.w));
      if (s > 0) r = fma4(s3, P[(size_t)lr * n + j], r);
      P[(size_t)lr * n + j] = r;
    }
    cluster.sync();  // every band of the new level is final
    if (rank > 0) {
      const float4* up = cluster.map_shared_rank(P, rank - 1);
      for (int j = t; j < n; j += nt) P[j] = up[(size_t)rows_above * n + j];
    }
    if (rank < kClu - 1) {
      const float4* dn = cluster.map_shared_rank(P, rank + 1);
      for (int j = t; j < n; j += nt) P[(size_t)(rows + 1) * n + j] = dn[(size_t)n + j];
    }
    __syncthreads();
    float4* tmp = C;
    C = P;
    P = tmp;
  }
  for (int e = t; e < rows * n; e += nt) {
    const int q = e / n, j = e - q * n;
    st4(out + (size_t)((r0 + q) * n + j) * ldo + cg4, C[(size_t)(q + 1) * n + j]);
  }
  // no CTA may leave while a neighbour can still read its shared memory
  cluster.sync();
}

// The defect-corrected recurrence Z_{i+1} = s1 A Z_i + s2 Z_i + s3 Z_{i-1} + s1 R diag(y_i),
// Z_0 = 0, resident the same way: per 4-column group, the cluster's bands keep both Z levels,
// the band of R and the stencil coefficients in shared memory; coef: [m][3] step scalars,
// ytab: [m][ncols] scalar values y_i. Columns >= ncols of the last group are padding.
template <int kClu>
__global__ void __launch_bounds__(1024)
dc_filter_cluster_kernel(Stencil32 A, const float* __restrict__ R, int ldr, int ncols,
                         const float* __restrict__ ytab, const float* __restrict__ coef, int m,
                         float* __restrict__ out, int ldo, const int* __restrict__ gdeg) {
  // per-column-group degree (all CTAs of a cluster share blockIdx.y, so the step count, and
  // with it the number of cluster barriers, is uniform within the cluster)
  if (gdeg) m = min(m, max(gdeg[blockIdx.y], 1));
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int n = A.n;
  const int r0 = band_begin<kClu>(rank, n), r1 = band_begin<kClu>(rank + 1, n);
  const int rows = r1 - r0;
  const int hrm = (n + kClu - 1) / kClu + 2;
  const int c0 = 4 * blockIdx.y;
  const int t = threadIdx.x, nt = blockDim.x;
  extern __shared__ float4 sm4[];
  float4* L0 = sm4;
  float4* L1 = sm4 + (size_t)hrm * n;
  float4* Rb = sm4 + 2 * (size_t)hrm * n;                                    // rows x n
  float* cd = reinterpret_cast<float*>(sm4 + (size_t)(3 * hrm - 2) * n);    // rows x n
  float* cwe = cd + (size_t)(hrm - 2) * n;                                  // (rows+1) x n
  float* cwn = cwe + (size_t)(hrm - 1) * n;                                 // rows x n
  // the float section is padded to whole float4s so that yt stays 16-byte aligned
  const size_t fl = ((size_t)(3 * (hrm - 2) + 1) * n + 3) & ~(size_t)3;
  float4* yt = reinterpret_cast<float4*>(cd + fl);                          // m
  for (int e = t; e < rows * n; e += nt) {
    const int I = r0 * n + e;
    cd[e] = A.d[I];
    cwn[e] = A.wn[I];
    const float* rr = R + (size_t)I * ldr + c0;
    Rb[e] = make_float4(rr[0], (c0 + 1 < ncols) ? rr[1] : 0.f, (c0 + 2 < ncols) ? rr[2] : 0.f,
                        (c0 + 3 < ncols) ? rr[3] : 0.f);
  }
  for (int e = t; e < (rows + 1) * n; e += nt) {
    const int gi = r0 - 1 + e / n;
    cwe[e] = (gi >= 0) ? A.we[gi * n + (e - (e / n) * n)] : 0.f;
  }
  for (int i = t; i < m; i += nt) {
    const float* y = ytab + (size_t)i * ncols + c0;
    yt[i] = make_float4(y[0], (c0 + 1 < ncols) ? y[1] : 0.f, (c0 + 2 < ncols) ? y[2] : 0.f,
                        (c0 + 3 < ncols) ? y[3] : 0.f);
  }
  for (int e = t; e < (rows + 2) * n; e += nt) L0[e] = make_float4(0.f, 0.f, 0.f, 0.f);  // Z_0
  __syncthreads();
  float4* C = L0;
  float4* P = L1;
  const int rows_above = (rank > 0) ? r0 - band_begin<kClu>(rank - 1, n) : 0;
  for (int s = 0; s < m; ++s) {
    const float s1 = coef[3 * s], s2 = coef[3 * s + 1], s3 = coef[3 * s + 2];
    const float4 ys = yt[s];
    for (int e = t; e < rows * n; e += nt) {
      const int q = e / n, j = e - q * n, lr = q + 1, gi = r0 + q;
      const float4* row = C + (size_t)lr * n + j;
      const float4 z = row[0];
      float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
      if (gi < n - 1) acc = fma4(cwe[(size_t)(q + 1) * n + j], row[n], acc);
      if (gi > 0) acc = fma4(cwe[(size_t)q * n + j], row[-n], acc);
      if (j < n - 1) acc = fma4(cwn[e], row[1], acc);
      if (j > 0) acc = fma4(cwn[e - 1], row[-1], acc);
      const float diag = fmaf(s1, cd[e], s2);
      const float4 rv = Rb[e];
      float4 r = make_float4(fmaf(-s1, acc.x, fmaf(diag, z.x, s1 * rv.x * ys.x)),
                             fmaf(-s1, acc.y, fmaf(diag, z.y, s1 * rv.y * ys.y)),
                             fmaf(-s1, acc.z, fmaf(diag, z.z, s1 * rv.z * ys.z)),
                             fmaf(-s1, acc.w, fmaf(diag, z.w, s1 * rv.w * ys.w)));
      if (s > 0) r = fma4(s3, P[(size_t)lr * n + j], r);
      P[(size_t)lr * n + j] = r;
    }
    cluster.sync();
    if (rank > 0) {
      const float4* up = cluster.map_shared_rank(P, rank - 1);
      for (int j = t; j < n; j += nt) P[j] = up[(size_t)rows_above * n + j];
    }
    if (rank < kClu - 1) {
      const float4* dn = cluster.map_shared_rank(P, rank + 1);
      for (int j = t; j < n; j += nt) P[(size_t)(rows + 1) * n + j] = dn[(size_t)n + j];
    }
    __syncthreads();
    float4* tmp = C;
    C = P;
    P = tmp;
  }
  for (int e = t; e < rows * n; e += nt) {
    const int q = e / n, j = e - q * n;
    const float4 v = C[(size_t)(q + 1) * n + j];
    float* o = out + (size_t)((r0 + q) * n + j) * ldo + c0;
    o[0] = v.x;
    if (c0 + 1 < ncols) o[1] = v.y;
    if (c0 + 2 < ncols) o[2] = v.z;
    if (c0 + 3 < ncols) o[3] = v.w;
  }
  cluster.sync();
}

template <int kClu>
size_t cluster_dc_smem(int n, int m) {
  const size_t hrm = (size_t)(n + kClu - 1) / kClu + 2;
  const size_t fl = ((3 * (hrm - 2) + 1) * (size_t)n + 3) & ~(size_t)3;
  return (3 * hrm - 2) * n * sizeof(float4) + fl * sizeof(float) + (size_t)m * sizeof(float4);
}

template <int kClu>
size_t cluster_filter_smem(int n) {
  const size_t hrm = (size_t)(n + kClu - 1) / kClu + 2;
  return 2 * hrm * n * sizeof(float4) + (3 * (hrm - 2) + 1) * (size_t)n * sizeof(float);
}

// Register-resident strips for both cluster-resident filters. The cluster's bands split the
// grid rows as above; inside a band every thread owns a vertical strip of kStripV rows of one
// grid column and keeps, in registers, the current recurrence level of its 4-column float4
// entries and their stencil coefficients. A step then reads from shared memory only the row
// above and the row below the strip, the horizontal neighbours and the level before (which
// the new level overwrites in place): 2 + 3 kStripV float4 loads per kStripV entries, against
// 6 float4 and 5 coefficient loads per entry when everything lives in shared memory.
// kDc: the defect-corrected remainder Z (Z_0 = 0, driven by s1 R diag(y_i), R in shared
// memory); otherwise the filter itself from Y_0 = X. Halos are exchanged through DSMEM after
// each step as in the kernels above; rows outside the grid stay zero (zero coefficients).
constexpr int kStripV = 4;

template <int kClu, bool kDc>
__global__ void __launch_bounds__(1024)
strip_filter_cluster_kernel(Stencil32 A, const float* __restrict__ X, int ldx, int ncols,
                            const float* __restrict__ ytab, const float* __restrict__ coef, int m,
                            float* __restrict__ out, int ldo, const int* __restrict__ gdeg) {
  if (kDc && gdeg) m = min(m, max(gdeg[blockIdx.y], 1));  // uniform within the cluster
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int n = A.n;
  const int r0 = band_begin<kClu>(rank, n), r1 = band_begin<kClu>(rank + 1, n);
  const int rows = r1 - r0;
  const int hrm = (n + kClu - 1) / kClu + 2;  // local rows incl. halos (same on every rank)
  const int c0 = 4 * blockIdx.y;
  const int t = threadIdx.x, nt = blockDim.x;
  extern __shared__ float4 sm4[];
  float4* L0 = sm4;
  float4* L1 = sm4 + (size_t)hrm * n;
  float4* Rb = sm4 + 2 * (size_t)hrm * n;           // kDc: own rows x n
  float4* yt = Rb + (size_t)(hrm - 2) * n;           // kDc: m step values
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int e = t; e < hrm * n; e += nt) {
    L0[e] = z4;
    L1[e] = z4;
  }
  __syncthreads();
  if (!kDc) {  // Y_0: own rows and both halo rows; local row lr <-> global r0 - 1 + lr
    for (int e = t; e < (rows + 2) * n; e += nt) {
      const int lr = e / n, j = e - lr * n, gi = r0 - 1 + lr;
      if (gi >= 0 && gi < n) L0[e] = ld4(X + (size_t)(gi * n + j) * ldx + c0);
    }
  } else {
    for (int e = t; e < rows * n; e += nt) {
      const float* rr = X + (size_t)(r0 * n + e) * ldx + c0;
      Rb[e] = make_float4(rr[0], (c0 + 1 < ncols) ? rr[1] : 0.f, (c0 + 2 < ncols) ? rr[2] : 0.f,
                          (c0 + 3 < ncols) ? rr[3] : 0.f);
    }
    for (int i = t; i < m; i += nt) {
      const float* y = ytab + (size_t)i * ncols + c0;
      yt[i] = make_float4(y[0], (c0 + 1 < ncols) ? y[1] : 0.f, (c0 + 2 < ncols) ? y[2] : 0.f,
                          (c0 + 3 < ncols) ? y[3] : 0.f);
    }
  }
  // this thread's strip: column j, own rows q0 .. q0 + kStripV - 1 (those below rows unused)
  const int j = t % n, q0 = (t / n) * kStripV;
  const bool active = q0 < rows;
  float4 cur[kStripV];
  float cd[kStripV], cs[kStripV], ce[kStripV], cw[kStripV], cn0 = 0.f;
#pragma unroll
  for (int v = 0; v < kStripV; ++v) {
    const int q = q0 + v, gi = r0 + q, I = gi * n + j;
    const bool own = active && q < rows;
    cd[v] = own ? A.d[I] : 0.f;
    cs[v] = (own && gi < n - 1) ? A.we[I] : 0.f;      // coupling to the row below
    ce[v] = (own && j < n - 1) ? A.wn[I] : 0.f;       // to the right
    cw[v] = (own && j > 0) ? A.wn[I - 1] : 0.f;       // to the left
    if (v == 0) cn0 = (own && gi > 0) ? A.we[I - n] : 0.f;  // to the row above the strip
  }
  __syncthreads();
#pragma unroll
  for (int v = 0; v < kStripV; ++v)
    cur[v] = (!kDc && active && q0 + v < rows) ? L0[(size_t)(q0 + v + 1) * n + j] : z4;
  float4* C = L0;
  float4* P = L1;
  const int rows_above = (rank > 0) ? r0 - band_begin<kClu>(rank - 1, n) : 0;
  for (int s = 0; s < m; ++s) {
    const float s1 = coef[3 * s], s2 = coef[3 * s + 1], s3 = coef[3 * s + 2];
    if (active) {
      const float4 ys = kDc ? yt[s] : z4;
      float4 up = C[(size_t)q0 * n + j];  // the row above the strip (a halo for q0 = 0)
      float cn = cn0;                     // coupling to it
#pragma unroll
      for (int v = 0; v < kStripV; ++v) {
        const int q = q0 + v;
        if (q < rows) {
          const size_t at = (size_t)(q + 1) * n + j;
          const float4 y = cur[v];
          const float4 dn = (v + 1 < kStripV && q + 1 < rows) ? cur[(v + 1) % kStripV] : C[at + n];
          const float4 ea = C[at + 1], we = C[at - 1];  // in bounds; zero weight off the grid
          float4 acc = make_float4(cs[v] * dn.x, cs[v] * dn.y, cs[v] * dn.z, cs[v] * dn.w);
          acc = fma4(cn, up, acc);
          acc = fma4(ce[v], ea, acc);
          acc = fma4(cw[v], we, acc);
          const float diag = fmaf(s1, cd[v], s2);
          const float4 pv = P[at];  // the level before (zero at the first step)
          float4 r = make_float4(fmaf(-s1, acc.x, fmaf(diag, y.x, s3 * pv.x)),
                                 fmaf(-s1, acc.y, fmaf(diag, y.y, s3 * pv.y)),
                                 fmaf(-s1, acc.z, fmaf(diag, y.z, s3 * pv.z)),
                                 fmaf(-s1, acc.w, fmaf(diag, y.w, s3 * pv.w)));
          if (kDc) {
            const float4 rv = Rb[at - n];
            r = make_float4(fmaf(s1 * rv.x, ys.x, r.x), fmaf(s1 * rv.y, ys.y, r.y),
                            fmaf(s1 * rv.z, ys.z, r.z), fmaf(s1 * rv.w, ys.w, r.w));
          }
          P[at] = r;
          cur[v] = r;
          up = y;
          cn = cs[v];  // the next row's coupling upwards is this row's coupling downwards
        }
      }
    }
    cluster.sync();  // every band of the new level is final
    if (rank > 0) {
      const float4* upr = cluster.map_shared_rank(P, rank - 1);
      for (int jj = t; jj < n; jj += nt) P[jj] = upr[(size_t)rows_above * n + jj];
    }
    if (rank < kClu - 1) {
      const float4* dnr = cluster.map_shared_rank(P, rank + 1);
      for (int jj = t; jj < n; jj += nt) P[(size_t)(rows + 1) * n + jj] = dnr[(size_t)n + jj];
    }
    __syncthreads();
    float4* tmp = C;
    C = P;
    P = tmp;
  }
  if (active) {
#pragma unroll
    for (int v = 0; v < kStripV; ++v) {
      const int q = q0 + v;
      if (q < rows) {
        float* o = out + (size_t)((r0 + q) * n + j) * ldo + c0;
        const bool vec = (ldo & 3) == 0 && (reinterpret_cast<uintptr_t>(out) & 15) == 0;
        if (!kDc || (vec && c0 + 3 < ncols)) {
          st4(o, cur[v]);
        } else {
          o[0] = cur[v].x;
          if (c0 + 1 < ncols) o[1] = cur[v].y;
          if (c0 + 2 < ncols) o[2] = cur[v].z;
          if (c0 + 3 < ncols) o[3] = cur[v].w;
        }
      }
    }
  }
  // no CTA may leave while a neighbour can still read its shared memory
  cluster.sync();
}

// Threads of a strip launch (0: the band does not fit one CTA's 1024 threads).
template <int kClu>
int strip_threads(int n) {
  const int hmax = (n + kClu - 1) / kClu;
  const int th = n * ((hmax + kStripV - 1) / kStripV);
  return (th <= 1024) ? ((th + 31) / 32) * 32 : 0;
}

template <int kClu>
size_t strip_smem(int n, bool dc, int m) {
  const size_t hrm = (size_t)(n + kClu - 1) / kClu + 2;
  return (2 * hrm * n + (dc ? (hrm - 2) * n + (size_t)m : 0)) * sizeof(float4);
}

// ---- defect-corrected filter ------------------------------------------------
// The filter's three-term recurrence Y_{i+1} = s1 A Y_i + s2 Y_i + s3 Y_{i-1} started
// from Y_0 = X splits exactly as Y_i = X diag(y_i) + Z_i: y_i(theta_j) is the same
// recurrence on the scalar theta_j, and with A X = X diag(theta) + R the remainder obeys
// Z_{i+1} = s1 A Z_i + s2 Z_i + s3 Z_{i-1} + s1 R diag(y_i), Z_0 = 0. Near convergence
// Z is of the size of R, so it is computed in FP32 while X diag(y_m) stays in FP64:
// the result has FP64 accuracy at the cost of an FP32 stencil sweep.

// One thread per column: y_i(theta_j) for the steps [i0, i0 + count) of the filter,
// y_{i+1} = (s1_i theta + s2_i) y_i + s3_i y_{i-1} with the filter's own (host-computed)
// coefficients. y_i goes to ytab row i (FP32); state [2][ncols] carries (y_{i-1}, y_i)
// in FP64 from chunk to chunk, and after the last chunk state[1] holds y_m. With per-group
// degrees (gdeg), ysel[j] = y_d (FP64) at the degree d of column j's group.
__global__ void dc_ytab_kernel(const double* __restrict__ theta, int ncols, DcSteps P,
                               float* __restrict__ ytab, double* __restrict__ state,
                               const int* __restrict__ gdeg, double* __restrict__ ysel) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= ncols) return;
  const double t = theta[j];
  const int d = gdeg ? gdeg[j / 4] : -1;
  double yp = (P.i0 == 0) ? 0.0 : state[j];
  double y = (P.i0 == 0) ? 1.0 : state[ncols + j];
  for (int q = 0; q < P.count; ++q) {
    ytab[(size_t)(P.i0 + q) * ncols + j] = (float)y;
    if (P.i0 + q == d) ysel[j] = y;
    const double yn = fma(fma(P.s1[q], t, P.s2[q]), y, P.s3[q] * yp);
    yp = y;
    y = yn;
  }
  if (P.i0 + P.count == d) ysel[j] = y;
  state[j] = yp;
  state[ncols + j] = y;
}

constexpr int kDcRows = 8;
constexpr int kDcUnroll = 4;  // column chunks of 32 in flight per thread
template <bool kCur, bool kPrev>
__global__ void __launch_bounds__(32 * kDcRows)
cheb_step_dc_kernel(Stencil32 A, const float* __restrict__ cur, const float* __restrict__ prev,
                    int ld, const float* __restrict__ R, int ldr, const float* __restrict__ ycol,
                    float* __restrict__ out, int ncols, float s1, float s2, float s3) {
  const int n = A.n, N = n * n;
  for (int I = blockIdx.x * kDcRows + threadIdx.y; I < N; I += gridDim.x * kDcRows) {
    const int i = I / n, j = I - i * n;
    float d = 0.f, wS = 0.f, wN = 0.f, wE = 0.f, wW = 0.f;
    if (kCur) {
      d = A.d[I];
      wS = (i < n - 1) ? A.we[I] : 0.f;
      wN = (i > 0) ? A.we[I - n] : 0.f;
      wE = (j < n - 1) ? A.wn[I] : 0.f;
      wW = (j > 0) ? A.wn[I - 1] : 0.f;
    }
    const size_t o = (size_t)I * ld;
    const float* rrow = R + (size_t)I * ldr;
    for (int c0 = threadIdx.x; c0 < ncols; c0 += 32 * kDcUnroll) {
      // all loads of kDcUnroll chunks first, then the arithmetic and the stores
      float rv[kDcUnroll], yc[kDcUnroll], y0[kDcUnroll], ys[kDcUnroll], yn[kDcUnroll],
          ye[kDcUnroll], yw[kDcUnroll], yp[kDcUnroll];
#pragma unroll
      for (int u = 0; u < kDcUnroll; ++u) {
        const int c = c0 + 32 * u;
        const bool ok = c < ncols;
        rv[u] = ok ? rrow[c] : 0.f;
        yc[u] = ok ? ycol[c] : 0.f;
        if (kCur) {
          const float* row = cur + o + c;
          y0[u] = ok ? row[0] : 0.f;
          ys[u] = (ok && i < n - 1) ? row[(size_t)n * ld] : 0.f;
          yn[u] = (ok && i > 0) ? row[-(long long)n * ld] : 0.f;
          ye[u] = (ok && j < n - 1) ? row[ld] : 0.f;
          yw[u] = (ok && j > 0) ? row[-(long long)ld] : 0.f;
        }
        if (kPrev) yp[u] = ok ? prev[o + c] : 0.f;
      }
#pragma unroll
      for (int u = 0; u < kDcUnroll; ++u) {
        const int c = c0 + 32 * u;
        if (c >= ncols) break;
        float r = s1 * rv[u] * yc[u];
        if (kCur) {
          const float acc = fmaf(wW, yw[u], fmaf(wE, ye[u], fmaf(wN, yn[u], wS * ys[u])));
          r = fmaf(s1, fmaf(d, y0[u], -acc), fmaf(s2, y0[u], r));
        }
        if (kPrev) r = fmaf(s3, yp[u], r);
        out[o + c] = r;
      }
    }
  }
}

__global__ void dc_combine_kernel(int rows, int ncols, const double* __restrict__ X, int ldx,
                                  const double* __restrict__ ym, const float* __restrict__ Z, int ldz,
                                  double* __restrict__ Y, int ldy) {
  const long long tot = (long long)rows * ncols;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const int I = (int)(e / ncols), c = (int)(e - (long long)I * ncols);
    Y[(size_t)I * ldy + c] = fma(X[(size_t)I * ldx + c], ym[c], (double)Z[(size_t)I * ldz + c]);
  }
}

// Per-column ||(A X)_j - theta_j X_j||^2 and ||(A X)_j||^2 (FP32 products, FP64 sums).
// blockIdx.y selects a slice of kSmallBlockWidth columns.
constexpr int kRows32 = 8;
__global__ void __launch_bounds__(32 * kRows32)
residual_norms_f32_kernel(Stencil32 A, const float* __restrict__ X, int ldx, int ncols,
                          const double* __restrict__ theta, double* __restrict__ partials) {
  constexpr int kChunks = kSmallBlockWidth / 32;
  const int n = A.n, N = n * n;
  const int c0 = blockIdx.y * kSmallBlockWidth;
  double rr[kChunks], aa[kChunks];
  float th[kChunks];
#pragma unroll
  for (int q = 0; q < kChunks; ++q) {
    rr[q] = aa[q] = 0.0;
    const int c = c0 + threadIdx.x + 32 * q;
    th[q] = (c < ncols) ? (float)theta[c] : 0.f;
  }
  for (int I = blockIdx.x * kRows32 + threadIdx.y; I < N; I += gridDim.x * kRows32) {
    const int i = I / n, j = I - i * n;
    const float d = A.d[I], wE = A.we[I], wW = (i > 0) ? A.we[I - n] : 0.f, wN = A.wn[I],
                wS = (j > 0) ? A.wn[I - 1] : 0.f;
    const float* row = X + (size_t)I * ldx;
#pragma unroll
    for (int q = 0; q < kChunks; ++q) {
      const int c = c0 + threadIdx.x + 32 * q;
      if (c < ncols) {
        const float x = row[c];
        float off = 0.f;
        if (i < n - 1) off = fmaf(wE, row[(size_t)n * ldx + c], off);
        if (i > 0) off = fmaf(wW, row[-(ptrdiff_t)((size_t)n * ldx) + c], off);
        if (j < n - 1) off = fmaf(wN, row[ldx + c], off);
        if (j > 0) off = fmaf(wS, row[-(ptrdiff_t)ldx + c], off);
        const float ax = fmaf(d, x, -off);
        const float r = fmaf(-th[q], x, ax);
        rr[q] += (double)r * r;
        aa[q] += (double)ax * ax;
      }
    }
  }
  __shared__ double s_r[kRows32][kSmallBlockWidth];
  __shared__ double s_a[kRows32][kSmallBlockWidth];
#pragma unroll
  for (int q = 0; q < kChunks; ++q) {
    const int lc = threadIdx.x + 32 * q;
    s_r[threadIdx.y][lc] = rr[q];
    s_a[threadIdx.y][lc] = aa[q];
  }
  __syncthreads();
  if (threadIdx.y == 0) {
    for (int lc = threadIdx.x; lc < kSmallBlockWidth && c0 + lc < ncols; lc += 32) {
      double sr = 0.0, sa = 0.0;
      for (int y = 0; y < kRows32; ++y) {
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
__global__ void colsum_reduce_kernel(const double* __restrict__ partials, int nb,
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

// C = A^T B (FP32 products, FP32 per-chunk sums, FP64 final sum), 64 x 64 tiles,
// split over rows; symmetric: only upper tiles, mirrored in the reduction.
constexpr int TT = 64;
__global__ void __launch_bounds__(256)
gemm_tn_f32_partial_kernel(int rows, int m, int n, const float* __restrict__ A, int lda,
                           const float* __restrict__ B, int ldb, bool symmetric, int chunk_rows,
                           float* __restrict__ partials) {
  __shared__ float As[16][TT + 4];
  __shared__ float Bs[16][TT + 4];
  int ti, tj;
  if (symmetric) {
    int t = blockIdx.x, T = (m + TT - 1) / TT;
    ti = 0;
    while (t >= T - ti) {
      t -= T - ti;
      ++ti;
    }
    tj = ti + t;
  } else {
    const int tn = (n + TT - 1) / TT;
    ti = blockIdx.x / tn;
    tj = blockIdx.x - ti * tn;
  }
  const int i0 = ti * TT, j0 = tj * TT;
  const int r_begin = blockIdx.y * chunk_rows;
  const int r_end = min(rows, r_begin + chunk_rows);
  const int t = threadIdx.x, ty = t >> 4, tx = t & 15;  // 4 x 4 outputs per thread
  float acc[4][4] = {};
  for (int r0 = r_begin; r0 < r_end; r0 += 16) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = t + 256 * q;  // 0..1023 = 16 rows x 64 cols
      const int rr = e >> 6, cc = e & 63;
      const int r = r0 + rr;
      const bool rin = r < r_end;
      As[rr][cc] = (rin && i0 + cc < m) ? A[(size_t)r * lda + i0 + cc] : 0.f;
      Bs[rr][cc] = (rin && j0 + cc < n) ? B[(size_t)r * ldb + j0 + cc] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int rr = 0; rr < 16; ++rr) {
      float a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        a[u] = As[rr][ty + 16 * u];
        b[u] = Bs[rr][tx + 16 * u];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(a[u], b[v], acc[u][v]);
    }
    __syncthreads();
  }
  float* P = partials + (size_t)blockIdx.y * m * n;
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int i = i0 + ty + 16 * u, j = j0 + tx + 16 * v;
      if (i < m && j < n) P[(size_t)i * n + j] = acc[u][v];
    }
}

__global__ void gemm_tn_f32_reduce_kernel(int m, int n, int nchunk, bool symmetric,
                                          const float* __restrict__ partials, double* __restrict__ C,
                                          int ldc) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m * n) return;
  int i = e / n, j = e - i * n;
  int si = i, sj = j;
  if (symmetric && i > j) {
    si = j;
    sj = i;
  }
  // compensated FP32 sum of the chunk partials (the FP64 pipe is 1/60 of FP32 on GB300)
  float s = 0.f, comp = 0.f;
  for (int c = 0; c < nchunk; ++c) {
    const float y = partials[(size_t)c * m * n + (size_t)si * n + sj] - comp;
    const float t = s + y;
    comp = (t - s) - y;
    s = t;
  }
  C[(size_t)i * ldc + j] = (double)s;
}

struct Plan32 {
  int ntiles, nchunk, chunk_rows;
};

Plan32 plan32(int rows, int m, int n, bool symmetric) {
  Plan32 p;
  const int tm = (m + TT - 1) / TT, tn = (n + TT - 1) / TT;
  p.ntiles = symmetric ? tm * (tm + 1) / 2 : tm * tn;
  const int max_chunks = std::max(1, (rows + 15) / 16);
  int want = (kSplitTarget + p.ntiles - 1) / p.ntiles;
  want = std::max(1, std::min(want, max_chunks));
  int cr = (rows + want - 1) / want;
  cr = ((cr + 15) / 16) * 16;
  p.chunk_rows = std::max(cr, 16);
  p.nchunk = (rows + p.chunk_rows - 1) / p.chunk_rows;
  return p;
}

// C[rows x n] = alpha A[rows x K] M[K x n] + beta C (M FP64 in memory, used as FP32).
__global__ void __launch_bounds__(256)
gemm_nn_f32_kernel(int rows, int K, int n, float alpha, const float* __restrict__ A, int lda,
                   const double* __restrict__ M, int ldm, float beta, float* C, int ldc, bool upper) {
  __shared__ float As[64][17];
  __shared__ float Ms[16][TT + 4];
  const int r0 = blockIdx.y * 64, j0 = blockIdx.x * TT;
  const int t = threadIdx.x, ty = t >> 4, tx = t & 15;
  float acc[4][4] = {};
  const int k_end = upper ? min(K, j0 + TT) : K;
  for (int k0 = 0; k0 < k_end; k0 += 16) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = t + 256 * q;  // 64 rows x 16 k
      const int rr = e >> 4, kk = e & 15;
      const int r = r0 + rr, kc = k0 + kk;
      As[rr][kk] = (r < rows && kc < K) ? A[(size_t)r * lda + kc] : 0.f;
      const int kk2 = e >> 6, jj = e & 63;  // 16 k x 64 cols
      const int kc2 = k0 + kk2, j = j0 + jj;
      Ms[kk2][jj] = (kc2 < K && j < n) ? (float)M[(size_t)kc2 * ldm + j] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        a[u] = As[ty + 16 * u][kk];
        b[u] = Ms[kk][tx + 16 * u];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(a[u], b[v], acc[u][v]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int r = r0 + ty + 16 * u, j = j0 + tx + 16 * v;
      if (r < rows && j < n) {
        float* c = C + (size_t)r * ldc + j;
        *c = (beta == 0.f) ? alpha * acc[u][v] : fmaf(alpha, acc[u][v], beta * (*c));
      }
    }
}

unsigned blocks_for(long long count, int threads) { return (unsigned)((count + threads - 1) / threads); }

}  // namespace

cudaError_t launch_to_f32(const double* in, float* out, long long count, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  to_f32_kernel<<<blocks_for(count, kThreads), kThreads, 0, st>>>(in, out, count);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_block_f32_to_f64(int rows, int cols, const float* in, int ld_in, double* out,
                                    int ld_out, cudaStream_t st) {
  const long long tot = (long long)rows * cols;
  if (tot <= 0) return cudaSuccess;
  block_f32_to_f64_kernel<<<blocks_for(tot, kThreads), kThreads, 0, st>>>(rows, cols, in, ld_in,
                                                                           out, ld_out);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_block_f64_to_f32(int rows, int cols, const double* in, int ld_in, float* out,
                                    int ld_out, cudaStream_t st) {
  const long long tot = (long long)rows * cols;
  if (tot <= 0) return cudaSuccess;
  block_f64_to_f32_kernel<<<blocks_for(tot, kThreads), kThreads, 0, st>>>(rows, cols, in, ld_in,
                                                                           out, ld_out);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_cheb_step_f32(const Stencil32& A, const float* cur, int ldc, const float* prev,
                                 int ldp, float* out, int ldo, int ncols, float s1, float s2,
                                 float s3, cudaStream_t st, int threads) {
  if (ncols % 4 || ldc % 4 || ldo % 4 || (prev && ldp % 4)) return cudaErrorInvalidValue;
  if (threads < 32 || threads > 1024 || threads % 32) return cudaErrorInvalidValue;
  const int quads = ncols / 4;
  const long long tot = (long long)A.n * A.n * quads;
  cheb_step_f32_kernel<<<blocks_for(tot, threads), threads, 0, st>>>(
      A, cur, ldc, (s3 != 0.f) ? prev : nullptr, ldp, out, ldo, quads, s1, s2, s3);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_cheb_step_f32_tab(const Stencil32& A, const float* cur, int ldc,
                                     const float* prev, int ldp, float* out, int ldo, int ncols,
                                     const float* coef, int threads, cudaStream_t st) {
  if (ncols % 4 || ldc % 4 || ldo % 4 || (prev && ldp % 4)) return cudaErrorInvalidValue;
  if (threads < 32 || threads > 1024 || threads % 32) return cudaErrorInvalidValue;
  const int quads = ncols / 4;
  const long long tot = (long long)A.n * A.n * quads;
  cheb_step_f32_tab_kernel<<<blocks_for(tot, threads), threads, 0, st>>>(A, cur, ldc, prev, ldp,
                                                                         out, ldo, quads, coef);
  return cudaGetLastError();
}

cudaError_t launch_residual_norms_f32(const Stencil32& A, const float* X, int ldx, int ncols,
                                      const double* theta, double* partials, double* out2,
                                      cudaStream_t st) {
  if (ncols > kMaxBlockWidth) return cudaErrorInvalidValue;
  const int nb = resid_blocks(A.n);
  const dim3 grid(nb, (ncols + kSmallBlockWidth - 1) / kSmallBlockWidth);
  residual_norms_f32_kernel<<<grid, dim3(32, kRows32), 0, st>>>(A, X, ldx, ncols, theta, partials);
  note_launch();
  colsum_reduce_kernel<<<(2 * ncols + 3) / 4, 128, 0, st>>>(partials, nb, ncols, out2);
  note_launch();
  return cudaGetLastError();
}

size_t gemm_tn_f32_partials(int rows, int m, int n, bool symmetric) {
  const Plan32 p = plan32(rows, m, n, symmetric);
  return (size_t)p.nchunk * m * n;
}

cudaError_t launch_gemm_tn_f32(int rows, int m, int n, const float* A, int lda, const float* B,
                               int ldb, double* C, int ldc, bool symmetric, float* partials,
                               cudaStream_t st) {
  if (m <= 0 || n <= 0) return cudaSuccess;
  if (symmetric && m != n) return cudaErrorInvalidValue;
  const Plan32 p = plan32(rows, m, n, symmetric);
  gemm_tn_f32_partial_kernel<<<dim3(p.ntiles, p.nchunk), 256, 0, st>>>(rows, m, n, A, lda, B, ldb,
                                                                       symmetric, p.chunk_rows,
                                                                       partials);
  note_launch();
  gemm_tn_f32_reduce_kernel<<<(m * n + 255) / 256, 256, 0, st>>>(m, n, p.nchunk, symmetric, partials,
                                                               C, ldc);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_gemm_nn_f32(int rows, int k, int n, float alpha, const float* A, int lda,
                               const double* M, int ldm, float beta, float* C, int ldc, bool upper,
                               cudaStream_t st) {
  if (rows <= 0 || n <= 0) return cudaSuccess;
  dim3 grid((n + TT - 1) / TT, (rows + 63) / 64);
  gemm_nn_f32_kernel<<<grid, 256, 0, st>>>(rows, k, n, alpha, A, lda, M, ldm, beta, C, ldc, upper);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_dc_ytab(const double* theta, int ncols, const DcSteps& P, float* ytab,
                           double* state, cudaStream_t st, const int* gdeg, double* ysel) {
  if (ncols < 1 || P.count < 1 || P.count > kDcChunk || (gdeg && !ysel)) return cudaErrorInvalidValue;
  dc_ytab_kernel<<<(ncols + 127) / 128, 128, 0, st>>>(theta, ncols, P, ytab, state, gdeg, ysel);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_cheb_step_dc(const Stencil32& A, const float* cur, const float* prev, int ld,
                                const float* R, int ldr, const float* ycol, float* out,
                                int ncols, float s1, float s2, float s3, cudaStream_t st) {
  if (ncols < 1 || ld < ncols || ldr < ncols) return cudaErrorInvalidValue;
  const long long N = (long long)A.n * A.n;
  const int nb = (int)std::min<long long>((N + kDcRows - 1) / kDcRows, 152LL * 16);
  const dim3 block(32, kDcRows);
  if (!cur)
    cheb_step_dc_kernel<false, false><<<nb, block, 0, st>>>(A, cur, nullptr, ld, R, ldr, ycol, out,
                                                             ncols, s1, s2, s3);
  else if (!prev || s3 == 0.f)
    cheb_step_dc_kernel<true, false><<<nb, block, 0, st>>>(A, cur, nullptr, ld, R, ldr, ycol, out,
                                                            ncols, s1, s2, s3);
  else
    cheb_step_dc_kernel<true, true><<<nb, block, 0, st>>>(A, cur, prev, ld, R, ldr, ycol, out, ncols,
                                                           s1, s2, s3);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_dc_combine(int rows, int ncols, const double* X, int ldx, const double* ym,
                              const float* Z, int ldz, double* Y, int ldy, cudaStream_t st) {
  const long long tot = (long long)rows * ncols;
  const int nb = (int)std::min<long long>((tot + 255) / 256, 152LL * 16);
  dc_combine_kernel<<<nb, 256, 0, st>>>(rows, ncols, X, ldx, ym, Z, ldz, Y, ldy);
  note_launch();
  return cudaGetLastError();
}

// ---- the resident filters: variants and the shape tuner ------------------------------
namespace {

// Variant v of a resident filter: v & 1 selects the cluster size (4 or 8 CTAs), v >> 1 the
// kernel (0: register strips, 1: both levels in shared memory). cudaErrorNotSupported when the
// band does not fit (threads or shared memory) or the device cannot place the cluster shape.
constexpr int kResidentVariants = 4;

cudaError_t launch_cluster(const void* fn, int clu, int groups, int threads, size_t smem,
                           cudaStream_t st, void** args) {
  cudaError_t e = ensure_dynamic_smem(fn, smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(clu, groups, 1);
  cfg.blockDim = dim3(threads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = clu;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelExC(&cfg, fn, args);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cudaErrorNotSupported;
  }
  note_launch();
  return cudaGetLastError();
}

template <bool kDc>
cudaError_t launch_resident_variant(int v, const Stencil32& A, const float* X, int ldx, int ncols,
                                    const float* ytab, const float* coef, int m, float* out,
                                    int ldo, const int* gdeg, cudaStream_t st) {
  constexpr size_t kMaxSmem = 227 * 1024;
  const int n = A.n, clu = (v & 1) ? 8 : 4, groups = (ncols + 3) / 4;
  if (n < 2 * clu) return cudaErrorNotSupported;
  Stencil32 a = A;
  const float* x = X;
  const float* yt = ytab;
  const float* cf = coef;
  float* o = out;
  const int* gd = gdeg;
  if ((v >> 1) == 0) {  // register strips
    const int threads = (clu == 4) ? strip_threads<4>(n) : strip_threads<8>(n);
    const size_t smem = (clu == 4) ? strip_smem<4>(n, kDc, m) : strip_smem<8>(n, kDc, m);
    if (threads == 0 || smem > kMaxSmem) return cudaErrorNotSupported;
    void* args[] = {&a, &x, &ldx, &ncols, &yt, &cf, &m, &o, &ldo, &gd};
    const void* fn = (clu == 4) ? (const void*)strip_filter_cluster_kernel<4, kDc>
                                : (const void*)strip_filter_cluster_kernel<8, kDc>;
    return launch_cluster(fn, clu, groups, threads, smem, st, args);
  }
  if (kDc) {
    const size_t smem = (clu == 4) ? cluster_dc_smem<4>(n, m) : cluster_dc_smem<8>(n, m);
    if (smem > kMaxSmem) return cudaErrorNotSupported;
    void* args[] = {&a, &x, &ldx, &ncols, &yt, &cf, &m, &o, &ldo, &gd};
    const void* fn = (clu == 4) ? (const void*)dc_filter_cluster_kernel<4>
                                : (const void*)dc_filter_cluster_kernel<8>;
    return launch_cluster(fn, clu, groups, 1024, smem, st, args);
  }
  const size_t smem = (clu == 4) ? cluster_filter_smem<4>(n) : cluster_filter_smem<8>(n);
  if (smem > kMaxSmem) return cudaErrorNotSupported;
  void* args[] = {&a, &x, &ldx, &o, &ldo, &m, &cf};
  const void* fn = (clu == 4) ? (const void*)cheb_filter_f32_cluster_kernel<4>
                              : (const void*)cheb_filter_f32_cluster_kernel<8>;
  return launch_cluster(fn, clu, groups, 1024, smem, st, args);
}

// Shape tuner: the first call for a (filter, n, column groups) shape on a stream that is not
// being captured times every applicable variant once on the call's own buffers (CUDA events on
// the caller's stream; every variant computes the same recurrence and writes only `out`),
// keeps the fastest (the default, the first variant that applies, unless another is 10 %
// faster) for the process and finishes with it; later calls run the cached choice
// (a call that finds the shape being tuned by another thread waits for the choice; under
// stream capture an untuned shape runs the first variant that applies). The choice is per
// process, so solves of the same shape in a process use the same kernel.
struct ResidentShape {
  bool dc;
  int n, groups;
  bool operator<(const ResidentShape& o) const {
    return dc != o.dc ? dc < o.dc : n != o.n ? n < o.n : groups < o.groups;
  }
};

template <bool kDc>
cudaError_t launch_resident_tuned(const Stencil32& A, const float* X, int ldx, int ncols,
                                  const float* ytab, const float* coef, int m, float* out,
                                  int ldo, const int* gdeg, cudaStream_t st) {
  static std::mutex mu;
  static std::condition_variable cv;
  static std::map<ResidentShape, int> best;  // -1: no variant applies
  static std::set<ResidentShape> busy;
  const ResidentShape key{kDc, A.n, (ncols + 3) / 4};
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  const bool capturing = cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone;
  bool tune = false;
  {
    std::unique_lock<std::mutex> g(mu);
    if (!capturing) cv.wait(g, [&] { return busy.count(key) == 0; });
    auto it = best.find(key);
    if (it != best.end()) {
      const int v = it->second;
      g.unlock();
      if (v < 0) return cudaErrorNotSupported;
      return launch_resident_variant<kDc>(v, A, X, ldx, ncols, ytab, coef, m, out, ldo, gdeg, st);
    }
    if (!capturing) {
      busy.insert(key);
      tune = true;
    }
  }
  if (!tune) {  // first applicable variant
    for (int v = 0; v < kResidentVariants; ++v) {
      const cudaError_t e =
          launch_resident_variant<kDc>(v, A, X, ldx, ncols, ytab, coef, m, out, ldo, gdeg, st);
      if (e != cudaErrorNotSupported) return e;
    }
    return cudaErrorNotSupported;
  }
  int pick = -1;
  float pick_ms = INFINITY;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t err = cudaSuccess;
  if ((err = cudaEventCreate(&e0)) == cudaSuccess && (err = cudaEventCreate(&e1)) == cudaSuccess) {
    for (int v = 0; v < kResidentVariants && err == cudaSuccess; ++v) {
      for (int rep = 0; rep < 2 && err == cudaSuccess; ++rep) {  // best of two
        if ((err = cudaEventRecord(e0, st)) != cudaSuccess) break;
        const cudaError_t lv =
            launch_resident_variant<kDc>(v, A, X, ldx, ncols, ytab, coef, m, out, ldo, gdeg, st);
        if (lv == cudaErrorNotSupported) break;
        if ((err = lv) != cudaSuccess) break;
        float ms = INFINITY;
        if ((err = cudaEventRecord(e1, st)) != cudaSuccess ||
            (err = cudaEventSynchronize(e1)) != cudaSuccess ||
            (err = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess)
          break;
        // the first variant that applies is the default; another replaces it only when 10 %
        // faster, so that timing noise (other streams share the GPU) does not flip choices
        if (pick < 0 ? true : (v == pick ? ms < pick_ms : ms < 0.9f * pick_ms)) {
          pick_ms = ms;
          pick = v;
        }
      }
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  {
    std::lock_guard<std::mutex> g(mu);
    busy.erase(key);
    if (err == cudaSuccess) best[key] = pick;
  }
  cv.notify_all();
  if (err != cudaSuccess) return err;
  if (pick < 0) return cudaErrorNotSupported;
  return launch_resident_variant<kDc>(pick, A, X, ldx, ncols, ytab, coef, m, out, ldo, gdeg, st);
}

}  // namespace

cudaError_t launch_cheb_filter_f32_resident(const Stencil32& A, const float* Y0, int ld0, float* out,
                                            int ldo, int ncols, int m, const float* coef,
                                            cudaStream_t st) {
  if (ncols % 4 || ld0 % 4 || ldo % 4 || m < 1) return cudaErrorNotSupported;
  return launch_resident_tuned<false>(A, Y0, ld0, ncols, nullptr, coef, m, out, ldo, nullptr, st);
}

cudaError_t launch_dc_filter_resident(const Stencil32& A, const float* R, int ldr, int ncols,
                                      const float* ytab, const float* coef, int m, float* out,
                                      int ldo, cudaStream_t st, const int* gdeg) {
  if (ncols < 1 || m < 1) return cudaErrorNotSupported;
  return launch_resident_tuned<true>(A, R, ldr, ncols, ytab, coef, m, out, ldo, gdeg, st);
}

}  // namespace scsf
