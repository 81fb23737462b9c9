// Dense start of the reduced eigensolve (included by eig.cu, inside its anonymous namespace).
//
// For the trailing block B = S[t0:k, t0:k] (m = k - t0 columns; t0 from the probe), in FP32:
//   trd_reduce_kernel   one CTA: B = Q T Q^T by m - 2 Householder reflections (three barriers a
//                       column), T = tridiag(d, e); reflector j (unit vector, rows > j) in Hv[j];
//   trd_eigval_kernel   one warp per eigenvalue of T: 32-point multisection on Sturm counts;
//   trd_eigvec_kernel   one warp per cluster of eigenvalues closer than 1e-3 ||T||: inverse
//                       iteration (tridiagonal LU with partial pivoting, three solves from a fixed
//                       start) with Gram-Schmidt against the cluster's earlier vectors;
//   trd_back_kernel     one warp per eigenvector: Z = Q V (the reflections applied in reverse).
// The result is an FP32-accurate eigenbasis of B; the FP64 refinement takes it from there.
// Compared with cyclic Jacobi in one CTA (k - 1 rounds of two barriers per sweep, 6-8 sweeps)
// the single-CTA part here needs three barriers per column once.
#pragma once

constexpr float kTrdClusterTol = 1e-3f;
constexpr int kTrdWarpsPerBlock = 2;  // inverse iteration: per-warp arrays in shared memory

template <bool kWide>
__global__ void __launch_bounds__(1024)
trd_reduce_kernel(int k, const double* __restrict__ S, const int* __restrict__ start,
                  double* __restrict__ Z, int ldz, double* __restrict__ lam, float* __restrict__ wide,
                  float* __restrict__ Hv, float* __restrict__ dd, float* __restrict__ ee,
                  int* __restrict__ skip) {
  extern __shared__ float smt[];
  __shared__ float vsh[kMaxBlockWidth], psh[kMaxBlockWidth];
  __shared__ int s_skip;
  const int t0 = start ? min(max(*start, 0), k) : 0;
  const int m = k - t0;
  const int t = threadIdx.x, nt = blockDim.x, lane = t & 31, warp = t >> 5, nwarps = nt >> 5;
  // the leading block [0, t0) keeps the identity (it is already nearly diagonal)
  for (int e = t; e < k * k; e += nt) {
    const int i = e / k, j = e - i * k;
    if (i < t0 || j < t0) Z[(size_t)i * ldz + j] = (i == j) ? 1.0 : 0.0;
  }
  if (lam)
    for (int i = t; i < t0; i += nt) lam[i] = S[(size_t)i * k + i];
  if (m <= 0) return;
  const int ms = m + 1;
  float* A = kWide ? wide : smt;  // m x ms
  for (int e = t; e < m * m; e += nt) {
    const int i = e / m, j = e - i * m;
    A[i * ms + j] = (float)S[(size_t)(t0 + i) * k + t0 + j];
  }
  __syncthreads();
  for (int j = 0; j + 2 < m; ++j) {
    const int L = m - j - 1;  // x = A[j+1 .. m-1][j]
    if (warp == 0) {
      float ss = 0.f;
      for (int r = lane; r < L; r += 32) {
        const float x = A[(j + 1 + r) * ms + j];
        ss = fmaf(x, x, ss);
      }
      for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
      const float x0 = A[(j + 1) * ms + j];
      const float xn = sqrtf(ss);
      const float alpha = (x0 > 0.f) ? -xn : xn;
      const float vn2 = 2.f * (ss - alpha * x0);  // |x - alpha e_1|^2
      const bool sk = !(vn2 > 1e-30f) || !(ss > 0.f);
      const float inv = sk ? 0.f : rsqrtf(vn2);
      for (int r = lane; r < L; r += 32) {
        const float x = A[(j + 1 + r) * ms + j];
        const float v = sk ? 0.f : ((r == 0) ? (x - alpha) : x) * inv;
        vsh[r] = v;
        Hv[(size_t)j * m + j + 1 + r] = v;
      }
      if (lane == 0) {
        dd[j] = A[j * ms + j];
        ee[j] = sk ? x0 : alpha;
        skip[j] = sk ? 1 : 0;
        s_skip = sk ? 1 : 0;
      }
    }
    __syncthreads();
    if (s_skip) {  // nothing to reflect; the barrier keeps warp 0 from rewriting s_skip early
      __syncthreads();
      continue;
    }
    // p = B_sub v, one row per warp pass (lanes over columns)
    for (int r = warp; r < L; r += nwarps) {
      const float* row = A + (j + 1 + r) * ms + j + 1;
      float acc = 0.f;
      for (int c = lane; c < L; c += 32) acc = fmaf(row[c], vsh[c], acc);
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) psh[r] = acc;
    }
    __syncthreads();
    // K = v^T p (every warp forms it), then B_sub -= 2 (v w^T + w v^T), w = p - K v
    float K = 0.f;
    for (int c = lane; c < L; c += 32) K = fmaf(vsh[c], psh[c], K);
    for (int o = 16; o > 0; o >>= 1) K += __shfl_xor_sync(0xffffffffu, K, o);
    for (int r = warp; r < L; r += nwarps) {
      const float vr = vsh[r], wr = psh[r] - K * vr;
      float* row = A + (j + 1 + r) * ms + j + 1;
      for (int c = lane; c < L; c += 32) {
        const float wc = psh[c] - K * vsh[c];
        row[c] -= 2.f * (vr * wc + wr * vsh[c]);
      }
    }
    __syncthreads();
  }
  if (t == 0) {
    if (m >= 2) {
      dd[m - 2] = A[(m - 2) * ms + m - 2];
      ee[m - 2] = A[(m - 1) * ms + m - 2];
      skip[m - 2] = 1;
    }
    dd[m - 1] = A[(m - 1) * ms + m - 1];
    ee[m - 1] = 0.f;
    skip[m - 1] = 1;
  }
}

// Number of eigenvalues of tridiag(d, e) below x (Sturm sequence, pivots kept off zero).
__device__ __forceinline__ int trd_count(const float* d, const float* e, int m, float x) {
  float q = d[0] - x;
  int c = q < 0.f;
  for (int i = 1; i < m; ++i) {
    if (fabsf(q) < 1e-30f) q = -1e-30f;
    q = (d[i] - x) - e[i - 1] * (e[i - 1] / q);
    c += q < 0.f;
  }
  return c;
}

__global__ void __launch_bounds__(256)
trd_eigval_kernel(int k, const int* __restrict__ start, const float* __restrict__ dd,
                  const float* __restrict__ ee, float* __restrict__ lamt) {
  __shared__ float d[kMaxBlockWidth], e[kMaxBlockWidth];
  const int t0 = start ? min(max(*start, 0), k) : 0;
  const int m = k - t0;
  if (m <= 0) return;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    d[i] = dd[i];
    e[i] = ee[i];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (i >= m) return;
  // Gershgorin interval of T
  float lo = INFINITY, hi = -INFINITY;
  for (int r = lane; r < m; r += 32) {
    const float rad = ((r > 0) ? fabsf(e[r - 1]) : 0.f) + ((r + 1 < m) ? fabsf(e[r]) : 0.f);
    lo = fminf(lo, d[r] - rad);
    hi = fmaxf(hi, d[r] + rad);
  }
  for (int o = 16; o > 0; o >>= 1) {
    lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  const float pad = 1e-6f * (hi - lo) + 1e-30f;
  lo -= pad;
  hi += pad;
  // 32-point multisection: lane l tests lo + (hi - lo)(l + 1)/33; the eigenvalue of index i
  // lies between the last point with at most i eigenvalues below it and the first with more
  for (int it = 0; it < 12; ++it) {
    const float x = lo + (hi - lo) * ((float)(lane + 1) / 33.f);
    const int c = trd_count(d, e, m, x);
    const unsigned above = __ballot_sync(0xffffffffu, c > i);
    const int f = above ? __ffs(above) - 1 : 32;
    const float xf = __shfl_sync(0xffffffffu, x, f & 31);
    const float xp = __shfl_sync(0xffffffffu, x, (f + 31) & 31);
    const float nhi = (f < 32) ? xf : hi;
    const float nlo = (f > 0) ? xp : lo;
    lo = nlo;
    hi = nhi;
    if (hi - lo <= 2e-7f * fmaxf(fabsf(lo), fabsf(hi))) break;
  }
  if (lane == 0) lamt[i] = 0.5f * (lo + hi);
}

// LU with partial pivoting of T - lambda I (U: diagonal u0, superdiagonals u1, u2; row
// interchanges in piv), run by one lane on the warp's shared arrays. A zero pivot is replaced
// by `tiny` (inverse iteration only needs a large solution, not an exact one).
__device__ void trd_lu(const float* d, const float* e, int m, float lam, float tiny, float* l,
                       float* u0, float* u1, float* u2, int* piv) {
  float b = d[0] - lam, c = (m > 1) ? e[0] : 0.f;  // current row: columns i, i + 1
  for (int i = 0; i + 1 < m; ++i) {
    const float a = e[i];                           // T[i+1][i]
    const float bn = d[i + 1] - lam;                // T[i+1][i+1]
    const float cn = (i + 2 < m) ? e[i + 1] : 0.f;  // T[i+1][i+2]
    if (fabsf(b) >= fabsf(a)) {                     // pivot on the current row
      const float bb = (b == 0.f) ? tiny : b;
      const float f = a / bb;
      l[i] = f;
      piv[i] = 0;
      u0[i] = bb;
      u1[i] = c;
      u2[i] = 0.f;
      b = bn - f * c;
      c = cn;
    } else {                                        // interchange with row i + 1
      const float f = b / a;
      l[i] = f;
      piv[i] = 1;
      u0[i] = a;
      u1[i] = bn;
      u2[i] = cn;
      b = c - f * bn;
      c = -f * cn;
    }
  }
  u0[m - 1] = (b == 0.f) ? tiny : b;
  u1[m - 1] = 0.f;
  u2[m - 1] = 0.f;
}

// (T - lambda I) x = y in place with the factors of trd_lu.
__device__ void trd_solve(int m, const float* l, const float* u0, const float* u1, const float* u2,
                          const int* piv, float* y) {
  for (int i = 0; i + 1 < m; ++i) {
    if (piv[i]) {
      const float tmp = y[i];
      y[i] = y[i + 1];
      y[i + 1] = tmp - l[i] * y[i];
    } else {
      y[i + 1] -= l[i] * y[i];
    }
  }
  for (int i = m - 1; i >= 0; --i) {
    float s = y[i];
    if (i + 1 < m) s -= u1[i] * y[i + 1];
    if (i + 2 < m) s -= u2[i] * y[i + 2];
    y[i] = s / u0[i];
  }
}

__global__ void __launch_bounds__(32 * kTrdWarpsPerBlock)
trd_eigvec_kernel(int k, const int* __restrict__ start, const float* __restrict__ dd,
                  const float* __restrict__ ee, const float* __restrict__ lamt,
                  float* __restrict__ V) {
  extern __shared__ float smv[];
  __shared__ int pivs[kTrdWarpsPerBlock][kMaxBlockWidth];
  const int t0 = start ? min(max(*start, 0), k) : 0;
  const int m = k - t0;
  if (m <= 0) return;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int i0 = blockIdx.x * kTrdWarpsPerBlock + w;
  if (i0 >= m) return;
  // norm of T and the cluster rule
  float tn = 0.f;
  for (int r = lane; r < m; r += 32) tn = fmaxf(tn, fabsf(dd[r]) + 2.f * fabsf(ee[r]));
  for (int o = 16; o > 0; o >>= 1) tn = fmaxf(tn, __shfl_xor_sync(0xffffffffu, tn, o));
  const float ortol = kTrdClusterTol * fmaxf(tn, 1e-30f);
  if (i0 > 0 && lamt[i0] - lamt[i0 - 1] <= ortol) return;  // not the first of its cluster
  int i1 = i0 + 1;
  while (i1 < m && lamt[i1] - lamt[i1 - 1] <= ortol) ++i1;
  float* base = smv + (size_t)w * 7 * m;
  float *d = base, *e = base + m, *l = base + 2 * m, *u0 = base + 3 * m, *u1 = base + 4 * m,
        *u2 = base + 5 * m, *y = base + 6 * m;
  int* piv = pivs[w];
  for (int r = lane; r < m; r += 32) {
    d[r] = dd[r];
    e[r] = ee[r];
  }
  __syncwarp();
  const float tiny = 1e-14f * fmaxf(tn, 1e-30f);
  for (int i = i0; i < i1; ++i) {
    if (lane == 0) trd_lu(d, e, m, lamt[i], tiny, l, u0, u1, u2, piv);
    // a fixed start with no structure in common with T's eigenvectors
    for (int r = lane; r < m; r += 32)
      y[r] = 0.5f + (float)((unsigned)(r * 2654435761u + (unsigned)i * 97u) % 1000u) * 1e-3f;
    __syncwarp();
    for (int it = 0; it < 3; ++it) {
      if (lane == 0) trd_solve(m, l, u0, u1, u2, piv, y);
      __syncwarp();
      float mx = 0.f;
      for (int r = lane; r < m; r += 32) mx = fmaxf(mx, fabsf(y[r]));
      for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      const float sc = (mx > 0.f && mx < INFINITY) ? 1.f / mx : 1.f;
      for (int r = lane; r < m; r += 32) y[r] *= sc;
      __syncwarp();
      // Gram-Schmidt against the cluster's earlier vectors (rows i0 .. i-1 of V)
      for (int p = i0; p < i; ++p) {
        const float* vp = V + (size_t)p * m;
        float dot = 0.f;
        for (int r = lane; r < m; r += 32) dot = fmaf(vp[r], y[r], dot);
        for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
        for (int r = lane; r < m; r += 32) y[r] -= dot * vp[r];
        __syncwarp();
      }
      float nn = 0.f;
      for (int r = lane; r < m; r += 32) nn = fmaf(y[r], y[r], nn);
      for (int o = 16; o > 0; o >>= 1) nn += __shfl_xor_sync(0xffffffffu, nn, o);
      const float inv = (nn > 0.f) ? rsqrtf(nn) : 0.f;
      for (int r = lane; r < m; r += 32) y[r] *= inv;
      __syncwarp();
    }
    for (int r = lane; r < m; r += 32) V[(size_t)i * m + r] = y[r];
    __syncwarp();
  }
}

// Z[t0 + r][t0 + i] = (Q v_i)_r, Q = H_0 H_1 ... H_{m-3}: one warp per eigenvector, the vector
// in registers (lane l holds rows l + 32 q), reflections applied from the last to the first.
__global__ void __launch_bounds__(256)
trd_back_kernel(int k, const int* __restrict__ start, const float* __restrict__ Hv,
                const int* __restrict__ skip, const float* __restrict__ V,
                const float* __restrict__ lamt, double* __restrict__ Z, int ldz,
                double* __restrict__ lam) {
  constexpr int R = (kMaxBlockWidth + 31) / 32;
  const int t0 = start ? min(max(*start, 0), k) : 0;
  const int m = k - t0;
  if (m <= 0) return;
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (i >= m) return;
  float y[R];
#pragma unroll
  for (int q = 0; q < R; ++q) {
    const int r = lane + 32 * q;
    y[q] = (r < m) ? V[(size_t)i * m + r] : 0.f;
  }
  for (int j = m - 3; j >= 0; --j) {
    if (skip[j]) continue;
    const float* h = Hv + (size_t)j * m;
    float s = 0.f;
#pragma unroll
    for (int q = 0; q < R; ++q) {
      const int r = lane + 32 * q;
      if (r > j && r < m) s = fmaf(h[r], y[q], s);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
#pragma unroll
    for (int q = 0; q < R; ++q) {
      const int r = lane + 32 * q;
      if (r > j && r < m) y[q] -= 2.f * s * h[r];
    }
  }
#pragma unroll
  for (int q = 0; q < R; ++q) {
    const int r = lane + 32 * q;
    if (r < m) Z[(size_t)(t0 + r) * ldz + t0 + i] = (double)y[q];
  }
  if (lam && lane == 0) lam[t0 + i] = (double)lamt[i];
}
