// Upper end of the spectrum for the filter's damped interval [alpha, beta] (Sec. 3.2).
//
// The filter needs beta >= lambda_max(A): components above beta are amplified instead of damped.
// The Gershgorin bound (computed with the assembly) is rigorous but loose on these operators;
// a short Lanczos run gives a much closer estimate (the bound the paper keeps commented out).
// Following Zhou and Li ("Bounding the spectrum of large Hermitian matrices", 2011): after K
// Lanczos steps from a random start, theta_max(T_K) + |beta_K| (the largest Ritz value plus the
// norm of the last Lanczos residual) bounds lambda_max in practice. The run here is one CTA in
// FP32 (an estimate needs no FP64; the relative margin below covers its rounding); the chain
// takes min(estimate, Gershgorin bound).
#include "kernels.cuh"

namespace scsf {
namespace {

constexpr int kLanczosMax = 32;
constexpr float kLanczosMargin = 2e-3f;  // relative safety margin on the estimate

// (A v)_I in FP32 for a stencil (d, we, wn) or CSR operator.
__device__ __forceinline__ float apply_row(const Stencil& A, const float* __restrict__ v, int I) {
  if (A.rp) {
    float s = 0.f;
    for (int p = A.rp[I]; p < A.rp[I + 1]; ++p) s = fmaf((float)A.val[p], v[A.ci[p]], s);
    return s;
  }
  const int n = A.n, N = n * n;
  const int i = I / n, j = I - i * n;
  float s = (float)A.d[I] * v[I];
  if (i < n - 1) s = fmaf(-(float)A.we[I], v[I + n], s);
  if (i > 0) s = fmaf(-(float)A.we[I - n], v[I - n], s);
  if (j < n - 1) s = fmaf(-(float)A.wn[I], v[I + 1], s);
  if (j > 0) s = fmaf(-(float)A.wn[I - 1], v[I - 1], s);
  (void)N;
  return s;
}

__device__ __forceinline__ float block_sum(float x, float* red) {
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = x;
  __syncthreads();
  float s = 0.f;
  for (int w = 0; w < nw; ++w) s += red[w];
  return s;
}

// Number of eigenvalues of tridiag(a, b) (m x m) below x.
__device__ int tri_count(const double* a, const double* b, int m, double x) {
  double q = a[0] - x;
  int c = q < 0.0;
  for (int i = 1; i < m; ++i) {
    if (fabs(q) < 1e-300) q = -1e-300;
    q = (a[i] - x) - b[i - 1] * (b[i - 1] / q);
    c += q < 0.0;
  }
  return c;
}

// K Lanczos steps (one CTA) from a hashed uniform start; out[0] = theta_max(T_K) + |beta_K|,
// widened by the margin, and at most `cap` (the Gershgorin bound). vecs: 3 N floats.
__global__ void __launch_bounds__(1024)
lanczos_bound_kernel(Stencil A, int K, unsigned long long seed, float* __restrict__ vecs,
                     double cap, double* __restrict__ out) {
  __shared__ float red[32];
  __shared__ double al[kLanczosMax], be[kLanczosMax];
  const int N = stencil_rows(A);
  const int t = threadIdx.x, nt = blockDim.x;
  float* vp = vecs;          // v_{j-1}
  float* v = vecs + N;       // v_j
  float* w = vecs + 2 * N;   // A v_j - ...
  float nn = 0.f;
  for (int I = t; I < N; I += nt) {
    unsigned long long z = seed + 0x9E3779B97F4A7C15ull * (unsigned long long)(I + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    const float u = (float)(z >> 40) * (1.0f / 16777216.0f) - 0.5f;
    v[I] = u;
    vp[I] = 0.f;
    nn = fmaf(u, u, nn);
  }
  const float inv0 = rsqrtf(fmaxf(block_sum(nn, red), 1e-30f));
  for (int I = t; I < N; I += nt) v[I] *= inv0;
  __syncthreads();
  float beta_prev = 0.f;
  int m = 0;
  for (int j = 0; j < K; ++j) {
    float ad = 0.f;
    for (int I = t; I < N; I += nt) {
      const float x = apply_row(A, v, I);
      w[I] = x;
      ad = fmaf(x, v[I], ad);
    }
    const float alpha = block_sum(ad, red);
    float bn = 0.f;
    for (int I = t; I < N; I += nt) {
      const float x = w[I] - alpha * v[I] - beta_prev * vp[I];
      w[I] = x;
      bn = fmaf(x, x, bn);
    }
    const float beta = sqrtf(block_sum(bn, red));
    if (t == 0) {
      al[j] = alpha;
      be[j] = beta;
    }
    m = j + 1;
    if (!(beta > 1e-30f)) break;  // invariant subspace: T_m holds exact eigenvalues
    const float ib = 1.f / beta;
    for (int I = t; I < N; I += nt) {
      vp[I] = v[I];
      v[I] = w[I] * ib;
    }
    __syncthreads();
    beta_prev = beta;
  }
  __syncthreads();
  if (t == 0) {
    // largest eigenvalue of T_m by bisection on Sturm counts (m <= 32, FP64)
    double lo = INFINITY, hi = -INFINITY;
    for (int i = 0; i < m; ++i) {
      const double r = ((i > 0) ? fabs(be[i - 1]) : 0.0) + ((i + 1 < m) ? fabs(be[i]) : 0.0);
      lo = fmin(lo, al[i] - r);
      hi = fmax(hi, al[i] + r);
    }
    for (int it = 0; it < 100 && hi - lo > 1e-12 * fmax(fabs(lo), fabs(hi)); ++it) {
      const double mid = 0.5 * (lo + hi);
      if (tri_count(al, be, m, mid) >= m) hi = mid;  // all eigenvalues below mid
      else lo = mid;
    }
    const double est = (hi + fabs(be[m - 1])) * (1.0 + kLanczosMargin) + 1e-30;
    out[0] = (isfinite(est) && est < cap) ? est : cap;
  }
}

}  // namespace

size_t lanczos_scratch_bytes(long long N) { return align256((size_t)3 * N * sizeof(float)); }

cudaError_t launch_lanczos_bound(const Stencil& A, int steps, unsigned long long seed, float* vecs,
                                 double cap, double* out, cudaStream_t st) {
  if (steps < 1 || steps > kLanczosMax) return cudaErrorInvalidValue;
  lanczos_bound_kernel<<<1, 1024, 0, st>>>(A, steps, seed, vecs, cap, out);
  note_launch();
  return cudaGetLastError();
}

}  // namespace scsf
