// Reduced symmetric eigensolve G W = W Lambda (Alg. 3 line 6) for k <= 160.
//
// GB300 runs FP32 about 60x faster than FP64, so the decomposition is found
// in FP32 and then refined to FP64 accuracy:
//   1. parallel cyclic Jacobi in FP32, one CTA, both k x k matrices in shared
//      memory, round-robin (circle method) pair ordering: k/2 disjoint
//      rotations per round, k-1 rounds per sweep;
//   2. Ogita-Aishima iterative refinement in FP64 (X' = X + X E with
//      R = I - X^T X, S = X^T G X, lambda_i = s_ii/(1 - r_ii), E_ij =
//      (s_ij + lambda_j r_ij)/(lambda_j - lambda_i), or r_ij/2 for pairs closer
//      than delta = max(2(||S - D|| + ||G|| ||R||), 3e-3 ||G||)); each step squares
//      the error. The k^3 products run on the FP64 block kernels spread over all SMs;
//   3. exact FP64 Jacobi rotations for the pairs left coupled in step 2 (close
//      pairs, where the first-order update does not converge from FP32 accuracy);
//      only significant off-diagonal entries rotate, so this is one scan when
//      nothing is left;
//   4. ascending sort of the pairs.
#include <algorithm>

#include "kernels.cuh"

namespace scsf {
namespace {

constexpr int kOaSteps = 3;
constexpr double kClusterFloor = 3e-3;  // relative gap below which pairs go to FP64 Jacobi
constexpr int kJacobiSweeps = 30;

// Pair (p < q) handled by slot `pr` in round `round` of the circle method over
// kp (even) players: position 0 is fixed, positions 1..kp-1 rotate.
__device__ __forceinline__ void circle_pair(int pr, int round, int kp, int& p, int& q) {
  const int pos_b = kp - 1 - pr;
  const int pa = (pr == 0) ? 0 : 1 + (pr - 1 + round) % (kp - 1);
  const int pb = 1 + (pos_b - 1 + round) % (kp - 1);
  p = min(pa, pb);
  q = max(pa, pb);
}

__global__ void __launch_bounds__(1024)
jacobi_f32_kernel(int k, const double* __restrict__ S, double* __restrict__ Z, int max_sweeps) {
  extern __shared__ float sm[];
  float* A = sm;          // k*k, row-major
  float* V = sm + k * k;  // k*k, eigenvectors in columns
  __shared__ float cs[kMaxBlockWidth + 1], sn[kMaxBlockWidth + 1];
  __shared__ float red_off[32], red_all[32];
  __shared__ int stop;
  __shared__ float prev_off;
  const int t = threadIdx.x, nt = blockDim.x;
  for (int e = t; e < k * k; e += nt) {
    const int i = e / k, j = e - (e / k) * k;
    A[e] = (float)S[e];
    V[e] = (i == j) ? 1.0f : 0.0f;
  }
  if (t == 0) prev_off = INFINITY;
  __syncthreads();
  const int kp = (k + 1) & ~1;  // index k is a dummy player when k is odd
  const int npairs = kp / 2;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    float off = 0.f, all = 0.f;
    for (int e = t; e < k * k; e += nt) {
      const int i = e / k, j = e - (e / k) * k;
      const float a = A[e];
      all += a * a;
      if (i != j) off += a * a;
    }
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_xor_sync(0xffffffffu, off, o);
      all += __shfl_xor_sync(0xffffffffu, all, o);
    }
    if ((t & 31) == 0) {
      red_off[t >> 5] = off;
      red_all[t >> 5] = all;
    }
    __syncthreads();
    if (t == 0) {
      float so = 0.f, sa = 0.f;
      for (int w = 0; w < (nt + 31) / 32; ++w) {
        so += red_off[w];
        sa += red_all[w];
      }
      // converged to FP32 resolution, or stalled at the rounding floor (Jacobi converges
      // linearly at first, so a stall only counts once the off-diagonal part is tiny).
      // The refinement's cluster threshold scales with this residue, so it must be small.
      stop = (so <= 1e-13f * sa || (so < 1e-10f * sa && so > 0.5f * prev_off)) ? 1 : 0;
      prev_off = so;
    }
    __syncthreads();
    if (stop) break;
    for (int round = 0; round < kp - 1; ++round) {
      if (t < npairs) {
        int p, q;
        circle_pair(t, round, kp, p, q);
        float c = 1.f, s = 0.f;
        if (q < k) {
          const float apq = A[p * k + q];
          if (apq != 0.f) {
            const float app = A[p * k + p], aqq = A[q * k + q];
            const float theta = (aqq - app) / (2.f * apq);
            const float tt = copysignf(1.f, theta) / (fabsf(theta) + sqrtf(theta * theta + 1.f));
            c = rsqrtf(tt * tt + 1.f);
            s = tt * c;
          }
        }
        cs[p] = c;
        sn[p] = s;
      }
      __syncthreads();
      // rows p, q of A: (J^T A)
      for (int e = t; e < npairs * k; e += nt) {
        const int pr = e / k, col = e - (e / k) * k;
        int p, q;
        circle_pair(pr, round, kp, p, q);
        if (q < k) {
          const float c = cs[p], s = sn[p];
          const float ap = A[p * k + col], aq = A[q * k + col];
          A[p * k + col] = c * ap - s * aq;
          A[q * k + col] = s * ap + c * aq;
        }
      }
      __syncthreads();
      // columns p, q of A and V: (A J), (V J)
      for (int e = t; e < npairs * k; e += nt) {
        const int pr = e / k, row = e - (e / k) * k;
        int p, q;
        circle_pair(pr, round, kp, p, q);
        if (q < k) {
          const float c = cs[p], s = sn[p];
          const float ap = A[row * k + p], aq = A[row * k + q];
          A[row * k + p] = c * ap - s * aq;
          A[row * k + q] = s * ap + c * aq;
          const float vp = V[row * k + p], vq = V[row * k + q];
          V[row * k + p] = c * vp - s * vq;
          V[row * k + q] = s * vp + c * vq;
        }
      }
      __syncthreads();
    }
  }
  for (int e = t; e < k * k; e += nt) Z[e] = (double)V[e];
}

// Element-wise part of one Ogita-Aishima step (single CTA).
// P = Z^T S Z, Q = Z^T Z (k x k, compact); writes E (k x k) and lam (k).
__global__ void __launch_bounds__(1024)
oa_update_kernel(int k, const double* __restrict__ P, const double* __restrict__ Q,
                 double* __restrict__ E, double* __restrict__ lam, double cluster_floor) {
  __shared__ double s_lam[kMaxBlockWidth];
  __shared__ double red[3][32];
  __shared__ double delta;
  const int t = threadIdx.x, nt = blockDim.x;
  for (int i = t; i < k; i += nt) s_lam[i] = P[i * k + i] / Q[i * k + i];  // s_ii / (1 - r_ii)
  __syncthreads();
  double off2 = 0.0, r2 = 0.0, nrm = 0.0;
  for (int e = t; e < k * k; e += nt) {
    const int i = e / k, j = e - (e / k) * k;
    const double r = ((i == j) ? 1.0 : 0.0) - Q[e];
    const double sd = P[e] - ((i == j) ? s_lam[i] : 0.0);
    off2 = fma(sd, sd, off2);
    r2 = fma(r, r, r2);
  }
  for (int i = t; i < k; i += nt) nrm = fmax(nrm, fabs(s_lam[i]));
  for (int o = 16; o > 0; o >>= 1) {
    off2 += __shfl_xor_sync(0xffffffffu, off2, o);
    r2 += __shfl_xor_sync(0xffffffffu, r2, o);
    nrm = fmax(nrm, __shfl_xor_sync(0xffffffffu, nrm, o));
  }
  if ((t & 31) == 0) {
    red[0][t >> 5] = off2;
    red[1][t >> 5] = r2;
    red[2][t >> 5] = nrm;
  }
  __syncthreads();
  if (t == 0) {
    double a = 0, b = 0, c = 0;
    for (int w = 0; w < (nt + 31) / 32; ++w) {
      a += red[0][w];
      b += red[1][w];
      c = fmax(c, red[2][w]);
    }
    // pairs closer than cluster_floor * ||S|| are left to the FP64 Jacobi pass:
    // the first-order update only converges when the error is below gap/||S||
    delta = fmax(2.0 * (sqrt(a) + c * sqrt(b)), cluster_floor * c);
  }
  __syncthreads();
  const double dl = delta;
  for (int e = t; e < k * k; e += nt) {
    const int i = e / k, j = e - (e / k) * k;
    const double r = ((i == j) ? 1.0 : 0.0) - Q[e];
    const double gap = s_lam[j] - s_lam[i];
    E[e] = (i != j && fabs(gap) > dl) ? (P[e] + s_lam[j] * r) / gap : 0.5 * r;
  }
  for (int i = t; i < k; i += nt) lam[i] = s_lam[i];
}

// Exact FP64 Jacobi on P = Z^T S Z after the refinement, for the pairs it left
// coupled (clusters closer than the refinement's floor). Only rotations with
// |P_pq| > max(1e-14 |P_pp - P_qq|, 1e-15 ||S||) are applied, so a resolved P
// costs one scan. Rotations are applied to P (shared memory) and to the
// columns of Z (global). Writes lam = diag(P).
__global__ void __launch_bounds__(1024)
jacobi_f64_cleanup_kernel(int k, const double* __restrict__ Pin, double* __restrict__ Z,
                          double* __restrict__ lam, int max_sweeps) {
  extern __shared__ double P[];  // k*k
  __shared__ double cs[kMaxBlockWidth + 1], sn[kMaxBlockWidth + 1];
  __shared__ int active[kMaxBlockWidth + 1];
  __shared__ int nsig;
  __shared__ double nrm;
  const int t = threadIdx.x, nt = blockDim.x;
  for (int e = t; e < k * k; e += nt) P[e] = Pin[e];
  if (t == 0) {
    double m = 0.0;
    for (int i = 0; i < k; ++i) m = fmax(m, fabs(Pin[i * k + i]));
    nrm = m;
  }
  __syncthreads();
  const int kp = (k + 1) & ~1;
  const int npairs = kp / 2;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    if (t == 0) nsig = 0;
    __syncthreads();
    int local = 0;
    for (int e = t; e < k * k; e += nt) {
      const int i = e / k, j = e - (e / k) * k;
      if (j > i) {
        const double apq = fabs(P[e]);
        if (apq > fmax(1e-14 * fabs(P[i * k + i] - P[j * k + j]), 1e-15 * nrm)) ++local;
      }
    }
    if (local) atomicAdd(&nsig, local);
    __syncthreads();
    if (nsig == 0) break;
    for (int round = 0; round < kp - 1; ++round) {
      if (t < npairs) {
        int p, q;
        circle_pair(t, round, kp, p, q);
        double c = 1.0, s = 0.0;
        int act = 0;
        if (q < k) {
          const double apq = P[p * k + q];
          const double app = P[p * k + p], aqq = P[q * k + q];
          if (fabs(apq) > fmax(1e-14 * fabs(app - aqq), 1e-15 * nrm)) {
            const double theta = (aqq - app) / (2.0 * apq);
            const double tt = copysign(1.0, theta) / (fabs(theta) + sqrt(theta * theta + 1.0));
            c = 1.0 / sqrt(tt * tt + 1.0);
            s = tt * c;
            act = 1;
          }
        }
        cs[p] = c;
        sn[p] = s;
        active[p] = act;
      }
      __syncthreads();
      for (int e = t; e < npairs * k; e += nt) {
        const int pr = e / k, col = e - (e / k) * k;
        int p, q;
        circle_pair(pr, round, kp, p, q);
        if (q < k && active[p]) {
          const double c = cs[p], s = sn[p];
          const double ap = P[p * k + col], aq = P[q * k + col];
          P[p * k + col] = c * ap - s * aq;
          P[q * k + col] = s * ap + c * aq;
        }
      }
      __syncthreads();
      for (int e = t; e < npairs * k; e += nt) {
        const int pr = e / k, row = e - (e / k) * k;
        int p, q;
        circle_pair(pr, round, kp, p, q);
        if (q < k && active[p]) {
          const double c = cs[p], s = sn[p];
          const double ap = P[row * k + p], aq = P[row * k + q];
          P[row * k + p] = c * ap - s * aq;
          P[row * k + q] = s * ap + c * aq;
          const double zp = Z[row * k + p], zq = Z[row * k + q];
          Z[row * k + p] = c * zp - s * zq;
          Z[row * k + q] = s * zp + c * zq;
        }
      }
      __syncthreads();
    }
  }
  for (int i = t; i < k; i += nt) lam[i] = P[i * k + i];
}

// S_out = (S + S^T)/2 (compact k x k): the projected matrix is symmetric only up to rounding.
__global__ void symmetrize_kernel(int k, const double* __restrict__ S, int lds,
                                  double* __restrict__ out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= k * k) return;
  const int i = e / k, j = e - (e / k) * k;
  out[e] = 0.5 * (S[(size_t)i * lds + j] + S[(size_t)j * lds + i]);
}

// Ascending order of lam (ties by index) and matching column permutation of Z.
__global__ void __launch_bounds__(1024)
sort_pairs_kernel(int k, const double* __restrict__ lam, const double* __restrict__ Zin,
                  double* __restrict__ evals, double* __restrict__ Zout, int ldz) {
  __shared__ int rank[kMaxBlockWidth];
  const int t = threadIdx.x, nt = blockDim.x;
  for (int i = t; i < k; i += nt) {
    const double li = lam[i];
    int r = 0;
    for (int j = 0; j < k; ++j) {
      const double lj = lam[j];
      r += (lj < li || (lj == li && j < i)) ? 1 : 0;
    }
    rank[i] = r;
    evals[r] = li;
  }
  __syncthreads();
  for (int e = t; e < k * k; e += nt) {
    const int row = e / k, i = e - (e / k) * k;
    Zout[(size_t)row * ldz + rank[i]] = Zin[e];
  }
}

struct EighScratch {
  double *S, *Z, *Z2, *T, *P, *Q, *E, *lam, *partials;
};

template <typename C>
EighScratch carve_eigh(C& c, int k) {
  EighScratch s{};
  const size_t kk = (size_t)k * k;
  s.S = c.template take<double>(kk);
  s.Z = c.template take<double>(kk);
  s.Z2 = c.template take<double>(kk);
  s.T = c.template take<double>(kk);
  s.P = c.template take<double>(kk);
  s.Q = c.template take<double>(kk);
  s.E = c.template take<double>(kk);
  s.lam = c.template take<double>(k);
  s.partials = c.template take<double>(
      std::max(gemm_tn_partials(k, k, k, false), gemm_tn_partials(k, k, k, true)));
  return s;
}

struct SizeOnly {
  size_t used = 0;
  template <typename T>
  T* take(size_t count) {
    used += align256(count * sizeof(T));
    return nullptr;
  }
};

}  // namespace

size_t small_eigh_scratch_bytes(int k) {
  SizeOnly s;
  carve_eigh(s, k);
  return s.used;
}

cudaError_t launch_small_eigh(int k, const double* S, int lds, double* evals, double* Zout, int ldz,
                              void* scratch, cudaStream_t st) {
  if (k <= 0 || k > kMaxBlockWidth) return cudaErrorInvalidValue;
  Carve c(scratch, small_eigh_scratch_bytes(k));
  EighScratch w = carve_eigh(c, k);
  if (!c.ok) return cudaErrorInvalidValue;
  cudaError_t e;
  symmetrize_kernel<<<(k * k + 255) / 256, 256, 0, st>>>(k, S, lds, w.S);
  note_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const size_t smem = 2 * (size_t)k * k * sizeof(float);
  if ((e = cudaFuncSetAttribute(jacobi_f32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem)) != cudaSuccess)
    return e;
  jacobi_f32_kernel<<<1, 1024, smem, st>>>(k, w.S, w.Z, kJacobiSweeps);
  note_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  double* Z = w.Z;
  double* Z2 = w.Z2;
  for (int step = 0; step < kOaSteps; ++step) {
    // T = S Z, P = Z^T T, Q = Z^T Z
    if ((e = launch_gemm_nn(k, k, k, 1.0, w.S, k, Z, k, 0.0, w.T, k, false, st)) != cudaSuccess)
      return e;
    if ((e = launch_gemm_tn(k, k, k, Z, k, w.T, k, w.P, k, false, w.partials, st)) != cudaSuccess)
      return e;
    if ((e = launch_gemm_tn(k, k, k, Z, k, Z, k, w.Q, k, true, w.partials, st)) != cudaSuccess)
      return e;
    oa_update_kernel<<<1, 1024, 0, st>>>(k, w.P, w.Q, w.E, w.lam, kClusterFloor);
  note_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // Z2 = Z + Z E
    if ((e = launch_copy2d(k, k, Z, k, Z2, k, st)) != cudaSuccess) return e;
    if ((e = launch_gemm_nn(k, k, k, 1.0, Z, k, w.E, k, 1.0, Z2, k, false, st)) != cudaSuccess)
      return e;
    std::swap(Z, Z2);
  }
  // exact FP64 rotations for the pairs the refinement treated as clusters
  if ((e = launch_gemm_nn(k, k, k, 1.0, w.S, k, Z, k, 0.0, w.T, k, false, st)) != cudaSuccess)
    return e;
  if ((e = launch_gemm_tn(k, k, k, Z, k, w.T, k, w.P, k, false, w.partials, st)) != cudaSuccess)
    return e;
  symmetrize_kernel<<<(k * k + 255) / 256, 256, 0, st>>>(k, w.P, k, w.Q);
  note_launch();
  const size_t smem64 = (size_t)k * k * sizeof(double);
  if ((e = cudaFuncSetAttribute(jacobi_f64_cleanup_kernel,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem64)) != cudaSuccess)
    return e;
  jacobi_f64_cleanup_kernel<<<1, 1024, smem64, st>>>(k, w.Q, Z, w.lam, 6);
  note_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  sort_pairs_kernel<<<1, 1024, 0, st>>>(k, w.lam, Z, evals, Zout, ldz);
  note_launch();
  return cudaGetLastError();
}

}  // namespace scsf
