// Truncated-FFT greedy sort (Alg. 2, Sec. 3.1).
//
// Features: F[k1][k2] = (1/p) sum_{x,y} P[x][y] w^(k1 x + k2 y), w = exp(-2 pi i/p),
// 0 <= k1, k2 < p0. Only p0 x p0 of the p x p coefficients are kept, so the
// kernel evaluates the truncated DFT directly in two passes instead of a full
// FFT: G[x][k2] = sum_y P[x][y] w^(k2 y) (p * p0 outputs, in shared memory),
// then F[k1][k2] = (1/p) sum_x w^(k1 x) G[x][k2]. Twiddles come from one
// table of the p roots of unity indexed by (k * y) mod p. One CTA per problem.
//
// Greedy chain: one CTA walks the n_ops - 1 steps. Each step computes the
// squared distance from the tail to every remaining problem in a fixed order
// (k1, k2, re, im) with explicitly rounded FP64 operations (no contraction),
// and takes the lexicographic minimum of (distance, index), so equal
// distances go to the smaller index.
#include "kernels.cuh"

namespace scsf {
namespace {

constexpr int kFeatThreads = 256;
constexpr int kChainThreads = 1024;

__global__ void __launch_bounds__(kFeatThreads)
dft_features_kernel(const double* __restrict__ fields, int p, int p0, double* __restrict__ feats) {
  extern __shared__ double sm[];
  double* twc = sm;              // [p]
  double* tws = sm + p;          // [p]
  double* G = sm + 2 * p;        // [p][p0][2]
  const double* P = fields + (size_t)blockIdx.x * p * p;
  const int t = threadIdx.x;
  for (int j = t; j < p; j += blockDim.x) {
    double s, c;
    sincospi(2.0 * (double)j / (double)p, &s, &c);
    twc[j] = c;
    tws[j] = s;
  }
  __syncthreads();
  // pass 1 over y (rows of P are contiguous)
  for (int item = t; item < p * p0; item += blockDim.x) {
    const int x = item / p0, k2 = item - (item / p0) * p0;
    const double* row = P + (size_t)x * p;
    double re = 0.0, im = 0.0;
    int idx = 0;  // (k2 * y) mod p
    for (int y = 0; y < p; ++y) {
      const double v = row[y];
      re = fma(v, twc[idx], re);
      im = fma(-v, tws[idx], im);
      idx += k2;
      if (idx >= p) idx -= p;
    }
    G[2 * item] = re;
    G[2 * item + 1] = im;
  }
  __syncthreads();
  // pass 2 over x
  const double inv_p = 1.0 / (double)p;
  double* F = feats + (size_t)blockIdx.x * p0 * p0 * 2;
  for (int item = t; item < p0 * p0; item += blockDim.x) {
    const int k1 = item / p0, k2 = item - (item / p0) * p0;
    double re = 0.0, im = 0.0;
    int idx = 0;  // (k1 * x) mod p
    for (int x = 0; x < p; ++x) {
      const double gr = G[2 * (x * p0 + k2)], gi = G[2 * (x * p0 + k2) + 1];
      const double c = twc[idx], s = tws[idx];
      // (c - i s)(gr + i gi) = (c gr + s gi) + i (c gi - s gr)
      re = fma(c, gr, fma(s, gi, re));
      im = fma(c, gi, fma(-s, gr, im));
      idx += k1;
      if (idx >= p) idx -= p;
    }
    F[2 * item] = re * inv_p;
    F[2 * item + 1] = im * inv_p;
  }
}

__device__ __forceinline__ bool lex_less(double da, int ja, double db, int jb) {
  return (da < db) || (da == db && ja < jb);
}

__global__ void __launch_bounds__(kChainThreads)
greedy_chain_kernel(const double* __restrict__ feats, int n_ops, int flen, int start,
                    unsigned char* __restrict__ visited, int32_t* __restrict__ perm,
                    double* __restrict__ dist) {
  extern __shared__ double tail[];  // [flen]
  __shared__ double red_d[32];
  __shared__ int red_j[32];
  __shared__ int s_tail;
  const int t = threadIdx.x, nt = blockDim.x;
  for (int j = t; j < n_ops; j += nt) visited[j] = 0;
  if (t == 0) {
    s_tail = start;
    perm[0] = start;
    if (dist) dist[0] = 0.0;
  }
  __syncthreads();
  if (t == 0) visited[start] = 1;
  __syncthreads();
  for (int step = 1; step < n_ops; ++step) {
    const int cur = s_tail;
    for (int m = t; m < flen; m += nt) tail[m] = feats[(size_t)cur * flen + m];
    __syncthreads();
    double best = INFINITY;
    int bj = 0x7fffffff;
    for (int j = t; j < n_ops; j += nt) {
      if (visited[j]) continue;
      const double* f = feats + (size_t)j * flen;
      double d = 0.0;
      for (int m = 0; m < flen; ++m) {
        const double diff = __dsub_rn(tail[m], f[m]);
        d = __dadd_rn(d, __dmul_rn(diff, diff));
      }
      if (lex_less(d, j, best, bj)) {
        best = d;
        bj = j;
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double od = __shfl_xor_sync(0xffffffffu, best, o);
      const int oj = __shfl_xor_sync(0xffffffffu, bj, o);
      if (lex_less(od, oj, best, bj)) {
        best = od;
        bj = oj;
      }
    }
    if ((t & 31) == 0) {
      red_d[t >> 5] = best;
      red_j[t >> 5] = bj;
    }
    __syncthreads();
    if (t == 0) {
      double b = red_d[0];
      int jb = red_j[0];
      for (int w = 1; w < (nt + 31) / 32; ++w)
        if (lex_less(red_d[w], red_j[w], b, jb)) {
          b = red_d[w];
          jb = red_j[w];
        }
      perm[step] = jb;
      if (dist) dist[step] = b;
      visited[jb] = 1;
      s_tail = jb;
    }
    __syncthreads();
  }
}

}  // namespace

size_t sort_workspace_bytes(int64_t n_ops, int p0) {
  return align256((size_t)n_ops * p0 * p0 * 2 * sizeof(double)) + align256((size_t)n_ops);
}

cudaError_t launch_sort(const double* fields, int64_t n_ops, int p, int p0, int start,
                        void* workspace, int32_t* perm, cudaStream_t st, double* dist) {
  double* feats = static_cast<double*>(workspace);
  unsigned char* visited = reinterpret_cast<unsigned char*>(
      static_cast<char*>(workspace) + align256((size_t)n_ops * p0 * p0 * 2 * sizeof(double)));
  const size_t smem = (size_t)(2 * p + 2 * p * p0) * sizeof(double);
  cudaError_t e = ensure_dynamic_smem((const void*)dft_features_kernel, smem);
  if (e != cudaSuccess) return e;
  dft_features_kernel<<<(unsigned)n_ops, kFeatThreads, smem, st>>>(fields, p, p0, feats);
  note_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const int flen = 2 * p0 * p0;
  greedy_chain_kernel<<<1, kChainThreads, flen * sizeof(double), st>>>(feats, (int)n_ops, flen,
                                                                       start, visited, perm, dist);
  note_launch();
  return cudaGetLastError();
}

}  // namespace scsf
