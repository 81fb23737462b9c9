// Reduced symmetric eigensolve G W = W Lambda (Alg. 3, reduced eigensolve) for k <= 512
// (shared-memory kernels up to k = 160, global-memory variants above).
//
// GB300 runs FP32 about 60x faster than FP64, and one SM runs FP64 at about 2 FMA/clk, so
// the decomposition is found cheaply and then refined to FP64 accuracy on all SMs:
//   0. a probe (one CTA, FP32) decides whether G is already nearly diagonal: every pair
//      whose diagonal entries differ by more than the cluster floor has |g_ij| below
//      1e-2 of that difference. In a warm-started chain this holds for every Rayleigh-Ritz
//      matrix after the first of a problem (the block is already close to the Ritz
//      vectors), and then the start is the identity;
//   1. otherwise an FP32 eigenbasis of the trailing block that holds the strongly coupled
//      pairs (the probe returns its first index; the leading block keeps the identity):
//      Householder tridiagonalisation in one CTA, then eigenvalues by multisection, vectors
//      by inverse iteration and the back-transformation on many warps (trd.cuh);
//   2. Ogita-Aishima refinement steps in FP64 (X' = X (I + E) with
//      R = I - X^T X, S = X^T G X, lambda_i = s_ii/(1 - r_ii), E_ij =
//      (s_ij + lambda_j r_ij)/(lambda_j - lambda_i), or r_ij/2 for pairs closer
//      than delta = max(2(||S - D|| + ||G|| ||R||), 3e-3 ||G||)); each step squares
//      the error. X^T [G X | X] is one split-K product over all SMs, the element-wise
//      update runs on many CTAs after a one-CTA norm pass;
//   3. the pairs the refinement left coupled (eigenvalues closer than delta) form runs of
//      consecutive eigenvalues; each run (cluster) is diagonalised exactly by one warp
//      (cyclic FP64 Jacobi on its small block) and its columns of X rotated along. Runs
//      longer than kClusterMax fall back to exact FP64 round-robin Jacobi sweeps over
//      the whole matrix (one CTA, circle-method pair order: the k/2 disjoint rotations of
//      a round applied as one similarity transform over 2 x 2 blocks);
//   4. ascending sort of the pairs.
#include <algorithm>

#include "kernels.cuh"

namespace scsf {
namespace {

// Refinement steps (each squares the error): from the probe's start (couplings below 1e-2
// of the gaps, or the FP32 dense start's accuracy) three reach FP64, two the FP32 phase's
// accuracy; the FP32 dense start of a wide matrix carries more accumulated rounding, so it
// gets one more.
constexpr int kOaSteps = 3;
constexpr int kOaStepsF32 = 1;
constexpr int kOaStepsWide = 4;
constexpr float kNearDiag = 1e-2f;  // probe: largest |g_ij| / |g_jj - g_ii| of separated pairs
constexpr int kClusterMax = 16;     // longest run one warp diagonalises
constexpr int kClusterWarps = 8;    // warps that take runs (static shared memory: 35 KB)
constexpr double kClusterFloor = 3e-3;  // relative gap below which pairs go to FP64 Jacobi
constexpr double kCleanupTol = 1e-13;   // |P_pq| / ||G|| below which a pair counts as resolved

__host__ __device__ __forceinline__ int odd_stride(int k) { return (k % 2 == 0) ? k + 1 : k; }

// Pair (p < q) handled by slot `pr` in round `round` of the circle method over
// kp (even) players: position 0 is fixed, positions 1..kp-1 rotate.
__device__ __forceinline__ void circle_pair(int pr, int round, int kp, int& p, int& q) {
  const int pos_b = kp - 1 - pr;
  const int pa = (pr == 0) ? 0 : 1 + (pr - 1 + round) % (kp - 1);
  const int pb = 1 + (pos_b - 1 + round) % (kp - 1);
  p = min(pa, pb);
  q = max(pa, pb);
}

template <typename T>
__device__ __forceinline__ void jacobi_angle(T app, T aqq, T apq, T& c, T& s) {
  const T theta = (aqq - app) / (T(2) * apq);
  const T tt = copysign(T(1), theta) / (fabs(theta) + sqrt(theta * theta + T(1)));
  c = T(1) / sqrt(tt * tt + T(1));
  s = tt * c;
}

// One round of the circle method (k/2 disjoint rotations) applied as one similarity
// step A' = J^T A J, V' = V J (A k x k with stride ks, V's columns with stride ldv), all k/2
// rotations of the round forming J: for i, j with partners i', j' and coefficients
// (alpha, beta) -- row_i' = alpha_i row_i + beta_i row_i'(partner), so alpha = c and
// beta = -s for the first index of a pair, +s for the second, (1, 0) when the pair does
// not rotate -- A'_ij = alpha_i alpha_j A_ij + alpha_i beta_j A_ij' + beta_i alpha_j A_i'j
// + beta_i beta_j A_i'j'. Every thread updates whole 2 x 2 blocks (pair a x pair b, a <= b,
// mirrored), so the round needs only the angle pass, one barrier, the block pass and a
// second barrier, with all 1024 threads busy in the block pass.
template <typename T, typename Keep>
__device__ __forceinline__ void jacobi_round_blocks(T* A, int ks, T* V, int ldv, int k, int kp,
                                                    int round, Keep keep, T* al, T* be, int* plist,
                                                    int* nrot = nullptr) {
  const int t = threadIdx.x, nt = blockDim.x;
  const int lane = t & 31, warp = t >> 5, nwarps = nt >> 5;
  const int npairs = kp / 2;
  for (int pr = t; pr < npairs; pr += nt) {
    int p, q;
    circle_pair(pr, round, kp, p, q);
    plist[2 * pr] = p;
    plist[2 * pr + 1] = q;
    T c = T(1), sn = T(0);
    bool act = false;
    if (q < k) {
      const T apq = A[p * ks + q], app = A[p * ks + p], aqq = A[q * ks + q];
      if (keep(apq, app, aqq)) {
        jacobi_angle(app, aqq, apq, c, sn);
        act = true;
        if (nrot) atomicAdd(nrot, 1);
      }
    }
    al[p] = act ? c : T(1);
    be[p] = act ? -sn : T(0);
    if (q < k) {
      al[q] = act ? c : T(1);
      be[q] = act ? sn : T(0);
    }
  }
  __syncthreads();
  // the npairs (npairs + 1) / 2 blocks a <= b, dealt evenly over all threads: block index
  // idx = b (b + 1) / 2 + a with 0 <= a <= b
  const int nblk = npairs * (npairs + 1) / 2;
  for (int idx = t; idx < nblk; idx += nt) {
    int b = (int)((sqrtf(8.f * (float)idx + 1.f) - 1.f) * 0.5f);
    while (b * (b + 1) / 2 > idx) --b;
    while ((b + 1) * (b + 2) / 2 <= idx) ++b;
    const int a = idx - b * (b + 1) / 2;
    const int pa = plist[2 * a], qa = plist[2 * a + 1];
    const bool ha = qa < k;
    const T a_p = al[pa], b_p = be[pa];
    const T a_q = ha ? al[qa] : T(1), b_q = ha ? be[qa] : T(0);
    {
      const int pb = plist[2 * b], qb = plist[2 * b + 1];
      const bool hb = qb < k;
      const T c_p = al[pb], d_p = be[pb];
      // a block between two pairs that do not rotate stays as it is
      if (b_p == T(0) && d_p == T(0)) continue;
      const T c_q = hb ? al[qb] : T(1), d_q = hb ? be[qb] : T(0);
      const T s_pp = A[pa * ks + pb];
      const T s_pq = hb ? A[pa * ks + qb] : T(0);
      const T s_qp = ha ? A[qa * ks + pb] : T(0);
      const T s_qq = (ha && hb) ? A[qa * ks + qb] : T(0);
      const T n_pp = a_p * (c_p * s_pp + d_p * s_pq) + b_p * (c_p * s_qp + d_p * s_qq);
      const T n_pq = a_p * (c_q * s_pq + d_q * s_pp) + b_p * (c_q * s_qq + d_q * s_qp);
      const T n_qp = a_q * (c_p * s_qp + d_p * s_qq) + b_q * (c_p * s_pp + d_p * s_pq);
      const T n_qq = a_q * (c_q * s_qq + d_q * s_qp) + b_q * (c_q * s_pq + d_q * s_pp);
      if (a == b) {  // the pair's own block: the rotation annihilates its off-diagonal entry
        const bool act = ha && b_q != T(0);
        A[pa * ks + pa] = n_pp;
        if (ha) {
          A[qa * ks + qa] = n_qq;
          A[pa * ks + qa] = act ? T(0) : n_pq;
          A[qa * ks + pa] = act ? T(0) : n_qp;
        }
      } else {
        A[pa * ks + pb] = n_pp;
        A[pb * ks + pa] = n_pp;
        if (hb) {
          A[pa * ks + qb] = n_pq;
          A[qb * ks + pa] = n_pq;
        }
        if (ha) {
          A[qa * ks + pb] = n_qp;
          A[pb * ks + qa] = n_qp;
        }
        if (ha && hb) {
          A[qa * ks + qb] = n_qq;
          A[qb * ks + qa] = n_qq;
        }
      }
    }
  }
  // V' = V J: column pairs, rows across the lanes (odd stride: conflict-free)
  for (int b = warp; b < npairs; b += nwarps) {
    const int pb = plist[2 * b], qb = plist[2 * b + 1];
    if (qb >= k || be[qb] == T(0)) continue;
    const T c_p = al[pb], d_p = be[pb], c_q = al[qb], d_q = be[qb];
    for (int r = lane; r < k; r += 32) {
      const T vp = V[r * ldv + pb], vq = V[r * ldv + qb];
      V[r * ldv + pb] = c_p * vp + d_p * vq;
      V[r * ldv + qb] = c_q * vq + d_q * vp;
    }
  }
  __syncthreads();
}

#include "trd.cuh"

// Norm pass of one Ogita-Aishima step, over many CTAs: lambda_i = s_ii / (1 - r_ii), and into
// state (zeroed before) the sums of squares of the off-diagonal of P and of R = I - Q, and
// max |lambda_i| (as the bits of a non-negative float), from PQ = Z^T [S Z | Z] (k x 2k;
// P = left half, Q = right half). The apply pass forms the cluster threshold from them.
__global__ void __launch_bounds__(256)
oa_norms_kernel(int k, const double* __restrict__ PQ, double* __restrict__ lam,
                float* __restrict__ state) {
  __shared__ float red[3][8];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int ld = 2 * k;
  // the norms only set the cluster threshold: FP32 sums (one SM's FP64 pipe is narrow)
  float off2 = 0.f, r2 = 0.f, nrm = 0.f;
  for (int e = blockIdx.x * blockDim.x + t; e < k * k; e += gridDim.x * blockDim.x) {
    const int i = e / k, j = e - i * k;
    const float r = (float)(((i == j) ? 1.0 : 0.0) - PQ[i * ld + k + j]);
    const float sd = (i == j) ? 0.f : (float)PQ[i * ld + j];
    off2 = fmaf(sd, sd, off2);
    r2 = fmaf(r, r, r2);
    if (i == j) {
      const double li = PQ[i * ld + i] / PQ[i * ld + k + i];
      lam[i] = li;
      nrm = fmaxf(nrm, (float)fabs(li));
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    off2 += __shfl_xor_sync(0xffffffffu, off2, o);
    r2 += __shfl_xor_sync(0xffffffffu, r2, o);
    nrm = fmaxf(nrm, __shfl_xor_sync(0xffffffffu, nrm, o));
  }
  if (lane == 0) {
    red[0][warp] = off2;
    red[1][warp] = r2;
    red[2][warp] = nrm;
  }
  __syncthreads();
  if (t == 0) {
    float a = 0.f, b = 0.f, c = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      a += red[0][w];
      b += red[1][w];
      c = fmaxf(c, red[2][w]);
    }
    atomicAdd(&state[0], a);
    atomicAdd(&state[1], b);
    atomicMax(reinterpret_cast<int*>(&state[2]), __float_as_int(c));
  }
}

// Element-wise part of the step on many CTAs: Eplus = I + E. Pairs closer than
// delta = max(2 (||S - D|| + ||G|| ||R||), cluster_floor ||G||) keep E = R / 2 (left to the
// cluster pass: the first-order update only converges when the error is below gap / ||S||).
__global__ void oa_apply_kernel(int k, const double* __restrict__ PQ, const double* __restrict__ lam,
                                const float* __restrict__ state, double cluster_floor,
                                double* __restrict__ Eplus) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= k * k) return;
  const double c = (double)state[2];
  const double dl =
      fmax(2.0 * (sqrt((double)state[0]) + c * sqrt((double)state[1])), cluster_floor * c);
  const int ld = 2 * k;
  const int i = e / k, j = e - i * k;
  const double r = ((i == j) ? 1.0 : 0.0) - PQ[i * ld + k + j];
  const double li = lam[i], lj = lam[j];
  const double gap = lj - li;
  const double v = (i != j && fabs(gap) > dl) ? (PQ[i * ld + j] + lj * r) / gap : 0.5 * r;
  Eplus[e] = v + ((i == j) ? 1.0 : 0.0);
}

// Probe (one CTA, FP32): the pairs of S whose diagonal entries differ by more than
// floor * max|s_ii| are "separated"; a separated pair with |s_ij| > kNearDiag |s_jj - s_ii| is
// "far". start[0] = the smallest index of any far pair (k when there is none): the FP32
// Jacobi then only has to diagonalise the trailing block [start, k), and the refinement
// converges from there. In a warm-started chain the far pairs, if any, are the couplings
// among the top (guard) columns, which converge last.
__global__ void __launch_bounds__(1024)
eig_probe_kernel(int k, const double* __restrict__ S, double floor, int* __restrict__ start) {
  __shared__ float red[32];
  __shared__ int first;
  const int t = threadIdx.x, nt = blockDim.x;
  float nrm = 0.f;
  for (int i = t; i < k; i += nt) nrm = fmaxf(nrm, fabsf((float)S[(size_t)i * k + i]));
  for (int o = 16; o > 0; o >>= 1) nrm = fmaxf(nrm, __shfl_xor_sync(0xffffffffu, nrm, o));
  if ((t & 31) == 0) red[t >> 5] = nrm;
  if (t == 0) first = k;
  __syncthreads();
  float m = 0.f;
  for (int w = 0; w < (nt + 31) / 32; ++w) m = fmaxf(m, red[w]);
  const float dl = (float)floor * m;
  int local = k;
  for (int e = t; e < k * k; e += nt) {
    const int i = e / k, j = e - i * k;
    if (j <= i) continue;
    const float gap = fabsf((float)S[(size_t)j * k + j] - (float)S[(size_t)i * k + i]);
    const float sij = fabsf((float)S[e]);
    if ((gap > dl && sij > kNearDiag * gap) || !(sij == sij)) local = min(local, i);
  }
  if (local < k) atomicMin(&first, local);
  __syncthreads();
  if (t == 0) start[0] = first;
}

// Exact diagonalisation of the clusters the refinement left coupled (one CTA). P = Z^T S Z
// is the left half of PQ. Pairs with |P_ij| > tol (tol = kCleanupTol max|P_ii|) join the run
// of consecutive eigenvalues between them (positions in ascending order of diag(P)); each
// run of length 2..kClusterMax is diagonalised by one warp (cyclic FP64 Jacobi on its small
// block to below tol) and its columns of Z (ld ldz) rotated along. lam = diag(P) updated.
// A run longer than kClusterMax: with fallback non-null, fallback[0] = 1 and nothing changes
// (exact round-robin sweeps take over); with fallback null such runs keep their columns of Z
// (the FP32 phase, whose start vectors already resolve them to FP32 accuracy).
__global__ void __launch_bounds__(1024)
cluster_jacobi_kernel(int k, const double* __restrict__ PQ, double* __restrict__ Z, int ldz,
                      double* __restrict__ lam, int* __restrict__ fallback) {
  __shared__ int pos[kMaxBlockWidth], idx[kMaxBlockWidth], reach[kMaxBlockWidth];
  __shared__ int run_start[kMaxBlockWidth], nruns, too_long;
  __shared__ double nrm;
  __shared__ double blk[kClusterWarps][kClusterMax][kClusterMax + 1];
  __shared__ double W[kClusterWarps][kClusterMax][kClusterMax + 1];
  const int t = threadIdx.x, nt = blockDim.x, lane = t & 31, warp = t >> 5;
  const int ld = 2 * k;
  __shared__ double mred[32];
  double m = 0.0;
  for (int i = t; i < k; i += nt) m = fmax(m, fabs(PQ[i * ld + i]));
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) mred[warp] = m;
  __syncthreads();
  if (t == 0) {
    double mm = 0.0;
    for (int w = 0; w < nt / 32; ++w) mm = fmax(mm, mred[w]);
    nrm = mm;
    nruns = 0;
    too_long = 0;
  }
  // ascending positions of the diagonal (ties by index), from a shared copy of it
  __shared__ double dg[kMaxBlockWidth];
  for (int i = t; i < k; i += nt) dg[i] = PQ[i * ld + i];
  __syncthreads();
  for (int i = t; i < k; i += nt) {
    const double li = dg[i];
    int r = 0;
    for (int j = 0; j < k; ++j) {
      const double lj = dg[j];
      r += (lj < li || (lj == li && j < i)) ? 1 : 0;
    }
    pos[i] = r;
    idx[r] = i;
    reach[r] = r;
  }
  __syncthreads();
  const double tol = kCleanupTol * nrm;
  for (int e = t; e < k * k; e += nt) {
    const int i = e / k, j = e - i * k;
    if (j <= i) continue;
    const double pij = 0.5 * (PQ[i * ld + j] + PQ[j * ld + i]);
    if (fabs(pij) > tol) {
      const int a = min(pos[i], pos[j]), b = max(pos[i], pos[j]);
      atomicMax(&reach[a], b);
    }
  }
  __syncthreads();
  if (t == 0) {  // runs: maximal intervals joined by some coupled pair
    int r = 0;
    while (r < k) {
      int end = reach[r];
      int q = r;
      while (q < end) {
        ++q;
        end = max(end, reach[q]);
      }
      if (end > r) {
        if (end - r + 1 > kClusterMax) too_long = 1;
        run_start[nruns++] = r;
      }
      reach[r] = end;  // end of the run starting at r
      r = end + 1;
    }
  }
  __syncthreads();
  if (too_long && fallback) {
    if (t == 0) fallback[0] = 1;
    return;
  }
  for (int i = t; i < k; i += nt) lam[i] = dg[i];
  __syncthreads();
  if (warp >= kClusterWarps) return;
  for (int c = warp; c < nruns; c += kClusterWarps) {
    const int r0 = run_start[c], n = reach[r0] - r0 + 1;
    if (n > kClusterMax) continue;
    double(*A)[kClusterMax + 1] = blk[warp];
    double(*V)[kClusterMax + 1] = W[warp];
    for (int e = lane; e < n * n; e += 32) {
      const int a = e / n, b = e - a * n;
      const int ia = idx[r0 + a], ib = idx[r0 + b];
      A[a][b] = 0.5 * (PQ[ia * ld + ib] + PQ[ib * ld + ia]);
      V[a][b] = (a == b) ? 1.0 : 0.0;
    }
    __syncwarp();
    for (int sweep = 0; sweep < 12; ++sweep) {
      double off = 0.0;
      for (int e = lane; e < n * n; e += 32) {
        const int a = e / n, b = e - a * n;
        if (a != b) off = fmax(off, fabs(A[a][b]));
      }
      for (int o = 16; o > 0; o >>= 1) off = fmax(off, __shfl_xor_sync(0xffffffffu, off, o));
      if (off <= 0.1 * tol) break;
      for (int p = 0; p < n - 1; ++p)
        for (int q = p + 1; q < n; ++q) {
          const double apq = A[p][q];
          double cs = 1.0, sn = 0.0;
          if (fabs(apq) > 0.1 * tol) jacobi_angle(A[p][p], A[q][q], apq, cs, sn);
          __syncwarp();
          if (sn != 0.0) {
            // A' = J^T A J on rows / columns p, q; V' = V J
            if (lane < n) {
              const double ap = A[p][lane], aq = A[q][lane];
              A[p][lane] = cs * ap - sn * aq;
              A[q][lane] = sn * ap + cs * aq;
            }
            __syncwarp();
            if (lane < n) {
              const double ap = A[lane][p], aq = A[lane][q];
              A[lane][p] = cs * ap - sn * aq;
              A[lane][q] = sn * ap + cs * aq;
              const double vp = V[lane][p], vq = V[lane][q];
              V[lane][p] = cs * vp - sn * vq;
              V[lane][q] = sn * vp + cs * vq;
            }
            __syncwarp();
          }
        }
    }
    for (int a = lane; a < n; a += 32) lam[idx[r0 + a]] = A[a][a];
    // Z[:, run] = Z[:, run] V, row by row
    for (int row = lane; row < k; row += 32) {
      double z[kClusterMax];
      for (int a = 0; a < n; ++a) z[a] = Z[(size_t)row * ldz + idx[r0 + a]];
      for (int b = 0; b < n; ++b) {
        double v = 0.0;
        for (int a = 0; a < n; ++a) v = fma(z[a], V[a][b], v);
        Z[(size_t)row * ldz + idx[r0 + b]] = v;
      }
    }
    __syncwarp();
  }
}

// Exact FP64 Jacobi on P = Z^T S Z (left half of PQ, symmetrised on load) for
// the pairs the refinement left coupled. Rotates the columns of Z (global, ld
// ldz) along. Writes lam = diag(P).
template <bool kWide>
__global__ void __launch_bounds__(1024)
jacobi_f64_cleanup_kernel(int k, const double* __restrict__ PQ, double* __restrict__ Z, int ldz,
                          double* __restrict__ lam, int max_sweeps, double* __restrict__ wide,
                          const int* __restrict__ only_if) {
  if (only_if && !*only_if) return;  // the cluster pass resolved every coupled pair
  extern __shared__ double smd[];
  const int ks = odd_stride(k);
  double* P = kWide ? wide : smd;  // k x ks
  __shared__ double nrm;
  __shared__ int nsig;
  __shared__ double s_al[kMaxBlockWidth + 1], s_be[kMaxBlockWidth + 1];
  __shared__ int s_pl[kMaxBlockWidth + 2];
  const int t = threadIdx.x, nt = blockDim.x;
  const int ld = 2 * k;
  for (int e = t; e < k * k; e += nt) {
    const int i = e / k, j = e - i * k;
    P[i * ks + j] = 0.5 * (PQ[i * ld + j] + PQ[j * ld + i]);
  }
  __syncthreads();
  if (t == 0) {
    double m = 0.0;
    for (int i = 0; i < k; ++i) m = fmax(m, fabs(P[i * ks + i]));
    nrm = m;
  }
  __syncthreads();
  const double tol = kCleanupTol * nrm;
  const int kp = (k + 1) & ~1;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    if (t == 0) nsig = 0;
    __syncthreads();
    int local = 0;
    for (int e = t; e < k * k; e += nt) {
      const int i = e / k, j = e - i * k;
      if (j > i && fabs(P[i * ks + j]) > tol) ++local;
    }
    if (local) atomicAdd(&nsig, local);
    __syncthreads();
    if (nsig == 0) break;
    for (int round = 0; round < kp - 1; ++round)
      jacobi_round_blocks<double>(P, ks, Z, ldz, k, kp, round,
                                  [tol](double apq, double, double) { return fabs(apq) > tol; },
                                  s_al, s_be, s_pl);
  }
  for (int i = t; i < k; i += nt) lam[i] = P[i * ks + i];
}

// S_out = (S + S^T)/2 (compact k x k): the projected matrix is symmetric only up to rounding.
__global__ void symmetrize_kernel(int k, const double* __restrict__ S, int lds,
                                  double* __restrict__ out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= k * k) return;
  const int i = e / k, j = e - i * k;
  out[e] = 0.5 * (S[(size_t)i * lds + j] + S[(size_t)j * lds + i]);
}

// Ascending order of lam (ties by index) and matching column permutation of Z.
__global__ void __launch_bounds__(1024)
sort_pairs_kernel(int k, const double* __restrict__ lam, const double* __restrict__ Zin, int ldzin,
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
    const int row = e / k, i = e - row * k;
    Zout[(size_t)row * ldz + rank[i]] = Zin[(size_t)row * ldzin + i];
  }
}

// Scratch: S (k x k); two k x 2k panels [T | Z]; PQ (k x 2k); Eplus (k x k); lam; partials.
struct EighScratch {
  double *S, *TZ0, *TZ1, *PQ, *E, *lam, *partials, *state;
  int* flags;  // [0] near-diagonal (probe), [1] cluster pass fell back
  float *Hv, *dd, *ee, *lamt, *V32;  // tridiagonal start: reflectors, T, eigenpairs of T
  int* skip;
  float* trdA;     // k > kSmallBlockWidth: the FP32 block being reduced (k (k + 1))
  double* wide64;  // k > kSmallBlockWidth: the FP64 clean-up matrix (k ks)
};

template <typename C>
EighScratch carve_eigh(C& c, int k) {
  EighScratch s{};
  const size_t kk = (size_t)k * k;
  s.S = c.template take<double>(kk);
  s.TZ0 = c.template take<double>(2 * kk);
  s.TZ1 = c.template take<double>(2 * kk);
  s.PQ = c.template take<double>(2 * kk);
  s.E = c.template take<double>(kk);
  s.lam = c.template take<double>(k);
  s.partials = c.template take<double>(gemm_tn_partials(k, k, 2 * k, false));
  s.state = c.template take<double>(4);
  s.flags = c.template take<int>(4);
  s.Hv = c.template take<float>(kk);
  s.V32 = c.template take<float>(kk);
  s.dd = c.template take<float>(k);
  s.ee = c.template take<float>(k);
  s.lamt = c.template take<float>(k);
  s.skip = c.template take<int>(k);
  s.trdA = nullptr;
  s.wide64 = nullptr;
  if (k > kSmallBlockWidth) {
    s.trdA = c.template take<float>((size_t)k * (k + 1));
    s.wide64 = c.template take<double>((size_t)k * odd_stride(k));
  }
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

cudaError_t set_smem(const void* fn, size_t bytes) {
  return ensure_dynamic_smem(fn, bytes);
}


// Dense start on the trailing block the probe selected (Householder tridiagonalisation,
// multisection, inverse iteration, back-transformation); the leading block gets the identity.
cudaError_t run_trd(int k, const double* S, double* Z, int ldz, double* lam, const EighScratch& w,
                    cudaStream_t st, const int* start) {
  cudaError_t e;
  if (k <= kSmallBlockWidth) {
    const size_t smem = (size_t)k * (k + 1) * sizeof(float);
    if ((e = set_smem((const void*)trd_reduce_kernel<false>, smem)) != cudaSuccess) return e;
    trd_reduce_kernel<false><<<1, 1024, smem, st>>>(k, S, start, Z, ldz, lam, nullptr, w.Hv, w.dd,
                                                     w.ee, w.skip);
  } else {
    trd_reduce_kernel<true><<<1, 1024, 0, st>>>(k, S, start, Z, ldz, lam, w.trdA, w.Hv, w.dd, w.ee,
                                                w.skip);
  }
  note_launch();
  trd_eigval_kernel<<<(k + 7) / 8, 256, 0, st>>>(k, start, w.dd, w.ee, w.lamt);
  note_launch();
  const size_t vsmem = (size_t)kTrdWarpsPerBlock * 7 * k * sizeof(float);
  trd_eigvec_kernel<<<(k + kTrdWarpsPerBlock - 1) / kTrdWarpsPerBlock, 32 * kTrdWarpsPerBlock,
                      vsmem, st>>>(k, start, w.dd, w.ee, w.lamt, w.V32);
  note_launch();
  trd_back_kernel<<<(k + 7) / 8, 256, 0, st>>>(k, start, w.Hv, w.skip, w.V32, w.lamt, Z, ldz, lam);
  note_launch();
  return cudaGetLastError();
}

// Cluster pass; with `exact`, runs too long for it fall back to round-robin FP64 sweeps.
cudaError_t run_cleanup_f64(int k, const double* PQ, double* Z, int ldz, double* lam,
                            const EighScratch& w, cudaStream_t st, bool exact) {
  cudaError_t e;
  if ((e = cudaMemsetAsync(w.flags + 1, 0, sizeof(int), st)) != cudaSuccess) return e;
  cluster_jacobi_kernel<<<1, 1024, 0, st>>>(k, PQ, Z, ldz, lam, exact ? w.flags + 1 : nullptr);
  note_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (!exact) return cudaSuccess;
  if (k <= kSmallBlockWidth) {
    const size_t smem64 = (size_t)k * odd_stride(k) * sizeof(double);
    if ((e = set_smem((const void*)jacobi_f64_cleanup_kernel<false>, smem64)) != cudaSuccess) return e;
    jacobi_f64_cleanup_kernel<false><<<1, 1024, smem64, st>>>(k, PQ, Z, ldz, lam, 6, nullptr,
                                                               w.flags + 1);
  } else {
    jacobi_f64_cleanup_kernel<true><<<1, 1024, 0, st>>>(k, PQ, Z, ldz, lam, 10, w.wide64,
                                                        w.flags + 1);
  }
  note_launch();
  return cudaGetLastError();
}

// Start (probe, then the FP32 dense start on the block it selects) and `steps` refinement steps on the
// symmetrised w.S; the eigenvectors end in the right half of the returned panel (ld 2k),
// PQ = Z^T [S Z | Z] of the final Z in w.PQ.
cudaError_t eigh_refined(int k, const EighScratch& w, int steps, double** TZout, cudaStream_t st) {
  cudaError_t e;
  const int ld2 = 2 * k;
  eig_probe_kernel<<<1, 1024, 0, st>>>(k, w.S, kClusterFloor, w.flags);
  note_launch();
  double* TZ = w.TZ0;
  double* TZn = w.TZ1;
  if ((e = run_trd(k, w.S, TZ + k, ld2, nullptr, w, st, w.flags)) != cudaSuccess) return e;
  for (int step = 0; step <= steps; ++step) {
    // T = S Z into the left half; PQ = Z^T [T | Z]
    if ((e = launch_gemm_nn(k, k, k, 1.0, w.S, k, TZ + k, ld2, 0.0, TZ, ld2, false, st)) != cudaSuccess)
      return e;
    if ((e = launch_gemm_tn(k, k, 2 * k, TZ + k, ld2, TZ, ld2, w.PQ, ld2, false, w.partials, st)) !=
        cudaSuccess)
      return e;
    if (step == steps) break;
    float* nst = reinterpret_cast<float*>(w.state);
    if ((e = cudaMemsetAsync(nst, 0, 3 * sizeof(float), st)) != cudaSuccess) return e;
    oa_norms_kernel<<<std::min(64, (k * k + 255) / 256), 256, 0, st>>>(k, w.PQ, w.lam, nst);
    note_launch();
    oa_apply_kernel<<<(k * k + 255) / 256, 256, 0, st>>>(k, w.PQ, w.lam, nst, kClusterFloor, w.E);
    note_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // Z' = Z (I + E) into the next panel's right half
    if ((e = launch_gemm_nn(k, k, k, 1.0, TZ + k, ld2, w.E, k, 0.0, TZn + k, ld2, false, st)) !=
        cudaSuccess)
      return e;
    std::swap(TZ, TZn);
  }
  *TZout = TZ;
  return cudaSuccess;
}
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
  const int ld2 = 2 * k;
  symmetrize_kernel<<<(k * k + 255) / 256, 256, 0, st>>>(k, S, lds, w.S);
  note_launch();
  double* TZ = nullptr;
  const int oa_steps = (k > kSmallBlockWidth) ? kOaStepsWide : kOaSteps;
  if ((e = eigh_refined(k, w, oa_steps, &TZ, st)) != cudaSuccess) return e;
  // exact FP64 rotations for the pairs the refinement treated as clusters
  if ((e = run_cleanup_f64(k, w.PQ, TZ + k, ld2, w.lam, w, st, true)) != cudaSuccess) return e;
  sort_pairs_kernel<<<1, 1024, 0, st>>>(k, w.lam, TZ + k, ld2, evals, Zout, ldz);
  note_launch();
  return cudaGetLastError();
}

}  // namespace scsf

namespace scsf {

cudaError_t launch_small_eigh_f32(int k, const double* S, int lds, double* evals, double* Zout,
                                  int ldz, void* scratch, cudaStream_t st) {
  if (k <= 0 || k > kMaxBlockWidth) return cudaErrorInvalidValue;
  Carve c(scratch, small_eigh_scratch_bytes(k));
  EighScratch w = carve_eigh(c, k);
  if (!c.ok) return cudaErrorInvalidValue;
  cudaError_t e;
  symmetrize_kernel<<<(k * k + 255) / 256, 256, 0, st>>>(k, S, lds, w.S);
  note_launch();
  // FP32-phase accuracy (about 1e-7): one refinement step from the probe's start (none cost
  // more FP32 iterations, two measured no better)
  double* TZ = nullptr;
  if ((e = eigh_refined(k, w, kOaStepsF32, &TZ, st)) != cudaSuccess) return e;
  if ((e = run_cleanup_f64(k, w.PQ, TZ + k, 2 * k, w.lam, w, st, false)) != cudaSuccess) return e;
  sort_pairs_kernel<<<1, 1024, 0, st>>>(k, w.lam, TZ + k, 2 * k, evals, Zout, ldz);
  note_launch();
  return cudaGetLastError();
}

}  // namespace scsf
