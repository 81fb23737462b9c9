// Seeded Gaussian block for the head of a chain (Sec. 3.2: the first problem
// starts from a random subspace). Counter-based Philox4x32-10 (Salmon, Moraes,
// Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11) feeding a
// Box-Muller transform, so every element depends only on (seed, index).
#include "kernels.cuh"

namespace scsf {
namespace {

struct U4 {
  uint32_t x, y, z, w;
};

__device__ __forceinline__ U4 philox_round(U4 c, uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
  const uint32_t hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
  return U4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
}

__device__ __forceinline__ U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1) {
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    c = philox_round(c, k0, k1);
    k0 += W0;
    k1 += W1;
  }
  return c;
}

// uniform in (0, 1) with 53 random bits
__device__ __forceinline__ double u53(uint32_t a, uint32_t b) {
  const uint64_t m = ((uint64_t)(a >> 5) << 26) | (uint64_t)(b >> 6);
  return ((double)m + 0.5) * (1.0 / 9007199254740992.0);
}

__global__ void philox_normal_kernel(double* __restrict__ out, int rows, int cols, int ld,
                                     uint64_t seed) {
  const long long total = (long long)rows * cols;
  const long long pair = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long e0 = 2 * pair;
  if (e0 >= total) return;
  const U4 r = philox4x32_10(U4{(uint32_t)pair, (uint32_t)(pair >> 32), 0u, 0u}, (uint32_t)seed,
                             (uint32_t)(seed >> 32));
  const double u1 = u53(r.x, r.y), u2 = u53(r.z, r.w);
  const double rad = sqrt(-2.0 * log(u1));
  double s, c;
  sincospi(2.0 * u2, &s, &c);
  const long long e1 = e0 + 1;
  out[(size_t)(e0 / cols) * ld + (e0 % cols)] = rad * c;
  if (e1 < total) out[(size_t)(e1 / cols) * ld + (e1 % cols)] = rad * s;
}

}  // namespace

cudaError_t launch_philox_normal(double* out, int rows, int cols, int ld, uint64_t seed,
                                 cudaStream_t st) {
  const long long pairs = ((long long)rows * cols + 1) / 2;
  if (pairs <= 0) return cudaSuccess;
  philox_normal_kernel<<<(unsigned)((pairs + 255) / 256), 256, 0, st>>>(out, rows, cols, ld, seed);
  note_launch();
  return cudaGetLastError();
}

}  // namespace scsf
