// Block products of Alg. 3 (Gram matrices of the orthonormalisation, the Rayleigh-Ritz
// projection Q^T (A Q), the rotation Q Z and the triangular solve X R^{-1}) on the
// fifth-generation tensor cores, with FP64 accuracy from BF16 operands.
//
// Method: the error-free splitting of Ozaki, Ogita and Oishi ("Error-free transformations
// of matrix multiplication by using fast routines of matrix multiplication", 2012), in
// the form Mukunoki, Ozaki, Ogita and Imamura used on FP16 tensor cores with FP32
// accumulation ("DGEMM using Tensor Cores, and Its Accurate and Reproducible Versions",
// 2020). Every row of the left operand and every column of the right operand is scaled
// by a power of two 2^E (E from its largest magnitude) and cut into S signed base-128
// digits: x = 2^E sum_p d_p 128^-p with d_1 in [0, 128] and d_p in [-64, 63] for p > 1
// (rounded at the last digit). Digits are small integers, exact in BF16. The product
// of two digit planes is a BF16 matrix product whose partial sums are integers of at most
// 2.36e6 over a K-chunk of 64 rows, so tcgen05.mma accumulates OZ_GROUP = 4 chunks (below
// 9.5e6 < 2^24) EXACTLY in FP32 tensor memory. Plane pairs (p, q) with p + q <= S + 1 are
// kept and summed per "level" p + q; the tensor-memory level sums are read out after every
// 4 chunks and added as integers, and the output is assembled from the exact integer level sums as a
// correctly rounded FP64 value (no FP64 arithmetic on the way; GB300's FP64 pipe is
// 1/60 of its FP32 rate). With S = 7 (28 BF16 products) the result carries ~49 bits of
// each operand, i.e. an error of a few 1e-15 of |a_i| |b_j| per term; S = 4 (10 products)
// gives FP32-class products for the mixed form's FP32 phase.
//
// Kernel (one CTA per SM, 320 threads):
//   warp 8   TMA producer: for each 64-row chunk, S stages of {A digit plane tile
//            128 x 64, B digit plane tile 32 x 64} (BF16, K-major, 128-byte swizzle)
//            into an 11-stage shared-memory ring, completion on mbarriers;
//   warp 9   allocates tensor memory and issues tcgen05.mma (M = 128, N = 32, K = 16)
//            from one thread, level sums double-buffered in tensor memory (2 x S x 32
//            columns), tcgen05.commit releases ring stages and hands every 4 chunks to readout;
//   warps 0-7 read the level sums (tcgen05.ld 32x32b.x16, lane quarter = warp % 4,
//            column half = warp / 4), add them as integers, and write the tile.
// Every wait is bounded (clock64 limit); a CTA that gives up sets a shared abort flag that
// ends the other roles' waits, drains its own copies and MMAs, frees its tensor memory and
// reports through the caller's error flag.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "kernels.cuh"

namespace scsf {
namespace {

constexpr int OZ_BM = 128;                          // output rows of a tile (MMA M)
constexpr int OZ_BN = 32;                           // output columns of a tile (MMA N)
constexpr int OZ_BK = 64;                           // K rows of a chunk (one 128-byte swizzle atom)
constexpr int OZ_A_BYTES = OZ_BM * OZ_BK * 2;       // 16 KiB
constexpr int OZ_B_BYTES = OZ_BN * OZ_BK * 2;       // 4 KiB
constexpr int OZ_STAGE = OZ_A_BYTES + OZ_B_BYTES;   // 20 KiB, multiple of 1024
constexpr int OZ_RING = 11;
constexpr int OZ_THREADS = 320;
constexpr int OZ_SMEM = OZ_RING * OZ_STAGE + 1024;  // + alignment slack
constexpr int OZ_GROUP = 4;  // 64-row chunks summed in tensor memory between readouts
constexpr int OZ_MAX_CHUNKS_PER_CTA = 512;          // keeps int32 level sums below 2^31
constexpr int OZ_NONFINITE = 0x7fff;                // exponent marker: the row/column has NaN/Inf
constexpr long long OZ_SPIN_CYCLES = 2000000000ll;  // ~1 s at 2 GHz per wait

// ---- PTX wrappers ----------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}
// D[tmem] (+)= A[smem] * B[smem]^T, BF16 in, FP32 accumulate
__device__ __forceinline__ void umma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   bar)
               : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
        "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Shared-memory matrix descriptor of a K-major BF16 tile written by TMA with the 128-byte
// swizzle: rows of 128 bytes, 8-row groups 1024 bytes apart (stride byte offset), the
// leading byte offset unused for this layout, descriptor version 1, swizzle mode 2.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) |
         ((uint64_t)(1024 >> 4) << 32) | ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
// Instruction descriptor: D FP32, A and B BF16, both K-major, N = 32, M = 128.
constexpr uint32_t OZ_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(OZ_BN >> 3) << 17) |
                              ((uint32_t)(OZ_BM >> 4) << 24);

// Bounded wait; a timeout or an abort raised by another role returns false.
// kSleep: back off between tries (the readout and producer warps); the MMA issuer, on the
// critical path, retries at once (mbarrier.try_wait itself suspends for a while).
template <bool kSleep = true>
__device__ __forceinline__ bool oz_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  for (;;) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*abort_flag) return false;
    if (clock64() - t0 > OZ_SPIN_CYCLES) {
      *abort_flag = 1;
      return false;
    }
    if (kSleep) __nanosleep(20);
  }
}
// Bounded wait that ignores the abort flag (draining own copies / MMAs before exit).
__device__ __forceinline__ void oz_wait_drain(uint32_t bar, uint32_t parity) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > OZ_SPIN_CYCLES) return;
    __nanosleep(20);
  }
}

// ---- exact integer -> FP64 --------------------------------------------------------
// T * 2^e rounded to nearest (ties to even); |T| < 2^127.
__device__ double oz_to_double(__int128 T, int e) {
  if (T == 0) return 0.0;
  const bool neg = T < 0;
  const unsigned __int128 a = neg ? (unsigned __int128)(-T) : (unsigned __int128)T;
  const unsigned long long hi = (unsigned long long)(a >> 64), lo = (unsigned long long)a;
  const int msb = hi ? 127 - __clzll((long long)hi) : 63 - __clzll((long long)lo);
  int sh = msb - 52;
  unsigned long long mant;
  if (sh <= 0) {
    mant = lo << (-sh);
  } else {
    const unsigned __int128 q = a >> sh;
    const unsigned __int128 rem = a - (q << sh);
    const unsigned __int128 half = (unsigned __int128)1 << (sh - 1);
    mant = (unsigned long long)q;
    if (rem > half || (rem == half && (mant & 1ull))) {
      ++mant;
      if (mant >> 53) {
        mant >>= 1;
        ++sh;
      }
    }
  }
  const int be = sh + e + 52 + 1023;
  if (be >= 1 && be <= 2046) {
    const unsigned long long bits = ((unsigned long long)be << 52) | (mant & 0xFFFFFFFFFFFFFull) |
                                    (neg ? (1ull << 63) : 0ull);
    return __longlong_as_double((long long)bits);
  }
  const double v = ldexp((double)mant, sh + e);  // subnormal or overflowing result (rare)
  return neg ? -v : v;
}

// ---- operand decoding and digits -------------------------------------------------
// |x| = mant * 2^e2 with mant an integer (< 2^53); returns the bits of |x| as a double for
// the column maxima (order of magnitudes = order of bit patterns).
__device__ __forceinline__ void oz_decode(double x, unsigned long long& mant, int& e2, bool& neg) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  neg = (b >> 63) != 0;
  const int ef = (int)((b >> 52) & 0x7FF);
  mant = b & 0xFFFFFFFFFFFFFull;
  if (ef) mant |= 1ull << 52;
  e2 = (ef ? ef : 1) - 1075;
}
__device__ __forceinline__ void oz_decode(float x, unsigned long long& mant, int& e2, bool& neg) {
  const uint32_t b = __float_as_uint(x);
  neg = (b >> 31) != 0;
  const int ef = (int)((b >> 23) & 0xFF);
  mant = b & 0x7FFFFFu;
  if (ef) mant |= 1ull << 23;
  e2 = (ef ? ef : 1) - 150;
}
// Magnitude keys ordered like |x|: the bits of |x| (FP64), or of |x| as FP32 (FP32 inputs,
// turned into FP64 bits once per column by oz_key_to_bits).
__device__ __forceinline__ unsigned long long oz_key(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
}
__device__ __forceinline__ unsigned long long oz_key(float x) {
  return (unsigned long long)(__float_as_uint(x) & 0x7FFFFFFFu);
}
template <typename T>
__device__ __forceinline__ unsigned long long oz_key_to_bits(unsigned long long key) {
  if constexpr (sizeof(T) == 8) {
    return key;
  } else {
    const float f = __uint_as_float((uint32_t)key);
    if (!(f <= 3.402823466e38f)) return 0x7FF8000000000000ull;  // NaN / Inf
    return (unsigned long long)__double_as_longlong((double)f);
  }
}

// Scale exponent of a row/column from the bits of its largest magnitude: the smallest E with
// max < 2^E (0 for an all-zero vector, OZ_NONFINITE for NaN / Inf).
__device__ __forceinline__ int oz_exponent(unsigned long long maxbits) {
  if (maxbits == 0) return 0;
  if (maxbits >= 0x7FF0000000000000ull) return OZ_NONFINITE;
  return ilogb(__longlong_as_double((long long)maxbits)) + 1;
}

// Digits of x / 2^E in base 128: d[0] in [0, 128], d[p] in [-64, 63], sign applied.
template <int S, typename T>
__device__ __forceinline__ void oz_digits(T x, int E, int (&d)[S]) {
  unsigned long long mant;
  int e2;
  bool neg;
  oz_decode(x, mant, e2, neg);
  long long V = 0;  // round(|x| 2^(7S - E)) < 2^(7S) + 1
  if (E != OZ_NONFINITE && mant) {
    const int sh = e2 + 7 * S - E;
    if (sh >= 0) V = (long long)(mant << sh);
    else if (sh > -60) V = (long long)((mant + (1ull << (-sh - 1))) >> (-sh));
  }
#pragma unroll
  for (int p = S - 1; p >= 1; --p) {
    const int r = (int)(V & 127);
    V >>= 7;
    if (r >= 64) {
      d[p] = r - 128;
      V += 1;
    } else {
      d[p] = r;
    }
  }
  d[0] = (int)V;
  if (neg)
#pragma unroll
    for (int p = 0; p < S; ++p) d[p] = -d[p];
}

__device__ __forceinline__ uint32_t bf16_bits_of_int(int v) {
  return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn((float)v));
}

// ---- preparation kernels ----------------------------------------------------------
// cmax[i] = max over rows of |X[r][i]| (as bits of a double), i < m. cmax zeroed before.
template <typename T>
__global__ void __launch_bounds__(256)
oz_colmax_kernel(int rows, int m, const T* __restrict__ X, int ld,
                 unsigned long long* __restrict__ cmax) {
  __shared__ unsigned long long red[8][32];
  const int lane = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int i = blockIdx.x * 32 + lane;
  unsigned long long best = 0;
  if (i < m) {
    const int step = 8 * gridDim.y;
    int r = blockIdx.y * 8 + ty;
    for (; r + 3 * step < rows; r += 4 * step) {  // four independent loads in flight
      const T x0 = X[(size_t)r * ld + i], x1 = X[(size_t)(r + step) * ld + i];
      const T x2 = X[(size_t)(r + 2 * step) * ld + i], x3 = X[(size_t)(r + 3 * step) * ld + i];
      best = max(max(best, max(oz_key(x0), oz_key(x1))), max(oz_key(x2), oz_key(x3)));
    }
    for (; r < rows; r += step) best = max(best, oz_key(X[(size_t)r * ld + i]));
  }
  red[ty][lane] = best;
  __syncthreads();
  if (ty == 0) {
#pragma unroll
    for (int t = 1; t < 8; ++t) best = max(best, red[t][lane]);
    if (i < m && best) atomicMax(&cmax[i], oz_key_to_bits<T>(best));
  }
}

// Digit planes of X^T: planes[s][i][k] = digit s of X[k][i] / 2^E_i (BF16), i < Mpad,
// k < Kp (zero outside rows x m). E_i from cmax; written to e_out by the first K tile.
template <typename T, int S>
__global__ void __launch_bounds__(256)
oz_split_cols_kernel(int rows, int m, const T* __restrict__ X, int ld,
                     const unsigned long long* __restrict__ cmax, int Mpad, int Kp,
                     uint32_t* __restrict__ planes, int* __restrict__ e_out) {
  __shared__ T tile[64][33];
  const int i0 = blockIdx.x * 32, k0 = blockIdx.y * 64;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int r = ty; r < 64; r += 8) {
    const int k = k0 + r, i = i0 + tx;
    tile[r][tx] = (k < rows && i < m) ? X[(size_t)k * ld + i] : T(0);
  }
  __syncthreads();
  for (int c = ty; c < 32; c += 8) {
    const int i = i0 + c;
    const int E = (i < m) ? oz_exponent(cmax[i]) : 0;
    if (blockIdx.y == 0 && tx == 0) e_out[i] = E;
    int d0[S], d1[S];
    oz_digits<S>(tile[2 * tx][c], E, d0);
    oz_digits<S>(tile[2 * tx + 1][c], E, d1);
#pragma unroll
    for (int s = 0; s < S; ++s)
      planes[((size_t)(s * Mpad + i) * Kp + k0 + 2 * tx) >> 1] =
          bf16_bits_of_int(d0[s]) | (bf16_bits_of_int(d1[s]) << 16);
  }
}

// Digit planes of X by rows: planes[s][r][c] = digit s of X[r][c] / 2^E_r, r < Mpad, c < Kp,
// E_r from the row's largest magnitude (one warp per row).
template <typename T, int S>
__global__ void __launch_bounds__(256)
oz_split_rows_kernel(int rows, int k, const T* __restrict__ X, int ld, int Mpad, int Kp,
                     uint32_t* __restrict__ planes, int* __restrict__ e_out) {
  const int lane = threadIdx.x & 31;
  const int r = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (r >= Mpad) return;
  const bool live = r < rows;
  unsigned long long best = 0;
  if (live)
    for (int c = lane; c < k; c += 32) best = max(best, oz_key(X[(size_t)r * ld + c]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) best = max(best, __shfl_xor_sync(0xffffffffu, best, o));
  const int E = oz_exponent(best ? oz_key_to_bits<T>(best) : 0ull);
  if (lane == 0) e_out[r] = E;
  for (int c = 2 * lane; c < Kp; c += 64) {
    const T x0 = (live && c < k) ? X[(size_t)r * ld + c] : T(0);
    const T x1 = (live && c + 1 < k) ? X[(size_t)r * ld + c + 1] : T(0);
    int d0[S], d1[S];
    oz_digits<S>(x0, E, d0);
    oz_digits<S>(x1, E, d1);
#pragma unroll
    for (int s = 0; s < S; ++s)
      planes[((size_t)(s * Mpad + r) * Kp + c) >> 1] =
          bf16_bits_of_int(d0[s]) | (bf16_bits_of_int(d1[s]) << 16);
  }
}

// ---- the tensor-core product --------------------------------------------------------
struct OzArgs {
  int Ma, Nb;        // rows per digit plane of the A / B operand tensors
  int tm, tn, sym;   // tile grid; sym: only tiles touching the upper triangle
  int m, n;          // output extent
  int nchunks, cps;  // 64-row K chunks in total, per CTA
  const int* ea;     // [Ma] row exponents of A
  const int* eb;     // [Nb] row exponents of B
  int mode;          // 0: exact int128 partial tiles; 1: FP64 C = alpha v + beta C; 2: FP32 C
  __int128* part;    // mode 0: [splits][m][n]
  double* out;       // mode 1
  float* outf;       // mode 2
  int ldo;
  double alpha, beta;
  int* err;
};

__device__ __forceinline__ void oz_tile(int idx, const OzArgs& a, int& mt, int& nt) {
  if (!a.sym) {
    mt = idx / a.tn;
    nt = idx - mt * a.tn;
    return;
  }
  mt = 0;
  for (;;) {
    const int cnt = a.tn - 4 * mt;  // tiles with 32 nt + 31 >= 128 mt
    if (idx < cnt) {
      nt = 4 * mt + idx;
      return;
    }
    idx -= cnt;
    ++mt;
  }
}

template <int S>
__global__ void __launch_bounds__(OZ_THREADS, 1)
oz_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
               const OzArgs args) {
  constexpr uint32_t TMEM_COLS = (2 * S * OZ_BN <= 256) ? 256u : 512u;
  static_assert(2 * S * OZ_BN <= 512, "level sums must fit tensor memory twice");
  __shared__ __align__(8) uint64_t full_bar[OZ_RING];
  __shared__ __align__(8) uint64_t empty_bar[OZ_RING];
  __shared__ __align__(8) uint64_t accf_bar[2];
  __shared__ __align__(8) uint64_t acce_bar[2];
  __shared__ __align__(8) uint64_t drain_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  extern __shared__ uint8_t oz_smem[];
  const uint32_t sbase = (smem_u32(oz_smem) + 1023u) & ~1023u;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int mt, nt;
  oz_tile(blockIdx.x, args, mt, nt);
  const int c0 = blockIdx.y * args.cps;
  const int nloc = max(0, min(args.nchunks, c0 + args.cps) - c0);

  if (threadIdx.x == 0) {
    for (int i = 0; i < OZ_RING; ++i) {
      mbar_init(smem_u32(&full_bar[i]), 1);
      mbar_init(smem_u32(&empty_bar[i]), 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(smem_u32(&accf_bar[i]), 1);
      mbar_init(smem_u32(&acce_bar[i]), 8);
    }
    mbar_init(smem_u32(&drain_bar), 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 9) tmem_alloc(smem_u32(&tmem_slot), TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  volatile int* abort_v = &abort_flag;

  if (warp == 8) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
      int issued = 0;
      bool ok = true;
      for (int tl = 0; tl < nloc && ok; ++tl) {
        const int kx = (c0 + tl) * OZ_BK;
        for (int j = 0; j < S; ++j) {
          const int g = tl * S + j, slot = g % OZ_RING, round = g / OZ_RING;
          if (round > 0 && !oz_wait(smem_u32(&empty_bar[slot]), (round - 1) & 1, abort_v)) {
            ok = false;
            break;
          }
          const uint32_t fb = smem_u32(&full_bar[slot]);
          const uint32_t dst = sbase + slot * OZ_STAGE;
          mbar_expect_tx(fb, OZ_STAGE);
          tma_load_2d(dst, &tmA, kx, j * args.Ma + mt * OZ_BM, fb);
          tma_load_2d(dst + OZ_A_BYTES, &tmB, kx, j * args.Nb + nt * OZ_BN, fb);
          ++issued;
        }
      }
      // every copy this CTA issued has landed before its shared memory is released
      for (int s = 0; s < OZ_RING && s < issued; ++s) {
        const int g_last = s + OZ_RING * ((issued - 1 - s) / OZ_RING);
        oz_wait_drain(smem_u32(&full_bar[s]), (g_last / OZ_RING) & 1);
      }
    }
  } else if (warp == 9) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      bool ok = true;
      for (int tl = 0; tl < nloc && ok; ++tl) {
        // OZ_GROUP chunks accumulate in one tensor-memory buffer before it is read out
        const int grp = tl / OZ_GROUP, tb = grp & 1;
        const bool first = tl % OZ_GROUP == 0;
        const bool last = tl % OZ_GROUP == OZ_GROUP - 1 || tl == nloc - 1;
        if (first && grp >= 2 &&
            !oz_wait<false>(smem_u32(&acce_bar[tb]), ((grp >> 1) - 1) & 1, abort_v)) {
          ok = false;
          break;
        }
        tc_fence_after();
        uint32_t started = first ? 0u : ~0u;
#pragma unroll
        for (int j = 0; j < S; ++j) {
          if (!ok) break;
          const int g = tl * S + j;
          if (!oz_wait<false>(smem_u32(&full_bar[g % OZ_RING]), (g / OZ_RING) & 1, abort_v)) {
            ok = false;
            break;
          }
          tc_fence_after();
          // plane pairs (p, q) whose later plane arrived with this stage
#pragma unroll
          for (int p = 1; p <= S; ++p)
#pragma unroll
            for (int q = 1; q <= S; ++q) {
              if ((p > q ? p : q) != j + 1 || p + q > S + 1) continue;
              const int l = p + q - 2;
              const uint32_t a_base = sbase + (uint32_t)((tl * S + p - 1) % OZ_RING) * OZ_STAGE;
              const uint32_t b_base =
                  sbase + (uint32_t)((tl * S + q - 1) % OZ_RING) * OZ_STAGE + OZ_A_BYTES;
              const uint32_t d = tmem + (uint32_t)(tb * S * OZ_BN + l * OZ_BN);
#pragma unroll
              for (int kk = 0; kk < OZ_BK / 16; ++kk)
                umma_bf16(d, sw128_desc(a_base + 32 * kk), sw128_desc(b_base + 32 * kk), OZ_IDESC,
                          ((started >> l) & 1u) | (kk > 0 ? 1u : 0u));
              started |= 1u << l;
            }
        }
        if (!ok) break;
        for (int j = 0; j < S; ++j) umma_commit(smem_u32(&empty_bar[(tl * S + j) % OZ_RING]));
        if (last) umma_commit(smem_u32(&accf_bar[tb]));
      }
      // no MMA may still write tensor memory when it is released
      umma_commit(smem_u32(&drain_bar));
      oz_wait_drain(smem_u32(&drain_bar), 0);
    }
    __syncwarp();
  } else {
    // ---------------- readout warps 0..7 ----------------
    const int quarter = warp & 3, half = warp >> 2;
    uint32_t acc[S][16];
#pragma unroll
    for (int l = 0; l < S; ++l)
#pragma unroll
      for (int c = 0; c < 16; ++c) acc[l][c] = 0u;
    bool ok = true;
    const int ngrp = (nloc + OZ_GROUP - 1) / OZ_GROUP;
    for (int gi = 0; gi < ngrp; ++gi) {
      const int tb = gi & 1;
      int got = 0;
      if (lane == 0) got = oz_wait(smem_u32(&accf_bar[tb]), (gi >> 1) & 1, abort_v) ? 1 : 0;
      got = __shfl_sync(0xffffffffu, got, 0);
      if (!got) {
        ok = false;
        break;
      }
      tc_fence_after();
#pragma unroll
      for (int l = 0; l < S; ++l) {
        uint32_t v[16];
        tmem_ld16(tmem + ((uint32_t)(32 * quarter) << 16) +
                      (uint32_t)(tb * S * OZ_BN + l * OZ_BN + 16 * half),
                  v);
#pragma unroll
        for (int c = 0; c < 16; ++c)
          acc[l][c] += (uint32_t)__float2int_rn(__uint_as_float(v[c]));  // an exact integer
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&acce_bar[tb]));
    }
    if (ok) {
      const int i = mt * OZ_BM + 32 * quarter + lane;
      const int jb = nt * OZ_BN + 16 * half;
      if (i < args.m) {
        const int Ea = args.ea[i];
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          const int j = jb + c;
          if (j >= args.n) break;
          __int128 T = 0;
#pragma unroll
          for (int l = 0; l < S; ++l)
            T += (__int128)(int)acc[l][c] * ((__int128)1 << (7 * (S - 1 - l)));
          if (args.mode == 0) {
            args.part[(size_t)blockIdx.y * args.m * args.n + (size_t)i * args.n + j] = T;
          } else {
            const int Eb = args.eb[j];
            double v = (Ea == OZ_NONFINITE || Eb == OZ_NONFINITE)
                           ? __longlong_as_double(0x7FF8000000000000ll)
                           : oz_to_double(T, Ea + Eb - 7 * (S + 1));
            if (args.alpha != 1.0) v *= args.alpha;
            if (args.mode == 1) {
              double* o = args.out + (size_t)i * args.ldo + j;
              *o = (args.beta == 0.0) ? v : v + args.beta * *o;
            } else {
              float* o = args.outf + (size_t)i * args.ldo + j;
              *o = (args.beta == 0.0) ? (float)v : (float)v + (float)args.beta * *o;
            }
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 9) {
    tc_fence_after();
    tmem_dealloc(tmem, TMEM_COLS);
  }
  if (threadIdx.x == 0 && abort_flag) atomicExch(args.err, 1);
}

// C[i][j] = sum over splits of the exact partials, rounded once (symmetric: mirrored).
__global__ void oz_reduce_kernel(int m, int n, int splits, bool sym, const __int128* __restrict__ part,
                                 const int* __restrict__ ea, const int* __restrict__ eb, int S,
                                 double* __restrict__ C, int ldc) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m * n) return;
  const int i = e / n, j = e - (e / n) * n;
  if (sym && i > j) return;  // written with its mirror by (j, i)
  const __int128* src = part + (size_t)i * n + j;
  const size_t stride = (size_t)m * n;
  __int128 T = 0;
  int s = 0;
  for (; s + 4 <= splits; s += 4)  // four independent loads in flight
    T += (src[s * stride] + src[(s + 1) * stride]) + (src[(s + 2) * stride] + src[(s + 3) * stride]);
  for (; s < splits; ++s) T += src[s * stride];
  const int Ea = ea[i], Eb = eb[j];
  const double v = (Ea == OZ_NONFINITE || Eb == OZ_NONFINITE)
                       ? __longlong_as_double(0x7FF8000000000000ll)
                       : oz_to_double(T, Ea + Eb - 7 * (S + 1));
  C[(size_t)i * ldc + j] = v;
  if (sym && i < j) C[(size_t)j * ldc + i] = v;
}

// ---- host side ------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static std::once_flag once;
  static EncodeTiledFn fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  return fn;
}

// 2-D BF16 tensor [rows_total][Kp] (K fastest), boxes of box_rows x 64, 128-byte swizzle.
cudaError_t make_map(CUtensorMap* map, const void* base, int Kp, long long rows_total,
                     int box_rows) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return cudaErrorNotSupported;
  if (reinterpret_cast<uintptr_t>(base) % 16 != 0 || Kp % OZ_BK != 0) return cudaErrorInvalidValue;
  cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)rows_total};
  cuuint64_t strides[1] = {(cuuint64_t)Kp * 2};
  cuuint32_t box[2] = {(cuuint32_t)OZ_BK, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims,
                         strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

inline int ru(int x, int q) { return (x + q - 1) / q * q; }

int sm_count() {
  static int cached[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 148;
  if (!cached[dev]) {
    int c = 0;
    cached[dev] = (cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && c > 0)
                      ? c
                      : 148;
  }
  return cached[dev];
}

struct OzPlan {
  int Ma, Nb, Kp, tm, tn, ntiles, nchunks, cps, splits;
};

// sym: only tiles touching the upper triangle (C symmetric); same: B is A (shared planes)
OzPlan plan_tn(int rows, int m, int n, bool sym, bool same, int sms) {
  OzPlan p;
  p.Ma = ru(m, OZ_BM);
  p.Kp = ru(std::max(rows, 1), OZ_BK);
  p.tm = p.Ma / OZ_BM;
  p.tn = ru(n, OZ_BN) / OZ_BN;
  p.Nb = same ? p.Ma : ru(n, OZ_BN);
  if (sym) {
    p.ntiles = 0;
    for (int mt = 0; mt < p.tm; ++mt) p.ntiles += std::max(0, p.tn - 4 * mt);
  } else {
    p.ntiles = p.tm * p.tn;
  }
  p.nchunks = p.Kp / OZ_BK;
  int want = std::max(1, sms / std::max(1, p.ntiles));
  want = std::max(want, (p.nchunks + OZ_MAX_CHUNKS_PER_CTA - 1) / OZ_MAX_CHUNKS_PER_CTA);
  want = std::min(want, p.nchunks);
  p.cps = (p.nchunks + want - 1) / want;
  p.splits = (p.nchunks + p.cps - 1) / p.cps;
  return p;
}

OzPlan plan_nn(int rows, int k, int n) {
  OzPlan p;
  p.Ma = ru(rows, OZ_BM);
  p.Nb = ru(n, OZ_BN);
  p.Kp = ru(std::max(k, 1), OZ_BK);
  p.tm = p.Ma / OZ_BM;
  p.tn = p.Nb / OZ_BN;
  p.ntiles = p.tm * p.tn;
  p.nchunks = p.Kp / OZ_BK;
  p.cps = p.nchunks;
  p.splits = 1;
  return p;
}

size_t planes_bytes(int S, int R, int Kp) { return align256((size_t)S * R * Kp * 2); }

// Scratch carving shared by sizing and launch.
struct OzScratch {
  uint32_t *pa, *pb;
  int *ea, *eb;
  unsigned long long* cmax;
  __int128* part;
  size_t used;
};

template <typename Cv>
void carve_tn(Cv& c, const OzPlan& p, int m, int n, bool same, int S, OzScratch& s) {
  s.pa = c.template take<uint32_t>(planes_bytes(S, p.Ma, p.Kp) / 4);
  s.pb = same ? s.pa : c.template take<uint32_t>(planes_bytes(S, p.Nb, p.Kp) / 4);
  s.ea = c.template take<int>(p.Ma);
  s.eb = same ? s.ea : c.template take<int>(p.Nb);
  s.cmax = c.template take<unsigned long long>((size_t)m + n);
  s.part = c.template take<__int128>((size_t)p.splits * m * n);
}
template <typename Cv>
void carve_nn(Cv& c, const OzPlan& p, int k, int n, int S, OzScratch& s) {
  s.pa = c.template take<uint32_t>(planes_bytes(S, p.Ma, p.Kp) / 4);
  s.pb = c.template take<uint32_t>(planes_bytes(S, p.Nb, p.Kp) / 4);
  s.ea = c.template take<int>(p.Ma);
  s.eb = c.template take<int>(p.Nb);
  s.cmax = c.template take<unsigned long long>((size_t)n);
  s.part = nullptr;
}

struct NullCarve {
  size_t used = 0;
  template <typename T>
  T* take(size_t count) {
    used += align256(count * sizeof(T));
    return nullptr;
  }
};

template <int S>
cudaError_t launch_oz_gemm(const OzPlan& p, const uint32_t* pa, const uint32_t* pb, OzArgs args,
                           cudaStream_t st) {
  CUtensorMap ma, mb;
  cudaError_t e = make_map(&ma, pa, p.Kp, (long long)S * p.Ma, OZ_BM);
  if (e != cudaSuccess) return e;
  e = make_map(&mb, pb, p.Kp, (long long)S * p.Nb, OZ_BN);
  if (e != cudaSuccess) return e;
  e = ensure_dynamic_smem(reinterpret_cast<const void*>(&oz_gemm_kernel<S>), OZ_SMEM);
  if (e != cudaSuccess) return e;
  args.Ma = p.Ma;
  args.Nb = p.Nb;
  args.tm = p.tm;
  args.tn = p.tn;
  args.nchunks = p.nchunks;
  args.cps = p.cps;
  dim3 grid(p.ntiles, p.splits);
  oz_gemm_kernel<S><<<grid, OZ_THREADS, OZ_SMEM, st>>>(ma, mb, args);
  note_launch();
  return cudaGetLastError();
}

template <int S, typename T>
cudaError_t gemm_tn_oz_impl(int rows, int m, int n, const T* A, int lda, const T* B, int ldb,
                            double* C, int ldc, bool sym, void* scratch, size_t scratch_bytes,
                            int* err, cudaStream_t st) {
  if (m <= 0 || n <= 0) return cudaSuccess;
  if (sym && m != n) return cudaErrorInvalidValue;
  const bool same = A == B && lda == ldb && m == n;
  const OzPlan p = plan_tn(rows, m, n, sym, same, sm_count());
  Carve cv(scratch, scratch_bytes);
  OzScratch s;
  carve_tn(cv, p, m, n, same, S, s);
  if (!cv.ok) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(s.cmax, 0, sizeof(unsigned long long) * ((size_t)m + n), st);
  if (e != cudaSuccess) return e;
  const dim3 mgrid((m + 31) / 32, std::min(128, std::max(1, (rows + 7) / 8)));
  oz_colmax_kernel<T><<<mgrid, 256, 0, st>>>(rows, m, A, lda, s.cmax);
  note_launch();
  oz_split_cols_kernel<T, S><<<dim3(p.Ma / 32, p.Kp / 64), 256, 0, st>>>(rows, m, A, lda, s.cmax,
                                                                         p.Ma, p.Kp, s.pa, s.ea);
  note_launch();
  if (!same) {
    const dim3 ngrid((n + 31) / 32, std::min(128, std::max(1, (rows + 7) / 8)));
    oz_colmax_kernel<T><<<ngrid, 256, 0, st>>>(rows, n, B, ldb, s.cmax + m);
    note_launch();
    oz_split_cols_kernel<T, S><<<dim3(p.Nb / 32, p.Kp / 64), 256, 0, st>>>(
        rows, n, B, ldb, s.cmax + m, p.Nb, p.Kp, s.pb, s.eb);
    note_launch();
  }
  OzArgs a{};
  a.sym = sym ? 1 : 0;
  a.m = m;
  a.n = n;
  a.ea = s.ea;
  a.eb = s.eb;
  a.mode = 0;
  a.part = s.part;
  a.alpha = 1.0;
  a.beta = 0.0;
  a.err = err;
  if ((e = launch_oz_gemm<S>(p, s.pa, s.pb, a, st)) != cudaSuccess) return e;
  oz_reduce_kernel<<<(m * n + 255) / 256, 256, 0, st>>>(m, n, p.splits, sym, s.part, s.ea, s.eb, S,
                                                        C, ldc);
  note_launch();
  return cudaGetLastError();
}

template <int S, typename T, typename TO>
cudaError_t gemm_nn_oz_impl(int rows, int k, int n, double alpha, const T* A, int lda,
                            const double* M, int ldm, double beta, TO* C, int ldc, void* scratch,
                            size_t scratch_bytes, int* err, cudaStream_t st) {
  if (rows <= 0 || n <= 0) return cudaSuccess;
  const OzPlan p = plan_nn(rows, k, n);
  Carve cv(scratch, scratch_bytes);
  OzScratch s;
  carve_nn(cv, p, k, n, S, s);
  if (!cv.ok) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(s.cmax, 0, sizeof(unsigned long long) * (size_t)n, st);
  if (e != cudaSuccess) return e;
  // B operand: M^T by rows of M's columns (K-major), scaled per column of M
  oz_colmax_kernel<double><<<dim3((n + 31) / 32, std::min(128, std::max(1, (k + 7) / 8))), 256, 0,
                             st>>>(k, n, M, ldm, s.cmax);
  note_launch();
  oz_split_cols_kernel<double, S><<<dim3(p.Nb / 32, p.Kp / 64), 256, 0, st>>>(k, n, M, ldm, s.cmax,
                                                                              p.Nb, p.Kp, s.pb, s.eb);
  note_launch();
  oz_split_rows_kernel<T, S><<<(p.Ma + 7) / 8, 256, 0, st>>>(rows, k, A, lda, p.Ma, p.Kp, s.pa,
                                                             s.ea);
  note_launch();
  OzArgs a{};
  a.sym = 0;
  a.m = rows;
  a.n = n;
  a.ea = s.ea;
  a.eb = s.eb;
  a.alpha = alpha;
  a.beta = beta;
  a.ldo = ldc;
  a.err = err;
  if constexpr (sizeof(TO) == 8) {
    a.mode = 1;
    a.out = reinterpret_cast<double*>(C);
  } else {
    a.mode = 2;
    a.outf = reinterpret_cast<float*>(C);
  }
  return launch_oz_gemm<S>(p, s.pa, s.pb, a, st);
}

}  // namespace

size_t oz_scratch_bytes(int rows, int kmax, int slices) {
  if (rows <= 0 || kmax <= 0) return 0;
  const int sms = 160;  // sizing bound: at least the SM count of the device
  // TN products C[m x n] = A^T B for every m, n <= kmax. Within a run of widths that give
  // the same tile count, planes and split partials grow with the width, so the ends of
  // the runs (multiples of the tile width 32) and kmax are the candidates.
  std::vector<int> ws;
  for (int v = OZ_BN; v < kmax; v += OZ_BN) ws.push_back(v);
  ws.push_back(kmax);
  size_t best = 0;
  for (int m : ws)
    for (int n : ws)
      for (int mode = 0; mode < 3; ++mode) {  // general, symmetric, symmetric with B = A
        if (mode > 0 && m != n) continue;
        const OzPlan p = plan_tn(rows, m, n, mode > 0, mode == 2, sms);
        NullCarve c;
        OzScratch s;
        carve_tn(c, p, m, n, mode == 2, slices, s);
        best = std::max(best, c.used);
      }
  const OzPlan p = plan_nn(rows, kmax, kmax);
  NullCarve c;
  OzScratch s;
  carve_nn(c, p, kmax, kmax, slices, s);
  best = std::max(best, c.used);
  return best + 256;
}

cudaError_t launch_gemm_tn_oz(int rows, int m, int n, const double* A, int lda, const double* B,
                              int ldb, double* C, int ldc, bool symmetric, int slices,
                              void* scratch, size_t scratch_bytes, int* err, cudaStream_t st) {
  if (slices == 7)
    return gemm_tn_oz_impl<7>(rows, m, n, A, lda, B, ldb, C, ldc, symmetric, scratch,
                              scratch_bytes, err, st);
  if (slices == 8)
    return gemm_tn_oz_impl<8>(rows, m, n, A, lda, B, ldb, C, ldc, symmetric, scratch,
                              scratch_bytes, err, st);
  if (slices == 4)
    return gemm_tn_oz_impl<4>(rows, m, n, A, lda, B, ldb, C, ldc, symmetric, scratch,
                              scratch_bytes, err, st);
  return cudaErrorInvalidValue;
}

cudaError_t time_gemm_tn_oz(int rows, int m, const double* A, int lda, int slices, void* scratch,
                            size_t scratch_bytes, int* err, int reps, cudaStream_t st,
                            float* ms_out) {
  if (slices != 8 || m <= 0 || rows <= 0 || reps < 1) return cudaErrorInvalidValue;
  constexpr int S = 8;
  const OzPlan p = plan_tn(rows, m, m, true, true, sm_count());
  Carve cv(scratch, scratch_bytes);
  OzScratch s;
  carve_tn(cv, p, m, m, true, S, s);
  if (!cv.ok) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(s.cmax, 0, sizeof(unsigned long long) * 2 * (size_t)m, st);
  if (e != cudaSuccess) return e;
  oz_colmax_kernel<double><<<dim3((m + 31) / 32, std::min(128, std::max(1, (rows + 7) / 8))), 256, 0,
                             st>>>(rows, m, A, lda, s.cmax);
  note_launch();
  oz_split_cols_kernel<double, S><<<dim3(p.Ma / 32, p.Kp / 64), 256, 0, st>>>(rows, m, A, lda, s.cmax,
                                                                              p.Ma, p.Kp, s.pa, s.ea);
  note_launch();
  OzArgs a{};
  a.sym = 1;
  a.m = m;
  a.n = m;
  a.ea = s.ea;
  a.eb = s.ea;
  a.mode = 0;
  a.part = s.part;
  a.alpha = 1.0;
  a.err = err;
  if ((e = launch_oz_gemm<S>(p, s.pa, s.pa, a, st)) != cudaSuccess) return e;  // warm
  cudaEvent_t e0, e1;
  if ((e = cudaEventCreate(&e0)) != cudaSuccess) return e;
  if ((e = cudaEventCreate(&e1)) != cudaSuccess) {
    cudaEventDestroy(e0);
    return e;
  }
  cudaEventRecord(e0, st);
  for (int r = 0; r < reps && e == cudaSuccess; ++r) e = launch_oz_gemm<S>(p, s.pa, s.pa, a, st);
  cudaEventRecord(e1, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e == cudaSuccess) *ms_out = ms / reps;
  return e;
}

cudaError_t launch_gemm_tn_oz_f32(int rows, int m, int n, const float* A, int lda, const float* B,
                                  int ldb, double* C, int ldc, bool symmetric, void* scratch,
                                  size_t scratch_bytes, int* err, cudaStream_t st) {
  return gemm_tn_oz_impl<kOzSlicesF32>(rows, m, n, A, lda, B, ldb, C, ldc, symmetric, scratch,
                                       scratch_bytes, err, st);
}

cudaError_t launch_gemm_nn_oz(int rows, int k, int n, double alpha, const double* A, int lda,
                              const double* M, int ldm, double beta, double* C, int ldc,
                              int slices, void* scratch, size_t scratch_bytes, int* err,
                              cudaStream_t st) {
  if (slices == 7)
    return gemm_nn_oz_impl<7>(rows, k, n, alpha, A, lda, M, ldm, beta, C, ldc, scratch,
                              scratch_bytes, err, st);
  if (slices == 8)
    return gemm_nn_oz_impl<8>(rows, k, n, alpha, A, lda, M, ldm, beta, C, ldc, scratch,
                              scratch_bytes, err, st);
  if (slices == 4)
    return gemm_nn_oz_impl<4>(rows, k, n, alpha, A, lda, M, ldm, beta, C, ldc, scratch,
                              scratch_bytes, err, st);
  return cudaErrorInvalidValue;
}

cudaError_t launch_gemm_nn_oz_f32(int rows, int k, int n, float alpha, const float* A, int lda,
                                  const double* M, int ldm, float beta, float* C, int ldc,
                                  void* scratch, size_t scratch_bytes, int* err, cudaStream_t st) {
  return gemm_nn_oz_impl<kOzSlicesF32>(rows, k, n, (double)alpha, A, lda, M, ldm, (double)beta, C,
                                       ldc, scratch, scratch_bytes, err, st);
}

}  // namespace scsf
