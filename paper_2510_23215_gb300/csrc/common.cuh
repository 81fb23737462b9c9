// Shared device/host helpers for the SCSF CUDA library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

namespace scsf {

// Largest block width k_b = k + nex accepted by the solver (the 256 x 256, k = 400
// workload needs 480).
constexpr int kMaxBlockWidth = 512;
// Up to this width the reduced eigensolve and the Cholesky factor keep their k_b x k_b
// matrices in one CTA's shared memory; wider blocks take the global-memory variants.
constexpr int kSmallBlockWidth = 160;

constexpr int kGemmTile = 32;     // output tile side of the FP64 block GEMMs
constexpr int kSplitTarget = 304; // CTAs targeted by split-K Gram launches (2 per SM)

// Stencil coefficients of the 5-point operator in row-major node order.
//   (A y)_I = d[I] y_I - we[I] y_{I+n} - we[I-n] y_{I-n} - wn[I] y_{I+1} - wn[I-1] y_{I-1}
// we[I] is the coupling of node I to its +i neighbour (zero on the last i row),
// wn[I] the coupling to its +j neighbour (zero on the last j column).
// A general sparse operator in CSR form (row_ptr [rows + 1], col / val [nnz], symmetric)
// travels in the same struct: when rp is non-null the kernels apply A from CSR and ignore
// d / we / wn.
struct Stencil {
  const double* d;
  const double* we;
  const double* wn;
  int n;
  const int* rp = nullptr;
  const int* ci = nullptr;
  const double* val = nullptr;
  int rows = 0;
};

__host__ __device__ inline int stencil_rows(const Stencil& A) { return A.rp ? A.rows : A.n * A.n; }

// FP32 copy of the stencil coefficients (mixed-precision path).
struct Stencil32 {
  const float* d;
  const float* we;
  const float* wn;
  int n;
};

// Process-wide count of kernels this library has launched (for benchmarks).
void note_launch();

inline size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// Bump allocator over a caller-owned device workspace.
struct Carve {
  char* base;
  size_t cap;
  size_t used = 0;
  bool ok = true;
  Carve(void* p, size_t c) : base(static_cast<char*>(p)), cap(c) {}
  template <typename T>
  T* take(size_t count) {
    size_t bytes = align256(count * sizeof(T));
    if (used + bytes > cap) { ok = false; return nullptr; }
    T* p = reinterpret_cast<T*>(base + used);
    used += bytes;
    return p;
  }
};

// Sizing-only twin of Carve.
struct CarveSize {
  size_t used = 0;
  template <typename T>
  void take(size_t count) { used += align256(count * sizeof(T)); }
};

}  // namespace scsf
