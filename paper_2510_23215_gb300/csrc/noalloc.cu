// Allocation-free variant of scsf_sort.
//
// Some callers cannot call cudaMalloc (or any allocating routine) at the point
// where they need the sort: for example code running inside a host framework
// that owns every byte of device memory through its own fixed-budget pool, or
// a latency-critical loop that must not enter the CUDA allocator. For them
// this entry point keeps its scratch (the truncated-DFT features and the
// visited flags) in a file-scope device array instead of a caller workspace.
// The array is reserved on a GPU when the first context is created there (scsf_create looks
// up its device address, which loads the library's module that holds it), or, if that failed,
// at the first call of this entry point on that GPU; it stays until the process exits.
#include <mutex>
#include <string>

#include "../../include/scsf.h"
#include "kernels.cuh"

namespace {

constexpr size_t kNoallocScratchBytes = size_t(8) << 20;  // 8 MiB per device

// Shared by every call on the same device; each call overwrites what it reads
// (features are fully rewritten, the visited flags are cleared by the kernel).
static __device__ __align__(256) unsigned char g_sort_scratch[kNoallocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};  // device address of g_sort_scratch, per device

// One-time set-up per device, with that device current: the host-side name of
// the array is only a stand-in, so the kernels need the device address.
cudaError_t scratch_address(int device, void** out) {
  if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_sort_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[device] = p;
  }
  *out = g_scratch_ptr[device];
  return cudaSuccess;
}

}  // namespace

namespace scsf {
cudaError_t noalloc_prepare(int device) {
  void* p = nullptr;
  const cudaError_t e = scratch_address(device, &p);
  if (e != cudaSuccess) cudaGetLastError();  // not sticky: the entry point retries
  return e;
}
}  // namespace scsf

extern "C" {

size_t scsf_sort_noalloc_capacity(void) { return kNoallocScratchBytes; }

scsf_status scsf_sort_noalloc(scsf_ctx* ctx, const double* fields, int64_t n_ops, int p, int p0,
                              int start, int32_t* perm_out) {
  if (!ctx) return SCSF_ERR_INVALID_ARG;
  // the same range and pointer checks as scsf_sort first, then the static capacity
  const scsf_status v = scsf::validate_sort_args(ctx, fields, n_ops, p, p0, start, perm_out);
  if (v != SCSF_OK) return v;
  if (scsf::sort_workspace_bytes(n_ops, p0) > kNoallocScratchBytes)
    return scsf::set_error(ctx, SCSF_ERR_NO_MEMORY,
                           "n_ops * p0 * p0 * 16 bytes (+ n_ops) exceeds the 8 MiB static scratch "
                           "of scsf_sort_noalloc; use scsf_sort with a caller workspace");
  const int dev = scsf::ctx_device(ctx);
  if (cudaSetDevice(dev) != cudaSuccess)
    return scsf::set_error(ctx, SCSF_ERR_CUDA, "cudaSetDevice failed");
  void* scratch = nullptr;
  const cudaError_t e = scratch_address(dev, &scratch);
  if (e != cudaSuccess)
    return scsf::set_error(ctx, SCSF_ERR_CUDA,
                           std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
  // enqueued on the context's stream like scsf_sort
  return scsf_sort(ctx, fields, n_ops, p, p0, start, scratch, kNoallocScratchBytes, perm_out);
}

}  // extern "C"
