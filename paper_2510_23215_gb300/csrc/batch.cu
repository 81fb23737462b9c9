// Batched solve: many independent chains (App. D.6: the dataset is cut into
// chunks, each solved by its own SCSF instance) in flight on one GPU.
//
// One outer iteration of a chain is a sequence of kernels, several of them
// latency-bound on one SM (Jacobi, Cholesky, triangular inverse) or a handful of
// SMs, plus a host decision (lock / stop). Running many chains at once, each on
// its own stream, overlaps those phases across the 152 SMs. Worker threads (one
// per concurrency slot) each own a stream, a staging context and a slice of the
// caller's workspace, and pull chains from a shared queue, largest first.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "../../include/scsf.h"
#include "kernels.cuh"

namespace {

size_t chain_bytes(const scsf_batch_chain& c) {
  if (!c.ops || c.n_ops < 1) return 0;
  if (c.ops[0].kind == SCSF_OP_CSR) return scsf_solve_workspace_size_rows(&c.params, c.ops[0].rows);
  return scsf_solve_workspace_size(&c.params, c.ops[0].n);
}

double chain_cost(const scsf_batch_chain& c) {
  const double N = c.ops[0].kind == SCSF_OP_CSR ? (double)c.ops[0].rows
                                                : (double)c.ops[0].n * c.ops[0].n;
  const double kb = c.params.k * 1.2;
  return (double)c.n_ops * N * kb * (1.0 + kb / 64.0);
}

}  // namespace

extern "C" {

size_t scsf_batch_workspace_size(const scsf_batch_chain* chains, int n_chains, int concurrency) {
  if (!chains || n_chains < 1 || concurrency < 1) return 0;
  size_t slot = 0;
  for (int i = 0; i < n_chains; ++i) {
    const size_t b = chain_bytes(chains[i]);
    if (b == 0) return 0;
    slot = std::max(slot, b);
  }
  const int slots = std::min(concurrency, n_chains);
  return scsf::align256(slot) * (size_t)slots;
}

scsf_status scsf_solve_batched(scsf_ctx* ctx, scsf_batch_chain* chains, int n_chains,
                               int concurrency, void* workspace, size_t workspace_bytes) {
  if (!ctx) return SCSF_ERR_INVALID_ARG;
  if (!chains || n_chains < 1 || concurrency < 1 || !workspace)
    return scsf::set_error(ctx, SCSF_ERR_INVALID_ARG, "bad batch arguments");
  if (concurrency > 64) return scsf::set_error(ctx, SCSF_ERR_INVALID_ARG, "concurrency > 64");
  const size_t need = scsf_batch_workspace_size(chains, n_chains, concurrency);
  if (need == 0)
    return scsf::set_error(ctx, SCSF_ERR_INVALID_ARG,
                           "a chain has no operators or unsupported parameters");
  if (workspace_bytes < need)
    return scsf::set_error(ctx, SCSF_ERR_NO_MEMORY, "batch workspace too small");
  const int device = scsf::ctx_device(ctx);
  if (cudaSetDevice(device) != cudaSuccess)
    return scsf::set_error(ctx, SCSF_ERR_CUDA, "cudaSetDevice failed");
  // inputs were produced on the caller's stream: make every worker stream wait for it
  cudaEvent_t ready;
  if (cudaEventCreateWithFlags(&ready, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventRecord(ready, scsf::ctx_stream(ctx)) != cudaSuccess)
    return scsf::set_error(ctx, SCSF_ERR_CUDA, "event record on the caller stream failed");

  std::vector<int> order(n_chains);
  for (int i = 0; i < n_chains; ++i) {
    order[i] = i;
    chains[i].status = SCSF_OK;
  }
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return chain_cost(chains[a]) > chain_cost(chains[b]); });
  const int slots = std::min(concurrency, n_chains);
  size_t slot_bytes = 0;
  for (int i = 0; i < n_chains; ++i) slot_bytes = std::max(slot_bytes, chain_bytes(chains[i]));
  slot_bytes = scsf::align256(slot_bytes);

  std::atomic<int> next{0};
  std::vector<std::string> errors(slots);
  std::vector<int> setup_fail(slots, 0);
  auto worker = [&](int w) {
    cudaSetDevice(device);
    cudaStream_t s = nullptr;
    scsf_ctx* sub = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamWaitEvent(s, ready, 0) != cudaSuccess || scsf_create(&sub, device, s) != SCSF_OK) {
      setup_fail[w] = 1;
      if (s) cudaStreamDestroy(s);
      return;
    }
    scsf_set_timing(sub, scsf::ctx_timing(ctx) ? 1 : 0);
    char* ws = static_cast<char*>(workspace) + slot_bytes * (size_t)w;
    for (;;) {
      const int idx = next.fetch_add(1);
      if (idx >= n_chains) break;
      scsf_batch_chain& c = chains[order[idx]];
      c.status = scsf_solve(sub, c.ops, c.n_ops, &c.params, ws, slot_bytes, c.evals, c.resid,
                            c.evecs, c.stats);
      if (c.status != SCSF_OK && errors[w].empty())
        errors[w] = "chain " + std::to_string(order[idx]) + ": " + scsf_last_error(sub);
    }
    cudaStreamSynchronize(s);
    scsf_destroy(sub);
    cudaStreamDestroy(s);
  };
  std::vector<std::thread> pool;
  pool.reserve(slots);
  for (int w = 0; w < slots; ++w) pool.emplace_back(worker, w);
  for (auto& t : pool) t.join();
  cudaEventDestroy(ready);
  for (int w = 0; w < slots; ++w)
    if (setup_fail[w]) return scsf::set_error(ctx, SCSF_ERR_CUDA, "worker stream setup failed");
  scsf_status first = SCSF_OK;
  for (int i = 0; i < n_chains && first == SCSF_OK; ++i) first = (scsf_status)chains[i].status;
  if (first != SCSF_OK) {
    std::string msg;
    for (auto& e : errors)
      if (!e.empty()) {
        msg = e;
        break;
      }
    return scsf::set_error(ctx, first, msg);
  }
  return SCSF_OK;
}

}  // extern "C"
