// Shared engine of the batched launch, used by rad_batch and the server.
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "rad.h"
#include "rad_impl.h"

struct rad_ctx;

namespace radimpl {

struct BatchCore {
  static constexpr int kSlots = 2;  // pinned per-call tables in flight
  cudaStream_t stream = nullptr;    // the caller's stream (may be the legacy NULL stream)
  cudaStream_t work = nullptr;      // internal stream: launches and graph capture
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  bool stream_ok = false;
  int cap = 0;
  JobStatic* d_js = nullptr;
  unsigned long long* d_counter = nullptr;  // counter block (see init)
  size_t counter_bytes = 0;
  JobCall* h_calls[kSlots] = {nullptr, nullptr};
  JobCall* d_calls[kSlots] = {nullptr, nullptr};
  cudaEvent_t slot_done[kSlots] = {nullptr, nullptr};
  cudaGraph_t graph[kSlots] = {nullptr, nullptr};
  cudaGraphExec_t graph_exec[kSlots] = {nullptr, nullptr};
  std::vector<rad_step> sig[kSlots];
  std::vector<JobStatic> h_js;
  std::vector<rad_ctx*> cur_jobs;
  std::vector<long long> cur_gen;
  int cur_variant = -1;
  int slot = 0;

  ~BatchCore();
  rad_status init(int max_jobs, cudaStream_t s);
  void release();
  void invalidate_graphs();
  rad_status run(rad_ctx* const* jobs, const rad_step* steps, int n_jobs, bool use_graphs);
};

}  // namespace radimpl
