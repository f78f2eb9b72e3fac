// Host-side definition of a radiation context (opaque in the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "rad.h"
#include "rad_impl.h"

struct rad_ctx {
  int n_omega = 0, n_dir = 0, n_bins = 0;
  rad_ff ff{};
  int prec = RAD_PREC_MIXED;
  cudaStream_t stream = nullptr;
  rad_tile tile{};
  // device buffers
  double* d_omega = nullptr;
  double* d_om_turns = nullptr;
  float* d_om_tab = nullptr;
  double* d_dirs = nullptr;
  float* d_dir_tab = nullptr;
  double* d_ref = nullptr;
  int* d_status = nullptr;
  unsigned long long* d_counter = nullptr;
  radimpl::JobStatic* d_js = nullptr;
  double* d_spec = nullptr;      // [3][n_bins] readout staging for host outputs
  float* d_state = nullptr;      // MIXED: [16][n_bins]
  double* d_state64 = nullptr;   // FP64:  [12][n_bins]
  // in-situ coupling (rad_push_step): three step slots of r, beta, w and beta_dot
  double* d_push = nullptr;      // [3][7 n_push] doubles: r (3n), beta (3n), w (n) per slot
  double* d_push_bdot = nullptr; // [3 n_push]
  long long n_push = 0;          // particle count of the held steps (0: none)
  int push_held = 0;             // steps held (0, 1, 2)
  int push_slot[2] = {0, 1};     // slots of the older / newer held step
  double push_t[3] = {0, 0, 0}, push_dt[3] = {0, 0, 0};
  float* d_state_p = nullptr;    // literal mode: [8][n_bins]
  float* d_f2 = nullptr;         // literal mode: [n_omega] f(omega)^2
  unsigned* d_tile_cnt = nullptr;
  int tile_cnt_cap = 0;
  double* d_stage = nullptr;     // staging for host particle arrays
  size_t stage_cap = 0;
  radimpl::JobStatic h_js{};     // host mirror of d_js
  // kernel timing (rad_profile_*): event triples around pre-pass / accumulate
  bool prof_on = false;
  std::vector<cudaEvent_t> prof_ev;  // 3 per timed call
  size_t prof_used = 0;
  unsigned long long* d_prof_clk = nullptr;  // [2] cycles, ns of the accumulate CTAs
  long long generation = 0;      // bumped whenever d_js changes
  uint64_t grid_hash = 0;        // FNV-1a of the frequencies and unit directions
  int device = -1;               // the CUDA device current at rad_create
  rad_status last_err = RAD_OK;
  bool failed = false;
};

namespace radimpl {

// A named NVTX range for the enclosing scope (host side; shows the library's
// calls on a profiler timeline, a no-op when no tool is attached).
struct TraceRange {
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};

rad_status fail(rad_ctx* c, rad_status s);
// RAD_OK when the context's device is the calling thread's current device;
// otherwise RAD_EINVAL (its memory, stream and kernels belong to that device).
rad_status check_device(rad_ctx* c);
rad_status cuda_check(rad_ctx* c, cudaError_t e);
int default_omega_tile(int variant, int n_omega);
bool valid_omega_tile(int variant, int wt);
void fill_tiles(JobStatic& js, int variant, int wt);
int resident_ctas(int variant);
// fine_tail: the job's last tiles are fine-chunked (TailPlan), which allows longer items.
int auto_chunk_for(int variant, long long n, int n_tiles, bool fine_tail);
int auto_chunk(const rad_ctx* c, int variant, long long n, int n_tiles);
// Capacity for n particles, n_chunks coarse chunks and fine_floats floats of
// fine-tile partial sums (TailPlan::fine_floats).
rad_status ensure_capacity(rad_ctx* c, long long n, int n_chunks, long long fine_floats = 0);
rad_status enqueue_accumulate(rad_ctx* c, long long n, const double* r, const double* beta,
                              const double* bdot, const double* w, double t, double dt);
rad_status upload_static(rad_ctx* c);

}  // namespace radimpl
