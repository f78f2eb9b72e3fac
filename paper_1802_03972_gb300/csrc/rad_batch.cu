// Batched accumulation: one time step of many independent jobs in one
// persistent launch (pre-pass + accumulate), work items ordered largest job
// first, replayed from captured CUDA graphs while the job set is unchanged.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <numeric>
#include <vector>

#include "rad_batch_impl.h"
#include "rad_ctx.h"

using namespace radimpl;

namespace radimpl {

namespace {

bool same_signature(const std::vector<rad_step>& a, const rad_step* b, size_t n) {
  if (a.size() != n) return false;
  for (size_t i = 0; i < n; ++i)
    if (a[i].n != b[i].n || a[i].r != b[i].r || a[i].beta != b[i].beta ||
        a[i].beta_dot != b[i].beta_dot || a[i].w != b[i].w)
      return false;
  return true;
}

}  // namespace

BatchCore::~BatchCore() { release(); }

void BatchCore::release() {
  if (stream_ok) cudaStreamSynchronize(work);
  for (int s = 0; s < kSlots; ++s) {
    if (graph_exec[s]) cudaGraphExecDestroy(graph_exec[s]);
    if (graph[s]) cudaGraphDestroy(graph[s]);
    if (slot_done[s]) cudaEventDestroy(slot_done[s]);
    if (h_calls[s]) cudaFreeHost(h_calls[s]);
    if (d_calls[s]) cudaFree(d_calls[s]);
    graph_exec[s] = nullptr;
    graph[s] = nullptr;
    slot_done[s] = nullptr;
    h_calls[s] = nullptr;
    d_calls[s] = nullptr;
  }
  if (d_js) cudaFree(d_js);
  if (d_counter) cudaFree(d_counter);
  if (ev_in) cudaEventDestroy(ev_in);
  if (ev_out) cudaEventDestroy(ev_out);
  if (work) {
    cudaStreamSynchronize(work);
    cudaStreamDestroy(work);
  }
  d_js = nullptr;
  d_counter = nullptr;
  ev_in = ev_out = nullptr;
  work = nullptr;
  stream_ok = false;
  cudaGetLastError();
}

rad_status BatchCore::init(int max_jobs, cudaStream_t s) {
  stream = s;
  cap = max_jobs;
  // Graphs cannot be captured on the legacy NULL stream, so work runs on an
  // internal stream ordered after / before the caller's stream with events.
  if (cudaStreamCreateWithFlags(&work, cudaStreamNonBlocking) != cudaSuccess) return RAD_ECUDA;
  stream_ok = true;
  if (cudaEventCreateWithFlags(&ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ev_out, cudaEventDisableTiming) != cudaSuccess)
    return RAD_ECUDA;
  if (cudaMalloc(&d_js, sizeof(JobStatic) * cap) != cudaSuccess) return RAD_ENOMEM;
  // Counter block: the two kernels' item counters, the launch's wide flag, then
  // one wide flag (int) per job slot; zeroed before every round.
  counter_bytes = kCounterWords * sizeof(unsigned long long) + sizeof(int) * (size_t)cap;
  if (cudaMalloc(&d_counter, counter_bytes) != cudaSuccess) return RAD_ENOMEM;
  for (int k = 0; k < kSlots; ++k) {
    if (cudaMallocHost(&h_calls[k], sizeof(JobCall) * cap) != cudaSuccess) return RAD_ENOMEM;
    if (cudaMalloc(&d_calls[k], sizeof(JobCall) * cap) != cudaSuccess) return RAD_ENOMEM;
    if (cudaEventCreateWithFlags(&slot_done[k], cudaEventDisableTiming) != cudaSuccess)
      return RAD_ECUDA;
  }
  h_js.resize(cap);
  return RAD_OK;
}

void BatchCore::invalidate_graphs() {
  for (int s = 0; s < kSlots; ++s) {
    if (graph_exec[s]) cudaGraphExecDestroy(graph_exec[s]);
    if (graph[s]) cudaGraphDestroy(graph[s]);
    graph_exec[s] = nullptr;
    graph[s] = nullptr;
    sig[s].clear();
  }
}

// Enqueue one round.  jobs[i] receives steps[i]; n = 0 skips a job.
rad_status BatchCore::run(rad_ctx* const* jobs, const rad_step* steps, int n_jobs, bool use_graphs) {
  if (n_jobs > cap) return RAD_EINVAL;
  // Variant: the jobs' common variant, else the default one.
  int variant = jobs[0]->tile.variant;
  for (int i = 1; i < n_jobs; ++i)
    if (jobs[i]->tile.variant != variant) variant = kDefaultVariant;

  // Per-job chunking, capacities (may reallocate: drain this stream first).
  struct Plan { int job; long long n; int ck, n_chunks; TailPlan tail; long long cost; JobStatic js; };
  std::vector<Plan> plan;
  plan.reserve(n_jobs);
  bool drained = false;
  for (int i = 0; i < n_jobs; ++i) {
    rad_ctx* c = jobs[i];
    if (steps[i].n <= 0) continue;
    JobStatic js = c->h_js;
    if (c->tile.variant != variant)
      fill_tiles(js, variant, default_omega_tile(variant, c->n_omega));
    const int ck = auto_chunk(c, variant, steps[i].n, js.n_tiles);
    const int nch = (int)((steps[i].n + ck - 1) / ck);
    // chunked as the job alone would be (results equal bit for bit)
    const TailPlan tail = tail_plan(variant_tensor_core(variant) && !js.literal, steps[i].n,
                                    js.n_tiles, ck, nch, resident_ctas(variant));
    const long long fine = tail.fine_floats(js.nt * js.wt);
    if (steps[i].n > c->h_js.n_cap || nch > c->h_js.chunk_cap || fine > c->h_js.fine_cap) {
      if (!drained) {
        if (cudaStreamSynchronize(work) != cudaSuccess) return RAD_ECUDA;
        drained = true;
      }
      rad_status s = ensure_capacity(c, steps[i].n, nch, fine);
      if (s != RAD_OK) return s;
      if (cudaStreamSynchronize(c->stream) != cudaSuccess) return RAD_ECUDA;
      js.rec = c->h_js.rec;
      js.n_cap = c->h_js.n_cap;
      js.partials = c->h_js.partials;
      js.chunk_cap = c->h_js.chunk_cap;
      js.partials_f = c->h_js.partials_f;
      js.fine_cap = c->h_js.fine_cap;
      js.perm = c->h_js.perm;
      js.sort_counts = c->h_js.sort_counts;
      js.bucket_base = c->h_js.bucket_base;
      js.gref = c->h_js.gref;
    }
    plan.push_back({i, steps[i].n, ck, nch, tail, (long long)js.n_tiles * nch * (long long)ck, js});
  }
  if (plan.empty()) return RAD_OK;
  // Largest jobs first, so the dynamic scheduler's tail holds small items.
  std::stable_sort(plan.begin(), plan.end(),
                   [](const Plan& a, const Plan& b) { return a.cost > b.cost; });
  // Each job's wide flag is its slot in the batch's counter block.
  int* wide_flags = reinterpret_cast<int*>(d_counter + kCounterWords);
  for (size_t p = 0; p < plan.size(); ++p)
    plan[p].js.wide_flag = plan[p].js.wide_flag ? wide_flags + p : nullptr;

  // Static job table (re-uploaded when the set or any context changed).
  bool js_changed = plan.size() != cur_jobs.size() || variant != cur_variant;
  for (size_t p = 0; p < plan.size() && !js_changed; ++p)
    js_changed = cur_jobs[p] != jobs[plan[p].job] ||
                 cur_gen[p] != jobs[plan[p].job]->generation ||
                 memcmp(&h_js[p], &plan[p].js, sizeof(JobStatic)) != 0;
  if (js_changed) {
    if (cudaStreamSynchronize(work) != cudaSuccess) return RAD_ECUDA;
    cur_jobs.resize(plan.size());
    cur_gen.resize(plan.size());
    for (size_t p = 0; p < plan.size(); ++p) {
      h_js[p] = plan[p].js;
      cur_jobs[p] = jobs[plan[p].job];
      cur_gen[p] = jobs[plan[p].job]->generation;
    }
    cur_variant = variant;
    if (cudaMemcpy(d_js, h_js.data(), sizeof(JobStatic) * plan.size(), cudaMemcpyHostToDevice) !=
        cudaSuccess)
      return RAD_ECUDA;
    invalidate_graphs();
  }

  // Per-call table in the next pinned slot.
  const int s = slot;
  slot = (slot + 1) % kSlots;
  if (cudaEventSynchronize(slot_done[s]) != cudaSuccess) return RAD_ECUDA;
  long long items = 0;
  int blocks = 0, sort_blocks = 0;
  std::vector<rad_step> sorted(plan.size());
  for (size_t p = 0; p < plan.size(); ++p) {
    const rad_step& st = steps[plan[p].job];
    sorted[p] = st;
    JobCall& K = h_calls[s][p];
    memset(&K, 0, sizeof(K));
    K.n = st.n;
    K.r = st.r;
    K.beta = st.beta;
    K.bdot = st.beta_dot;
    K.w = st.w;
    K.t = st.t;
    K.dt = st.dt;
    K.ck = plan[p].ck;
    K.n_chunks = plan[p].n_chunks;
    set_tail(K, plan[p].tail);
    K.item_begin = items;
    K.block_begin = blocks;
    K.sort_block_begin = sort_blocks;
    items += plan[p].tail.items(plan[p].js.n_tiles, plan[p].n_chunks);
    blocks += (int)((st.n + 255) / 256);
    sort_blocks += (int)((st.n + kSortBlock - 1) / kSortBlock);
  }
  LaunchArgs a;
  memset(&a, 0, sizeof(a));
  a.js = d_js;
  a.jc = d_calls[s];
  a.n_jobs = (int)plan.size();
  a.use_inline = 0;
  a.n_items = items;
  a.item_counter = d_counter;
  a.any_wide = reinterpret_cast<int*>(d_counter + 2);
  const int grid = (int)std::min<long long>(items, resident_ctas(variant));
  const size_t call_bytes = sizeof(JobCall) * plan.size();

  auto enqueue = [&](cudaStream_t st) -> cudaError_t {
    cudaError_t e = cudaMemcpyAsync(d_calls[s], h_calls[s], call_bytes, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_counter, 0, counter_bytes, st);
    if (e == cudaSuccess) e = launch_prepass(a, blocks, st);
    if (e == cudaSuccess) e = launch_wide(a, sort_blocks, blocks, st);
    if (e == cudaSuccess) e = launch_accumulate(variant, a, grid, st);
    return e;
  };
  // kernels per round: pre-pass, the wide-call kernels, both accumulate kernels
  const int launches = 1 + kWideLaunches + 2;

  // Order after the caller's stream (its inputs), run on the internal stream.
  cudaError_t e = cudaEventRecord(ev_in, stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(work, ev_in, 0);
  if (e != cudaSuccess) return RAD_ECUDA;
  if (use_graphs && graph_exec[s] && same_signature(sig[s], sorted.data(), sorted.size())) {
    e = cudaGraphLaunch(graph_exec[s], work);
    count_launches(launches);
  } else if (use_graphs) {
    if (graph_exec[s]) cudaGraphExecDestroy(graph_exec[s]);
    if (graph[s]) cudaGraphDestroy(graph[s]);
    graph_exec[s] = nullptr;
    graph[s] = nullptr;
    e = cudaStreamBeginCapture(work, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t e2 = enqueue(work);
      count_launches(-launches);  // captured, not launched
      e = cudaStreamEndCapture(work, &graph[s]);
      if (e2 != cudaSuccess) e = e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&graph_exec[s], graph[s], 0);
    if (e == cudaSuccess) {
      sig[s] = sorted;
      e = cudaGraphLaunch(graph_exec[s], work);
      count_launches(launches);
    }
  } else {
    e = enqueue(work);
  }
  if (e != cudaSuccess) return RAD_ECUDA;
  if (cudaEventRecord(slot_done[s], work) != cudaSuccess) return RAD_ECUDA;
  // The caller's stream continues after this round.
  if (cudaEventRecord(ev_out, work) != cudaSuccess || cudaStreamWaitEvent(stream, ev_out, 0) != cudaSuccess)
    return RAD_ECUDA;
  return RAD_OK;
}

}  // namespace radimpl

struct rad_batch {
  std::vector<rad_ctx*> jobs;
  BatchCore core;
  bool failed = false;
};

extern "C" {

rad_status rad_batch_create(rad_ctx* const* ctxs, int32_t n_jobs, void* stream, rad_batch** out) {
  if (!out) return RAD_EINVAL;
  *out = nullptr;
  if (!ctxs || n_jobs < 1) return RAD_EINVAL;
  for (int i = 0; i < n_jobs; ++i) {
    if (!ctxs[i] || ctxs[i]->prec != RAD_PREC_MIXED || ctxs[i]->failed || ctxs[i]->h_js.literal)
      return RAD_EINVAL;
    if (check_device(ctxs[i]) != RAD_OK) return RAD_EINVAL;  // one device for the whole batch
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == ctxs[i]) return RAD_EINVAL;
  }
  rad_batch* b = new (std::nothrow) rad_batch();
  if (!b) return RAD_ENOMEM;
  b->jobs.assign(ctxs, ctxs + n_jobs);
  rad_status s = b->core.init(n_jobs, (cudaStream_t)stream);
  if (s != RAD_OK) {
    delete b;
    return s;
  }
  *out = b;
  return RAD_OK;
}

rad_status rad_batch_accumulate(rad_batch* b, const rad_step* steps) {
  if (!b || !steps) return RAD_EINVAL;
  if (b->failed) return RAD_ESTATE;
  for (size_t i = 0; i < b->jobs.size(); ++i) {
    const rad_step& st = steps[i];
    if (st.n < 0 || !isfinite(st.t) || !isfinite(st.dt) || !(st.dt > 0.0)) return RAD_EINVAL;
    if (st.n > 0 && (!st.r || !st.beta || !st.beta_dot || !st.w)) return RAD_EINVAL;
    if (b->jobs[i]->failed) return RAD_ESTATE;
    if (check_device(b->jobs[i]) != RAD_OK) return RAD_EINVAL;
  }
  TraceRange trace("rad_batch_accumulate");
  rad_status s = b->core.run(b->jobs.data(), steps, (int)b->jobs.size(), true);
  if (s == RAD_ECUDA) b->failed = true;
  return s;
}

rad_status rad_batch_sync(rad_batch* b) {
  if (!b) return RAD_EINVAL;
  if (b->failed) return RAD_ESTATE;
  if (cudaStreamSynchronize(b->core.work) != cudaSuccess ||
      cudaStreamSynchronize(b->core.stream) != cudaSuccess) {
    b->failed = true;
    return RAD_ECUDA;
  }
  return RAD_OK;
}

void rad_batch_destroy(rad_batch* b) { delete b; }

}  // extern "C"
