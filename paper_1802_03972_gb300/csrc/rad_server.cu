// Continuous-batching request loop for radiation-diagnostic jobs.
//
// Jobs arrive at any time.  A scheduler thread admits waiting jobs in arrival
// order while a slot is free and their device footprint fits the budget,
// keeps each admitted job's amplitudes resident on the device, and in every
// round takes the oldest pending step of admitted jobs and runs them all in one
// batched persistent launch (the same engine as rad_batch), so a job that
// arrives while others run joins the next round.  Which jobs a round takes is
// the policy (rad_server_set_policy): every job with a ready step, or jobs in
// arrival order, or in order of least work done so far, until the round holds
// a given number of amplitude updates.  Steps are copied into
// per-job device staging slots on a separate copy stream (overlapping the
// compute stream); a round waits only on the copies of the steps it uses.
// After a finished job's last step its spectrum is read out and its device
// memory is released for the next job.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "rad_batch_impl.h"
#include "rad_ctx.h"

using namespace radimpl;

namespace {

using Clock = std::chrono::steady_clock;

struct Slot {
  double* d = nullptr;       // [10 * max_particles]: r, beta, beta_dot, w
  cudaEvent_t ready = nullptr;
  bool busy = false;         // holds a queued step
};

struct QueuedStep {
  int slot = -1;                 // device slot, or -1 while held on the host
  std::vector<double> host;      // host copy while the job waits for admission
  long long n = 0;
  double t = 0, dt = 0;
};

enum class JobState { Waiting, Active, Done, Failed };

struct Job {
  rad_job_id id = 0;
  std::vector<double> omega, dirs;
  rad_ff ff{};
  long long max_particles = 0;
  int max_queued = 1;
  size_t footprint = 0;
  JobState state = JobState::Waiting;
  rad_ctx* ctx = nullptr;
  std::vector<Slot> slots;
  std::deque<QueuedStep> queue;
  bool finished = false;
  bool in_round = false;
  long long served = 0;  // amplitude updates done
  rad_status err = RAD_OK;
  std::vector<double> coh, inc, tot;
  Clock::time_point t_submit, t_ready;
};

size_t estimate_footprint(const rad_job_desc& d) {
  const size_t nb = (size_t)d.n_omega * d.n_dir;
  // Per-chunk partial sums (32 B per bin and chunk).  Automatic chunking aims
  // at kItemsPerCta work items per resident block with the fine-chunked tail
  // and kItemsPerCtaUniform (the larger) without it; with B bins per tile,
  // chunks x bins <= kItemsPerCtaUniform x resident blocks x B + bins.  There
  // are also never more chunks than 256-particle groups.
  const Variant v = variant_info(kDefaultVariant);
  const size_t bins_per_tile = (size_t)v.threads * v.w * v.passes;
  const size_t by_particles = nb * (size_t)((d.max_particles + kChunkAlign - 1) / kChunkAlign);
  const size_t by_items = (size_t)kItemsPerCtaUniform * resident_ctas(kDefaultVariant) * bins_per_tile + nb;
  const size_t partials = 32 * std::min(by_particles, by_items);
  // The fine-chunked last tiles' partial sums (TailPlan), 32 B per tile bin
  // and (tile, chunk).  Level 0: L0 <= grid / n_c + 2 tiles of n_0 <= 4 n_c
  // chunks, L0 n_0 <= 4 grid + 8 n_c; level 1: L1 <= grid / n_1 + 2 tiles of
  // n_1 <= 4 n_0 <= 16 n_c chunks, L1 n_1 <= grid + 32 n_c.  Together at most
  // 6 grid + 40 n_c (tile, chunk) pairs, with a few to spare.
  const size_t grid = (size_t)resident_ctas(kDefaultVariant);
  const size_t tiles_per_nb = std::max<size_t>(1, nb / bins_per_tile);
  const size_t fine = 32 * bins_per_tile * (6 * grid + 12) + 40 * partials / tiles_per_nb;
  // Records (80 B per particle), the sort buffers of wide calls (13 B) and the
  // queued steps' staging slots (80 B each).
  return nb * (64 + 24) + partials + fine +
         (size_t)d.max_particles * (80 + 13 + 80 * (size_t)d.max_queued) +
         (size_t)d.n_omega * 48 + (size_t)d.n_dir * 72 + (1 << 16) + 4 * (size_t)kSortBuckets;
}

}  // namespace

struct rad_server {
  int device = -1;  // the CUDA device current at rad_server_create; the worker runs on it
  size_t budget = 0;
  int max_slots = 1;
  cudaStream_t compute = nullptr;
  cudaStream_t copy = nullptr;
  bool own_compute = false;
  BatchCore core;
  std::mutex mu;
  std::condition_variable cv_sched, cv_done;
  std::thread worker;
  bool stop = false;
  rad_job_id next_id = 1;
  std::map<rad_job_id, std::unique_ptr<Job>> jobs;
  std::deque<rad_job_id> waiting;
  size_t footprint = 0, peak_footprint = 0;
  // The oldest job with bounded backfill, rounds of at least ~1 ms of GB300
  // work: measured on the job mix at 50-500 steps per job, it keeps the tail
  // latency of one-job-at-a-time FIFO service and lowers its median.
  int policy = RAD_SERVE_OLDEST_BACKFILL;
  long long round_updates = 2000000000LL;
  rad_server_stats st{};
  rad_status fatal = RAD_OK;

  void loop();
  rad_status admit_locked(Job& j);
  void release_job_locked(Job& j);
};

rad_status rad_server::admit_locked(Job& j) {
  rad_ctx* c = nullptr;
  rad_status s = rad_create(j.omega.data(), (int32_t)j.omega.size(), j.dirs.data(),
                            (int32_t)(j.dirs.size() / 3), j.ff, RAD_PREC_MIXED, compute, &c);
  if (s != RAD_OK) return s;
  j.ctx = c;
  j.slots.resize(j.max_queued);
  for (auto& sl : j.slots) {
    if (cudaMalloc(&sl.d, sizeof(double) * 10 * (size_t)j.max_particles) != cudaSuccess ||
        cudaEventCreateWithFlags(&sl.ready, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      return RAD_ENOMEM;
    }
  }
  // Steps fed while waiting move from host memory to device slots.
  int k = 0;
  for (auto& q : j.queue) {
    Slot& sl = j.slots[k];
    if (cudaMemcpyAsync(sl.d, q.host.data(), sizeof(double) * q.host.size(),
                        cudaMemcpyHostToDevice, copy) != cudaSuccess ||
        cudaEventRecord(sl.ready, copy) != cudaSuccess)
      return RAD_ECUDA;
    sl.busy = true;
    q.slot = k++;
  }
  if (cudaStreamSynchronize(copy) != cudaSuccess) return RAD_ECUDA;
  for (auto& q : j.queue) {
    q.host.clear();
    q.host.shrink_to_fit();
  }
  j.state = JobState::Active;
  return RAD_OK;
}

void rad_server::release_job_locked(Job& j) {
  for (auto& sl : j.slots) {
    if (sl.d) cudaFree(sl.d);
    if (sl.ready) cudaEventDestroy(sl.ready);
    sl.d = nullptr;
    sl.ready = nullptr;
  }
  j.slots.clear();
  if (j.ctx) rad_destroy(j.ctx);
  j.ctx = nullptr;
  footprint -= std::min(footprint, j.footprint);
  st.active = std::max(0, st.active - 1);
}

void rad_server::loop() {
  std::unique_lock<std::mutex> lk(mu);
  while (!stop) {
    // 1. admission, in arrival order, while slots and memory allow
    while (!waiting.empty()) {
      Job& j = *jobs[waiting.front()];
      if (st.active >= max_slots || footprint + j.footprint > budget) break;
      waiting.pop_front();
      footprint += j.footprint;
      peak_footprint = std::max(peak_footprint, footprint);
      st.active++;
      st.waiting = (int32_t)waiting.size();
      st.admitted++;
      rad_log(2, "server: job %lld admitted (%zu bytes, %d active)", (long long)j.id, j.footprint,
              st.active);
      const rad_status s = admit_locked(j);
      if (s != RAD_OK) {
        j.err = s;
        j.state = JobState::Failed;
        release_job_locked(j);
        cv_done.notify_all();
      }
    }
    // 2. one round: the oldest ready step of the jobs the policy picks
    std::vector<Job*> ready;
    for (auto& kv : jobs) {  // arrival order
      Job& j = *kv.second;
      if (j.state != JobState::Active || j.queue.empty() || j.queue.front().slot < 0) continue;
      ready.push_back(&j);
    }
    if (policy == RAD_SERVE_LEAST_SERVED)
      std::stable_sort(ready.begin(), ready.end(),
                       [](const Job* a, const Job* b) { return a->served < b->served; });
    // Oldest job with bounded backfill: the oldest ready job always gets its
    // step, and other jobs (least served first) join only while the round's
    // work stays within max(round_updates, 17/16 of the head's step).  The head
    // of the queue then runs at >= 16/17 of its own pace, as under FIFO, which
    // keeps the tail latency of a FIFO queue, while small jobs progress in the
    // margin instead of waiting behind large ones.
    const bool backfill = policy == RAD_SERVE_OLDEST_BACKFILL;
    long long budget = round_updates;
    if (backfill && !ready.empty()) {
      std::stable_sort(ready.begin() + 1, ready.end(),
                       [](const Job* a, const Job* b) { return a->served < b->served; });
      const long long head = ready[0]->queue.front().n * (long long)ready[0]->ctx->n_bins;
      budget = std::max(round_updates, head + head / 16);
    }
    if (policy == RAD_SERVE_LEAST_SERVED_AGED) {
      // Attained service minus a credit for the time since submission, at one
      // round's updates per 12 ms (about the GPU's rate): a job that has waited
      // t seconds competes like one that has had that much less work.
      const Clock::time_point now = Clock::now();
      const double credit = (double)round_updates / 0.012;
      std::vector<std::pair<double, Job*>> keyed;
      keyed.reserve(ready.size());
      for (Job* jp : ready)
        keyed.emplace_back((double)jp->served -
                               credit * std::chrono::duration<double>(now - jp->t_submit).count(),
                           jp);
      std::stable_sort(keyed.begin(), keyed.end(),
                       [](const auto& a, const auto& b) { return a.first < b.first; });
      for (size_t i = 0; i < keyed.size(); ++i) ready[i] = keyed[i].second;
    }
    std::vector<rad_ctx*> ctxs;
    std::vector<rad_step> steps;
    std::vector<Job*> in_round;
    long long round_work = 0;
    for (Job* jp : ready) {
      Job& j = *jp;
      QueuedStep& q = j.queue.front();
      const long long work = q.n * (long long)j.ctx->n_bins;
      if (backfill) {
        if (!in_round.empty() && round_work + work > budget) continue;
      } else if (policy != RAD_SERVE_ALL && !in_round.empty() && round_work >= round_updates) {
        break;
      }
      round_work += work;
      Slot& sl = j.slots[q.slot];
      const long long n = q.n;
      rad_step s;
      s.n = n;
      s.r = sl.d;
      s.beta = sl.d + 3 * n;
      s.beta_dot = sl.d + 6 * n;
      s.w = sl.d + 9 * n;
      s.t = q.t;
      s.dt = q.dt;
      cudaStreamWaitEvent(compute, sl.ready, 0);
      ctxs.push_back(j.ctx);
      steps.push_back(s);
      in_round.push_back(&j);
      j.in_round = true;
    }
    // 3. finished jobs with nothing queued: read out and release
    std::vector<Job*> to_read;
    for (auto& kv : jobs) {
      Job& j = *kv.second;
      if (j.state == JobState::Active && j.finished && j.queue.empty() && !j.in_round)
        to_read.push_back(&j);
    }
    if (ctxs.empty() && to_read.empty()) {
      cv_sched.wait_for(lk, std::chrono::milliseconds(20));
      continue;
    }
    lk.unlock();
    rad_status rs = RAD_OK;
    if (!ctxs.empty()) {
      TraceRange trace("rad_server round");
      rs = core.run(ctxs.data(), steps.data(), (int)ctxs.size(), false);
      if (rs == RAD_OK && cudaStreamSynchronize(compute) != cudaSuccess) rs = RAD_ECUDA;
    }
    for (Job* j : to_read) {
      const size_t nb = (size_t)j->ctx->n_bins;
      j->coh.resize(nb);
      j->inc.resize(nb);
      j->tot.resize(nb);
      j->err = rad_spectrum(j->ctx, j->coh.data(), j->inc.data(), j->tot.data());
    }
    lk.lock();
    if (!ctxs.empty()) {
      st.rounds++;
      for (size_t i = 0; i < in_round.size(); ++i) {
        Job& j = *in_round[i];
        j.in_round = false;
        QueuedStep& q = j.queue.front();
        j.slots[q.slot].busy = false;
        j.queue.pop_front();
        if (rs != RAD_OK) {
          j.err = rs;
          j.state = JobState::Failed;
        } else {
          st.updates += steps[i].n * (long long)j.ctx->n_bins;
          j.served += steps[i].n * (long long)j.ctx->n_bins;
        }
      }
      if (rs == RAD_ECUDA) fatal = RAD_ECUDA;
    }
    for (Job* j : to_read) {
      j->t_ready = Clock::now();
      j->state = (j->err == RAD_OK || j->err == RAD_EDATA) ? JobState::Done : JobState::Failed;
      st.completed++;
      rad_log(2, "server: job %lld %s after %.3f s", (long long)j->id,
              j->state == JobState::Done ? "done" : "failed",
              std::chrono::duration<double>(j->t_ready - j->t_submit).count());
      release_job_locked(*j);
    }
    cv_done.notify_all();
    cv_sched.notify_all();  // feeders waiting on full queues
  }
}

extern "C" {

rad_status rad_server_create(size_t hbm_budget, int32_t max_slots, void* stream, rad_server** out) {
  if (!out) return RAD_EINVAL;
  *out = nullptr;
  if (hbm_budget == 0 || max_slots < 1) return RAD_EINVAL;
  rad_server* s = new (std::nothrow) rad_server();
  if (!s) return RAD_ENOMEM;
  s->device = current_device();
  s->budget = hbm_budget;
  s->max_slots = max_slots;
  s->compute = (cudaStream_t)stream;
  if (!s->compute) {
    if (cudaStreamCreateWithFlags(&s->compute, cudaStreamNonBlocking) != cudaSuccess) {
      delete s;
      return RAD_ECUDA;
    }
    s->own_compute = true;
  }
  if (cudaStreamCreateWithFlags(&s->copy, cudaStreamNonBlocking) != cudaSuccess) {
    if (s->own_compute) cudaStreamDestroy(s->compute);
    delete s;
    return RAD_ECUDA;
  }
  rad_status st = s->core.init(max_slots, s->compute);
  if (st != RAD_OK) {
    s->core.release();
    cudaStreamDestroy(s->copy);
    if (s->own_compute) cudaStreamDestroy(s->compute);
    delete s;
    return st;
  }
  s->worker = std::thread([s] {
    if (s->device >= 0) cudaSetDevice(s->device);  // a new thread starts on device 0
    s->loop();
  });
  *out = s;
  return RAD_OK;
}

rad_status rad_server_set_policy(rad_server* s, int32_t policy, int64_t round_updates) {
  if (!s || policy < RAD_SERVE_ALL || policy > RAD_SERVE_OLDEST_BACKFILL) return RAD_EINVAL;
  if (policy != RAD_SERVE_ALL && round_updates < 1) return RAD_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  s->policy = policy;
  s->round_updates = round_updates;
  s->cv_sched.notify_all();
  return RAD_OK;
}

rad_status rad_job_submit(rad_server* s, const rad_job_desc* d, rad_job_id* id) {
  if (!s || !d || !id || !d->omega || !d->dirs) return RAD_EINVAL;
  if (d->n_omega < 1 || d->n_dir < 1 || d->max_particles < 1 || d->max_queued < 1)
    return RAD_EINVAL;
  if ((long long)d->n_omega * d->n_dir > 0x7fffffffLL) return RAD_EINVAL;
  if (d->ff.flags & RAD_FF_LITERAL) return RAD_EINVAL;  // literal contexts run on their own
  auto j = std::make_unique<Job>();
  j->omega.assign(d->omega, d->omega + d->n_omega);
  j->dirs.assign(d->dirs, d->dirs + 3 * (size_t)d->n_dir);
  j->ff = d->ff;
  j->max_particles = d->max_particles;
  j->max_queued = d->max_queued;
  j->footprint = estimate_footprint(*d);
  if (j->footprint > s->budget) return RAD_EINVAL;
  j->t_submit = Clock::now();
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->fatal != RAD_OK) return RAD_ESTATE;
  j->id = s->next_id++;
  *id = j->id;
  s->waiting.push_back(j->id);
  s->st.submitted++;
  s->st.waiting = (int32_t)s->waiting.size();
  s->jobs[j->id] = std::move(j);
  s->cv_sched.notify_all();
  return RAD_OK;
}

rad_status rad_job_feed(rad_server* s, rad_job_id id, const rad_step* step) {
  if (!s || !step) return RAD_EINVAL;
  if (current_device() != s->device) return RAD_EINVAL;  // the server's copies run on its device
  if (step->n < 0 || !isfinite(step->t) || !isfinite(step->dt) || !(step->dt > 0.0))
    return RAD_EINVAL;
  if (step->n > 0 && (!step->r || !step->beta || !step->beta_dot || !step->w)) return RAD_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->jobs.find(id);
  if (it == s->jobs.end()) return RAD_EINVAL;
  Job& j = *it->second;
  if (j.finished || j.state == JobState::Done) return RAD_ESTATE;
  if (j.state == JobState::Failed) return j.err == RAD_OK ? RAD_ESTATE : j.err;
  if (step->n == 0) return RAD_OK;
  if (step->n > j.max_particles) return RAD_EINVAL;
  if ((int)j.queue.size() >= j.max_queued) return RAD_EBUSY;
  const long long n = step->n;
  const double* src[4] = {step->r, step->beta, step->beta_dot, step->w};
  const size_t cnt[4] = {(size_t)3 * n, (size_t)3 * n, (size_t)3 * n, (size_t)n};
  QueuedStep q;
  q.n = n;
  q.t = step->t;
  q.dt = step->dt;
  if (j.state == JobState::Waiting) {
    q.host.resize((size_t)10 * n);
    size_t off = 0;
    for (int i = 0; i < 4; ++i) {
      if (cudaMemcpy(q.host.data() + off, src[i], cnt[i] * sizeof(double), cudaMemcpyDefault) !=
          cudaSuccess)
        return RAD_ECUDA;
      off += cnt[i];
    }
  } else {
    int k = 0;
    while (k < (int)j.slots.size() && j.slots[k].busy) ++k;
    if (k == (int)j.slots.size()) return RAD_EBUSY;
    // Reserve the slot, then copy without holding the lock, so the scheduler
    // keeps forming rounds meanwhile.  The job cannot be released while this
    // step is outstanding: it is not finished (checked above), and callers use
    // a server from one thread at a time.
    Slot& sl = j.slots[k];
    sl.busy = true;
    double* dst = sl.d;
    cudaEvent_t ready = sl.ready;
    lk.unlock();
    cudaError_t e = cudaSuccess;
    size_t off = 0;
    for (int i = 0; i < 4 && e == cudaSuccess; ++i) {
      e = cudaMemcpyAsync(dst + off, src[i], cnt[i] * sizeof(double), cudaMemcpyDefault, s->copy);
      off += cnt[i];
    }
    if (e == cudaSuccess) e = cudaEventRecord(ready, s->copy);
    // The caller may reuse its buffers on return, host or device.
    if (e == cudaSuccess) e = cudaEventSynchronize(ready);
    lk.lock();
    if (e != cudaSuccess || j.state != JobState::Active) {
      sl.busy = false;
      if (e != cudaSuccess) return RAD_ECUDA;
      return j.err == RAD_OK ? RAD_ESTATE : j.err;
    }
    q.slot = k;
  }
  j.queue.push_back(std::move(q));
  s->cv_sched.notify_all();
  return RAD_OK;
}

rad_status rad_job_finish(rad_server* s, rad_job_id id) {
  if (!s) return RAD_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->jobs.find(id);
  if (it == s->jobs.end()) return RAD_EINVAL;
  it->second->finished = true;
  s->cv_sched.notify_all();
  return RAD_OK;
}

rad_status rad_job_poll(rad_server* s, rad_job_id id, int32_t* done) {
  if (!s || !done) return RAD_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->jobs.find(id);
  if (it == s->jobs.end()) return RAD_EINVAL;
  const JobState js = it->second->state;
  *done = (js == JobState::Done || js == JobState::Failed) ? 1 : 0;
  return RAD_OK;
}

rad_status rad_job_result(rad_server* s, rad_job_id id, double timeout_s, double* coh,
                          double* inc, double* tot, double* latency_s) {
  if (!s) return RAD_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->jobs.find(id);
  if (it == s->jobs.end()) return RAD_EINVAL;
  Job& j = *it->second;
  auto ready = [&] { return j.state == JobState::Done || j.state == JobState::Failed; };
  if (timeout_s < 0) {
    s->cv_done.wait(lk, ready);
  } else if (!s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), ready)) {
    return RAD_ETIMEOUT;
  }
  rad_status r = j.state == JobState::Done ? j.err : (j.err == RAD_OK ? RAD_ESTATE : j.err);
  if (j.state == JobState::Done) {
    const size_t nb = j.coh.size();
    if (coh) memcpy(coh, j.coh.data(), nb * sizeof(double));
    if (inc) memcpy(inc, j.inc.data(), nb * sizeof(double));
    if (tot) memcpy(tot, j.tot.data(), nb * sizeof(double));
  }
  if (latency_s)
    *latency_s = std::chrono::duration<double>(j.t_ready - j.t_submit).count();
  s->jobs.erase(it);
  return r;
}

rad_status rad_server_stats_get(rad_server* s, rad_server_stats* out) {
  if (!s || !out) return RAD_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->st;
  out->footprint_bytes = (int64_t)s->footprint;
  out->peak_footprint_bytes = (int64_t)s->peak_footprint;
  out->waiting = (int32_t)s->waiting.size();
  return RAD_OK;
}

void rad_server_destroy(rad_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->cv_sched.notify_all();
  }
  if (s->worker.joinable()) s->worker.join();
  cudaStreamSynchronize(s->compute);
  cudaStreamSynchronize(s->copy);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    for (auto& kv : s->jobs) {
      Job& j = *kv.second;
      if (j.state == JobState::Active) s->release_job_locked(j);
    }
    s->jobs.clear();
  }
  s->core.release();
  cudaStreamDestroy(s->copy);
  if (s->own_compute) cudaStreamDestroy(s->compute);
  delete s;
}

}  // extern "C"
