// Device helpers shared by the radiation kernels: constants, MUFU sin/cos,
// mbarrier + TMA bulk copies with bounded waits, job lookup, float-float split.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "rad_impl.h"

namespace radimpl {
namespace dev {

// Debug builds (compiled with RAD_DEBUG_BOUNDS) check the global-memory
// indices that depend on host-side sizing (record capacity, partial-sum slots,
// bins): a failed check sets ST_BOUNDS in the job's status word and the access
// is skipped.  Release builds compile the checks away.
#ifdef RAD_DEBUG_BOUNDS
__device__ __forceinline__ bool bounds_ok(bool cond, int* status) {
  if (!cond) atomicOr(status, ST_BOUNDS);
  return cond;
}
#else
__device__ __forceinline__ bool bounds_ok(bool, int*) { return true; }
#endif

constexpr double kC = 299792458.0;
constexpr double kInvC = 1.0 / 299792458.0;
constexpr unsigned long long kWaitLimitNs = 1000000000ULL;  // 1 s bound on any wait

__device__ __forceinline__ float sin_approx(float x) {
  float y;
  asm("sin.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float cos_approx(float x) {
  float y;
  asm("cos.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Waits for the given phase parity of the barrier; gives up after limit_ns.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t phase,
                                          unsigned long long limit_ns = kWaitLimitNs) {
  const uint32_t a = smem_addr(bar);
  const unsigned long long t0 = global_ns();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done) : "r"(a), "r"(phase) : "memory");
    if (done) return true;
    if (global_ns() - t0 > limit_ns) return false;
  }
}
// One elected thread: bulk copy of `bytes` (multiple of 16, both addresses
// 16-byte aligned) from global to shared memory, completing on `bar`.
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, uint32_t bytes,
                                            uint64_t* bar) {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// Job of a global work item (jobs ordered by item_begin).
__device__ __forceinline__ int find_job(const LaunchArgs& a, long long item) {
  if (a.n_jobs == 1) return 0;
  int lo = 0, hi = a.n_jobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (a.jc[mid].item_begin <= item) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Job of a pre-pass block (jobs ordered by block_begin).
__device__ __forceinline__ int find_job_block(const LaunchArgs& a, int block) {
  if (a.n_jobs == 1) return 0;
  int lo = 0, hi = a.n_jobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (a.jc[mid].block_begin <= block) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Split a double into a float-float pair hi + lo.
__device__ __forceinline__ void split_ff(double x, float& hi, float& lo) {
  hi = __double2float_rn(x);
  lo = __double2float_rn(x - (double)hi);
}

}  // namespace dev
}  // namespace radimpl
