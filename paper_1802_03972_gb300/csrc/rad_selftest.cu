// Test-support entry points (include/rad_selftest.h): the accumulate kernel's
// stage 1 and phase arithmetic run on caller-given inputs, through the same
// device functions (rad_stage.cuh), and a bounded wait that nothing completes.
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "rad_ctx.h"
#include "rad_selftest.h"
#include "rad_stage.cuh"

namespace radimpl {
namespace {

using namespace dev;

__global__ void selftest_wait_kernel(unsigned long long limit_ns, int* timed_out,
                                     unsigned long long* waited_ns) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_fence_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned long long t0 = global_ns();
    const bool done = mbar_wait(&bar, 0u, limit_ns);  // nothing arrives on it
    *waited_ns = global_ns() - t0;
    *timed_out = done ? 0 : 1;
  }
}

__global__ void selftest_record_kernel(const float* __restrict__ rec, long long n,
                                       const float* __restrict__ dir_tab, int n_dir, int d,
                                       float tau_fast, float* __restrict__ out) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  float th = 0.f, tl = 0.f, a[4];
  const bool fast = compute_record(rec + k * kRecFields, dir_tab, n_dir, d, tau_fast, th, tl, a);
  float* o = out + 8 * k;
  o[0] = th;
  o[1] = tl;
  o[2] = a[0];
  o[3] = a[1];
  o[4] = a[2];
  o[5] = a[3];
  o[6] = fast ? 1.f : 0.f;
  o[7] = 0.f;
}

// om_tab rows: omega/2pi hi, 2pi hi, 2pi lo (floats); om_turns: omega/2pi (double).
__global__ void selftest_phase_kernel(const float* __restrict__ om_tab,
                                      const double* __restrict__ om_turns, int n_omega,
                                      const float* __restrict__ th, const float* __restrict__ tl,
                                      int n_tau, float* __restrict__ fast, float* __restrict__ wide) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)n_omega * n_tau) return;
  const int i = (int)(idx / n_tau), j = (int)(idx - (long long)i * n_tau);
  const float h = om_tab[i];
  const float wh = om_tab[n_omega + i], wl = om_tab[2 * n_omega + i];
  const float2 p = phase2(make_float2(h, h), make_float2(wh, wh), make_float2(wl, wl),
                          make_float2(th[j], th[j]), make_float2(tl[j], tl[j]));
  fast[idx] = p.x;
  wide[idx] = phase_wide(om_turns[i], th[j], tl[j]);
}

}  // namespace
}  // namespace radimpl

using namespace radimpl;

extern "C" {

rad_status rad_selftest_wait(int64_t limit_ns, int32_t* timed_out, double* waited_s) {
  if (!timed_out || !waited_s) return RAD_EINVAL;
  const unsigned long long lim =
      (unsigned long long)std::min<int64_t>(std::max<int64_t>(limit_ns, 1000000), 2000000000);
  int* d_flag = nullptr;
  unsigned long long* d_ns = nullptr;
  if (cudaMalloc(&d_flag, sizeof(int)) != cudaSuccess) return RAD_ECUDA;
  if (cudaMalloc(&d_ns, sizeof(unsigned long long)) != cudaSuccess) {
    cudaFree(d_flag);
    return RAD_ECUDA;
  }
  selftest_wait_kernel<<<1, 32>>>(lim, d_flag, d_ns);
  count_launches(1);
  int flag = 0;
  unsigned long long ns = 0;
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(&flag, d_flag, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(&ns, d_ns, sizeof(ns), cudaMemcpyDeviceToHost);
  cudaFree(d_flag);
  cudaFree(d_ns);
  if (e != cudaSuccess) return RAD_ECUDA;
  *timed_out = flag;
  *waited_s = 1e-9 * (double)ns;
  return RAD_OK;
}

rad_status rad_selftest_stage1(rad_ctx* c, int64_t n, const double* r, const double* beta,
                               const double* beta_dot, const double* w, double t, double dt,
                               int32_t dir, float* out, float* basis) {
  if (!c || !out || !basis || !r || !beta || !beta_dot || !w) return RAD_EINVAL;
  if (c->failed) return RAD_ESTATE;
  if (check_device(c) != RAD_OK) return RAD_EINVAL;
  if (c->prec != RAD_PREC_MIXED || n < 1 || n > (1 << 20) || dir < 0 || dir >= c->n_dir)
    return RAD_EINVAL;
  rad_status s = ensure_capacity(c, n, 1);
  if (s != RAD_OK) return s;
  LaunchArgs a;
  memset(&a, 0, sizeof(a));
  a.js = c->d_js;
  a.n_jobs = 1;
  a.use_inline = 1;
  JobCall& K = a.inline_call;
  K.n = n;
  K.r = r;
  K.beta = beta;
  K.bdot = beta_dot;
  K.w = w;
  K.t = t;
  K.dt = dt;
  K.ck = (int)std::min<int64_t>(n, 1 << 30);
  K.n_chunks = 1;
  s = cuda_check(c, launch_prepass(a, (int)((n + 255) / 256), c->stream));
  if (s != RAD_OK) return s;
  float* d_out = nullptr;
  s = cuda_check(c, cudaMalloc(&d_out, sizeof(float) * 8 * (size_t)n));
  if (s != RAD_OK) return s;
  const JobStatic& J = c->h_js;
  selftest_record_kernel<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(
      J.rec, n, J.dir_tab, c->n_dir, dir, J.tau_fast, d_out);
  count_launches(1);
  s = cuda_check(c, cudaGetLastError());
  if (s == RAD_OK)
    s = cuda_check(c, cudaMemcpyAsync(out, d_out, sizeof(float) * 8 * (size_t)n,
                                      cudaMemcpyDeviceToHost, c->stream));
  for (int i = 0; s == RAD_OK && i < 6; ++i)
    s = cuda_check(c, cudaMemcpyAsync(basis + i, J.dir_tab + (size_t)(6 + i) * c->n_dir + dir,
                                      sizeof(float), cudaMemcpyDeviceToHost, c->stream));
  if (s == RAD_OK) s = cuda_check(c, cudaStreamSynchronize(c->stream));
  cudaFree(d_out);
  return s;
}

rad_status rad_selftest_phase(rad_ctx* c, int32_t n_tau, const float* th, const float* tl,
                              float* fast, float* wide) {
  if (!c || !th || !tl || !fast || !wide) return RAD_EINVAL;
  if (c->failed) return RAD_ESTATE;
  if (check_device(c) != RAD_OK) return RAD_EINVAL;
  if (c->prec != RAD_PREC_MIXED || n_tau < 1 || n_tau > (1 << 20)) return RAD_EINVAL;
  const size_t m = (size_t)c->n_omega * (size_t)n_tau;
  float *d_th = nullptr, *d_tl = nullptr, *d_f = nullptr, *d_w = nullptr;
  rad_status s = cuda_check(c, cudaMalloc(&d_th, sizeof(float) * n_tau));
  if (s == RAD_OK) s = cuda_check(c, cudaMalloc(&d_tl, sizeof(float) * n_tau));
  if (s == RAD_OK) s = cuda_check(c, cudaMalloc(&d_f, sizeof(float) * m));
  if (s == RAD_OK) s = cuda_check(c, cudaMalloc(&d_w, sizeof(float) * m));
  if (s == RAD_OK)
    s = cuda_check(c, cudaMemcpyAsync(d_th, th, sizeof(float) * n_tau, cudaMemcpyHostToDevice, c->stream));
  if (s == RAD_OK)
    s = cuda_check(c, cudaMemcpyAsync(d_tl, tl, sizeof(float) * n_tau, cudaMemcpyHostToDevice, c->stream));
  if (s == RAD_OK) {
    selftest_phase_kernel<<<(unsigned)((m + 255) / 256), 256, 0, c->stream>>>(
        c->h_js.om_tab, c->h_js.om_turns, c->n_omega, d_th, d_tl, n_tau, d_f, d_w);
    count_launches(1);
    s = cuda_check(c, cudaGetLastError());
  }
  if (s == RAD_OK)
    s = cuda_check(c, cudaMemcpyAsync(fast, d_f, sizeof(float) * m, cudaMemcpyDeviceToHost, c->stream));
  if (s == RAD_OK)
    s = cuda_check(c, cudaMemcpyAsync(wide, d_w, sizeof(float) * m, cudaMemcpyDeviceToHost, c->stream));
  if (s == RAD_OK) s = cuda_check(c, cudaStreamSynchronize(c->stream));
  cudaFree(d_th);
  cudaFree(d_tl);
  cudaFree(d_f);
  cudaFree(d_w);
  return s;
}

}  // extern "C"
