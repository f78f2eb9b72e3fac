// In-situ coupling to a particle pusher: steps arrive with positions and
// velocities only; beta_dot comes from finite differences of consecutive
// steps held on the device (central in the interior, one-sided at the ends),
// and each step is then accumulated by the usual path (rad_accumulate).
#include <cuda_runtime.h>
#include <math.h>

#include "rad.h"
#include "rad_ctx.h"
#include "rad_impl.h"

using namespace radimpl;

namespace {

// out = (b_new - b_old) * inv_span over 3 n values.
__global__ void fd_kernel(long long n3, const double* __restrict__ b_old,
                          const double* __restrict__ b_new, double inv_span,
                          double* __restrict__ out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n3) return;
  out[i] = (b_new[i] - b_old[i]) * inv_span;
}

double* slot_r(rad_ctx* c, int s) { return c->d_push + (size_t)s * 7 * c->n_push; }
double* slot_beta(rad_ctx* c, int s) { return slot_r(c, s) + 3 * c->n_push; }
double* slot_w(rad_ctx* c, int s) { return slot_r(c, s) + 6 * c->n_push; }

// Accumulates held step `s` with beta_dot = (beta[b] - beta[a]) / (t[b] - t[a]).
rad_status accumulate_fd(rad_ctx* c, int s, int a, int b) {
  const double span = c->push_t[b] - c->push_t[a];
  if (!(span != 0.0) || !isfinite(span)) return fail(c, RAD_EINVAL);
  const long long n3 = 3 * c->n_push;
  fd_kernel<<<(unsigned)((n3 + 255) / 256), 256, 0, c->stream>>>(
      n3, slot_beta(c, a), slot_beta(c, b), 1.0 / span, c->d_push_bdot);
  count_launches(1);
  rad_status st = cuda_check(c, cudaGetLastError());
  if (st != RAD_OK) return st;
  return enqueue_accumulate(c, c->n_push, slot_r(c, s), slot_beta(c, s), c->d_push_bdot,
                            slot_w(c, s), c->push_t[s], c->push_dt[s]);
}

}  // namespace

extern "C" {

rad_status rad_push_step(rad_ctx* c, int64_t n, const double* r, const double* beta,
                         const double* w, double t, double dt) {
  if (!c) return RAD_EINVAL;
  if (c->failed) return RAD_ESTATE;
  if (check_device(c) != RAD_OK) return RAD_EINVAL;
  if (n < 1 || !r || !beta || !w || !isfinite(t) || !isfinite(dt) || !(dt > 0.0))
    return fail(c, RAD_EINVAL);
  if (c->push_held > 0 && n != c->n_push) return fail(c, RAD_EINVAL);
  if (c->push_held == 0 && n != c->n_push) {
    cudaStreamSynchronize(c->stream);
    if (c->d_push) cudaFree(c->d_push);
    if (c->d_push_bdot) cudaFree(c->d_push_bdot);
    c->d_push = c->d_push_bdot = nullptr;
    c->n_push = 0;
    if (cudaMalloc(&c->d_push, sizeof(double) * 21 * (size_t)n) != cudaSuccess ||
        cudaMalloc(&c->d_push_bdot, sizeof(double) * 3 * (size_t)n) != cudaSuccess) {
      cudaGetLastError();
      if (c->d_push) cudaFree(c->d_push);
      c->d_push = nullptr;
      return fail(c, RAD_ENOMEM);
    }
    c->n_push = n;
  }
  // The free slot of three: none held -> 0; one held -> the next; two -> the third.
  int fr;
  if (c->push_held == 0) fr = 0;
  else if (c->push_held == 1) fr = (c->push_slot[1] + 1) % 3;
  else fr = 3 - c->push_slot[0] - c->push_slot[1];
  const double* src[3] = {r, beta, w};
  double* dst[3] = {slot_r(c, fr), slot_beta(c, fr), slot_w(c, fr)};
  const size_t cnt[3] = {(size_t)3 * n, (size_t)3 * n, (size_t)n};
  for (int i = 0; i < 3; ++i) {
    rad_status s = cuda_check(c, cudaMemcpyAsync(dst[i], src[i], cnt[i] * sizeof(double),
                                                 cudaMemcpyDefault, c->stream));
    if (s != RAD_OK) return s;
  }
  c->push_t[fr] = t;
  c->push_dt[fr] = dt;
  rad_status s = RAD_OK;
  if (c->push_held == 0) {
    c->push_slot[1] = fr;
    c->push_held = 1;
  } else if (c->push_held == 1) {
    // first step: forward difference
    const int j = c->push_slot[1];
    s = accumulate_fd(c, j, j, fr);
    c->push_slot[0] = j;
    c->push_slot[1] = fr;
    c->push_held = 2;
  } else {
    // interior step: central difference over its neighbours
    const int older = c->push_slot[0], j = c->push_slot[1];
    s = accumulate_fd(c, j, older, fr);
    c->push_slot[0] = j;
    c->push_slot[1] = fr;
  }
  return s;
}

rad_status rad_push_flush(rad_ctx* c) {
  if (!c) return RAD_EINVAL;
  if (c->failed) return RAD_ESTATE;
  if (check_device(c) != RAD_OK) return RAD_EINVAL;
  rad_status s = RAD_OK;
  if (c->push_held == 2) {
    // last step: backward difference
    s = accumulate_fd(c, c->push_slot[1], c->push_slot[0], c->push_slot[1]);
  }
  c->push_held = 0;
  return s;
}

}  // extern "C"
