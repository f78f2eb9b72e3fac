/*
 * rad_selftest.h - test-support entry points of the radiation library.  They
 * run pieces of the accumulate kernel's device arithmetic on caller-given
 * inputs, so that tests can compare each piece with FP64 host values, and they
 * exercise a bounded device wait.  Nothing here is on the accumulation path.
 */
#ifndef RAD_SELFTEST_H
#define RAD_SELFTEST_H

#include <stdint.h>

#include "rad.h"

#ifdef __cplusplus
extern "C" {
#endif

/* rad_selftest_wait - launch one block that waits, with the kernels' bounded
 * wait, on an mbarrier that nothing arrives on, giving up after limit_ns
 * nanoseconds (clamped to [1e6, 2e9]).  *timed_out = 1 when the wait gave up
 * (the expected outcome), *waited_s = the time it waited on the device clock.
 * Both out pointers are host memory.  Synchronises the device.  Returns RAD_OK,
 * RAD_EINVAL for NULL outputs, or RAD_ECUDA. */
rad_status rad_selftest_wait(int64_t limit_ns, int32_t* timed_out, double* waited_s);

/* rad_selftest_stage1 - stage 1 of the accumulate kernel for one direction.
 * Runs the context's pre-pass on n particles (device arrays, the layout of
 * rad_accumulate; the reference point is particle 0) and then, for every
 * particle k, the per-(particle, direction) record computation for direction
 * index dir, writing to out[8 k .. 8 k + 7] (host floats):
 *   th, tl   the retarded-time offset -n.(r_k - r_0)/c as a float-float pair (s);
 *   a0..a3   (w dt a1, w dt a2, sqrt(w) dt a1, sqrt(w) dt a2), with a_i = e_i . A and
 *            A = n x ((n - beta) x beta_dot) / (1 - beta.n)^2 (Eq. 1);
 *   fast     1 when |th| is within the fast phase path's range, else 0;
 *   pad      0.
 * basis (host, 6 floats): the context's transverse unit vectors e1, e2 of that
 * direction.  Mixed-precision contexts only; 0 <= dir < n_dir; 1 <= n <= 2^20.
 * Leaves the accumulators unchanged.  Errors: RAD_EINVAL, RAD_ECUDA, RAD_ESTATE. */
rad_status rad_selftest_stage1(rad_ctx* ctx, int64_t n, const double* r, const double* beta,
                               const double* beta_dot, const double* w, double t, double dt,
                               int32_t dir, float* out, float* basis);

/* rad_selftest_phase - the phase of every (frequency of the context, offset)
 * pair as the accumulate kernel forms it: tau = th[j] + tl[j] (host float
 * arrays of n_tau), fast path (float-float product, exact reduction to
 * (-pi, pi] plus cross terms) into fast[i * n_tau + j] and the FP64 wide path
 * into wide[i * n_tau + j], both radians (host floats, n_omega x n_tau each).
 * Mixed-precision contexts only; 1 <= n_tau <= 2^20.  Errors: RAD_EINVAL,
 * RAD_ECUDA, RAD_ESTATE. */
rad_status rad_selftest_phase(rad_ctx* ctx, int32_t n_tau, const float* th, const float* tl,
                              float* fast, float* wide);

#ifdef __cplusplus
}
#endif

#endif /* RAD_SELFTEST_H */
