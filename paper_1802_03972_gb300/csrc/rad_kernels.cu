// Kernels around the accumulate kernel (which lives in rad_accumulate.cu):
// the per-particle FP64 pre-pass, the readout of the spectra, the plain FP64
// kernel and the state merge (Pausch et al. 2018, Eq. 1, Eq. 12, Eq. 13).
//
// pre-pass (one thread per particle, FP64): moves positions to a per-call
// reference point r_ref (the first particle), so that
//    t - n.r/c = tau_ref(n) + dtau,   tau_ref = t - n.r_ref/c,   dtau = -n.(r - r_ref)/c,
// and writes a compact 80-byte FP32 record per particle (array of structures):
// (r - r_ref)/c and beta as float-float pairs, beta_dot, 1/gamma^2 = 1 - |beta|^2
// (FP64 before rounding), w dt and sqrt(w) dt.  FP64 is used here once per
// particle, never per (particle, direction, frequency).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <atomic>

#include "rad_device.cuh"
#include "rad_impl.h"

namespace radimpl {

namespace {

using dev::kC;
using dev::kInvC;
// Physical prefactor q_e^2 / (16 pi^3 eps0 c) of Eq. 1, from the SI constants.
constexpr double kQe = 1.602176634e-19;
constexpr double kEps0 = 8.8541878128e-12;
constexpr double kPi = 3.14159265358979323846;

// ------------------------------------------------------------------ prepass
// Record layout (floats): 0-2 (r - r_ref)/c hi, 3-5 lo, 6-8 beta hi, 9-11 beta
// lo, 12-14 beta_dot, 15 1/gamma^2, 16 w dt, 17 sqrt(w) dt, 18 w - 1, 19 unused.
// Record of particle k with positions relative to rr; false for invalid data
// (the record then has zero weights and a harmless finite beta).
__device__ __forceinline__ bool make_record(const JobStatic& J, const JobCall& K, long long k,
                                            const double rr[3], float v[kRecFields]) {
  const long long n = K.n;
  const double x = K.r[k], y = K.r[n + k], z = K.r[2 * n + k];
  const double bx = K.beta[k], by = K.beta[n + k], bz = K.beta[2 * n + k];
  const double ax = K.bdot[k], ay = K.bdot[n + k], az = K.bdot[2 * n + k];
  const double w = K.w[k];
  const double g2 = 1.0 - (bx * bx + by * by + bz * bz);
  const bool valid = isfinite(x) && isfinite(y) && isfinite(z) && isfinite(bx) && isfinite(by) &&
                     isfinite(bz) && isfinite(ax) && isfinite(ay) && isfinite(az) && isfinite(w) &&
                     w > 0.0 && g2 > 0.0 && isfinite(K.dt) && isfinite(K.t);
  if (valid && !J.skip) {
    dev::split_ff((x - rr[0]) * kInvC, v[0], v[3]);
    dev::split_ff((y - rr[1]) * kInvC, v[1], v[4]);
    dev::split_ff((z - rr[2]) * kInvC, v[2], v[5]);
    dev::split_ff(bx, v[6], v[9]);
    dev::split_ff(by, v[7], v[10]);
    dev::split_ff(bz, v[8], v[11]);
    v[12] = __double2float_rn(ax);
    v[13] = __double2float_rn(ay);
    v[14] = __double2float_rn(az);
    v[15] = __double2float_rn(g2);
    v[16] = __double2float_rn(w * K.dt);
    // FP32 square root (the field is FP32; ~1e-7 relative): FP64's is slow on this GPU
    v[17] = sqrtf(__double2float_rn(w)) * __double2float_rn(K.dt);
    v[18] = __double2float_rn(w - 1.0);
  } else {
#pragma unroll
    for (int f = 0; f < 19; ++f) v[f] = 0.0f;
    v[8] = 0.5f;   // a harmless finite beta (zero weights)
    v[15] = 0.75f;
  }
  v[19] = 0.0f;
  return valid;
}

__device__ __forceinline__ void store_record(float* dst_rec, const float v[kRecFields]) {
  float4* dst = reinterpret_cast<float4*>(dst_rec);
#pragma unroll
  for (int q = 0; q < kRecFields / 4; ++q)
    dst[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
}

__global__ void __launch_bounds__(256) prepass_kernel(LaunchArgs a) {
  const int j = dev::find_job_block(a, blockIdx.x);
  const JobStatic& J = a.js[j];
  const JobCall K = a.use_inline ? a.inline_call : a.jc[j];
  const long long n = K.n;
  // Reference point: the first particle (origin if it is not finite).
  double rr[3] = {K.r[0], K.r[n], K.r[2 * n]};
  if (!(isfinite(rr[0]) && isfinite(rr[1]) && isfinite(rr[2]))) rr[0] = rr[1] = rr[2] = 0.0;
  const long long k = (long long)(blockIdx.x - K.block_begin) * blockDim.x + threadIdx.x;
  if (k == 0) {
    J.ref[0] = rr[0];
    J.ref[1] = rr[1];
    J.ref[2] = rr[2];
    J.ref[3] = K.t;
  }
  if (k >= n) return;
  float v[kRecFields];
  const bool valid = make_record(J, K, k, rr, v);
  if (!valid) atomicOr(J.status, ST_BAD_PARTICLE);
  // A particle that some direction of the grid may see beyond the fast phase
  // range makes the call wide (one atomic per warp that has one).  The bound
  // on |n . (r - r_ref)| over the grid: |axis . dr| + sin(largest angle from
  // the axis) |dr across the axis|.
  // A call of one sorted group or less gains nothing from sorting: never wide.
  // In FP32 on the record's (r - r_ref) / c (hi parts, seconds): the flag only
  // steers a call to the sorted path, and a call wrongly left unsorted still
  // runs correctly (its far tiles take the FP64 phase path).
  bool far = false;
  if (J.wide_flag && valid && !J.skip && n > kGroup && n < (1LL << 31)) {
    const float along = fmaf((float)J.axis[0], v[0], fmaf((float)J.axis[1], v[1], (float)J.axis[2] * v[2]));
    const float r2 = fmaf(v[0], v[0], fmaf(v[1], v[1], v[2] * v[2]));
    const float across = sqrtf(fmaxf(r2 - along * along, 0.0f));
    far = fabsf(along) + (float)J.cone_sin * across > 0.999f * J.tau_fast;
  }
  const unsigned far_lanes = __ballot_sync(__activemask(), far);
  if (far && (threadIdx.x & 31) == __ffs(far_lanes) - 1) {
    atomicOr(J.wide_flag, 1);
    if (a.any_wide && a.any_wide != J.wide_flag) atomicOr(a.any_wide, 1);
  }
  if (!dev::bounds_ok(k < J.n_cap, J.status)) return;
  store_record(J.rec + (size_t)k * kRecFields, v);
}

// ------------------------------------------------------------- wide calls
__device__ __forceinline__ bool call_is_wide(const JobStatic& J) {
  return J.wide_flag != nullptr && *J.wide_flag != 0;
}

// Bucket of particle k along the sort axis, centred on the call's reference.
// Explicit roundings: the histogram and the scatter kernels must agree bit for
// bit, whatever either compilation contracts into fused multiply-adds.
__device__ __forceinline__ int sort_bucket(const JobStatic& J, const JobCall& K, long long k) {
  const long long n = K.n;
  const double dx = __dsub_rn(K.r[k], J.ref[0]);
  const double dy = __dsub_rn(K.r[n + k], J.ref[1]);
  const double dz = __dsub_rn(K.r[2 * n + k], J.ref[2]);
  const double s = __fma_rn(J.axis[0], dx, __fma_rn(J.axis[1], dy, __dmul_rn(J.axis[2], dz)));
  const double q = __ddiv_rn(s, J.bucket_w);
  constexpr double kHalf = 0.5 * kSortBuckets;
  if (!(q > -kHalf)) return 0;  // also NaN
  if (!(q < kHalf)) return kSortBuckets - 1;
  return min(kSortBuckets - 1, (int)floor(q + kHalf));
}

// Job of a sort-histogram block (jobs ordered by sort_block_begin).
__device__ __forceinline__ int find_job_sort_block(const LaunchArgs& a, int block) {
  if (a.n_jobs == 1) return 0;
  int lo = 0, hi = a.n_jobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (a.jc[mid].sort_block_begin <= block) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Per kSortBlock particles: bucket counts.
__global__ void __launch_bounds__(256) wide_hist_kernel(LaunchArgs a) {
  const int j = find_job_sort_block(a, blockIdx.x);
  const JobStatic& J = a.js[j];
  if (!call_is_wide(J)) return;
  const JobCall K = a.use_inline ? a.inline_call : a.jc[j];
  __shared__ int hist[kSortBuckets];
  for (int b = threadIdx.x; b < kSortBuckets; b += blockDim.x) hist[b] = 0;
  __syncthreads();
  const long long blk = blockIdx.x - K.sort_block_begin;
  const long long k0 = blk * kSortBlock;
  for (int i = threadIdx.x; i < kSortBlock; i += blockDim.x)
    if (k0 + i < K.n) atomicAdd(&hist[sort_bucket(J, K, k0 + i)], 1);
  __syncthreads();
  int* out = J.sort_counts + (size_t)blk * kSortBuckets;
  for (int b = threadIdx.x; b < kSortBuckets; b += blockDim.x) out[b] = hist[b];
}

// One block per job: per bucket, the prefix of the counts over the histogram
// blocks (in place), and the first sorted position of every bucket.
__global__ void __launch_bounds__(1024) wide_scan_kernel(LaunchArgs a) {
  const JobStatic& J = a.js[blockIdx.x];
  if (!call_is_wide(J)) return;
  const JobCall K = a.use_inline ? a.inline_call : a.jc[blockIdx.x];
  __shared__ int tot[kSortBuckets];
  __shared__ int wsum[32];
  const int nblk = (int)((K.n + kSortBlock - 1) / kSortBlock);
  for (int b = threadIdx.x; b < kSortBuckets; b += 1024) {
    int run = 0;
    int* c = J.sort_counts + b;
    int blk = 0;
    // eight independent loads in flight per step, then their prefix
    for (; blk + 8 <= nblk; blk += 8) {
      int v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = c[(size_t)(blk + u) * kSortBuckets];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        c[(size_t)(blk + u) * kSortBuckets] = run;
        run += v[u];
      }
    }
    for (; blk < nblk; ++blk) {
      const int v = c[(size_t)blk * kSortBuckets];
      c[(size_t)blk * kSortBuckets] = run;
      run += v;
    }
    tot[b] = run;
  }
  __syncthreads();
  static_assert(kSortBuckets == 4 * 1024, "four buckets per thread");
  const int t = threadIdx.x, lane = t & 31;
  const int v0 = tot[4 * t], v1 = tot[4 * t + 1], v2 = tot[4 * t + 2], v3 = tot[4 * t + 3];
  const int s = v0 + v1 + v2 + v3;
  int x = s;
  for (int off = 1; off < 32; off <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, off);
    if (lane >= off) x += y;
  }
  if (lane == 31) wsum[t >> 5] = x;
  __syncthreads();
  if (t < 32) {
    int w = wsum[t];
    for (int off = 1; off < 32; off <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, w, off);
      if (t >= off) w += y;
    }
    wsum[t] = w;
  }
  __syncthreads();
  const int excl = x - s + ((t >> 5) ? wsum[(t >> 5) - 1] : 0);
  J.bucket_base[4 * t] = excl;
  J.bucket_base[4 * t + 1] = excl + v0;
  J.bucket_base[4 * t + 2] = excl + v0 + v1;
  J.bucket_base[4 * t + 3] = excl + v0 + v1 + v2;
}

// Per kSortBlock particles: the sorted position of every particle, stable
// (particles of one bucket keep their order), so the order is a function of
// the input alone.  The block computes the buckets into shared memory, then
// one warp hands out the positions in particle order.
__global__ void __launch_bounds__(256) wide_scatter_kernel(LaunchArgs a) {
  const int j = find_job_sort_block(a, blockIdx.x);
  const JobStatic& J = a.js[j];
  if (!call_is_wide(J)) return;
  const JobCall K = a.use_inline ? a.inline_call : a.jc[j];
  __shared__ int cnt[kSortBuckets];
  __shared__ int bkt[kSortBlock];
  const long long blk = blockIdx.x - K.sort_block_begin;
  const long long k0 = blk * kSortBlock;
  const int* pre = J.sort_counts + (size_t)blk * kSortBuckets;
  for (int b = threadIdx.x; b < kSortBuckets; b += blockDim.x) cnt[b] = J.bucket_base[b] + pre[b];
  for (int i = threadIdx.x; i < kSortBlock; i += blockDim.x)
    bkt[i] = k0 + i < K.n ? sort_bucket(J, K, k0 + i) : -1;
  __syncthreads();
  if (threadIdx.x >= 32) return;
  const int lane = threadIdx.x;
  const unsigned below = (1u << lane) - 1u;
  for (int it = 0; it < kSortBlock / 32; ++it) {
    const long long k = k0 + it * 32 + lane;
    const bool in = k < K.n;
    const int b = bkt[it * 32 + lane];
    const unsigned peers = __match_any_sync(0xffffffffu, b);
    const int pos = in ? cnt[b] + __popc(peers & below) : 0;
    __syncwarp();
    if (in) {
      // positions are in [0, n) by construction; an inconsistency is reported
      // (the context then fails) instead of written
      if (pos >= 0 && pos < K.n) J.perm[pos] = (int)k;
      else atomicOr(J.status, ST_BOUNDS);
      if (lane == 31 - __clz(peers)) cnt[b] += __popc(peers);
    }
    __syncwarp();
  }
}

// Records in sorted order, positions relative to the first particle of each
// kGroup-particle group (its reference point); the group references relative
// to the call's reference go to gref.
__global__ void __launch_bounds__(256) wide_records_kernel(LaunchArgs a) {
  const int j = dev::find_job_block(a, blockIdx.x);
  const JobStatic& J = a.js[j];
  if (!call_is_wide(J)) return;
  const JobCall K = a.use_inline ? a.inline_call : a.jc[j];
  static_assert(kGroup == 256, "one block per group");
  const long long p0 = (long long)(blockIdx.x - K.block_begin) * kGroup;
  const long long p = p0 + threadIdx.x;
  if (p >= K.n) return;
  const long long n = K.n;
  int k = J.perm[p], k0 = J.perm[p0];
  if (k < 0 || k >= n || k0 < 0 || k0 >= n) {  // never, for a consistent sort
    atomicOr(J.status, ST_BOUNDS);
    k = k0 = 0;
  }
  double R[3] = {K.r[k0], K.r[n + k0], K.r[2 * n + k0]};
  if (!(isfinite(R[0]) && isfinite(R[1]) && isfinite(R[2]))) {
    R[0] = J.ref[0];
    R[1] = J.ref[1];
    R[2] = J.ref[2];
  }
  float v[kRecFields];
  make_record(J, K, k, R, v);  // invalid data was reported by the pre-pass
  if (!dev::bounds_ok(p < J.n_cap, J.status)) return;
  store_record(J.rec + (size_t)p * kRecFields, v);
  if (threadIdx.x == 0) {
    double* g = J.gref + 3 * (p0 / kGroup);
    g[0] = R[0] - J.ref[0];
    g[1] = R[1] - J.ref[1];
    g[2] = R[2] - J.ref[2];
  }
}

// ------------------------------------------------------------------ readout
__device__ double sinc(double x) { return x == 0.0 ? 1.0 : sin(x) / x; }

// Amplitude form factor of Table 1, normalised to f(0) = 1.
__device__ double form_factor(int kind, double width, double omega) {
  const double x = omega * width * (0.5 * kInvC);
  switch (kind) {
    case RAD_FF_CIC: return sinc(x);
    case RAD_FF_TSC: { const double s = sinc(x); return s * s; }
    case RAD_FF_QSC: { const double s = sinc(x); return s * s * s; }
    case RAD_FF_GAUSS: { const double g = omega * width * kInvC; return exp(-0.5 * g * g); }
    default: return 1.0;
  }
}

// With RAD_FF_3D, box shapes are axis-aligned 3-D products: f = prod_d f_1(omega n_d).
__device__ double form_factor_dir(int kind, int flags, double width, double omega,
                                  const double* n) {
  if (!(flags & RAD_FF_3D) || kind == RAD_FF_POINT || kind == RAD_FF_GAUSS)
    return form_factor(kind, width, omega);
  return form_factor(kind, width, omega * n[0]) * form_factor(kind, width, omega * n[1]) *
         form_factor(kind, width, omega * n[2]);
}

__global__ void readout_kernel(const float* __restrict__ state, const double* __restrict__ state64,
                               int mixed, int n_omega, int n_bins, const double* __restrict__ omega,
                               const double* __restrict__ dirs, int kind, int flags, double width,
                               double k0, double* coh, double* inc, double* tot) {
  const int bin = blockIdx.x * blockDim.x + threadIdx.x;
  if (bin >= n_bins) return;
  double u2 = 0.0, v2 = 0.0;
  if (mixed) {
#pragma unroll
    for (int c = 0; c < kComps; ++c) {
      const double x = (double)state[(size_t)c * n_bins + bin] -
                       (double)state[(size_t)(kComps + c) * n_bins + bin];
      if (c < 4) u2 += x * x;
      else v2 += x * x;
    }
  } else {
#pragma unroll
    for (int c = 0; c < 12; ++c) {
      const double x = state64[(size_t)c * n_bins + bin];
      if (c < 6) u2 += x * x;
      else v2 += x * x;
    }
  }
  const int d = bin / n_omega;
  const double f = form_factor_dir(kind, flags, width, omega[bin - d * n_omega], dirs + 3 * d);
  const double f2 = f * f;
  const double ic = k0 * f2 * u2, ii = k0 * (1.0 - f2) * v2;
  if (coh) coh[bin] = ic;
  if (inc) inc[bin] = ii;
  if (tot) tot[bin] = ic + ii;
}

__global__ void readout_species_kernel(SpeciesArgs a, int n_omega, int n_bins,
                                       const double* __restrict__ omega,
                                       const double* __restrict__ dirs, double k0, double* coh,
                                       double* inc, double* tot) {
  const int bin = blockIdx.x * blockDim.x + threadIdx.x;
  if (bin >= n_bins) return;
  const int d = bin / n_omega;
  const double om = omega[bin - d * n_omega];
  const int nu = a.mixed ? 4 : 6;  // real components of U (and of V)
  double u[6] = {0, 0, 0, 0, 0, 0};
  double ii = 0.0;
  for (int s = 0; s < a.n_species; ++s) {
    const double f = form_factor_dir(a.kind[s], a.flags[s], a.width[s], om, dirs + 3 * d);
    double v2 = 0.0;
    for (int c = 0; c < 2 * nu; ++c) {
      double x;
      if (a.mixed)
        x = (double)a.state[s][(size_t)c * n_bins + bin] -
            (double)a.state[s][(size_t)(kComps + c) * n_bins + bin];
      else
        x = a.state64[s][(size_t)c * n_bins + bin];
      if (c < nu) u[c] += f * x;  // amplitudes add across species before |.|^2
      else v2 += x * x;
    }
    ii += (1.0 - f * f) * v2;
  }
  double u2 = 0.0;
  for (int c = 0; c < nu; ++c) u2 += u[c] * u[c];
  const double ic = k0 * u2;
  ii *= k0;
  if (coh) coh[bin] = ic;
  if (inc) inc[bin] = ii;
  if (tot) tot[bin] = ic + ii;
}

// ----------------------------------------------------------- plain FP64 K5
// One thread per (direction, frequency) bin; every particle's amplitude and
// phase in FP64 with the library sincos, summed in FP64 (Eq. 1, Eq. 13).
__global__ void __launch_bounds__(128) fp64_kernel(const double* __restrict__ omega,
                                                   const double* __restrict__ dirs, int n_omega,
                                                   int n_dir, long long n, const double* __restrict__ r,
                                                   const double* __restrict__ beta,
                                                   const double* __restrict__ bdot,
                                                   const double* __restrict__ w, double t, double dt,
                                                   double* __restrict__ state, int* status) {
  const int n_bins = n_omega * n_dir;
  const int bin = blockIdx.x * blockDim.x + threadIdx.x;
  if (bin >= n_bins) return;
  const int di = bin / n_omega;
  const double om = omega[bin - di * n_omega];
  const double nx = dirs[3 * di], ny = dirs[3 * di + 1], nz = dirs[3 * di + 2];
  double u[6] = {0, 0, 0, 0, 0, 0}, v[6] = {0, 0, 0, 0, 0, 0};
  bool bad = false;
  for (long long k = 0; k < n; ++k) {
    const double bx = beta[k], by = beta[n + k], bz = beta[2 * n + k];
    const double ax = bdot[k], ay = bdot[n + k], az = bdot[2 * n + k];
    const double wk = w[k];
    const double g2 = 1.0 - (bx * bx + by * by + bz * bz);
    if (!(wk > 0.0) || !(g2 > 0.0) || !isfinite(wk) || !isfinite(ax + ay + az) ||
        !isfinite(r[k] + r[n + k] + r[2 * n + k])) {
      bad = true;
      continue;
    }
    const double ux = nx - bx, uy = ny - by, uz = nz - bz;
    const double cx = uy * az - uz * ay, cy = uz * ax - ux * az, cz = ux * ay - uy * ax;
    const double mx = ny * cz - nz * cy, my = nz * cx - nx * cz, mz = nx * cy - ny * cx;
    const double dd = 1.0 - (bx * nx + by * ny + bz * nz);
    const double id2 = 1.0 / (dd * dd);
    const double phi = om * (t - (nx * r[k] + ny * r[n + k] + nz * r[2 * n + k]) * kInvC);
    double sp, cp;
    sincos(phi, &sp, &cp);
    const double a[3] = {mx * id2, my * id2, mz * id2};
    const double ww = wk * dt, sw = sqrt(wk) * dt;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      u[2 * c] += ww * a[c] * cp;
      u[2 * c + 1] += ww * a[c] * sp;
      v[2 * c] += sw * a[c] * cp;
      v[2 * c + 1] += sw * a[c] * sp;
    }
  }
  if (bad) atomicOr(status, ST_BAD_PARTICLE);
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    state[(size_t)c * n_bins + bin] += u[c];
    state[(size_t)(6 + c) * n_bins + bin] += v[c];
  }
}

// Literal spectrum K0 |P|^2 from the compensated P.e1, P.e2 sums.
__global__ void readout_literal_kernel(const float* __restrict__ state_p, int n_bins, double k0,
                                       double* out) {
  const int bin = blockIdx.x * blockDim.x + threadIdx.x;
  if (bin >= n_bins) return;
  double p2 = 0.0;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const double x = (double)state_p[(size_t)c * n_bins + bin] -
                     (double)state_p[(size_t)(4 + c) * n_bins + bin];
    p2 += x * x;
  }
  out[bin] = k0 * p2;
}

// Adds another accumulator array into state with compensation.  Both hold
// n_comps sums followed by their n_comps compensations per bin.
__global__ void state_add_kernel(float* __restrict__ state, const float* __restrict__ other,
                                 int n_bins, int n_comps) {
  const int bin = blockIdx.x * blockDim.x + threadIdx.x;
  if (bin >= n_bins) return;
  // other holds (sum, comp) pairs; add its value sum - comp with compensation.
  for (int c = 0; c < n_comps; ++c) {
    const float x = __fsub_rn(other[(size_t)c * n_bins + bin], other[(size_t)(n_comps + c) * n_bins + bin]);
    float* sum = &state[(size_t)c * n_bins + bin];
    float* cmp = &state[(size_t)(n_comps + c) * n_bins + bin];
    const float y = __fsub_rn(x, *cmp);
    const float tt = __fadd_rn(*sum, y);
    *cmp = __fsub_rn(__fsub_rn(tt, *sum), y);
    *sum = tt;
  }
}

__global__ void state64_add_kernel(double* __restrict__ state, const double* __restrict__ other,
                                   int n_bins) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 12 * n_bins) return;
  state[i] += other[i];
}

std::atomic<long long> g_launches{0};

}  // namespace

void count_launches(int n) { g_launches.fetch_add(n); }

cudaError_t launch_prepass(const LaunchArgs& a, int total_blocks, cudaStream_t s) {
  if (total_blocks <= 0) return cudaSuccess;
  prepass_kernel<<<total_blocks, 256, 0, s>>>(a);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_wide(const LaunchArgs& a, int sort_blocks, int prepass_blocks, cudaStream_t s) {
  if (sort_blocks <= 0 || prepass_blocks <= 0) return cudaSuccess;
  wide_hist_kernel<<<sort_blocks, 256, 0, s>>>(a);
  wide_scan_kernel<<<a.n_jobs, 1024, 0, s>>>(a);
  wide_scatter_kernel<<<sort_blocks, 256, 0, s>>>(a);
  wide_records_kernel<<<prepass_blocks, 256, 0, s>>>(a);
  count_launches(kWideLaunches);
  return cudaGetLastError();
}

void wide_geometry(const double* nd, int n_dir, float tau_fast, double axis[3], double* cone_sin,
                   double* bucket_w) {
  double m[3] = {0.0, 0.0, 0.0};
  for (int d = 0; d < n_dir; ++d)
    for (int i = 0; i < 3; ++i) m[i] += nd[3 * d + i];
  double len = sqrt(m[0] * m[0] + m[1] * m[1] + m[2] * m[2]);
  // A grid spread over all directions has no useful mean: sort along z.
  if (!(len > 0.5 * n_dir)) {
    m[0] = m[1] = 0.0;
    m[2] = len = 1.0;
  }
  for (int i = 0; i < 3; ++i) axis[i] = m[i] / len;
  double cos_min = 1.0;
  for (int d = 0; d < n_dir; ++d)
    cos_min = std::min(cos_min, axis[0] * nd[3 * d] + axis[1] * nd[3 * d + 1] + axis[2] * nd[3 * d + 2]);
  *cone_sin = cos_min <= 0.0 ? 1.0 : sqrt(std::max(0.0, 1.0 - cos_min * cos_min));
  // A group of sorted particles spans about two buckets along the axis: an
  // eighth of the fast range keeps it well inside.
  *bucket_w = (double)tau_fast * kC / 8.0;
}

cudaError_t launch_readout(const float* state, int mixed, const double* state64, int n_omega,
                           int n_bins, const double* omega, const double* dirs, rad_ff ff,
                           double* coh, double* inc, double* tot, cudaStream_t s) {
  const double k0 = kQe * kQe / (16.0 * kPi * kPi * kPi * kEps0 * kC);
  readout_kernel<<<(n_bins + 255) / 256, 256, 0, s>>>(state, state64, mixed, n_omega, n_bins,
                                                       omega, dirs, ff.kind, ff.flags, ff.width,
                                                       k0, coh, inc, tot);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_readout_species(const SpeciesArgs& a, int n_omega, int n_bins,
                                   const double* omega, const double* dirs, double* coh,
                                   double* inc, double* tot, cudaStream_t s) {
  const double k0 = kQe * kQe / (16.0 * kPi * kPi * kPi * kEps0 * kC);
  readout_species_kernel<<<(n_bins + 255) / 256, 256, 0, s>>>(a, n_omega, n_bins, omega, dirs, k0,
                                                              coh, inc, tot);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_fp64(const double* omega, const double* dirs, int n_omega, int n_dir,
                        long long n, const double* r, const double* beta, const double* bdot,
                        const double* w, double t, double dt, double* state64, int* status,
                        cudaStream_t s) {
  const int n_bins = n_omega * n_dir;
  fp64_kernel<<<(n_bins + 127) / 128, 128, 0, s>>>(omega, dirs, n_omega, n_dir, n, r, beta, bdot,
                                                    w, t, dt, state64, status);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_state_add(float* state, const float* other, int n_bins, int n_comps,
                             cudaStream_t s) {
  state_add_kernel<<<(n_bins + 255) / 256, 256, 0, s>>>(state, other, n_bins, n_comps);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_readout_literal(const float* state_p, int n_bins, double* out, cudaStream_t s) {
  const double k0 = kQe * kQe / (16.0 * kPi * kPi * kPi * kEps0 * kC);
  readout_literal_kernel<<<(n_bins + 255) / 256, 256, 0, s>>>(state_p, n_bins, k0, out);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_state64_add(double* state, const double* other, int n_bins, cudaStream_t s) {
  state64_add_kernel<<<(12 * n_bins + 255) / 256, 256, 0, s>>>(state, other, n_bins);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace radimpl

extern "C" int64_t rad_kernel_launch_count(void) { return radimpl::g_launches.load(); }
