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
  const double x = K.r[k], y = K.r[n + k], z = K.r[2 * n + k];
  const double bx = K.beta[k], by = K.beta[n + k], bz = K.beta[2 * n + k];
  const double ax = K.bdot[k], ay = K.bdot[n + k], az = K.bdot[2 * n + k];
  const double w = K.w[k];
  const double g2 = 1.0 - (bx * bx + by * by + bz * bz);
  const bool valid = isfinite(x) && isfinite(y) && isfinite(z) && isfinite(bx) && isfinite(by) &&
                     isfinite(bz) && isfinite(ax) && isfinite(ay) && isfinite(az) && isfinite(w) &&
                     w > 0.0 && g2 > 0.0 && isfinite(K.dt) && isfinite(K.t);
  const bool ok = valid && !J.skip;
  float v[kRecFields];
  if (ok) {
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
    v[17] = __double2float_rn(sqrt(w) * K.dt);
    v[18] = __double2float_rn(w - 1.0);
  } else {
    if (!valid) atomicOr(J.status, ST_BAD_PARTICLE);
#pragma unroll
    for (int f = 0; f < 19; ++f) v[f] = 0.0f;
    v[8] = 0.5f;   // a harmless finite beta (zero weights)
    v[15] = 0.75f;
  }
  v[19] = 0.0f;
  if (!dev::bounds_ok(k < J.n_cap, J.status)) return;
  float4* dst = reinterpret_cast<float4*>(J.rec + (size_t)k * kRecFields);
#pragma unroll
  for (int q = 0; q < kRecFields / 4; ++q)
    dst[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
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
