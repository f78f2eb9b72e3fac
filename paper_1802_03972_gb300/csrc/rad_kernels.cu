// Kernels of the far-field radiation sum (Pausch et al. 2018, Eq. 1, Eq. 13).
//
// Per call (one time step t, dt of N macro-particles) the mixed-precision path
// runs two kernels:
//
//  1. prepass (one thread per particle, FP64): moves positions to a per-call
//     reference point r_ref (the first particle), so that
//        t - n.r/c = tau_ref(n) + dtau,   tau_ref = t - n.r_ref/c,
//        dtau = -n.(r - r_ref)/c,
//     and writes a compact 80-byte FP32 record per particle (array of
//     structures): (r - r_ref)/c and beta as float-float pairs, beta_dot,
//     1/gamma^2 = 1 - |beta|^2 (FP64 before rounding), w dt, sqrt(w) dt.  FP64
//     is used here once per particle, never per (particle, direction, frequency).
//
//  2. accumulate (persistent: one CTA per resident slot; dynamic work items of
//     (job, bin tile, particle chunk)).  The particle records of a chunk stream
//     through shared memory in tiles of THREADS / NT particles (NT = directions
//     per bin tile), fetched by TMA bulk copies (cp.async.bulk + mbarrier) two
//     tiles ahead of use.  Per tile:
//     stage 1, one (particle, direction) record per thread, FP32: dtau as a
//       float-float pair and the transverse amplitude components a_i = e_i . A
//       in a basis (e1, e2) perpendicular to n.  Since n . A = 0 (Eq. 1) these
//       two carry |A|^2; with u = n - beta, n x (u x bdot) = u (n.bdot) - bdot D,
//       D = 1 - beta.n = (1/gamma^2 + b1^2 + b2^2) / (1 + beta.n) and e_i.u = -b_i,
//       so a_i = -(b_i (n.bdot) + (e_i.bdot) D) / D^2 without cancellation at
//       high gamma.  Records are double-buffered: one barrier per tile.
//     stage 2, per (particle, direction, frequency) "amplitude update": the
//       phase in turns p = (omega/2pi) dtau is reduced exactly with one fused
//       multiply-add against 1.5 * 2^23 (no FRND, which shares the MUFU pipe),
//       the float-float cross terms are added in radians, sin/cos come from the
//       MUFU (2 per update), and 8 packed FMAs add w dt a_i e^{i phi} and
//       sqrt(w) dt a_i e^{i phi} into register accumulators.  Frequencies are
//       processed in pairs with the packed f32x2 instructions of sm_100+.
//     Each work item writes its partial sums; the last item of a bin tile to
//     finish (an arrival counter, no float atomics) adds the partials in chunk
//     order, multiplies by e^{i omega tau_ref(n)} (reduced in FP64) and adds
//     the result into the resident state with compensated (Kahan) FP32 sums.
//     Results are deterministic for a given tile configuration.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <atomic>

#include "rad_impl.h"

namespace radimpl {

namespace {

constexpr double kC = 299792458.0;
constexpr double kInvC = 1.0 / 299792458.0;
// Physical prefactor q_e^2 / (16 pi^3 eps0 c) of Eq. 1, from the SI constants.
constexpr double kQe = 1.602176634e-19;
constexpr double kEps0 = 8.8541878128e-12;
constexpr double kPi = 3.14159265358979323846;
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

// ---------------------------------------------------------- mbarrier / TMA
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
// Waits for the given phase of the barrier; gives up after kWaitLimitNs.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t phase) {
  const uint32_t a = smem_addr(bar);
  const unsigned long long t0 = global_ns();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done) : "r"(a), "r"(phase) : "memory");
    if (done) return true;
    if (global_ns() - t0 > kWaitLimitNs) return false;
  }
}
// One elected thread: bulk copy of `bytes` (multiple of 16, both addresses
// 16-byte aligned) from global to shared memory, completing on `bar`.
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
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

// ------------------------------------------------------------------ prepass
// Record layout (floats): 0-2 (r - r_ref)/c hi, 3-5 lo, 6-8 beta hi, 9-11 beta
// lo, 12-14 beta_dot, 15 1/gamma^2, 16 w dt, 17 sqrt(w) dt, 18-19 unused.
__global__ void __launch_bounds__(256) prepass_kernel(LaunchArgs a) {
  const int j = find_job_block(a, blockIdx.x);
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
  const bool ok = isfinite(x) && isfinite(y) && isfinite(z) && isfinite(bx) && isfinite(by) &&
                  isfinite(bz) && isfinite(ax) && isfinite(ay) && isfinite(az) && isfinite(w) &&
                  w > 0.0 && g2 > 0.0 && isfinite(K.dt) && isfinite(K.t);
  float v[kRecFields];
  if (ok) {
    split_ff((x - rr[0]) * kInvC, v[0], v[3]);
    split_ff((y - rr[1]) * kInvC, v[1], v[4]);
    split_ff((z - rr[2]) * kInvC, v[2], v[5]);
    split_ff(bx, v[6], v[9]);
    split_ff(by, v[7], v[10]);
    split_ff(bz, v[8], v[11]);
    v[12] = __double2float_rn(ax);
    v[13] = __double2float_rn(ay);
    v[14] = __double2float_rn(az);
    v[15] = __double2float_rn(g2);
    v[16] = __double2float_rn(w * K.dt);
    v[17] = __double2float_rn(sqrt(w) * K.dt);
  } else {
    atomicOr(J.status, ST_BAD_PARTICLE);
#pragma unroll
    for (int f = 0; f < 18; ++f) v[f] = 0.0f;
    v[8] = 0.5f;   // a harmless finite beta (zero weights)
    v[15] = 0.75f;
  }
  v[18] = 0.0f;
  v[19] = 0.0f;
  float4* dst = reinterpret_cast<float4*>(J.rec + (size_t)k * kRecFields);
#pragma unroll
  for (int q = 0; q < kRecFields / 4; ++q)
    dst[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
}

// -------------------------------------------------------------- accumulate
// Stage 1 record of (particle, direction): three float4 in shared memory, each
// value duplicated for the packed (f32x2) stage-2 arithmetic:
//   r0 = (tau_h, tau_h, tau_l, tau_l)  dtau = -n.(r - r_ref)/c as hi + lo
//   r1 = (aw1, aw1, aw2, aw2)          w dt a_i
//   r2 = (av1, av1, av2, av2)          sqrt(w) dt a_i
// raw: the particle's 80-byte record.  Returns false when |dtau| is beyond the
// fast phase path's range.
__device__ __forceinline__ bool make_record(const float* __restrict__ raw,
                                            const float* __restrict__ dt_, int n_dir, int d,
                                            float tau_fast, float4* out) {
  const float4 q0 = *reinterpret_cast<const float4*>(raw);
  const float4 q1 = *reinterpret_cast<const float4*>(raw + 4);
  const float4 q2 = *reinterpret_cast<const float4*>(raw + 8);
  const float4 q3 = *reinterpret_cast<const float4*>(raw + 12);
  const float2 q4 = *reinterpret_cast<const float2*>(raw + 16);
  const float sh0 = q0.x, sh1 = q0.y, sh2 = q0.z, sl0 = q0.w, sl1 = q1.x, sl2 = q1.y;
  const float bh0 = q1.z, bh1 = q1.w, bh2 = q2.x, bl0 = q2.y, bl1 = q2.z, bl2 = q2.w;
  const float ad0 = q3.x, ad1 = q3.y, ad2 = q3.z, g2 = q3.w, ww = q4.x, sw = q4.y;
  const float nh0 = __ldg(dt_ + 0 * n_dir + d), nh1 = __ldg(dt_ + 1 * n_dir + d), nh2 = __ldg(dt_ + 2 * n_dir + d);
  const float nl0 = __ldg(dt_ + 3 * n_dir + d), nl1 = __ldg(dt_ + 4 * n_dir + d), nl2 = __ldg(dt_ + 5 * n_dir + d);
  const float e10 = __ldg(dt_ + 6 * n_dir + d), e11 = __ldg(dt_ + 7 * n_dir + d), e12 = __ldg(dt_ + 8 * n_dir + d);
  const float e20 = __ldg(dt_ + 9 * n_dir + d), e21 = __ldg(dt_ + 10 * n_dir + d), e22 = __ldg(dt_ + 11 * n_dir + d);

  // n . s in float-float: exact products (TwoProduct via fma) and exact sums
  // (Knuth TwoSum) of the hi parts, all first-order lo terms added in FP32.
  const float p0 = __fmul_rn(nh0, sh0), p1 = __fmul_rn(nh1, sh1), p2 = __fmul_rn(nh2, sh2);
  float lo = __fadd_rn(__fadd_rn(fmaf(nh0, sh0, -p0), fmaf(nh1, sh1, -p1)), fmaf(nh2, sh2, -p2));
  lo = fmaf(nh0, sl0, lo);
  lo = fmaf(nh1, sl1, lo);
  lo = fmaf(nh2, sl2, lo);
  lo = fmaf(nl0, sh0, lo);
  lo = fmaf(nl1, sh1, lo);
  lo = fmaf(nl2, sh2, lo);
  const float s1 = __fadd_rn(p0, p1);
  float bb = __fsub_rn(s1, p0);
  const float er1 = __fadd_rn(__fsub_rn(p0, __fsub_rn(s1, bb)), __fsub_rn(p1, bb));
  const float s2 = __fadd_rn(s1, p2);
  bb = __fsub_rn(s2, s1);
  const float er2 = __fadd_rn(__fsub_rn(s1, __fsub_rn(s2, bb)), __fsub_rn(p2, bb));
  lo = __fadd_rn(lo, __fadd_rn(er1, er2));
  const float hi = __fadd_rn(s2, lo);
  const float lo2 = __fsub_rn(lo, __fsub_rn(hi, s2));
  const float th = -hi, tl = -lo2;

  // Transverse amplitude (see the file comment).
  const float b1 = fmaf(e10, bh0, fmaf(e11, bh1, e12 * bh2)) + fmaf(e10, bl0, fmaf(e11, bl1, e12 * bl2));
  const float b2 = fmaf(e20, bh0, fmaf(e21, bh1, e22 * bh2)) + fmaf(e20, bl0, fmaf(e21, bl1, e22 * bl2));
  const float bn = fmaf(nh0, bh0, fmaf(nh1, bh1, nh2 * bh2));
  const float d1 = fmaf(e10, ad0, fmaf(e11, ad1, e12 * ad2));
  const float d2 = fmaf(e20, ad0, fmaf(e21, ad1, e22 * ad2));
  const float dn = fmaf(nh0, ad0, fmaf(nh1, ad1, nh2 * ad2));
  const float D = (g2 + fmaf(b1, b1, b2 * b2)) / (1.0f + bn);
  const float iD = 1.0f / D;
  const float iD2 = iD * iD;
  const float a1 = -fmaf(b1, dn, d1 * D) * iD2;
  const float a2 = -fmaf(b2, dn, d2 * D) * iD2;
  const float aw1 = ww * a1, aw2 = ww * a2, av1 = sw * a1, av2 = sw * a2;
  out[0] = make_float4(th, th, tl, tl);
  out[1] = make_float4(aw1, aw1, aw2, aw2);
  out[2] = make_float4(av1, av1, av2, av2);
  return fabsf(th) <= tau_fast;  // false for NaN as well
}

// Shared memory of the accumulate kernel: two raw tiles (THREADS particles x
// 80 B) filled by TMA, two record buffers (THREADS records x 48 B).
template <int THREADS>
struct Smem {
  static constexpr size_t raw_bytes = (size_t)THREADS * kRecFields * sizeof(float);
  static constexpr size_t rec_bytes = (size_t)THREADS * 3 * sizeof(float4);
  static constexpr size_t bytes = 2 * raw_bytes + 2 * rec_bytes;
};

template <int THREADS>
__device__ __forceinline__ float* raw_buf(unsigned char* smem, int b) {
  return reinterpret_cast<float*>(smem + (size_t)b * Smem<THREADS>::raw_bytes);
}
template <int THREADS>
__device__ __forceinline__ float4* rec_buf(unsigned char* smem, int b) {
  return reinterpret_cast<float4*>(smem + 2 * Smem<THREADS>::raw_bytes +
                                   (size_t)b * Smem<THREADS>::rec_bytes);
}

// phase: bit b is the parity to wait for on bars[b].
template <int THREADS, int W>
__device__ __forceinline__ bool process_item(const JobStatic& J, const JobCall& K, int tile,
                                             int chunk, unsigned char* __restrict__ smem,
                                             uint64_t* bars, uint32_t& phase, int* s_flag) {
  constexpr int NP = W / 2;
  const int WT = J.wt;
  const int NT = J.nt;
  const int KT = THREADS / NT;  // particles per shared-memory tile
  const int lanes_per_dir = WT / W;
  const int tile_d = tile / J.tiles_om, tile_o = tile - tile_d * J.tiles_om;
  const int d0 = tile_d * NT, o0 = tile_o * WT;
  const int my_dl = threadIdx.x / lanes_per_dir;
  const int my_slot = threadIdx.x - my_dl * lanes_per_dir;
  const int my_d_raw = d0 + my_dl;
  const int my_d = min(my_d_raw, J.n_dir - 1);
  const int om_first = o0 + my_slot * W;
  const int n_om = J.n_omega;
  // stage-1 assignment: thread -> (direction s1_dl, particle s1_kk) of a tile
  const int s1_dl = threadIdx.x / KT, s1_kk = threadIdx.x - s1_dl * KT;
  const int s1_d = min(d0 + s1_dl, J.n_dir - 1);

  float2 omh[NP], nomh[NP], wh[NP], wl[NP];
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    const int i0 = min(om_first + 2 * p, n_om - 1), i1 = min(om_first + 2 * p + 1, n_om - 1);
    omh[p] = make_float2(__ldg(J.om_tab + i0), __ldg(J.om_tab + i1));
    nomh[p] = make_float2(__ldg(J.om_tab + n_om + i0), __ldg(J.om_tab + n_om + i1));
    wh[p] = make_float2(__ldg(J.om_tab + 2 * n_om + i0), __ldg(J.om_tab + 2 * n_om + i1));
    wl[p] = make_float2(__ldg(J.om_tab + 3 * n_om + i0), __ldg(J.om_tab + 3 * n_om + i1));
  }
  float2 acc1[NP][kComps], acc2[NP][kComps];
#pragma unroll
  for (int p = 0; p < NP; ++p)
#pragma unroll
    for (int c = 0; c < kComps; ++c) acc1[p][c] = acc2[p][c] = make_float2(0.f, 0.f);

  const float2 kMag = make_float2(12582912.0f, 12582912.0f);      // 1.5 * 2^23
  const float2 kNegMag = make_float2(-12582912.0f, -12582912.0f);
  const float2 k2Pi = make_float2(6.28318530717958647692f, 6.28318530717958647692f);

  const long long k_begin = (long long)chunk * K.ck;
  const long long k_end = min(k_begin + (long long)K.ck, K.n);
  const int n_kt = (int)((k_end - k_begin + KT - 1) / KT);
  const uint32_t tile_bytes = (uint32_t)KT * kRecFields * sizeof(float);
  // Whole tiles are copied: k_begin is a multiple of KT and the record buffer
  // holds at least round_up(n, 256) particles, so the copy stays in bounds.
  if (threadIdx.x == 0) {
    tma_load_1d(raw_buf<THREADS>(smem, 0), J.rec + (size_t)k_begin * kRecFields, tile_bytes, &bars[0]);
    if (n_kt > 1)
      tma_load_1d(raw_buf<THREADS>(smem, 1), J.rec + (size_t)(k_begin + KT) * kRecFields, tile_bytes,
                  &bars[1]);
  }
  for (int it = 0; it < n_kt; ++it) {
    const int b = it & 1;
    const long long kt = k_begin + (long long)it * KT;
    const int kn = (int)min((long long)KT, k_end - kt);
    const bool landed = mbar_wait(&bars[b], (phase >> b) & 1u);
    phase ^= 1u << b;
    bool slow = false;
    if (landed && s1_kk < kn)
      slow = !make_record(raw_buf<THREADS>(smem, b) + s1_kk * kRecFields, J.dir_tab, J.n_dir, s1_d,
                          J.tau_fast, rec_buf<THREADS>(smem, b) + (s1_kk * NT + s1_dl) * 3);
    const int flags = __syncthreads_or((slow ? 1 : 0) | (landed ? 0 : 2));
    if (flags & 2) {
      // A TMA copy did not complete within the bound: record it, wait (bounded)
      // for the other buffer's copy still in flight, and leave.
      if (threadIdx.x == 0) {
        atomicOr(J.status, ST_TIMEOUT);
        if (it + 1 < n_kt) mbar_wait(&bars[b ^ 1], (phase >> (b ^ 1)) & 1u);
      }
      return false;
    }
    if (threadIdx.x == 0 && it + 2 < n_kt)
      tma_load_1d(raw_buf<THREADS>(smem, b), J.rec + (size_t)(kt + 2 * KT) * kRecFields, tile_bytes,
                  &bars[b]);
    const float4* rc = rec_buf<THREADS>(smem, b) + my_dl * 3;
    if (!(flags & 1)) {
#pragma unroll 4
      for (int kk = 0; kk < kn; ++kk) {
        const float4 r0 = rc[kk * NT * 3 + 0];
        const float4 r1 = rc[kk * NT * 3 + 1];
        const float4 r2 = rc[kk * NT * 3 + 2];
        const float2 th = make_float2(r0.x, r0.y), tl = make_float2(r0.z, r0.w);
        const float2 aw1 = make_float2(r1.x, r1.y), aw2 = make_float2(r1.z, r1.w);
        const float2 av1 = make_float2(r2.x, r2.y), av2 = make_float2(r2.z, r2.w);
#pragma unroll
        for (int p = 0; p < NP; ++p) {
          // p_turns = (omega/2pi) dtau: exact reduction of the hi product.
          const float2 t0 = __ffma2_rn(nomh[p], th, kMag);     // 1.5*2^23 - rint(x)
          const float2 q = __fadd2_rn(t0, kNegMag);             // -rint(x), exact
          const float2 f0 = __ffma2_rn(omh[p], th, q);         // x - rint(x), one rounding
          const float2 c1 = __fmul2_rn(wl[p], th);             // cross terms, radians
          const float2 c2 = __ffma2_rn(wh[p], tl, c1);
          const float2 ph = __ffma2_rn(f0, k2Pi, c2);          // phase in (-pi, pi] + tiny
          const float2 cc = make_float2(cos_approx(ph.x), cos_approx(ph.y));
          const float2 ss = make_float2(sin_approx(ph.x), sin_approx(ph.y));
          acc1[p][0] = __ffma2_rn(aw1, cc, acc1[p][0]);
          acc1[p][1] = __ffma2_rn(aw1, ss, acc1[p][1]);
          acc1[p][2] = __ffma2_rn(aw2, cc, acc1[p][2]);
          acc1[p][3] = __ffma2_rn(aw2, ss, acc1[p][3]);
          acc1[p][4] = __ffma2_rn(av1, cc, acc1[p][4]);
          acc1[p][5] = __ffma2_rn(av1, ss, acc1[p][5]);
          acc1[p][6] = __ffma2_rn(av2, cc, acc1[p][6]);
          acc1[p][7] = __ffma2_rn(av2, ss, acc1[p][7]);
        }
      }
    } else {
      // Wide path: some |dtau| exceed the fast range in this tile.  The phase
      // of every update is formed in FP64 from the float-float dtau and
      // omega / 2pi (exact for any magnitude the pair represents).
      if (threadIdx.x == 0) atomicOr(J.status, ST_SLOW_PHASE);
      double omt[W];
#pragma unroll
      for (int i = 0; i < W; ++i) omt[i] = J.om_turns[min(om_first + i, n_om - 1)];
      for (int kk = 0; kk < kn; ++kk) {
        const float4 r0 = rc[kk * NT * 3 + 0];
        const float4 r1 = rc[kk * NT * 3 + 1];
        const float4 r2 = rc[kk * NT * 3 + 2];
        const double tau = (double)r0.x + (double)r0.z;
#pragma unroll
        for (int p = 0; p < NP; ++p) {
          double x0 = omt[2 * p] * tau, x1 = omt[2 * p + 1] * tau;
          x0 -= rint(x0);
          x1 -= rint(x1);
          const float2 ph = make_float2((float)(x0 * 6.283185307179586), (float)(x1 * 6.283185307179586));
          const float2 cc = make_float2(cos_approx(ph.x), cos_approx(ph.y));
          const float2 ss = make_float2(sin_approx(ph.x), sin_approx(ph.y));
          acc1[p][0] = __ffma2_rn(make_float2(r1.x, r1.y), cc, acc1[p][0]);
          acc1[p][1] = __ffma2_rn(make_float2(r1.x, r1.y), ss, acc1[p][1]);
          acc1[p][2] = __ffma2_rn(make_float2(r1.z, r1.w), cc, acc1[p][2]);
          acc1[p][3] = __ffma2_rn(make_float2(r1.z, r1.w), ss, acc1[p][3]);
          acc1[p][4] = __ffma2_rn(make_float2(r2.x, r2.y), cc, acc1[p][4]);
          acc1[p][5] = __ffma2_rn(make_float2(r2.x, r2.y), ss, acc1[p][5]);
          acc1[p][6] = __ffma2_rn(make_float2(r2.z, r2.w), cc, acc1[p][6]);
          acc1[p][7] = __ffma2_rn(make_float2(r2.z, r2.w), ss, acc1[p][7]);
        }
      }
    }
    // Two-level summation: the tile's sums join the chunk sums.
#pragma unroll
    for (int p = 0; p < NP; ++p)
#pragma unroll
      for (int c = 0; c < kComps; ++c) {
        acc2[p][c] = __fadd2_rn(acc2[p][c], acc1[p][c]);
        acc1[p][c] = make_float2(0.f, 0.f);
      }
  }

  // Partial sums of this work item.
  const bool d_ok = my_d_raw < J.n_dir;
  const int nb = J.n_bins;
  float* part = J.partials + (size_t)chunk * kComps * nb;
  if (d_ok) {
#pragma unroll
    for (int p = 0; p < NP; ++p)
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int o = om_first + 2 * p + e;
        if (o < n_om) {
          const int bin = my_d * n_om + o;
#pragma unroll
          for (int c = 0; c < kComps; ++c)
            part[(size_t)c * nb + bin] = e ? acc2[p][c].y : acc2[p][c].x;
        }
      }
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned prev = atomicAdd(&J.tile_cnt[tile], 1u);
    *s_flag = (prev == (unsigned)(K.n_chunks - 1));
    if (*s_flag) J.tile_cnt[tile] = 0u;  // ready for the next call
    __threadfence();
  }
  __syncthreads();
  if (!*s_flag || !d_ok) return true;

  // Last arrival: add the chunks in order, rotate by e^{i omega tau_ref(n)},
  // compensated add into the resident state.
  const double* nd = J.dirs + 3 * my_d;
  const double tref = J.ref[3] - (nd[0] * J.ref[0] + nd[1] * J.ref[1] + nd[2] * J.ref[2]) * kInvC;
#pragma unroll
  for (int i = 0; i < W; ++i) {
    const int o = om_first + i;
    if (o >= n_om) continue;
    const int bin = my_d * n_om + o;
    float s[kComps];
#pragma unroll
    for (int c = 0; c < kComps; ++c) s[c] = 0.0f;
    for (int ch = 0; ch < K.n_chunks; ++ch) {
      const float* pc = J.partials + (size_t)ch * kComps * nb;
#pragma unroll
      for (int c = 0; c < kComps; ++c) s[c] += __ldcg(&pc[(size_t)c * nb + bin]);
    }
    double psi = J.om_turns[o] * tref;
    psi -= rint(psi);
    float sp, cp;
    sincospif(2.0f * (float)psi, &sp, &cp);
    float* st = J.state;
#pragma unroll
    for (int c = 0; c < kComps; c += 2) {
      const float re = s[c] * cp - s[c + 1] * sp;
      const float im = s[c] * sp + s[c + 1] * cp;
      const float x2[2] = {re, im};
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        float* sum = &st[(size_t)(c + h) * nb + bin];
        float* cmp = &st[(size_t)(kComps + c + h) * nb + bin];
        const float y = __fsub_rn(x2[h], *cmp);
        const float tt = __fadd_rn(*sum, y);
        *cmp = __fsub_rn(__fsub_rn(tt, *sum), y);
        *sum = tt;
      }
    }
  }
  return true;
}

template <int THREADS, int W, int MINB>
__global__ void __launch_bounds__(THREADS, MINB) accumulate_kernel(LaunchArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t bars[2];
  __shared__ long long s_item[2];
  __shared__ int s_flag;
  if (threadIdx.x == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    mbar_fence_init();
  }
  __syncthreads();
  uint32_t phase = 0u;
  int buf = 0;
  for (;;) {
    if (threadIdx.x == 0) s_item[buf] = (long long)atomicAdd(a.item_counter, 1ULL);
    __syncthreads();
    const long long item = s_item[buf];
    buf ^= 1;
    if (item >= a.n_items) return;
    const int j = find_job(a, item);
    const JobStatic& J = a.js[j];
    const JobCall K = a.use_inline ? a.inline_call : a.jc[j];
    const long long local = item - K.item_begin;
    const int tile = (int)(local % J.n_tiles);
    const int chunk = (int)(local / J.n_tiles);
    if (!process_item<THREADS, W>(J, K, tile, chunk, smem, bars, phase, &s_flag)) return;
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

__global__ void readout_kernel(const float* __restrict__ state, const double* __restrict__ state64,
                               int mixed, int n_omega, int n_bins, const double* __restrict__ omega,
                               int kind, double width, double k0, double* coh, double* inc,
                               double* tot) {
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
  const double f = form_factor(kind, width, omega[bin % n_omega]);
  const double f2 = f * f;
  const double ic = k0 * f2 * u2, ii = k0 * (1.0 - f2) * v2;
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

__global__ void state_add_kernel(float* __restrict__ state, const float* __restrict__ other,
                                 int n_bins) {
  const int bin = blockIdx.x * blockDim.x + threadIdx.x;
  if (bin >= n_bins) return;
  // other holds (sum, comp) pairs; add its value sum - comp with compensation.
#pragma unroll
  for (int c = 0; c < kComps; ++c) {
    const float x = __fsub_rn(other[(size_t)c * n_bins + bin], other[(size_t)(kComps + c) * n_bins + bin]);
    float* sum = &state[(size_t)c * n_bins + bin];
    float* cmp = &state[(size_t)(kComps + c) * n_bins + bin];
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

template <int T, int W, int MINB>
static cudaError_t launch_acc(const LaunchArgs& a, int grid, cudaStream_t s) {
  const size_t smem = Smem<T>::bytes;
  static bool attr_set = false;  // the opt-in is per kernel and idempotent
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(accumulate_kernel<T, W, MINB>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  accumulate_kernel<T, W, MINB><<<grid, T, smem, s>>>(a);
  count_launches(1);
  return cudaGetLastError();
}

size_t accumulate_smem_bytes(int variant) {
  return variant_info(variant).threads == 128 ? Smem<128>::bytes : Smem<256>::bytes;
}

template <int T, int W, int MINB>
static int blocks_per_sm() {
  int nb = 0;
  const size_t smem = Smem<T>::bytes;
  cudaFuncSetAttribute(accumulate_kernel<T, W, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)smem);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, accumulate_kernel<T, W, MINB>, T, smem) !=
          cudaSuccess ||
      nb < 1)
    nb = 1;
  return nb;
}

int accumulate_blocks_per_sm(int variant) {
  static int cached[kNumVariants] = {0, 0, 0};
  if (variant < 0 || variant >= kNumVariants) variant = 0;
  if (cached[variant] == 0) {
    switch (variant) {
      case 1: cached[1] = blocks_per_sm<256, 4, 2>(); break;
      case 2: cached[2] = blocks_per_sm<128, 2, 6>(); break;
      default: cached[0] = blocks_per_sm<256, 2, 3>(); break;
    }
  }
  return cached[variant];
}

cudaError_t launch_accumulate(int variant, const LaunchArgs& a, int grid, cudaStream_t s) {
  switch (variant) {
    case 1: return launch_acc<256, 4, 2>(a, grid, s);
    case 2: return launch_acc<128, 2, 6>(a, grid, s);
    default: return launch_acc<256, 2, 3>(a, grid, s);
  }
}

cudaError_t launch_prepass(const LaunchArgs& a, int total_blocks, cudaStream_t s) {
  if (total_blocks <= 0) return cudaSuccess;
  prepass_kernel<<<total_blocks, 256, 0, s>>>(a);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_readout(const float* state, int mixed, const double* state64, int n_omega,
                           int n_bins, const double* omega, rad_ff ff, double* coh, double* inc,
                           double* tot, cudaStream_t s) {
  const double k0 = kQe * kQe / (16.0 * kPi * kPi * kPi * kEps0 * kC);
  readout_kernel<<<(n_bins + 255) / 256, 256, 0, s>>>(state, state64, mixed, n_omega, n_bins,
                                                       omega, ff.kind, ff.width, k0, coh, inc, tot);
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

cudaError_t launch_state_add(float* state, const float* other, int n_bins, cudaStream_t s) {
  state_add_kernel<<<(n_bins + 255) / 256, 256, 0, s>>>(state, other, n_bins);
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
