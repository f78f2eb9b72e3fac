// Per-(particle, direction) and per-update arithmetic of the accumulate
// kernel, shared with the self-test kernels that check it against FP64 host
// values: stage 1 (retarded-time offset and transverse amplitude of one
// particle record for one direction) and the exact phase reduction.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "rad_device.cuh"

namespace radimpl {
namespace dev {

// One direction's row of the direction table: n (hi, lo) and the transverse
// basis e1, e2.
struct DirRow {
  float nh0, nh1, nh2, nl0, nl1, nl2, e10, e11, e12, e20, e21, e22;
};

// Row d of the direction table dt_ ([12][n_dir] floats, global memory).
__device__ __forceinline__ DirRow dir_row(const float* __restrict__ dt_, int n_dir, int d) {
  DirRow r;
  r.nh0 = __ldg(dt_ + 0 * n_dir + d), r.nh1 = __ldg(dt_ + 1 * n_dir + d), r.nh2 = __ldg(dt_ + 2 * n_dir + d);
  r.nl0 = __ldg(dt_ + 3 * n_dir + d), r.nl1 = __ldg(dt_ + 4 * n_dir + d), r.nl2 = __ldg(dt_ + 5 * n_dir + d);
  r.e10 = __ldg(dt_ + 6 * n_dir + d), r.e11 = __ldg(dt_ + 7 * n_dir + d), r.e12 = __ldg(dt_ + 8 * n_dir + d);
  r.e20 = __ldg(dt_ + 9 * n_dir + d), r.e21 = __ldg(dt_ + 10 * n_dir + d), r.e22 = __ldg(dt_ + 11 * n_dir + d);
  return r;
}

// The same row staged in shared memory as 12 consecutive floats (16-byte aligned).
__device__ __forceinline__ DirRow dir_row_staged(const float* s) {
  const float4 a = reinterpret_cast<const float4*>(s)[0];
  const float4 b = reinterpret_cast<const float4*>(s)[1];
  const float4 c = reinterpret_cast<const float4*>(s)[2];
  return DirRow{a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, c.x, c.y, c.z, c.w};
}

// Stage 1: record of (particle, direction).  raw: the particle's 80-byte record.
// Returns false when |dtau| is beyond the fast phase path's range.
__device__ __forceinline__ bool compute_record(const float* __restrict__ raw, const DirRow& dr,
                                               float tau_fast, float& th, float& tl, float amp[4]) {
  const float4 q0 = *reinterpret_cast<const float4*>(raw);
  const float4 q1 = *reinterpret_cast<const float4*>(raw + 4);
  const float4 q2 = *reinterpret_cast<const float4*>(raw + 8);
  const float4 q3 = *reinterpret_cast<const float4*>(raw + 12);
  const float2 q4 = *reinterpret_cast<const float2*>(raw + 16);
  const float sh0 = q0.x, sh1 = q0.y, sh2 = q0.z, sl0 = q0.w, sl1 = q1.x, sl2 = q1.y;
  const float bh0 = q1.z, bh1 = q1.w, bh2 = q2.x, bl0 = q2.y, bl1 = q2.z, bl2 = q2.w;
  const float ad0 = q3.x, ad1 = q3.y, ad2 = q3.z, g2 = q3.w, ww = q4.x, sw = q4.y;
  const float nh0 = dr.nh0, nh1 = dr.nh1, nh2 = dr.nh2, nl0 = dr.nl0, nl1 = dr.nl1, nl2 = dr.nl2;
  const float e10 = dr.e10, e11 = dr.e11, e12 = dr.e12, e20 = dr.e20, e21 = dr.e21, e22 = dr.e22;

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
  th = -hi;
  tl = -lo2;

  // Transverse amplitude (see the file comment).
  const float b1 = fmaf(e10, bh0, fmaf(e11, bh1, e12 * bh2)) + fmaf(e10, bl0, fmaf(e11, bl1, e12 * bl2));
  const float b2 = fmaf(e20, bh0, fmaf(e21, bh1, e22 * bh2)) + fmaf(e20, bl0, fmaf(e21, bl1, e22 * bl2));
  const float bn = fmaf(nh0, bh0, fmaf(nh1, bh1, nh2 * bh2));
  const float d1 = fmaf(e10, ad0, fmaf(e11, ad1, e12 * ad2));
  const float d2 = fmaf(e20, ad0, fmaf(e21, ad1, e22 * ad2));
  const float dn = fmaf(nh0, ad0, fmaf(nh1, ad1, nh2 * ad2));
  // Approximate reciprocals (about 1 ulp): a relative error of a few 1e-7 in
  // the amplitude, far below what the TF32 and MUFU steps leave.
  const float D = (g2 + fmaf(b1, b1, b2 * b2)) * rcp_approx(1.0f + bn);
  const float iD = rcp_approx(D);
  const float iD2 = iD * iD;
  const float a1 = -fmaf(b1, dn, d1 * D) * iD2;
  const float a2 = -fmaf(b2, dn, d2 * D) * iD2;
  amp[0] = ww * a1;  // U . e1
  amp[1] = ww * a2;  // U . e2
  amp[2] = sw * a1;  // V . e1
  amp[3] = sw * a2;  // V . e2
  return fabsf(th) <= tau_fast;  // false for NaN as well
}

__device__ __forceinline__ bool compute_record(const float* __restrict__ raw,
                                               const float* __restrict__ dt_, int n_dir, int d,
                                               float tau_fast, float& th, float& tl, float amp[4]) {
  return compute_record(raw, dir_row(dt_, n_dir, d), tau_fast, th, tl, amp);
}

// Shared memory: one raw particle tile (THREADS x 80 B, TMA destination) and
// two record buffers.  FP32 variants: per record 3 float4 (values duplicated
// for packed arithmetic); tensor-core variants: float2 dtau + 8 floats of
// amplitude hi/lo parts; with the cross terms on tensor cores (variant 9),
// dtau hi + 8 floats of TF32 parts of dtau + 12 floats (8 used) of amplitude
// hi/lo parts.
// Tensor-core variants also keep their per-chunk (second-level) sums in
// shared memory: 8 floats per thread and 16-frequency block of a warp (16 or
// 32 per thread), one slot per thread and value.
// The literal variant adds a fourth float4 per record: (w - 1) duplicated.

// Phase of a frequency pair (packed) for one particle: returns radians in
// (-pi, pi] + a tiny cross-term excess.
__device__ __forceinline__ float2 phase2(float2 omh, float2 wh, float2 wl, float2 th, float2 tl) {
  const float2 kMag = make_float2(12582912.0f, 12582912.0f);  // 1.5 * 2^23
  const float2 k2Pi = make_float2(6.28318530717958647692f, 6.28318530717958647692f);
  const float2 t0 = __ffma2_rn(omh, th, kMag);                     // 1.5*2^23 + rint(x)
  const float2 q = __fadd2_rn(kMag, make_float2(-t0.x, -t0.y));   // -rint(x), exact
  const float2 f0 = __ffma2_rn(omh, th, q);                        // x - rint(x), one rounding
  const float2 c1 = __fmul2_rn(wl, th);                            // cross terms, radians
  const float2 c2 = __ffma2_rn(wh, tl, c1);
  return __ffma2_rn(f0, k2Pi, c2);
}

// Phase of one frequency for a particle pair (packed over the particles): om2
// holds omega/2pi (hi) in both halves, th2 the two particles' dtau hi parts, cr
// their cross terms 2pi (omega_lo th + omega_hi tl) in radians, formed
// elsewhere.  The turns om th are reduced exactly as in phase2.
__device__ __forceinline__ float2 phase2x(float2 om2, float2 th2, float2 cr) {
  const float2 kMag = make_float2(12582912.0f, 12582912.0f);  // 1.5 * 2^23
  const float2 k2Pi = make_float2(6.28318530717958647692f, 6.28318530717958647692f);
  const float2 t0 = __ffma2_rn(om2, th2, kMag);
  const float2 q = __fadd2_rn(kMag, make_float2(-t0.x, -t0.y));
  const float2 f0 = __ffma2_rn(om2, th2, q);
  return __ffma2_rn(f0, k2Pi, cr);
}

// Phase in FP64 (wide path): omega/2pi times the float-float dtau plus an
// offset (the tile group's reference time in a wide call), reduced.
__device__ __forceinline__ float phase_wide(double om_turns, float th, float tl, double off = 0.0) {
  double x = om_turns * ((double)th + (double)tl + off);
  x -= rint(x);
  return (float)(x * 6.283185307179586);
}

// e^{i 2 pi omega_turns tau} in FP32 (tau: a group's reference time in a wide
// call, up to ~1e-11 s), the phase reduced in FP64.
__device__ __forceinline__ void group_rotation(double om_turns, double tau, float& c, float& s) {
  double x = om_turns * tau;
  x -= rint(x);
  const float ph = (float)(x * 6.283185307179586);
  c = cos_approx(ph);
  s = sin_approx(ph);
}

// ---- the tensor-core update block (shared with the loop probe) ----

constexpr uint32_t kTf32Mask = 0xFFFFE000u;  // sign, exponent, 10 mantissa bits

__device__ __forceinline__ void mma_tf32(float d[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                         uint32_t a3, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t tf32_hi(float x) { return __float_as_uint(x) & kTf32Mask; }

// Splits a packed pair into TF32 hi bits and the exact FP32 rest.
__device__ __forceinline__ void split_pair(float2 v, uint32_t& h0, uint32_t& h1, float2& lo) {
  h0 = tf32_hi(v.x);
  h1 = tf32_hi(v.y);
  lo = __fadd2_rn(v, make_float2(-__uint_as_float(h0), -__uint_as_float(h1)));
}

// The TF32 value nearest to x (ties away from zero), as bits.
__device__ __forceinline__ uint32_t tf32_rna(float x) {
  uint32_t y;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(y) : "f"(x));
  return y;
}

// x ~ hi + lo, both TF32 values, |x - hi - lo| <= 2^-22 |x|.
__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
  hi = tf32_rna(x);
  lo = tf32_rna(__fsub_rn(x, __uint_as_float(hi)));
}

// d = A B (m16n8k8 TF32, zero accumulator).
__device__ __forceinline__ void mma_tf32_zero(float d[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                              uint32_t a3, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%10,%10,%10,%10};"
      : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1), "f"(0.0f));
}

// One 16-frequency x 8-particle MMA block: pA / pB are the phases of the
// frequency rows (r, r+8) for particles (c, c+4) of the fragment layout.
__device__ __forceinline__ void tc_block(float2 pA, float2 pB, uint32_t b0, uint32_t b1,
                                         float dre[4], float dim[4]) {
  const float2 cA = make_float2(cos_approx(pA.x), cos_approx(pA.y));
  const float2 sA = make_float2(sin_approx(pA.x), sin_approx(pA.y));
  const float2 cB = make_float2(cos_approx(pB.x), cos_approx(pB.y));
  const float2 sB = make_float2(sin_approx(pB.x), sin_approx(pB.y));
  uint32_t ca0, ca1, cb0, cb1, sa0, sa1, sb0, sb1;
  float2 caL, cbL, saL, sbL;
  split_pair(cA, ca0, ca1, caL);
  split_pair(cB, cb0, cb1, cbL);
  split_pair(sA, sa0, sa1, saL);
  split_pair(sB, sb0, sb1, sbL);
  // A fragment (m16n8k8 tf32): a0 = (row r, k c), a1 = (r+8, c), a2 = (r, c+4), a3 = (r+8, c+4)
  mma_tf32(dre, ca0, ca1, cb0, cb1, b0, b1);
  mma_tf32(dre, __float_as_uint(caL.x), __float_as_uint(caL.y), __float_as_uint(cbL.x),
           __float_as_uint(cbL.y), b0, b1);
  mma_tf32(dim, sa0, sa1, sb0, sb1, b0, b1);
  mma_tf32(dim, __float_as_uint(saL.x), __float_as_uint(saL.y), __float_as_uint(sbL.x),
           __float_as_uint(sbL.y), b0, b1);
}

}  // namespace dev
}  // namespace radimpl
