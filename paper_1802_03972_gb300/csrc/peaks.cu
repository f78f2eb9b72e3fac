// Pipe-throughput microbenchmarks for the roofline denominators of the
// radiation kernel: FP32 FMA (scalar and packed f32x2), MUFU sin/cos, FP64
// FMA, float rounding and f64<->f32 conversion, and one mixed loop with the
// op mix of the phase-accumulate inner loop (2 MUFU + packed FMAs).
//
// Each kernel runs independent dependency chains per thread so the pipe, not
// latency, limits it; a block records its start/end SM cycle counter, so the
// rates come out per SM clock cycle, independent of the clock the GPU ran at.
// Entry point: rad_probe_peaks() (C ABI), results in lane-ops / clk / SM.
#include <cuda_runtime.h>
#include <stdint.h>

#include "rad_stage.cuh"

namespace {

constexpr int kThreads = 512;

// Block b records its start and end SM cycle counts and the SM it ran on in
// cyc[3b .. 3b + 2]; the host rates each SM over the span of all its blocks.
__device__ __forceinline__ void stamp(long long* cyc, long long t0) {
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned sm;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(sm));
    cyc[3 * blockIdx.x] = t0;
    cyc[3 * blockIdx.x + 1] = clock64();
    cyc[3 * blockIdx.x + 2] = (long long)sm;
  }
}

__global__ void __launch_bounds__(kThreads) k_ffma(float* out, long long* cyc, int iters, float a, float b) {
  long long t0 = clock64();
  float x[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) x[i] = threadIdx.x * 1e-3f + i;
#pragma unroll 2
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = fmaf(x[i], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += x[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
  stamp(cyc, t0);
}

__global__ void __launch_bounds__(kThreads) k_ffma2(float* out, long long* cyc, int iters, float a, float b) {
  long long t0 = clock64();
  float2 x[8];
  const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
#pragma unroll
  for (int i = 0; i < 8; ++i) x[i] = make_float2(threadIdx.x * 1e-3f + i, i * 0.5f);
#pragma unroll 2
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = __ffma2_rn(x[i], a2, b2);
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += x[i].x + x[i].y;
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
  stamp(cyc, t0);
}

__device__ __forceinline__ float sin_approx(float x) {
  float y;
  asm volatile("sin.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float cos_approx(float x) {
  float y;
  asm volatile("cos.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__global__ void __launch_bounds__(kThreads) k_mufu(float* out, long long* cyc, int iters) {
  long long t0 = clock64();
  float x[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) x[i] = threadIdx.x * 1e-3f + i * 0.1f;
#pragma unroll 2
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; i += 2) {
      x[i] = sin_approx(x[i]);
      x[i + 1] = cos_approx(x[i + 1]);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += x[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
  stamp(cyc, t0);
}

__global__ void __launch_bounds__(kThreads) k_dfma(float* out, long long* cyc, int iters, double a, double b) {
  long long t0 = clock64();
  double x[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) x[i] = threadIdx.x * 1e-3 + i;
#pragma unroll 2
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = fma(x[i], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += x[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = (float)s;
  stamp(cyc, t0);
}

__global__ void __launch_bounds__(kThreads) k_frnd(float* out, long long* cyc, int iters, float a) {
  long long t0 = clock64();
  float x[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) x[i] = threadIdx.x * 1.3e-3f + i * 0.7f;
#pragma unroll 2
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      float r;
      asm volatile("cvt.rni.f32.f32 %0, %1;" : "=f"(r) : "f"(x[i]));
      x[i] = r + a;  // one FADD per round so the chain stays live
    }
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += x[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
  stamp(cyc, t0);
}

__global__ void __launch_bounds__(kThreads) k_cvt(float* out, long long* cyc, int iters) {
  long long t0 = clock64();
  double x[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) x[i] = threadIdx.x * 1e-3 + i;
#pragma unroll 2
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      float f = __double2float_rn(x[i]);   // cvt f64 -> f32
      x[i] = (double)(f * 1.0000001f);     // cvt f32 -> f64 (+1 FMUL)
    }
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += x[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = (float)s;
  stamp(cyc, t0);
}

// Mixed loop shaped like the phase-accumulate inner loop for one packed pair
// of frequencies: 2 sin + 2 cos MUFU ops and NF packed FMAs per iteration.
template <int NF>
__global__ void __launch_bounds__(kThreads) k_mix(float* out, long long* cyc, int iters, float a) {
  long long t0 = clock64();
  float2 acc[NF];
  float2 ph = make_float2(threadIdx.x * 1e-3f, threadIdx.x * 2e-3f);
  const float2 a2 = make_float2(a, a);
#pragma unroll
  for (int i = 0; i < NF; ++i) acc[i] = make_float2(0.f, 0.f);
#pragma unroll 2
  for (int it = 0; it < iters; ++it) {
    float2 c = make_float2(cos_approx(ph.x), cos_approx(ph.y));
    float2 s = make_float2(sin_approx(ph.x), sin_approx(ph.y));
#pragma unroll
    for (int i = 0; i < NF; i += 2) {
      acc[i] = __ffma2_rn(a2, c, acc[i]);
      acc[i + 1] = __ffma2_rn(a2, s, acc[i + 1]);
    }
    ph = __ffma2_rn(ph, a2, c);
  }
  float t = 0.f;
#pragma unroll
  for (int i = 0; i < NF; ++i) t += acc[i].x + acc[i].y;
  out[blockIdx.x * blockDim.x + threadIdx.x] = t;
  stamp(cyc, t0);
}


// ---- tensor pipes: legacy mma.sync and tcgen05.mma with A in tensor memory ----

constexpr unsigned long long kProbeWaitNs = 1000000000ULL;  // 1 s bound on any wait

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__global__ void __launch_bounds__(256) k_mma_sync(float* out, long long* cyc, int iters) {
  long long t0 = clock64();
  float d[4][4] = {};
  const uint32_t a = __float_as_uint(1.0001f + threadIdx.x), b = __float_as_uint(0.999f);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 4; ++j)
      asm volatile(
          "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
          "{%0,%1,%2,%3};"
          : "+f"(d[j][0]), "+f"(d[j][1]), "+f"(d[j][2]), "+f"(d[j][3])
          : "r"(a), "r"(a), "r"(a), "r"(a), "r"(b), "r"(b));
  }
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < 4; ++j) s += d[j][0] + d[j][1] + d[j][2] + d[j][3];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
  stamp(cyc, t0);
}

// Instruction descriptor of tcgen05.mma, dense, FP32 accumulator, K-major A and
// B: bits 4-5 D type (1 = F32), 7-9 / 10-12 A / B type (kind::f16: 0 = F16;
// kind::tf32: 2 = TF32), 17-22 N >> 3, 24-28 M >> 4.
__host__ __device__ constexpr uint32_t umma_idesc(bool tf32, int m, int n) {
  return (1u << 4) | ((tf32 ? 2u : 0u) << 7) | ((tf32 ? 2u : 0u) << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(m >> 4) << 24);
}

// One CTA of one warp per SM holds all 512 TMEM columns; lane 0 issues `n_mma`
// MMAs (M = 128, A from TMEM columns 0-63, D in columns 64.., B one 128-byte
// core matrix in shared memory read with zero strides) and times issue to
// completion with the SM cycle counter.
template <int N, bool TF32>
__global__ void __launch_bounds__(32, 1) k_umma(int n_mma, long long* cyc, int* err) {
  __shared__ __align__(128) float bcore[64];
  __shared__ __align__(8) uint64_t done;
  __shared__ uint32_t tbase;
  const int lane = threadIdx.x;
  for (int i = lane; i < 64; i += 32) bcore[i] = 1e-3f * (float)i;
  if (lane == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&done)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(su32(&tbase)) : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncwarp();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tb = tbase;
  if (lane == 0) {
    const uint64_t bdesc = (uint64_t)((su32(bcore) >> 4) & 0x3FFFu) | (1ull << 46);
    constexpr uint32_t id = umma_idesc(TF32, 128, N);
    const long long c0 = clock64();
    for (int i = 0; i < n_mma; ++i) {
      const uint32_t d = tb + 64u, a = tb + (uint32_t)((i & 7) * 8);
      if constexpr (TF32)
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d),
            "r"(a), "l"(bdesc), "r"(id), "r"(i > 0 ? 1 : 0)
            : "memory");
      else
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d),
            "r"(a), "l"(bdesc), "r"(id), "r"(i > 0 ? 1 : 0)
            : "memory");
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(&done))
                 : "memory");
    const unsigned long long t0 = globaltimer_ns();
    bool ok = false;
    while (!ok && globaltimer_ns() - t0 < kProbeWaitNs) {
      uint32_t r;
      asm volatile(
          "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}\n"
          : "=r"(r) : "r"(su32(&done)) : "memory");
      ok = r != 0;
    }
    if (!ok) atomicOr(err, 1);
    cyc[2 * blockIdx.x] = c0;
    cyc[2 * blockIdx.x + 1] = clock64();
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncwarp();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tb) : "memory");
}

// ---- the accumulate kernel's update loop with parts removed (timing only) ----
// One 256-particle tile of synthetic records in shared memory, swept `reps`
// times by 256 threads (2 blocks per SM, as the tensor-core kernels run), each
// warp holding four 16-frequency MMA blocks, the particle loop unrolled 8x, no
// barriers, no stage 1 and no epilogue.  MODE:
//   0  the variant-8 block: two packed phase reductions, the TF32 hi/lo split
//      and four mma.sync per 16-frequency x 8-particle block;
//   1  no split: the raw sin/cos bits go into the same four MMAs;
//   2  the split, no MMA: its outputs are folded by XOR (three-input LOP3s);
//   3  neither: sin/cos consumed by two packed FMAs;
//   4  the variant-9 block: the phase cross terms by one more mma.sync.
// The results are meaningless; only the pipes' throughput is of interest.
constexpr int kLoopNB = 4, kLoopKT = 256;

template <int MODE>
__device__ __forceinline__ void loop_block(float2 pA, float2 pB, uint32_t b0, uint32_t b1,
                                           float dre[4], float dim[4], uint32_t& xacc) {
  using namespace radimpl::dev;
  if constexpr (MODE == 0 || MODE == 4) {
    tc_block(pA, pB, b0, b1, dre, dim);
    return;
  }
  const float2 cA = make_float2(cos_approx(pA.x), cos_approx(pA.y));
  const float2 sA = make_float2(sin_approx(pA.x), sin_approx(pA.y));
  const float2 cB = make_float2(cos_approx(pB.x), cos_approx(pB.y));
  const float2 sB = make_float2(sin_approx(pB.x), sin_approx(pB.y));
  if constexpr (MODE == 1) {
    mma_tf32(dre, __float_as_uint(cA.x), __float_as_uint(cA.y), __float_as_uint(cB.x), __float_as_uint(cB.y), b0, b1);
    mma_tf32(dre, __float_as_uint(cA.y), __float_as_uint(cA.x), __float_as_uint(cB.y), __float_as_uint(cB.x), b0, b1);
    mma_tf32(dim, __float_as_uint(sA.x), __float_as_uint(sA.y), __float_as_uint(sB.x), __float_as_uint(sB.y), b0, b1);
    mma_tf32(dim, __float_as_uint(sA.y), __float_as_uint(sA.x), __float_as_uint(sB.y), __float_as_uint(sB.x), b0, b1);
  } else if constexpr (MODE == 3) {
    const float2 bb = make_float2(__uint_as_float(b0), __uint_as_float(b1));
    float2* r = reinterpret_cast<float2*>(dre);
    float2* i = reinterpret_cast<float2*>(dim);
    r[0] = __ffma2_rn(cA, bb, r[0]);
    r[1] = __ffma2_rn(cB, bb, r[1]);
    i[0] = __ffma2_rn(sA, bb, i[0]);
    i[1] = __ffma2_rn(sB, bb, i[1]);
  } else {
    uint32_t h[8];
    float2 lo[4];
    split_pair(cA, h[0], h[1], lo[0]);
    split_pair(cB, h[2], h[3], lo[1]);
    split_pair(sA, h[4], h[5], lo[2]);
    split_pair(sB, h[6], h[7], lo[3]);
    uint32_t x = xacc;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      asm("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(x) : "r"(x), "r"(h[2 * k]), "r"(h[2 * k + 1]));
      asm("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(x) : "r"(x), "r"(__float_as_uint(lo[k].x)), "r"(__float_as_uint(lo[k].y)));
    }
    xacc = x;
  }
}

template <int MODE>
__global__ void __launch_bounds__(256, 2) k_loop(float* out, long long* cyc, int reps) {
  using namespace radimpl::dev;
  __shared__ float2 tw[kLoopKT];
  __shared__ float aw[kLoopKT * 8];
  const int t = threadIdx.x;
  tw[t] = make_float2(6.0e-14f * (float)((t * 37) % 256 - 128) / 128.0f, 1.0e-21f * (float)(t % 7 - 3));
  for (int j = 0; j < 8; ++j) aw[t * 8 + j] = 1.0f + 0.01f * (float)((t + j) % 13);
  __syncthreads();
  const int warp = t >> 5, lane = t & 31, r = lane >> 2, c = lane & 3;
  float2 omh[kLoopNB], wh[kLoopNB], wl[kLoopNB], omr[kLoopNB], omr8[kLoopNB];
  uint32_t xa[kLoopNB][4];
  float dre[kLoopNB][4], dim[kLoopNB][4];
  for (int b = 0; b < kLoopNB; ++b) {
    const float f0 = 1.6e13f * __powf(1.0276f, (float)(warp * 64 + 16 * b + r)), f1 = f0 * 1.2456f;
    omh[b] = make_float2(f0, f1);
    wh[b] = make_float2(6.2831855f * f0, 6.2831855f * f1);
    wl[b] = make_float2(1e-7f * f0, 1e-7f * f1);
    omr[b] = make_float2(f0, f0);
    omr8[b] = make_float2(f1, f1);
    for (int i = 0; i < 4; ++i) xa[b][i] = tf32_hi(wl[b].x * (float)(1 + i));
    for (int e = 0; e < 4; ++e) dre[b][e] = dim[b][e] = 0.0f;
  }
  uint32_t xacc = 0;
  __syncthreads();
  const long long t0 = clock64();
  for (int rep = 0; rep < reps; ++rep) {
#pragma unroll 8
    for (int kk = 0; kk < kLoopKT; kk += 8) {
      if constexpr (MODE == 4) {
        const float2 th2 = make_float2(tw[kk + 2 * c].x, tw[kk + 2 * c + 1].x);
        const uint32_t r0 = tf32_hi(aw[(kk + r) * 8 + 2 * c]), r1 = tf32_hi(aw[(kk + r) * 8 + 2 * c + 1]);
        const uint32_t b0 = __float_as_uint(aw[(kk + 2 * c) * 8 + r]);
        const uint32_t b1 = __float_as_uint(aw[(kk + 2 * c + 1) * 8 + r]);
#pragma unroll
        for (int b = 0; b < kLoopNB; ++b) {
          float cr[4];
          mma_tf32_zero(cr, xa[b][0], xa[b][1], xa[b][2], xa[b][3], r0, r1);
          const float2 p0 = phase2x(omr[b], th2, make_float2(cr[0], cr[1]));
          const float2 p8 = phase2x(omr8[b], th2, make_float2(cr[2], cr[3]));
          loop_block<MODE>(make_float2(p0.x, p8.x), make_float2(p0.y, p8.y), b0, b1, dre[b], dim[b], xacc);
        }
      } else {
        const float2 tA = tw[kk + c], tB = tw[kk + c + 4];
        const uint32_t b0 = __float_as_uint(aw[(kk + c) * 8 + r]);
        const uint32_t b1 = __float_as_uint(aw[(kk + c + 4) * 8 + r]);
        const float2 thA = make_float2(tA.x, tA.x), tlA = make_float2(tA.y, tA.y);
        const float2 thB = make_float2(tB.x, tB.x), tlB = make_float2(tB.y, tB.y);
#pragma unroll
        for (int b = 0; b < kLoopNB; ++b) {
          const float2 pA = phase2(omh[b], wh[b], wl[b], thA, tlA);
          const float2 pB = phase2(omh[b], wh[b], wl[b], thB, tlB);
          loop_block<MODE>(pA, pB, b0, b1, dre[b], dim[b], xacc);
        }
      }
    }
  }
  const long long t1 = clock64();
  float sum = (float)xacc;
  for (int b = 0; b < kLoopNB; ++b)
    for (int e = 0; e < 4; ++e) sum += dre[b][e] + dim[b][e];
  out[blockIdx.x * blockDim.x + t] = sum;
  __syncthreads();
  if (t == 0) {
    unsigned sm;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(sm));
    cyc[3 * blockIdx.x] = t0;
    cyc[3 * blockIdx.x + 1] = t1;
    cyc[3 * blockIdx.x + 2] = (long long)sm;
  }
}

// Operations per SM clock and the effective clock (MHz) of a probe launch of
// nb blocks, each doing ops_per_block operations: every SM is timed from its
// first block's start to its last block's end, so blocks that an SM ran one
// after another are not counted as concurrent.
void rate_per_sm(const long long* h, int nb, double ops_per_block, float ms, int n_sm_max,
                 double* rate, double* mhz) {
  long long* first = new long long[n_sm_max];
  long long* last = new long long[n_sm_max];
  int* cnt = new int[n_sm_max];
  for (int i = 0; i < n_sm_max; ++i) {
    cnt[i] = 0;
    first[i] = last[i] = 0;
  }
  for (int b = 0; b < nb; ++b) {
    const long long sm = h[3 * b + 2];
    if (sm < 0 || sm >= n_sm_max) continue;
    if (cnt[sm] == 0 || h[3 * b] < first[sm]) first[sm] = h[3 * b];
    if (cnt[sm] == 0 || h[3 * b + 1] > last[sm]) last[sm] = h[3 * b + 1];
    cnt[sm]++;
  }
  double ops = 0.0, span = 0.0;
  int sms = 0;
  for (int i = 0; i < n_sm_max; ++i) {
    if (cnt[i] == 0) continue;
    ops += ops_per_block * cnt[i];
    span += (double)(last[i] - first[i]);
    sms++;
  }
  *rate = span > 0 ? ops / span : 0.0;
  *mhz = sms > 0 && ms > 0 ? span / sms / (ms * 1e-3) / 1e6 : 0.0;
  delete[] first;
  delete[] last;
  delete[] cnt;
}

}  // namespace

extern "C" {

// Runs every probe once (after one warm-up launch each) on the current device.
// out[] receives, per probe, lane-ops per SM clock cycle, then the effective SM
// clock in MHz seen by that probe:
//   [0,1] FFMA scalar      [2,3] FFMA2 (lane-ops = 2 per lane per instr)
//   [4,5] MUFU sin/cos     [6,7] DFMA
//   [8,9] FRND (+1 FADD)   [10,11] cvt f64->f32->f64 pairs (2 cvt per step)
//   [12,13] mixed, MUFU ops/clk/SM with 8 FFMA2 per 4 MUFU
//   [14,15] mixed, MUFU ops/clk/SM with 16 FFMA2 per 4 MUFU
// Returns 0 on success, otherwise the CUDA error code. n_out must be >= 16.
int rad_probe_peaks(double* out, int n_out) {
  if (out == nullptr || n_out < 16) return (int)cudaErrorInvalidValue;
  int dev = 0, n_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  // Every probe launches exactly one wave: n_sm x (its resident blocks per SM).
  const int max_per_sm = 2048 / kThreads;
  const int blocks = n_sm * max_per_sm;
  float* d_out = nullptr;
  long long* d_cyc = nullptr;
  cudaError_t e = cudaMalloc(&d_out, sizeof(float) * blocks * kThreads);
  if (e != cudaSuccess) return (int)e;
  e = cudaMalloc(&d_cyc, sizeof(long long) * 3 * blocks);
  if (e != cudaSuccess) { cudaFree(d_out); return (int)e; }
  long long* h_cyc = new long long[3 * blocks];
  int sm_ids = 0;  // %smid may exceed the SM count; bound it by the attribute
  cudaDeviceGetAttribute(&sm_ids, cudaDevAttrMultiProcessorCount, dev);
  sm_ids = 2 * sm_ids + 64;
  cudaEvent_t ev0, ev1;
  cudaEventCreate(&ev0);
  cudaEventCreate(&ev1);

  auto measure = [&](const void* kern, auto launch, double ops_per_thread, double* res) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, 0);
    if (per_sm < 1) per_sm = 1;
    if (per_sm > max_per_sm) per_sm = max_per_sm;
    const int nb = n_sm * per_sm;
    launch(nb);  // warm-up
    cudaEventRecord(ev0);
    launch(nb);
    cudaEventRecord(ev1);
    cudaEventSynchronize(ev1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev0, ev1);
    cudaMemcpy(h_cyc, d_cyc, sizeof(long long) * 3 * nb, cudaMemcpyDeviceToHost);
    rate_per_sm(h_cyc, nb, ops_per_thread * kThreads, ms, sm_ids, &res[0], &res[1]);
  };

  const int it = 1 << 14;
  measure((const void*)k_ffma, [&](int nb) { k_ffma<<<nb, kThreads>>>(d_out, d_cyc, it, 0.999f, 1e-3f); }, 8.0 * it, out + 0);
  measure((const void*)k_ffma2, [&](int nb) { k_ffma2<<<nb, kThreads>>>(d_out, d_cyc, it, 0.999f, 1e-3f); }, 16.0 * it, out + 2);
  measure((const void*)k_mufu, [&](int nb) { k_mufu<<<nb, kThreads>>>(d_out, d_cyc, it / 4); }, 8.0 * (it / 4), out + 4);
  measure((const void*)k_dfma, [&](int nb) { k_dfma<<<nb, kThreads>>>(d_out, d_cyc, it / 16, 0.999, 1e-3); }, 8.0 * (it / 16), out + 6);
  measure((const void*)k_frnd, [&](int nb) { k_frnd<<<nb, kThreads>>>(d_out, d_cyc, it / 4, 0.25f); }, 8.0 * (it / 4), out + 8);
  measure((const void*)k_cvt, [&](int nb) { k_cvt<<<nb, kThreads>>>(d_out, d_cyc, it / 16); }, 16.0 * (it / 16), out + 10);
  measure((const void*)k_mix<8>, [&](int nb) { k_mix<8><<<nb, kThreads>>>(d_out, d_cyc, it / 4, 0.999f); }, 4.0 * (it / 4), out + 12);
  measure((const void*)k_mix<16>, [&](int nb) { k_mix<16><<<nb, kThreads>>>(d_out, d_cyc, it / 4, 0.999f); }, 4.0 * (it / 4), out + 14);

  e = cudaGetLastError();
  cudaEventDestroy(ev0);
  cudaEventDestroy(ev1);
  delete[] h_cyc;
  cudaFree(d_out);
  cudaFree(d_cyc);
  return (int)e;
}


// Tensor pipes: out[0] legacy mma.sync m16n8k8 TF32 MACs / clk / SM; then SM
// cycles per tcgen05.mma (M = 128, A in tensor memory) for kind::tf32 at
// N = 16, 64, 128, 256 (out[1..4]) and kind::f16 at N = 16, 256 (out[5], out[6]);
// out[7] the effective clock (MHz) of the mma.sync probe.
int rad_probe_tensor(double* out, int n_out) {
  if (out == nullptr || n_out < 8) return (int)cudaErrorInvalidValue;
  int dev = 0, n_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  const int per_sm = 4, blocks = n_sm * per_sm;
  float* d_out = nullptr;
  long long* d_cyc = nullptr;
  int* d_err = nullptr;
  cudaError_t e = cudaMalloc(&d_out, sizeof(float) * blocks * 256);
  if (e == cudaSuccess) e = cudaMalloc(&d_cyc, sizeof(long long) * 3 * blocks);
  if (e == cudaSuccess) e = cudaMalloc(&d_err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(d_err, 0, sizeof(int));
  long long* h_cyc = new long long[3 * blocks];
  const int sm_ids = 2 * n_sm + 64;
  cudaEvent_t ev0, ev1;
  cudaEventCreate(&ev0);
  cudaEventCreate(&ev1);
  if (e == cudaSuccess) {
    const int iters = 4096;
    k_mma_sync<<<blocks, 256>>>(d_out, d_cyc, 16);
    cudaEventRecord(ev0);
    k_mma_sync<<<blocks, 256>>>(d_out, d_cyc, iters);
    cudaEventRecord(ev1);
    cudaEventSynchronize(ev1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev0, ev1);
    cudaMemcpy(h_cyc, d_cyc, sizeof(long long) * 3 * blocks, cudaMemcpyDeviceToHost);
    // multiply-adds per block: 8 warps x iters x 4 MMAs x (16 x 8 x 8)
    rate_per_sm(h_cyc, blocks, 8.0 * iters * 4 * 16 * 8 * 8, ms, sm_ids, &out[0], &out[7]);
  }
  auto umma = [&](auto kern, double* res) {
    if (e != cudaSuccess) return;
    const int n_mma = 4096;
    kern<<<n_sm, 32>>>(64, d_cyc, d_err);
    kern<<<n_sm, 32>>>(n_mma, d_cyc, d_err);
    e = cudaDeviceSynchronize();
    int err = 0;
    cudaMemcpy(&err, d_err, sizeof(int), cudaMemcpyDeviceToHost);
    cudaMemcpy(h_cyc, d_cyc, sizeof(long long) * 2 * n_sm, cudaMemcpyDeviceToHost);
    double cyc_sum = 0.0;
    for (int b = 0; b < n_sm; ++b) cyc_sum += (double)(h_cyc[2 * b + 1] - h_cyc[2 * b]);
    *res = err ? -1.0 : cyc_sum / n_sm / n_mma;
  };
  umma(k_umma<16, true>, out + 1);
  umma(k_umma<64, true>, out + 2);
  umma(k_umma<128, true>, out + 3);
  umma(k_umma<256, true>, out + 4);
  umma(k_umma<16, false>, out + 5);
  umma(k_umma<256, false>, out + 6);
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(ev0);
  cudaEventDestroy(ev1);
  delete[] h_cyc;
  cudaFree(d_out);
  cudaFree(d_cyc);
  cudaFree(d_err);
  return (int)e;
}

// The update loop with parts removed (k_loop): out[2 m], out[2 m + 1] = MUFU
// lane-ops per SM clock and the effective clock (MHz) of mode m = 0..4.
int rad_probe_loop(double* out, int n_out) {
  if (out == nullptr || n_out < 10) return (int)cudaErrorInvalidValue;
  int dev = 0, n_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = n_sm * 2;
  float* d_out = nullptr;
  long long* d_cyc = nullptr;
  cudaError_t e = cudaMalloc(&d_out, sizeof(float) * blocks * 256);
  if (e == cudaSuccess) e = cudaMalloc(&d_cyc, sizeof(long long) * 3 * blocks);
  long long* h_cyc = new long long[3 * blocks];
  const int sm_ids = 2 * n_sm + 64;
  cudaEvent_t ev0, ev1;
  cudaEventCreate(&ev0);
  cudaEventCreate(&ev1);
  const int reps = 200;
  // MUFU lane-ops per block: 256 threads x reps x 32 steps x 4 MMA blocks x 8
  const double ops = 256.0 * reps * (kLoopKT / 8) * kLoopNB * 8;
  auto run = [&](auto kern, double* res) {
    if (e != cudaSuccess) return;
    kern<<<blocks, 256>>>(d_out, d_cyc, 2);
    cudaEventRecord(ev0);
    kern<<<blocks, 256>>>(d_out, d_cyc, reps);
    cudaEventRecord(ev1);
    e = cudaEventSynchronize(ev1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev0, ev1);
    if (e == cudaSuccess) e = cudaMemcpy(h_cyc, d_cyc, sizeof(long long) * 3 * blocks, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) rate_per_sm(h_cyc, blocks, ops, ms, sm_ids, &res[0], &res[1]);
  };
  run(k_loop<0>, out + 0);
  run(k_loop<1>, out + 2);
  run(k_loop<2>, out + 4);
  run(k_loop<3>, out + 6);
  run(k_loop<4>, out + 8);
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(ev0);
  cudaEventDestroy(ev1);
  delete[] h_cyc;
  cudaFree(d_out);
  cudaFree(d_cyc);
  return (int)e;
}

}  // extern "C"
