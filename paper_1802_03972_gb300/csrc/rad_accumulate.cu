// The accumulate kernel of the far-field radiation sum (Pausch et al. 2018,
// Eq. 1 and the in-situ inner sum of Eq. 13).
//
// Persistent: one CTA per resident slot takes dynamic work items (job, bin
// tile, particle chunk).  A bin tile is NT directions x WT frequencies; the
// chunk's particle records (80 B each, written by the pre-pass) stream through
// shared memory in tiles of THREADS / NT particles, fetched by a TMA bulk copy
// (cp.async.bulk + mbarrier, time-bounded wait) one tile ahead of use.
//
// Stage 1, one (particle, direction) record per thread, FP32: the retarded-time
// offset dtau = -n.(r - r_ref)/c as a float-float pair (TwoProduct with fma,
// TwoSum), and the transverse amplitude components a_i = e_i . A in a basis
// (e1, e2) perpendicular to n.  n . A = 0 (Eq. 1), so these two carry |A|^2;
// with u = n - beta, n x (u x bdot) = u (n.bdot) - bdot D,
// D = 1 - beta.n = (1/gamma^2 + b1^2 + b2^2) / (1 + beta.n) and e_i.u = -b_i,
// a_i = -(b_i (n.bdot) + (e_i.bdot) D) / D^2, free of cancellation at high
// gamma.  Records are double-buffered, one barrier per particle tile.
//
// Stage 2, per (particle, direction, frequency), the "amplitude update": the
// phase in turns p = (omega/2pi) dtau is reduced exactly by one fused multiply-
// add against 1.5 * 2^23 (no FRND, which shares the MUFU pipe), the float-float
// cross terms are added in radians, and sin/cos come from the MUFU (2 per
// update).  The weighted sums U_i += w dt a_i e^{i phi}, V_i += sqrt(w) dt a_i
// e^{i phi} are then formed in one of two ways:
//  * FP32 variants: 8 packed FMAs (f32x2) per update into register accumulators,
//    two frequencies per packed lane pair;
//  * tensor-core variants: per warp, each 16-frequency x 8-particle block of
//    e^{i phi} (two or four blocks per warp) is the A operand of mma.sync
//    m16n8k8 TF32 and the 4 weighted amplitudes of the 8 particles are B.  Both are split into TF32 hi and lo
//    parts (hi = the top 19 bits, lo = the exact rest), B's hi and lo side by
//    side in the 8 N-columns, so two MMAs per cos/sin give all of
//    hi.hi + hi.lo + lo.hi + lo.lo with FP32 accumulation.  This takes the
//    accumulation FMAs off the FP32 pipe, which together with the phase
//    arithmetic and MUFU issue is what limits the FP32 variants.
// Wide calls (particles spread beyond the fast phase range about the call's
// reference point, sorted by the wide-call kernels) run in a second
// instantiation (WIDE): their records are relative to the first particle of
// each 256-particle group, so stage 1 and the update loop are unchanged, and
// each tile's sums are rotated by e^{i omega tau_group} before they join the
// chunk sums.
// Sums are two-level (per particle tile, then per chunk).  Each work item
// writes its partial sums; the last item of a bin tile to finish (an arrival
// counter, no float atomics) adds the partials in chunk order, multiplies by
// e^{i omega tau_ref(n)} (reduced in FP64) and adds the result into the
// resident state with compensated (Kahan) FP32 sums.  Results are
// deterministic for a given tile configuration.  Work items are handed out
// tile-major, so a tile's partials are still in L2 when they are added up;
// the tensor-core variants then drop those lines from L2 unwritten.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <atomic>

#include "rad_device.cuh"
#include "rad_impl.h"
#include "rad_stage.cuh"

namespace radimpl {

namespace {

using namespace dev;


template <int THREADS, bool TC, bool LIT = false, int PASSES = 1, bool XT = false>
struct Smem {
  static constexpr size_t raw_bytes = (size_t)THREADS * kRecFields * sizeof(float);
  static constexpr size_t rec_bytes = (size_t)THREADS * (XT ? 84 : TC ? 40 : (LIT ? 64 : 48));
  static constexpr size_t l2_bytes = TC ? (size_t)THREADS * 16 * sizeof(float) * PASSES : 0;
  // XT: the tile's direction rows (12 floats each; at most THREADS / 8 directions)
  static constexpr size_t dir_bytes = XT ? (size_t)(THREADS / 8) * 12 * sizeof(float) : 0;
  static constexpr size_t bytes = raw_bytes + 2 * rec_bytes + l2_bytes + dir_bytes;
};

struct TileGeom {
  int WT, NT, KT, d0, o0;
};

__device__ __forceinline__ TileGeom tile_geom(const JobStatic& J, int tile, int threads) {
  TileGeom g;
  g.WT = J.wt;
  g.NT = J.nt;
  g.KT = threads / g.NT;
  const int tile_d = tile / J.tiles_om;
  g.d0 = tile_d * g.NT;
  g.o0 = (tile - tile_d * J.tiles_om) * g.WT;
  return g;
}

// A work item: its tile and particle chunk, and the chunking of that tile.
// fine: the tile's index among the tiles of its fine-chunked level (TailPlan),
// -1 for the coarse tiles.  (The level itself follows from the tile and the
// call; the item, live across the whole particle loop, holds no more.)
struct ItemRef {
  int tile, chunk, ck, n_chunks, fine;
};

// Item `local` of a job: the coarse tiles' items tile-major, then level 0's
// fine tiles' items, then level 1's, each tile-major.  FINE = false: the
// FP32 variants, whose jobs are never fine-chunked (every item coarse).
template <bool FINE>
__device__ __forceinline__ ItemRef decode_item(const JobStatic& J, const JobCall& K,
                                               long long local) {
  static_assert(kTailLevels == 2, "two fine levels");
  ItemRef it;
  const int first0 = FINE ? J.n_tiles - K.tail_tiles[0] - K.tail_tiles[1] : J.n_tiles;
  const long long coarse = (long long)first0 * K.n_chunks;
  const long long fine0 = (long long)K.tail_tiles[0] * K.n_chunks_f[0];
  if (!FINE || local < coarse) {
    it.tile = (int)(local / K.n_chunks);
    it.chunk = (int)(local - (long long)it.tile * K.n_chunks);
    it.ck = K.ck;
    it.n_chunks = K.n_chunks;
    it.fine = -1;
  } else if (local - coarse < fine0) {
    const long long l = local - coarse;
    it.fine = (int)(l / K.n_chunks_f[0]);
    it.tile = first0 + it.fine;
    it.chunk = (int)(l - (long long)it.fine * K.n_chunks_f[0]);
    it.ck = K.ck_f[0];
    it.n_chunks = K.n_chunks_f[0];
  } else {
    const long long l = local - coarse - fine0;
    it.fine = (int)(l / K.n_chunks_f[1]);
    it.tile = first0 + K.tail_tiles[0] + it.fine;
    it.chunk = (int)(l - (long long)it.fine * K.n_chunks_f[1]);
    it.ck = K.ck_f[1];
    it.n_chunks = K.n_chunks_f[1];
  }
  return it;
}

// Where an item's partial sums live: component comp of chunk ch at
// base[ch * chunk_stride + comp * comp_stride + bin offset].  Coarse tiles:
// J.partials [chunk][comp][n_bins], the offset the bin; fine tiles: their
// level's region of J.partials_f, [chunk][comp][level tiles][NT WT], level 1's
// after level 0's, the offset the bin's index within the tile.  room: the
// floats from the start of the item's buffer or region.
struct PartMap {
  float* base;
  size_t chunk_stride, comp_stride;
  long long room;
};
__device__ __forceinline__ PartMap part_map(const JobStatic& J, const JobCall& K, const ItemRef& it,
                                            const TileGeom& g) {
  PartMap m;
  if (it.fine < 0) {
    m.base = J.partials;
    m.comp_stride = (size_t)J.n_bins;
    m.room = (long long)J.chunk_cap * kComps * J.n_bins;
  } else {
    const long long tb = (long long)g.NT * g.WT;
    const bool l1 = it.tile >= J.n_tiles - K.tail_tiles[1];
    const long long foff = l1 ? (long long)K.tail_tiles[0] * K.n_chunks_f[0] * kComps * tb : 0;
    m.base = J.partials_f + foff + (long long)it.fine * tb;
    m.comp_stride = (size_t)(l1 ? K.tail_tiles[1] : K.tail_tiles[0]) * tb;
    m.room = J.fine_cap - foff;
  }
  m.chunk_stride = (size_t)kComps * m.comp_stride;
  return m;
}
__device__ __forceinline__ size_t part_bin(const JobStatic& J, const ItemRef& it, const TileGeom& g,
                                           int d, int o) {
  return it.fine < 0 ? (size_t)d * J.n_omega + o : (size_t)(d - g.d0) * g.WT + (o - g.o0);
}

// Compensated (Kahan) add of x into sum with compensation cmp.
__device__ __forceinline__ void kahan_add(float* sum, float* cmp, float x) {
  const float y = __fsub_rn(x, *cmp);
  const float tt = __fadd_rn(*sum, y);
  *cmp = __fsub_rn(__fsub_rn(tt, *sum), y);
  *sum = tt;
}

// Arrival counter of the bin tile; true for the last work item of this call.
template <int THREADS>
__device__ __forceinline__ bool last_arrival(const JobStatic& J, const ItemRef& it, int* s_flag) {
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const int tile = it.tile;
    const unsigned prev = atomicAdd(&J.tile_cnt[tile], 1u);
    *s_flag = (prev == (unsigned)(it.n_chunks - 1));
    if (*s_flag) J.tile_cnt[tile] = 0u;  // ready for the next call
    __threadfence();
  }
  __syncthreads();
  return *s_flag != 0;
}

// Drops one 128-byte L2 line without writing it back (its contents become
// undefined; the line must not be read again before it is rewritten).
__device__ __forceinline__ void discard_l2_line(const void* p) {
  asm volatile("discard.global.L2 [%0], 128;" ::"l"(p) : "memory");
}

// The partial sums of a tile are dead once the last arrival has added them up,
// and every call rewrites each slot before reading it.  Dropping their L2
// lines saves the write-back to DRAM.  Arrays: n_arrays arrays from base, one
// every `stride` floats, each laid out as [n_bins] (fine: false) or as a fine
// level's [level tiles][NT WT] with base at this tile (fine: true); only
// whole lines inside the tile's bins of each direction are dropped, so the
// neighbouring tiles' partials are untouched.
template <int THREADS>
__device__ __forceinline__ void discard_tile_partials(const float* base, size_t stride,
                                                      long long n_arrays, const JobStatic& J,
                                                      const TileGeom& g, bool fine) {
  // Four arrays per warp, eight lanes per array: a 256-bin row is 8 lines.
  const int sub = threadIdx.x >> 3, l8 = threadIdx.x & 7;
  const int n_om = J.n_omega, o1 = min(g.o0 + g.WT, n_om);
  for (long long arr = sub; arr < n_arrays; arr += THREADS / 8) {
    const float* ap = base + (size_t)arr * stride;
    for (int dl = 0; dl < g.NT; ++dl) {
      const int d = g.d0 + dl;
      if (d >= J.n_dir) break;
      // rp + o: the partial of bin (d, o)
      const float* rp = fine ? ap + (size_t)dl * g.WT - g.o0 : ap + (size_t)d * n_om;
      const uintptr_t a0 = reinterpret_cast<uintptr_t>(rp + g.o0);
      const uintptr_t a1 = reinterpret_cast<uintptr_t>(rp + o1);
      for (uintptr_t line = ((a0 + 127) & ~(uintptr_t)127) + (uintptr_t)l8 * 128; line + 128 <= a1;
           line += 8 * 128)
        discard_l2_line(reinterpret_cast<const void*>(line));
    }
  }
}

// Last arrival: for every bin of the tile, add the chunks' partials in chunk
// order, rotate by e^{i omega tau_ref(n)} and add into the state (Kahan).
// DISCARD: then drop the partials' L2 lines (tensor-core variants; the FP32
// variants measured slower with it and keep the write-back).
// Whether an item's chunks fit the partial-sum buffer it writes.
__device__ __forceinline__ bool part_fits(const JobStatic& J, const ItemRef& it, const PartMap& m) {
  return it.fine < 0 ? it.n_chunks <= J.chunk_cap
                     : m.room >= (long long)it.n_chunks * (long long)m.chunk_stride;
}

// Rotation of a bin's chunk sums by e^{i omega tau_ref(n)} (psi in turns).
__device__ __forceinline__ void bin_rotation(const JobStatic& J, int d, int o, float& cp, float& sp) {
  const double* nd = J.dirs + 3 * d;
  const double tref = J.ref[3] - (nd[0] * J.ref[0] + nd[1] * J.ref[1] + nd[2] * J.ref[2]) * kInvC;
  double psi = J.om_turns[o] * tref;
  psi -= rint(psi);
  sincospif(2.0f * (float)psi, &sp, &cp);
}

// A fine tile's last arrival (TailPlan).  Its bins are contiguous in its
// level's region ([chunk][comp][level tiles][NT WT], NT WT a multiple of 4,
// 16-byte aligned), so the chunk sums are read four bins at a time: a unit is
// (bin quad, component pair), consecutive threads take consecutive quads, and
// each thread sums two units at once, keeping many loads in flight (a finest
// tile has over a hundred chunks, and the last of these sums ends the
// launch).  Every bin's components are still added in chunk order.
template <int THREADS>
__device__ __forceinline__ void fine_tile_sums(const JobStatic& J, const TileGeom& g, const PartMap& m,
                                               int n_chunks) {
  const int n_quads = g.NT * g.WT / 4, n_units = 4 * n_quads;
  const int nb = J.n_bins, n_om = J.n_omega;
  for (int ua = threadIdx.x; ua < n_units; ua += 2 * THREADS) {
    const int ub = min(ua + THREADS, n_units - 1);  // a repeat of ua's last unit when past the end
    const bool has_b = ua + THREADS < n_units;
    const int pa = ua / n_quads, qa = ua - pa * n_quads;
    const int pb = ub / n_quads, qb = ub - pb * n_quads;
    const float* ra = m.base + (size_t)(2 * pa) * m.comp_stride + 4 * qa;
    const float* rb = m.base + (size_t)(2 * pb) * m.comp_stride + 4 * qb;
    float4 are = make_float4(0.f, 0.f, 0.f, 0.f), aim = are, bre = are, bim = are;
#pragma unroll 4
    for (int ch = 0; ch < n_chunks; ++ch) {
      const size_t co = (size_t)ch * m.chunk_stride;
      const float4 x0 = __ldcg(reinterpret_cast<const float4*>(ra + co));
      const float4 x1 = __ldcg(reinterpret_cast<const float4*>(ra + co + m.comp_stride));
      const float4 y0 = __ldcg(reinterpret_cast<const float4*>(rb + co));
      const float4 y1 = __ldcg(reinterpret_cast<const float4*>(rb + co + m.comp_stride));
      are.x += x0.x; are.y += x0.y; are.z += x0.z; are.w += x0.w;
      aim.x += x1.x; aim.y += x1.y; aim.z += x1.z; aim.w += x1.w;
      bre.x += y0.x; bre.y += y0.y; bre.z += y0.z; bre.w += y0.w;
      bim.x += y1.x; bim.y += y1.y; bim.z += y1.z; bim.w += y1.w;
    }
    float* st = J.state;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (h == 1 && !has_b) break;
      const int p = h ? pb : pa, q = h ? qb : qa;
      const float re4[4] = {h ? bre.x : are.x, h ? bre.y : are.y, h ? bre.z : are.z, h ? bre.w : are.w};
      const float im4[4] = {h ? bim.x : aim.x, h ? bim.y : aim.y, h ? bim.z : aim.z, h ? bim.w : aim.w};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int i = 4 * q + k, dl = i / g.WT;
        const int d = g.d0 + dl, o = g.o0 + (i - dl * g.WT);
        if (d >= J.n_dir || o >= n_om) continue;
        const int bin = d * n_om + o, c = 2 * p;
        float cp, sp;
        bin_rotation(J, d, o, cp, sp);
        const float re = re4[k] * cp - im4[k] * sp;
        const float im = re4[k] * sp + im4[k] * cp;
        kahan_add(&st[(size_t)c * nb + bin], &st[(size_t)(kComps + c) * nb + bin], re);
        kahan_add(&st[(size_t)(c + 1) * nb + bin], &st[(size_t)(kComps + c + 1) * nb + bin], im);
      }
    }
  }
}

template <int THREADS, bool DISCARD>
__device__ __forceinline__ void tile_epilogue(const JobStatic& J, const JobCall& K,
                                              const ItemRef& it) {
  const int tile = it.tile;
  const TileGeom g = tile_geom(J, tile, THREADS);
  const PartMap m = part_map(J, K, it, g);
  const int nb = J.n_bins, n_om = J.n_omega;
  if (!bounds_ok(part_fits(J, it, m) && tile < J.n_tiles, J.status)) return;
  // (literal contexts run an FP32 variant: never fine tiles)
  const bool vec = it.fine >= 0 && !J.literal && ((g.NT * g.WT) & 3) == 0;
  if (vec) fine_tile_sums<THREADS>(J, g, m, it.n_chunks);
  for (int i = threadIdx.x; i < (vec ? 0 : g.NT * g.WT); i += THREADS) {
    const int dl = i / g.WT;
    const int d = g.d0 + dl, o = g.o0 + (i - dl * g.WT);
    if (d >= J.n_dir || o >= n_om) continue;
    const int bin = d * n_om + o;
    const size_t off = part_bin(J, it, g, d, o);
    float s[kComps];
#pragma unroll
    for (int c = 0; c < kComps; ++c) s[c] = 0.0f;
    // (unrolled so that several chunks' loads are in flight; the adds keep chunk order)
#pragma unroll 4
    for (int ch = 0; ch < it.n_chunks; ++ch) {
      const float* pc = m.base + (size_t)ch * m.chunk_stride;
#pragma unroll
      for (int c = 0; c < kComps; ++c) s[c] += __ldcg(&pc[(size_t)c * m.comp_stride + off]);
    }
    float sp, cp;
    bin_rotation(J, d, o, cp, sp);
    float* st = J.state;
#pragma unroll
    for (int c = 0; c < kComps; c += 2) {
      const float re = s[c] * cp - s[c + 1] * sp;
      const float im = s[c] * sp + s[c + 1] * cp;
      kahan_add(&st[(size_t)c * nb + bin], &st[(size_t)(kComps + c) * nb + bin], re);
      kahan_add(&st[(size_t)(c + 1) * nb + bin], &st[(size_t)(kComps + c + 1) * nb + bin], im);
    }
    if (J.literal) {  // (literal contexts run an FP32 variant: never fine tiles)
      float p[4] = {0.f, 0.f, 0.f, 0.f};
      for (int ch = 0; ch < it.n_chunks; ++ch) {
        const float* pc = J.partials_p + (size_t)ch * 4 * nb;
#pragma unroll
        for (int c = 0; c < 4; ++c) p[c] += __ldcg(&pc[(size_t)c * nb + bin]);
      }
      float* sp_ = J.state_p;
#pragma unroll
      for (int c = 0; c < 4; c += 2) {
        const float re = p[c] * cp - p[c + 1] * sp;
        const float im = p[c] * sp + p[c + 1] * cp;
        kahan_add(&sp_[(size_t)c * nb + bin], &sp_[(size_t)(4 + c) * nb + bin], re);
        kahan_add(&sp_[(size_t)(c + 1) * nb + bin], &sp_[(size_t)(4 + c + 1) * nb + bin], im);
      }
    }
  }
  if constexpr (DISCARD) {
    __syncthreads();  // every thread's reads of the partials are done
    discard_tile_partials<THREADS>(m.base, m.comp_stride, (long long)it.n_chunks * kComps, J, g,
                                   it.fine >= 0);
    if (J.literal)
      discard_tile_partials<THREADS>(J.partials_p, (size_t)nb, (long long)it.n_chunks * 4, J, g,
                                     false);
  }
}

__device__ __forceinline__ float sqrt_approx(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Reference time of a wide call's particle group (the group holding particle
// kt) seen from direction d: -n . (r_group - r_ref) / c.
__device__ __forceinline__ double group_tau(const JobStatic& J, long long kt, int d) {
  const double* D = J.gref + 3 * (kt / kGroup);
  const double* nd = J.dirs + 3 * d;
  return -(nd[0] * D[0] + nd[1] * D[1] + nd[2] * D[2]) * kInvC;
}

// Loads one raw particle tile; thread 0 only.
__device__ __forceinline__ void issue_tile(const JobStatic& J, long long k0, int KT, float* raw,
                                           uint64_t* bar) {
  // (skipped in a debug build when out of range: the block's bounded wait then gives up)
  if (!bounds_ok(k0 + KT <= J.n_cap, J.status)) return;
  tma_load_1d(raw, J.rec + (size_t)k0 * kRecFields, (uint32_t)KT * kRecFields * sizeof(float), bar);
}

// ------------------------------------------------------------ FP32 variant
// LIT: also the paper's literal sum P_i += sqrt(w) dt a_i g e^{i phi} with
// g = sqrt(1 + (w - 1) f(omega)^2), i.e. F_k(omega) dt a_i (Eq. 13 with Eq. 12).
template <int THREADS, int W, int UNROLL, bool LIT = false, bool WIDE = false>
__device__ __forceinline__ bool process_item_fma(const JobStatic& J, const JobCall& K,
                                                 const ItemRef& item, unsigned char* __restrict__ smem,
                                                 uint64_t* bar, uint32_t& phase, int* s_flag) {
  const int tile = item.tile, chunk = item.chunk;
  constexpr int NP = W / 2;
  constexpr int REC = LIT ? 4 : 3;                 // float4 per record
  constexpr int NC = kComps + (LIT ? 4 : 0);       // accumulated components per frequency
  using S = Smem<THREADS, false, LIT>;
  float* raw = reinterpret_cast<float*>(smem);
  const TileGeom g = tile_geom(J, tile, THREADS);
  const int lanes_per_dir = g.WT / W;
  const int my_dl = threadIdx.x / lanes_per_dir;
  const int my_d_raw = g.d0 + my_dl;
  const int my_d = min(my_d_raw, J.n_dir - 1);
  const int om_first = g.o0 + (threadIdx.x - my_dl * lanes_per_dir) * W;
  const int n_om = J.n_omega;
  const int s1_dl = threadIdx.x / g.KT, s1_kk = threadIdx.x - s1_dl * g.KT;
  const int s1_d = min(g.d0 + s1_dl, J.n_dir - 1);
  // WIDE: a wide call, whose records are relative to their group's reference point.
  constexpr bool wide = WIDE;

  float2 omh[NP], wh[NP], wl[NP];
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    const int i0 = min(om_first + 2 * p, n_om - 1), i1 = min(om_first + 2 * p + 1, n_om - 1);
    omh[p] = make_float2(__ldg(J.om_tab + i0), __ldg(J.om_tab + i1));
    wh[p] = make_float2(__ldg(J.om_tab + n_om + i0), __ldg(J.om_tab + n_om + i1));
    wl[p] = make_float2(__ldg(J.om_tab + 2 * n_om + i0), __ldg(J.om_tab + 2 * n_om + i1));
  }
  float2 f2[NP];
  if (LIT) {
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      const int i0 = min(om_first + 2 * p, n_om - 1), i1 = min(om_first + 2 * p + 1, n_om - 1);
      f2[p] = make_float2(__ldg(J.f2_tab + i0), __ldg(J.f2_tab + i1));
    }
  }
  float2 acc1[NP][NC], acc2[NP][NC];
#pragma unroll
  for (int p = 0; p < NP; ++p)
#pragma unroll
    for (int c = 0; c < NC; ++c) acc1[p][c] = acc2[p][c] = make_float2(0.f, 0.f);
  const float2 kOne = make_float2(1.0f, 1.0f);

  const long long k_begin = (long long)chunk * item.ck;
  const long long k_end = min(k_begin + (long long)item.ck, K.n);
  const int n_kt = (int)((k_end - k_begin + g.KT - 1) / g.KT);
  // Whole tiles are copied: k_begin is a multiple of KT and the record buffer
  // holds at least round_up(n, 256) particles, so every copy stays in bounds.
  if (threadIdx.x == 0) issue_tile(J, k_begin, g.KT, raw, bar);
  for (int it = 0; it < n_kt; ++it) {
    const long long kt = k_begin + (long long)it * g.KT;
    const int kn = (int)min((long long)g.KT, k_end - kt);
    float4* rec = reinterpret_cast<float4*>(smem + S::raw_bytes + (size_t)(it & 1) * S::rec_bytes);
    const bool landed = mbar_wait(bar, phase);
    phase ^= 1u;
    bool slow = false;
    if (landed && s1_kk < kn) {
      float th, tl, a[4];
      slow = !compute_record(raw + s1_kk * kRecFields, J.dir_tab, J.n_dir, s1_d, J.tau_fast, th,
                             tl, a);
      float4* out = rec + (s1_kk * g.NT + s1_dl) * REC;
      out[0] = make_float4(th, th, tl, tl);
      out[1] = make_float4(a[0], a[0], a[1], a[1]);
      out[2] = make_float4(a[2], a[2], a[3], a[3]);
      if (LIT) {
        const float wm1 = raw[s1_kk * kRecFields + 18];
        out[REC - 1] = make_float4(wm1, wm1, 0.f, 0.f);
      }
    }
    const int flags = __syncthreads_or((slow ? 1 : 0) | (landed ? 0 : 2));
    if (flags & 2) {
      // The copy did not land within the bound: record it, wait (bounded) once
      // more for that copy, and leave.
      if (threadIdx.x == 0) {
        atomicOr(J.status, ST_TIMEOUT);
        mbar_wait(bar, phase ^ 1u);
      }
      return false;
    }
    if (threadIdx.x == 0 && it + 1 < n_kt) issue_tile(J, kt + g.KT, g.KT, raw, bar);
    const float4* rc = rec + my_dl * REC;
    if (!(flags & 1)) {
      // kend particles at a record stride of nt; a full tile of one direction
      // instantiates it with both known at compile time.
      auto fast_loop = [&](const int kend, const int nt) {
#pragma unroll UNROLL
      for (int kk = 0; kk < kend; ++kk) {
        const float4 r0 = rc[kk * nt * REC + 0];
        const float4 r1 = rc[kk * nt * REC + 1];
        const float4 r2 = rc[kk * nt * REC + 2];
        const float2 th = make_float2(r0.x, r0.y), tl = make_float2(r0.z, r0.w);
        const float2 aw1 = make_float2(r1.x, r1.y), aw2 = make_float2(r1.z, r1.w);
        const float2 av1 = make_float2(r2.x, r2.y), av2 = make_float2(r2.z, r2.w);
#pragma unroll
        for (int p = 0; p < NP; ++p) {
          const float2 ph = phase2(omh[p], wh[p], wl[p], th, tl);
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
          if (LIT) {
            const float4 r3 = rc[kk * nt * REC + REC - 1];
            const float2 g2 = __ffma2_rn(make_float2(r3.x, r3.y), f2[p], kOne);
            const float2 gg = make_float2(sqrt_approx(g2.x), sqrt_approx(g2.y));
            const float2 pv1 = __fmul2_rn(av1, gg), pv2 = __fmul2_rn(av2, gg);
            acc1[p][NC - 4] = __ffma2_rn(pv1, cc, acc1[p][NC - 4]);
            acc1[p][NC - 3] = __ffma2_rn(pv1, ss, acc1[p][NC - 3]);
            acc1[p][NC - 2] = __ffma2_rn(pv2, cc, acc1[p][NC - 2]);
            acc1[p][NC - 1] = __ffma2_rn(pv2, ss, acc1[p][NC - 1]);
          }
        }
      }
      };
      if (g.NT == 1 && kn == THREADS) fast_loop(THREADS, 1);
      else fast_loop(kn, g.NT);
    } else {
      // Wide path: some |dtau| exceed the fast range in this tile; the phase of
      // every update is formed in FP64.
      if (threadIdx.x == 0) atomicOr(J.status, ST_SLOW_PHASE);
      double tau_g = 0.0;
      if constexpr (wide) tau_g = group_tau(J, kt, my_d);
      double omt[W];
#pragma unroll
      for (int i = 0; i < W; ++i) omt[i] = J.om_turns[min(om_first + i, n_om - 1)];
      for (int kk = 0; kk < kn; ++kk) {
        const float4 r0 = rc[kk * g.NT * REC + 0];
        const float4 r1 = rc[kk * g.NT * REC + 1];
        const float4 r2 = rc[kk * g.NT * REC + 2];
#pragma unroll
        for (int p = 0; p < NP; ++p) {
          const float2 ph = make_float2(phase_wide(omt[2 * p], r0.x, r0.z, tau_g),
                                        phase_wide(omt[2 * p + 1], r0.x, r0.z, tau_g));
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
          if (LIT) {
            const float4 r3 = rc[kk * g.NT * REC + REC - 1];
            const float2 g2 = __ffma2_rn(make_float2(r3.x, r3.y), f2[p], kOne);
            const float2 gg = make_float2(sqrt_approx(g2.x), sqrt_approx(g2.y));
            const float2 pv1 = __fmul2_rn(make_float2(r2.x, r2.y), gg);
            const float2 pv2 = __fmul2_rn(make_float2(r2.z, r2.w), gg);
            acc1[p][NC - 4] = __ffma2_rn(pv1, cc, acc1[p][NC - 4]);
            acc1[p][NC - 3] = __ffma2_rn(pv1, ss, acc1[p][NC - 3]);
            acc1[p][NC - 2] = __ffma2_rn(pv2, cc, acc1[p][NC - 2]);
            acc1[p][NC - 1] = __ffma2_rn(pv2, ss, acc1[p][NC - 1]);
          }
        }
      }
    }
    // Wide call, fast path: the tile's sums are relative to its group's
    // reference; rotate them by e^{i omega tau_g} (the FP64 path above already
    // has tau_g in every phase).
    if constexpr (wide) {
      if (!(flags & 1)) {
        const double tau_g = group_tau(J, kt, my_d);
#pragma unroll
        for (int p = 0; p < NP; ++p) {
          float2 cs, sn;
          group_rotation(J.om_turns[min(om_first + 2 * p, n_om - 1)], tau_g, cs.x, sn.x);
          group_rotation(J.om_turns[min(om_first + 2 * p + 1, n_om - 1)], tau_g, cs.y, sn.y);
#pragma unroll
          for (int c = 0; c < NC; c += 2) {
            const float2 re = acc1[p][c], im = acc1[p][c + 1];
            acc1[p][c] = __ffma2_rn(re, cs, __fmul2_rn(make_float2(-im.x, -im.y), sn));
            acc1[p][c + 1] = __ffma2_rn(re, sn, __fmul2_rn(im, cs));
          }
        }
      }
    }
    // Two-level summation: the tile's sums join the chunk sums.
#pragma unroll
    for (int p = 0; p < NP; ++p)
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        acc2[p][c] = __fadd2_rn(acc2[p][c], acc1[p][c]);
        acc1[p][c] = make_float2(0.f, 0.f);
      }
  }

  // Partial sums of this work item.  (FP32 variants never take fine-chunked
  // tiles, TailPlan: their items write the coarse partials directly, which
  // keeps the fine tiles' bookkeeping out of this loop's registers.)
  const int nb = J.n_bins;
  float* part = J.partials + (size_t)chunk * kComps * nb;
  if (my_d_raw < J.n_dir) {
#pragma unroll
    for (int p = 0; p < NP; ++p)
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int o = om_first + 2 * p + e;
        if (o < n_om && bounds_ok(chunk < J.chunk_cap && item.fine < 0, J.status)) {
          const int bin = my_d * n_om + o;
#pragma unroll
          for (int c = 0; c < kComps; ++c)
            part[(size_t)c * nb + bin] = e ? acc2[p][c].y : acc2[p][c].x;
          if (LIT) {
            float* pp = J.partials_p + (size_t)chunk * 4 * nb;
#pragma unroll
            for (int c = 0; c < 4; ++c)
              pp[(size_t)c * nb + bin] = e ? acc2[p][NC - 4 + c].y : acc2[p][NC - 4 + c].x;
          }
        }
      }
  }
  if (last_arrival<THREADS>(J, item, s_flag)) tile_epilogue<THREADS, false>(J, K, item);
  return true;
}

// ------------------------------------------------------ tensor-core variant
// Warp layout: warp w handles direction d0 + w / (WT/(16 NB)) and 16 NB
// frequencies (NB 16-row MMA blocks) starting at o0 + 16 NB (w % (WT/(16 NB))).
// XT: the phases' cross terms 2pi (omega_lo th + omega_hi tl) come from one
// more MMA per block (below), and the phase arithmetic is packed over particle
// pairs instead of frequency pairs.
template <int THREADS, int PASSES, int NB, bool WIDE = false, bool XT = false>
__device__ __forceinline__ bool process_item_tc(const JobStatic& J, const JobCall& K,
                                                const ItemRef& item, unsigned char* __restrict__ smem,
                                                uint64_t* bar, uint32_t& phase, int* s_flag) {
  const int tile = item.tile, chunk = item.chunk;
  // NB: 16-frequency blocks per warp; GQ: second-level float4 groups per pass
  constexpr int GQ = 2 * NB;
  using S = Smem<THREADS, true, false, PASSES * NB / 2, XT>;
  float* raw = reinterpret_cast<float*>(smem);
  const TileGeom g = tile_geom(J, tile, THREADS);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int r = lane >> 2, c = lane & 3;
  // The tile's frequencies are swept in PASSES passes of PW over the same
  // staged particle records (one stage 1 and one barrier per tile and pass set).
  const int PW = g.WT / PASSES;
  const int warps_per_dir = PW / (16 * NB);
  const int my_dl = warp / warps_per_dir;
  const int my_d_raw = g.d0 + my_dl;
  const int my_d = min(my_d_raw, J.n_dir - 1);
  const int o_warp0 = g.o0 + (warp - my_dl * warps_per_dir) * 16 * NB;
  const int n_om = J.n_omega;
  const int s1_dl = threadIdx.x / g.KT, s1_kk = threadIdx.x - s1_dl * g.KT;
  const int s1_d = min(g.d0 + s1_dl, J.n_dir - 1);
  // WIDE: a wide call, whose records are relative to their group's reference point.
  constexpr bool wide = WIDE;

  float2 omh[NB], wh[NB], wl[NB];
  // XT: omega/2pi (hi) of rows r and r + 8 of each block, each in both halves
  // of a pair, and the A fragment of the cross-term product.  That product has
  // eight terms t (A columns, B rows), with x ~ x_hi + x_lo split into TF32
  // values:  t = 0..7: wl_hi th_hi, wl_hi th_lo, wl_lo th_hi, wh_hi tl_hi,
  // wh_hi tl_lo, wh_lo tl_hi, wl_lo th_lo, wh_lo tl_lo  (wh, wl: 2pi omega hi
  // and lo in radians; th, tl: the particle's dtau hi and lo), which sum to
  // wl th + wh tl.
  float2 omr[NB], omr8[NB];
  uint32_t xa[NB][4];
  auto load_omega = [&](int o_warp) {
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const int i0 = min(o_warp + 16 * b + r, n_om - 1), i1 = min(o_warp + 16 * b + r + 8, n_om - 1);
      if constexpr (XT) {
        const float h0 = __ldg(J.om_tab + i0), h1 = __ldg(J.om_tab + i1);
        omr[b] = make_float2(h0, h0);
        omr8[b] = make_float2(h1, h1);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int i = h ? i1 : i0;
          uint32_t whh, whl, wlh, wll;
          split_tf32(__ldg(J.om_tab + n_om + i), whh, whl);
          split_tf32(__ldg(J.om_tab + 2 * n_om + i), wlh, wll);
          // a0/a1: column c of rows r / r + 8; a2/a3: column c + 4.
          xa[b][h] = c == 3 ? whh : (c == 2 ? wll : wlh);
          xa[b][2 + h] = c == 0 ? whh : (c == 2 ? wll : whl);
        }
      } else {
        omh[b] = make_float2(__ldg(J.om_tab + i0), __ldg(J.om_tab + i1));
        wh[b] = make_float2(__ldg(J.om_tab + n_om + i0), __ldg(J.om_tab + n_om + i1));
        wl[b] = make_float2(__ldg(J.om_tab + 2 * n_om + i0), __ldg(J.om_tab + 2 * n_om + i1));
      }
    }
  };
  load_omega(o_warp0);
  float dre[NB][4], dim[NB][4];
  // second-level sums of pass p: group q (q = b for the real parts of block b,
  // NB + b for the imaginary parts) of this thread at l2[(p * GQ + q) * THREADS + threadIdx.x]
  float4* l2 = reinterpret_cast<float4*>(smem + S::raw_bytes + 2 * S::rec_bytes);
#pragma unroll
  for (int b = 0; b < NB; ++b)
#pragma unroll
    for (int e = 0; e < 4; ++e) dre[b][e] = dim[b][e] = 0.0f;
#pragma unroll
  for (int v = 0; v < GQ * PASSES; ++v) l2[v * THREADS + threadIdx.x] = make_float4(0.f, 0.f, 0.f, 0.f);

  const long long k_begin = (long long)chunk * item.ck;
  const long long k_end = min(k_begin + (long long)item.ck, K.n);
  const int n_kt = (int)((k_end - k_begin + g.KT - 1) / g.KT);
  if (threadIdx.x == 0) issue_tile(J, k_begin, g.KT, raw, bar);
  // XT: the tile's direction rows, staged once per item for stage 1 (the
  // previous item's last reads of them precede its closing barriers).
  float* sdir = reinterpret_cast<float*>(smem + S::raw_bytes + 2 * S::rec_bytes + S::l2_bytes);
  if constexpr (XT) {
    for (int t = threadIdx.x; t < 12 * g.NT; t += THREADS) {
      const int dl = t / 12, k = t - dl * 12;
      sdir[t] = __ldg(J.dir_tab + (size_t)k * J.n_dir + min(g.d0 + dl, J.n_dir - 1));
    }
    __syncthreads();
  }
  for (int it = 0; it < n_kt; ++it) {
    const long long kt = k_begin + (long long)it * g.KT;
    const int kn = (int)min((long long)g.KT, k_end - kt);
    unsigned char* recb = smem + S::raw_bytes + (size_t)(it & 1) * S::rec_bytes;
    float2* tau2 = reinterpret_cast<float2*>(recb);                     // [NT][KT]
    float* ampb = reinterpret_cast<float*>(recb + (size_t)THREADS * 8);  // [NT][KT][8]
    // XT records: dtau hi [NT][KT]; the cross-term B rows [NT][KT][8] as four
    // pairs (terms c, c + 4), pair c of particle p at position c ^ 2 ((p >> 2) & 1)
    // (lane c reads its pair with one 8-byte load); the amplitudes' hi/lo parts
    // [NT][KT][12], 8 used.  The swizzle and the 12-word stride keep both the
    // stage-1 stores and the loop's loads free of bank conflicts.
    float* xth = reinterpret_cast<float*>(recb);
    float* xrt = reinterpret_cast<float*>(recb + (size_t)THREADS * 4);
    float* xam = reinterpret_cast<float*>(recb + (size_t)THREADS * 36);
    const bool landed = mbar_wait(bar, phase);
    phase ^= 1u;
    bool slow = false;
    if (landed) {
      float th = 0.f, tl = 0.f, a[4] = {0.f, 0.f, 0.f, 0.f};
      if (s1_kk < kn) {
        if constexpr (XT)
          slow = !compute_record(raw + s1_kk * kRecFields, dir_row_staged(sdir + 12 * s1_dl),
                                 J.tau_fast, th, tl, a);
        else
          slow = !compute_record(raw + s1_kk * kRecFields, J.dir_tab, J.n_dir, s1_d, J.tau_fast,
                                 th, tl, a);
      }
      // Particles past kn are zero padding of the last 8-particle MMA step.
      const int slot = s1_dl * g.KT + s1_kk;
      const uint32_t h0 = tf32_hi(a[0]), h1 = tf32_hi(a[1]), h2 = tf32_hi(a[2]), h3 = tf32_hi(a[3]);
      if constexpr (XT) {
        xth[slot] = th;
        uint32_t thh, thl, tlh, tll;
        split_tf32(th, thh, thl);
        split_tf32(tl, tlh, tll);
        float4* rp = reinterpret_cast<float4*>(xrt + (size_t)slot * 8);
        const int sw = (s1_kk >> 2) & 1;  // pairs 0, 1 and 2, 3 swap places
        rp[sw] = make_float4(__uint_as_float(thh), __uint_as_float(tll), __uint_as_float(thl),
                             __uint_as_float(tlh));
        rp[sw ^ 1] = make_float4(__uint_as_float(thh), __uint_as_float(thl),
                                 __uint_as_float(tlh), __uint_as_float(tll));
        float4* ap = reinterpret_cast<float4*>(xam + (size_t)slot * 12);
        ap[0] = make_float4(__uint_as_float(h0), __uint_as_float(h1), __uint_as_float(h2),
                            __uint_as_float(h3));
        ap[1] = make_float4(a[0] - __uint_as_float(h0), a[1] - __uint_as_float(h1),
                            a[2] - __uint_as_float(h2), a[3] - __uint_as_float(h3));
      } else {
        tau2[slot] = make_float2(th, tl);
        float4* ap = reinterpret_cast<float4*>(ampb + (size_t)slot * 8);
        ap[0] = make_float4(__uint_as_float(h0), __uint_as_float(h1), __uint_as_float(h2),
                            __uint_as_float(h3));
        ap[1] = make_float4(a[0] - __uint_as_float(h0), a[1] - __uint_as_float(h1),
                            a[2] - __uint_as_float(h2), a[3] - __uint_as_float(h3));
      }
    }
    const int flags = __syncthreads_or((slow ? 1 : 0) | (landed ? 0 : 2));
    if (flags & 2) {
      if (threadIdx.x == 0) {
        atomicOr(J.status, ST_TIMEOUT);
        mbar_wait(bar, phase ^ 1u);
      }
      return false;
    }
    if (threadIdx.x == 0 && it + 1 < n_kt) issue_tile(J, kt + g.KT, g.KT, raw, bar);
    const float2* tw = tau2 + my_dl * g.KT;
    const float* aw = ampb + (size_t)my_dl * g.KT * 8;
    const float* xtw = xth + my_dl * g.KT;
    const float* xrw = xrt + (size_t)my_dl * g.KT * 8;
    const float* xaw = xam + (size_t)my_dl * g.KT * 12;
    // this lane's cross-term pair within particle kk + r's row (kk % 8 == 0)
    const int xr_off = 2 * (c ^ ((r >> 1) & 2));
    // XT, the 8-particle step at kk: the main product's k = c and k = c + 4 are
    // particles kk + 2c and kk + 2c + 1 (the columns of the cross-term result
    // this lane holds).
    auto xamp = [&](int kk) {
      return make_uint2(__float_as_uint(xaw[(kk + 2 * c) * 12 + r]),
                        __float_as_uint(xaw[(kk + 2 * c + 1) * 12 + r]));
    };
    const int kn8 = (kn + 7) & ~7;
#pragma unroll 1
    for (int ps = 0; ps < PASSES; ++ps) {
      const int o_warp = o_warp0 + ps * PW;
      if (PASSES > 1) load_omega(o_warp);
      if (!(flags & 1)) {
        // Unrolled 2x with two 16-frequency blocks per warp, 8x with four (measured: 1, 2, 4, 8).
        constexpr int kUnroll = NB >= 4 ? 8 : 2;
        auto fast_loop = [&](const int kend) {
#pragma unroll kUnroll
          for (int kk = 0; kk < kend; kk += 8) {
            if constexpr (XT) {
              const float2 th2 = *reinterpret_cast<const float2*>(xtw + kk + 2 * c);
              const uint2 rt = *reinterpret_cast<const uint2*>(xrw + (size_t)(kk + r) * 8 + xr_off);
              const uint2 bb = xamp(kk);
#pragma unroll
              for (int b = 0; b < NB; ++b) {
                // cr: rows r, r + 8 x particles kk + 2c, kk + 2c + 1
                float cr[4];
                mma_tf32_zero(cr, xa[b][0], xa[b][1], xa[b][2], xa[b][3], rt.x, rt.y);
                const float2 p0 = phase2x(omr[b], th2, make_float2(cr[0], cr[1]));
                const float2 p8 = phase2x(omr8[b], th2, make_float2(cr[2], cr[3]));
                tc_block(make_float2(p0.x, p8.x), make_float2(p0.y, p8.y), bb.x, bb.y, dre[b],
                         dim[b]);
              }
              continue;
            }
            const float2 tA = tw[kk + c], tB = tw[kk + c + 4];
            const uint32_t b0 = __float_as_uint(aw[(kk + c) * 8 + r]);
            const uint32_t b1 = __float_as_uint(aw[(kk + c + 4) * 8 + r]);
            const float2 thA = make_float2(tA.x, tA.x), tlA = make_float2(tA.y, tA.y);
            const float2 thB = make_float2(tB.x, tB.x), tlB = make_float2(tB.y, tB.y);
#pragma unroll
            for (int b = 0; b < NB; ++b) {
              const float2 pA = phase2(omh[b], wh[b], wl[b], thA, tlA);
              const float2 pB = phase2(omh[b], wh[b], wl[b], thB, tlB);
              tc_block(pA, pB, b0, b1, dre[b], dim[b]);
            }
          }
        };
        // A full tile of one direction takes the loop with its trip count known at
        // compile time (measured ~1 % faster); ragged and multi-direction tiles
        // the runtime bound.
        if (kn8 == THREADS) fast_loop(THREADS);
        else fast_loop(kn8);
      } else {
        if (threadIdx.x == 0) atomicOr(J.status, ST_SLOW_PHASE);
        double tau_g = 0.0;
        if constexpr (wide) tau_g = group_tau(J, kt, my_d);
        double omt[NB][2];
#pragma unroll
        for (int b = 0; b < NB; ++b) {
          omt[b][0] = J.om_turns[min(o_warp + 16 * b + r, n_om - 1)];
          omt[b][1] = J.om_turns[min(o_warp + 16 * b + r + 8, n_om - 1)];
        }
        for (int kk = 0; kk < kn8; kk += 8) {
          float2 tA, tB;
          uint32_t b0, b1;
          if constexpr (XT) {
            // particles kk + 2c and kk + 2c + 1; tl = tl_hi + tl_lo (terms 3, 7:
            // pair 3, at position 3 ^ 2 ((p >> 2) & 1))
            const int pa = kk + 2 * c;
            auto tl_of = [&](int p) {
              const float* q = xrw + (size_t)p * 8 + 2 * (3 ^ (((p >> 2) & 1) << 1));
              return q[0] + q[1];
            };
            tA = make_float2(xtw[pa], tl_of(pa));
            tB = make_float2(xtw[pa + 1], tl_of(pa + 1));
            const uint2 bb = xamp(kk);
            b0 = bb.x;
            b1 = bb.y;
          } else {
            tA = tw[kk + c];
            tB = tw[kk + c + 4];
            b0 = __float_as_uint(aw[(kk + c) * 8 + r]);
            b1 = __float_as_uint(aw[(kk + c + 4) * 8 + r]);
          }
#pragma unroll
          for (int b = 0; b < NB; ++b) {
            const float2 pA = make_float2(phase_wide(omt[b][0], tA.x, tA.y, tau_g),
                                          phase_wide(omt[b][1], tA.x, tA.y, tau_g));
            const float2 pB = make_float2(phase_wide(omt[b][0], tB.x, tB.y, tau_g),
                                          phase_wide(omt[b][1], tB.x, tB.y, tau_g));
            tc_block(pA, pB, b0, b1, dre[b], dim[b]);
          }
        }
      }
      // Wide call, fast path: rotate the tile's sums by e^{i omega tau_g}.  The
      // warp's 16 NB frequencies are shared out: lane L reduces the phases of
      // frequencies L and L + 32 of the warp's range in FP64 (FP64 is narrow on
      // this GPU), and each lane takes the factors of its rows r and r + 8 of
      // every block from their owners by shuffles.
      if constexpr (wide) {
        if (!(flags & 1)) {
          const double tau_g = group_tau(J, kt, my_d);
          float cA, sA, cB = 1.0f, sB = 0.0f;
          group_rotation(J.om_turns[min(o_warp + lane, n_om - 1)], tau_g, cA, sA);
          if constexpr (NB > 2)
            group_rotation(J.om_turns[min(o_warp + lane + 32, n_om - 1)], tau_g, cB, sB);
#pragma unroll
          for (int b = 0; b < NB; ++b)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const int src = (16 * b + r + 8 * h) & 31;
              const float cs = __shfl_sync(0xffffffffu, b < 2 ? cA : cB, src);
              const float sn = __shfl_sync(0xffffffffu, b < 2 ? sA : sB, src);
#pragma unroll
              for (int e = 2 * h; e < 2 * h + 2; ++e) {
                const float re = dre[b][e], im = dim[b][e];
                dre[b][e] = fmaf(re, cs, -im * sn);
                dim[b][e] = fmaf(re, sn, im * cs);
              }
            }
        }
      }
      // Second level: after every particle tile the tile sums join the chunk
      // sums in shared memory, so the MMA accumulators never sum more than one
      // tile.  Longer runs would be faster (LWFA workload, variant 9: a flush
      // every second tile 0.2 % and every fourth 0.5 % less time per step) but
      // the MMA's FP32 accumulation error grows with the run's length: at every
      // fourth tile a 5000-particle workload read 1.3e-5 of row error against
      // the oracle (gate 1e-5), about four times that of a flush every tile.
      float4* l2p = l2 + ps * GQ * THREADS + threadIdx.x;
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        float4 x = l2p[b * THREADS], y = l2p[(NB + b) * THREADS];
        const float2 x01 = __fadd2_rn(make_float2(x.x, x.y), make_float2(dre[b][0], dre[b][1]));
        const float2 x23 = __fadd2_rn(make_float2(x.z, x.w), make_float2(dre[b][2], dre[b][3]));
        const float2 y01 = __fadd2_rn(make_float2(y.x, y.y), make_float2(dim[b][0], dim[b][1]));
        const float2 y23 = __fadd2_rn(make_float2(y.z, y.w), make_float2(dim[b][2], dim[b][3]));
        l2p[b * THREADS] = make_float4(x01.x, x01.y, x23.x, x23.y);
        l2p[(NB + b) * THREADS] = make_float4(y01.x, y01.y, y23.x, y23.y);
#pragma unroll
        for (int e = 0; e < 4; ++e) dre[b][e] = dim[b][e] = 0.0f;
      }
    }
  }

  // The D fragment holds rows (r, r+8) and columns (2c, 2c+1); columns 0-3 are
  // the hi parts of (U.e1, U.e2, V.e1, V.e2), columns 4-7 the lo parts: lane c
  // (c < 2) adds lane c+2's values.
  const PartMap pm = part_map(J, K, item, g);
  float* part = pm.base + (size_t)chunk * pm.chunk_stride;
#pragma unroll 1
  for (int ps = 0; ps < PASSES; ++ps)
#pragma unroll
  for (int b = 0; b < NB; ++b)
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const float* l2p = reinterpret_cast<const float*>(l2 + ps * GQ * THREADS + threadIdx.x);
      const float lre = l2p[4 * b * THREADS + e];
      const float lim = l2p[4 * (NB + b) * THREADS + e];
      const float re = lre + __shfl_xor_sync(0xffffffffu, lre, 2);
      const float im = lim + __shfl_xor_sync(0xffffffffu, lim, 2);
      const int o = o_warp0 + ps * PW + 16 * b + r + ((e >> 1) << 3);
      const int j = 2 * c + (e & 1);  // amplitude column
      if (c < 2 && my_d_raw < J.n_dir && o < n_om &&
          bounds_ok(chunk < item.n_chunks && part_fits(J, item, pm), J.status)) {
        const size_t off = part_bin(J, item, g, my_d, o);
        part[(size_t)(2 * j) * pm.comp_stride + off] = re;
        part[(size_t)(2 * j + 1) * pm.comp_stride + off] = im;
      }
    }
  if (last_arrival<THREADS>(J, item, s_flag)) tile_epilogue<THREADS, true>(J, K, item);
  return true;
}

// WIDE = false: the work items of jobs whose call is not wide; true: those of
// wide calls (exits at once when no job of the launch is wide).  The two run
// one after the other on the same stream, each with its own item counter, so
// the common path keeps its register allocation free of the wide-call code.
template <int THREADS, int W, int MINB, bool TC, bool LIT, int PASSES = 1, bool WIDE = false,
          bool XT = false>
__global__ void __launch_bounds__(THREADS, MINB) accumulate_kernel(LaunchArgs a) {
  // Whether any job of the launch is wide is final before either kernel starts:
  // the wide one leaves at once without, and the ordinary one then takes every
  // item without looking at the jobs' flags.
  const bool any_wide = a.any_wide != nullptr && *a.any_wide != 0;
  if (WIDE && !any_wide) return;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ long long s_item[2];
  __shared__ int s_flag;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_fence_init();
  }
  // Profiling: the block's start, kept in shared memory rather than in
  // registers live across the whole loop.
  __shared__ long long s_clk0;
  __shared__ unsigned long long s_ns0;
  if (a.prof_clk && threadIdx.x == 0) {
    s_clk0 = clock64();
    s_ns0 = global_ns();
  }
  __syncthreads();
  uint32_t phase = 0u;
  int buf = 0;
  for (;;) {
    if (threadIdx.x == 0) s_item[buf] = (long long)atomicAdd(a.item_counter + (WIDE ? 1 : 0), 1ULL);
    __syncthreads();
    const long long item = s_item[buf];
    buf ^= 1;
    if (item >= a.n_items) break;
    const int j = find_job(a, item);
    const JobStatic& J = a.js[j];
    if (any_wide && (J.wide_flag != nullptr && *J.wide_flag != 0) != WIDE) continue;  // the other kernel's
    const JobCall K = a.use_inline ? a.inline_call : a.jc[j];
    // Tile-major order: the chunks of one tile run close together in time, so
    // their partial sums are still in L2 when the tile's last arrival reads them.
    const ItemRef it = decode_item<TC>(J, K, item - K.item_begin);
    bool ok;
    if constexpr (TC)
      ok = process_item_tc<THREADS, PASSES, 2 * W, WIDE, XT>(J, K, it, smem, &bar, phase, &s_flag);
    else
      ok = process_item_fma<THREADS, W, 8, LIT, WIDE>(J, K, it, smem, &bar, phase, &s_flag);
    if (!ok) break;
  }
  if (a.prof_clk && threadIdx.x == 0) {
    atomicAdd(&a.prof_clk[0], (unsigned long long)(clock64() - s_clk0));
    atomicAdd(&a.prof_clk[1], global_ns() - s_ns0);
  }
}

template <int T, int W, int MINB, bool TC, bool LIT, int P = 1, bool XT = false>
cudaError_t launch_acc(const LaunchArgs& a, int grid, cudaStream_t s) {
  const size_t smem = Smem<T, TC, LIT, TC ? P * W : P, XT>::bytes;
  // The shared-memory opt-in is per kernel and device, and idempotent.
  static std::atomic<bool> attr_set[kMaxDevices];
  const int dev = current_device();
  if (dev < 0 || dev >= kMaxDevices || !attr_set[dev].load(std::memory_order_acquire)) {
    cudaError_t e = cudaFuncSetAttribute(accumulate_kernel<T, W, MINB, TC, LIT, P, false, XT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(accumulate_kernel<T, W, MINB, TC, LIT, P, true, XT>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < kMaxDevices) attr_set[dev].store(true, std::memory_order_release);
  }
  accumulate_kernel<T, W, MINB, TC, LIT, P, false, XT><<<grid, T, smem, s>>>(a);
  count_launches(1);
  if (a.any_wide != nullptr) {
    accumulate_kernel<T, W, MINB, TC, LIT, P, true, XT><<<grid, T, smem, s>>>(a);
    count_launches(1);
  }
  return cudaGetLastError();
}

template <int T, int W, int MINB, bool TC, bool LIT, int P = 1, bool XT = false>
int blocks_per_sm() {
  int nb = 0;
  const size_t smem = Smem<T, TC, LIT, TC ? P * W : P, XT>::bytes;
  cudaFuncSetAttribute(accumulate_kernel<T, W, MINB, TC, LIT, P, false, XT>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(
          &nb, accumulate_kernel<T, W, MINB, TC, LIT, P, false, XT>, T, smem) != cudaSuccess ||
      nb < 1)
    nb = 1;
  return nb;
}

}  // namespace

// Variants (rad_impl.h: variant_info): 0 FP32 256x2, 1 FP32 256x4, 2 FP32 128x2,
// 3 tensor-core 256 (3 CTAs/SM), 4 tensor-core 256 (4 CTAs/SM), 5 FP32 256x2 (4 CTAs/SM),
// 6 FP32 256x2 with the literal sum (2 CTAs/SM), 7 tensor-core 256 sweeping each staged
// particle tile in two frequency passes, 8 tensor-core 256 with four 16-frequency blocks
// per warp (512 frequencies per tile, 2 CTAs/SM), 9 as 8 with the phases' cross
// terms on tensor cores.
size_t accumulate_smem_bytes(int variant) {
  switch (variant) {
    case 2: return Smem<128, false>::bytes;
    case 3:
    case 4: return Smem<256, true>::bytes;
    case 6: return Smem<256, false, true>::bytes;
    case 7:
    case 8: return Smem<256, true, false, 2>::bytes;
    case 9: return Smem<256, true, false, 2, true>::bytes;
    default: return Smem<256, false>::bytes;
  }
}

int accumulate_blocks_per_sm(int variant) {
  static std::atomic<int> cached[kMaxDevices][kNumVariants];  // per device; 0 = not yet
  if (variant < 0 || variant >= kNumVariants) variant = 0;
  const int dev = current_device();
  const bool cache = dev >= 0 && dev < kMaxDevices;
  if (cache) {
    const int c = cached[dev][variant].load(std::memory_order_relaxed);
    if (c > 0) return c;
  }
  int nb;
  switch (variant) {
    case 1: nb = blocks_per_sm<256, 4, 2, false, false>(); break;
    case 2: nb = blocks_per_sm<128, 2, 6, false, false>(); break;
    case 3: nb = blocks_per_sm<256, 1, 3, true, false>(); break;
    case 4: nb = blocks_per_sm<256, 1, 4, true, false>(); break;
    case 5: nb = blocks_per_sm<256, 2, 4, false, false>(); break;
    case 6: nb = blocks_per_sm<256, 2, 2, false, true>(); break;
    case 7: nb = blocks_per_sm<256, 1, 3, true, false, 2>(); break;
    case 8: nb = blocks_per_sm<256, 2, 2, true, false>(); break;
    case 9: nb = blocks_per_sm<256, 2, 2, true, false, 1, true>(); break;
    default: nb = blocks_per_sm<256, 2, 3, false, false>(); break;
  }
  if (cache) cached[dev][variant].store(nb, std::memory_order_relaxed);
  return nb;
}

cudaError_t launch_accumulate(int variant, const LaunchArgs& a, int grid, cudaStream_t s) {
  switch (variant) {
    case 1: return launch_acc<256, 4, 2, false, false>(a, grid, s);
    case 2: return launch_acc<128, 2, 6, false, false>(a, grid, s);
    case 3: return launch_acc<256, 1, 3, true, false>(a, grid, s);
    case 4: return launch_acc<256, 1, 4, true, false>(a, grid, s);
    case 5: return launch_acc<256, 2, 4, false, false>(a, grid, s);
    case 6: return launch_acc<256, 2, 2, false, true>(a, grid, s);
    case 7: return launch_acc<256, 1, 3, true, false, 2>(a, grid, s);
    case 8: return launch_acc<256, 2, 2, true, false>(a, grid, s);
    case 9: return launch_acc<256, 2, 2, true, false, 1, true>(a, grid, s);
    default: return launch_acc<256, 2, 3, false, false>(a, grid, s);
  }
}

}  // namespace radimpl
