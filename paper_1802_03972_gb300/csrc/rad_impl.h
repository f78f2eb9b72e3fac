// Internal declarations of the radiation library (not part of the C ABI).
//
// Data layout in HBM, per job (one rad_ctx):
//   om_tab   float [3][n_omega]  omega/2pi (hi part), and 2pi times its hi and
//                                lo parts (rad/s) for the phase's cross terms
//   om_turns double [n_omega]    omega / 2pi (turns per second)
//   omega    double [n_omega]
//   dir_tab  float [12][n_dir]   n hi, n lo, transverse basis e1, e2
//   dirs     double [n_dir][3]
//   state    float [16][n_bins]  8 compensated sums + 8 compensations:
//                                U.e1 re/im, U.e2 re/im, V.e1 re/im, V.e2 re/im
//   partials float [chunks][8][n_bins]   per-work-item partial sums of a call
//   partials_f float  the same for the call's fine-chunked last tiles
//                     (TailPlan): per level l, [chunks_l][8][L_l][tile bins],
//                     level 1's region after level 0's
//   rec      float [n_cap][20]   per-particle records written by the pre-pass
// Bins are row-major: bin = direction * n_omega + frequency.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "rad.h"

namespace radimpl {

constexpr int kRecFields = 20;
constexpr int kComps = 8;
constexpr int kDirTab = 12;
constexpr int kOmTab = 3;
// Work items hold a multiple of 256 macro-particles: a whole number of
// shared-memory tiles (threads / directions-per-tile particles) for every
// kernel variant and tile shape.
constexpr int kChunkAlign = 256;
// Levels of fine-chunked last tiles (TailPlan).
constexpr int kTailLevels = 2;
// Automatic chunking aims at this many (coarse) work items per resident
// block when the job's last tiles are fine-chunked (TailPlan: tensor-core
// variants, not literal).  Each item has fixed costs (the first tile's exposed
// copy, zeroing and writing its partial sums, ~5 us), so fewer, longer items
// are cheaper; the end-of-launch tail they would leave is cut by the fine-
// chunked last tiles.  Measured with the tensor-core variant 9 on the LWFA workload
// (1e5 particles, 512 x 256 bins), kernel time per step: 8 items 6.858 ms, 6
// 6.916, 10 6.882, 16 6.880, 24 6.915, 4 6.984 (items of one size, 24: 6.957) ...
constexpr int kItemsPerCta = 8;
// ... and this many without the fine-chunked tail (FP32 variants, the literal
// sum, the allocation-free entry): there the blocks that finish last wait on at
// most one item, so shorter items shorten the tail (variant 8 before the fine
// tail: 24 items 7.13 ms per step, 16 items 7.19) ...
constexpr int kItemsPerCtaUniform = 24;
// ... but gives a work item at least this many particles, over which its fixed
// costs (the first tile's exposed copy, zeroing and writing its partial sums)
// spread: on the batched job mix of small jobs this measured 1 % faster.
constexpr int kMinChunk = 2048;
static_assert(kMinChunk % kChunkAlign == 0, "the minimum chunk is a whole number of tiles");

// Wide calls (particles farther than half the fast phase range from the
// call's reference point): a stable bucket sort along the grid's mean
// direction (kSortBuckets buckets of width bucket_w centred on the reference,
// kSortBlock particles per histogram block) puts nearby particles next to
// each other, and records are written relative to the first particle of
// each sorted kGroup-particle group; the accumulate kernel rotates each tile's
// sums by the group's reference phase.
constexpr int kSortBlock = 2048;
// A context's counter block (unsigned long long words, zeroed before every
// call): [0], [1] the two accumulate kernels' work-item counters, [2] the
// call's wide flag (an int).
constexpr int kCounterWords = 3;
constexpr int kSortBuckets = 4096;
constexpr int kGroup = 256;
static_assert(kGroup == kChunkAlign, "a work item holds whole sorted groups");

// Device status bits (per job).
// ST_BOUNDS: an index check of a debug build (RAD_DEBUG_BOUNDS) failed.
// ST_BAD_GRID: a frequency or direction given in device memory (the
// allocation-free entry) was not finite and positive / non-zero; the step was
// skipped.
enum : int { ST_BAD_PARTICLE = 1, ST_SLOW_PHASE = 2, ST_TIMEOUT = 4, ST_BOUNDS = 8, ST_BAD_GRID = 16 };

// Per-job data that does not change between calls.
struct JobStatic {
  int n_omega, n_dir, n_bins;
  int wt, nt;                     // tile: wt frequencies x nt directions
  int tiles_om, tiles_dir, n_tiles;
  float tau_fast;                 // |delta tau| bound of the fast phase path, s
  int chunk_cap;                  // capacity of partials, in chunks
  long long n_cap;                // capacity of rec, in particles
  const float* om_tab;
  const double* om_turns;
  const double* omega;
  const float* dir_tab;
  const double* dirs;
  float* state;
  float* partials;                // [chunk_cap][kComps][n_bins]
  // the fine-chunked last tiles of a call (see TailPlan): per level l,
  // [n_chunks_f[l]][kComps][tail_tiles[l]][nt * wt], level 1 after level 0;
  // fine_cap floats
  float* partials_f;
  long long fine_cap;
  unsigned* tile_cnt;             // [n_tiles] arrival counters (self-resetting)
  float* rec;
  double* ref;                    // [4]: reference position xyz, t (per call)
  int* status;
  // literal mode (RAD_FF_LITERAL): the paper's sum P with weights F_k(omega)
  int literal;
  int skip;                       // 1: the grid is invalid, every particle weighs zero
  const float* f2_tab;            // [n_omega] f(omega)^2 of the creation shape
  float* state_p;                 // [8][n_bins]: P.e1, P.e2 re/im sums, then compensations
  float* partials_p;              // [chunk_cap][4][n_bins]
  // wide calls (null wide_flag: never; the tiles of a spread call then take
  // the FP64 phase path)
  int* wide_flag;                 // per call: 1 if the call is wide (set by the pre-pass)
  double axis[3];                 // sort axis: the grid's mean direction (unit)
  double cone_sin;                // sine of the largest angle of a direction from the axis (1 past 90 deg)
  double bucket_w;                // bucket width along the axis, m
  int* perm;                      // [n_cap] sorted position -> particle index
  int* sort_counts;               // [ceil(n_cap / kSortBlock)][kSortBuckets]
  int* bucket_base;               // [kSortBuckets] first sorted position of each bucket
  double* gref;                   // [ceil(n_cap / kGroup)][3] group reference - call reference, m
};

// Per-call data of one job.
struct JobCall {
  long long n;
  const double* r;
  const double* beta;
  const double* bdot;
  const double* w;
  double t, dt;
  int ck;                // macro-particles per work item (multiple of kChunkAlign)
  int n_chunks;
  long long item_begin;  // first global work item of this job
  int block_begin;       // first pre-pass block of this job
  int sort_block_begin;  // first sort-histogram block of this job
  // Fine-chunked last tiles (TailPlan), level 0 then level 1 in tile order
  // (level 1 the job's last tail_tiles[1] tiles): tail_tiles[l] tiles with
  // chunks of ck_f[l] (n_chunks_f[l] per tile)
  int tail_tiles[kTailLevels];
  int ck_f[kTailLevels];
  int n_chunks_f[kTailLevels];
};

// Finer work items for the last tiles of a job (tensor-core variants).  With
// items of one size, the launch ends with the resident blocks finishing their
// last items at spread-out times, about half an item idle per block.  A job
// that fills the GPU at least twice over cuts its last L0 tiles into chunks of
// a quarter of the size, L0 = ceil(grid / n_chunks) + 1: enough fine work for
// every resident block to move on to it before the coarse items run out.  The
// fine items' ends are spread in turn, over one fine item: the L1 tiles after
// those, the job's last, take a quarter of the fine chunk, and
// L1 = ceil(grid / n_chunks_1) + 1 from their own chunk count, about one of
// these items per resident block, so the idle end is about half of the
// finest item.  Each level needs a chunk at least one particle tile
// (kChunkAlign) and smaller than the one before it, and all levels together at
// most half the job's tiles.  The plan depends on the job alone (its size and
// tiling) and the device's resident blocks, so a job is chunked alike alone,
// in a batch and in the server.
struct TailLevel {
  int tiles = 0;     // tiles of this level
  int ck = 0;        // their chunk, a multiple of kChunkAlign
  int n_chunks = 0;  // their chunks per tile
};
struct TailPlan {
  TailLevel lv[kTailLevels];
  int tiles() const {
    int t = 0;
    for (int l = 0; l < kTailLevels; ++l) t += lv[l].tiles;
    return t;
  }
  long long items(int n_tiles, int n_chunks_coarse) const {
    long long it = (long long)(n_tiles - tiles()) * n_chunks_coarse;
    for (int l = 0; l < kTailLevels; ++l) it += (long long)lv[l].tiles * lv[l].n_chunks;
    return it;
  }
  // floats of JobStatic::partials_f the levels before `level` take
  long long level_offset(int level, int bins_per_tile) const {
    long long f = 0;
    for (int l = 0; l < level; ++l) f += (long long)lv[l].n_chunks * kComps * lv[l].tiles * bins_per_tile;
    return f;
  }
  // floats of JobStatic::partials_f the plan needs
  long long fine_floats(int bins_per_tile) const { return level_offset(kTailLevels, bins_per_tile); }
};
inline TailPlan tail_plan(bool tensor_core, long long n, int n_tiles, int ck, int n_chunks,
                          long long grid) {
  TailPlan t;
  if (!tensor_core || n <= 0 || (long long)n_tiles * n_chunks < 2 * grid) return t;
  int tiles = 0;
  for (int l = 0; l < kTailLevels; ++l) {
    int ckf = (ck / 4 + kChunkAlign - 1) / kChunkAlign * kChunkAlign;
    if (ckf < kChunkAlign) ckf = kChunkAlign;
    if (ckf >= ck) break;
    const long long ncf = (n + ckf - 1) / ckf;
    const long long per = l == 0 ? n_chunks : ncf;  // chunks per tile L is counted in
    const long long L = (grid + per - 1) / per + 1;
    if (2 * (tiles + L) > n_tiles) break;
    t.lv[l].tiles = (int)L;
    t.lv[l].ck = ckf;
    t.lv[l].n_chunks = (int)ncf;
    tiles += (int)L;
    ck = ckf;
  }
  return t;
}
// The plan's fields of a call.
inline void set_tail(JobCall& K, const TailPlan& t) {
  for (int l = 0; l < kTailLevels; ++l) {
    K.tail_tiles[l] = t.lv[l].tiles;
    K.ck_f[l] = t.lv[l].ck;
    K.n_chunks_f[l] = t.lv[l].n_chunks;
  }
}

struct LaunchArgs {
  const JobStatic* js;   // device [n_jobs]
  const JobCall* jc;     // device [n_jobs] (unused when use_inline)
  int n_jobs;
  int use_inline;        // 1: single job, call passed by value below
  long long n_items;
  // [2] work-item counters: [0] the kernel for ordinary calls, [1] the kernel
  // for wide calls (both zeroed before the launch)
  unsigned long long* item_counter;
  JobCall inline_call;
  // Profiling only (else null): [0] SM clock cycles and [1] nanoseconds, each
  // summed over the accumulate CTAs' lifetimes.
  unsigned long long* prof_clk;
  // Set (non-zero) by the pre-pass when some job's call is wide; null when no
  // job can be (the wide kernels are then not launched).
  int* any_wide;
};

// Kernel variants of the mixed-precision accumulate kernel.
struct Variant {
  int threads;
  int w;       // frequencies per thread and pass
  int passes;  // frequency passes over each staged particle tile
};
// 0-2, 5: FP32-FMA accumulation, w frequencies per thread;
// 3-4: tensor-core accumulation, a warp covers 32 frequencies (w = 1 in the
// tiling rules: bins per tile = threads x w x passes, frequency tiles multiples
// of 32 w passes);
// 6: FP32-FMA with the paper's literal sum as well (literal contexts only);
// 7: tensor-core accumulation in two frequency passes per staged particle tile;
// 8: tensor-core accumulation, a warp covers 64 frequencies (w = 2), 2 CTAs/SM;
// 9: as 8, with the phases' float-float cross terms formed by an MMA per block.
constexpr int kNumVariants = 10;
constexpr int kLiteralVariant = 6;
constexpr int kDefaultVariant = 9;  // a new context's tile, and a mixed batch's
inline Variant variant_info(int v) {
  switch (v) {
    case 1: return {256, 4, 1};
    case 2: return {128, 2, 1};
    case 3:
    case 4: return {256, 1, 1};
    case 7: return {256, 1, 2};
    case 8:
    case 9: return {256, 2, 1};
    default: return {256, 2, 1};
  }
}
// Tensor-core (mma.sync) accumulation variants.
inline bool variant_tensor_core(int v) { return v == 3 || v == 4 || v == 7 || v == 8 || v == 9; }
cudaError_t launch_readout_literal(const float* state_p, int n_bins, double* out, cudaStream_t s);

// Launchers (rad_kernels.cu). All enqueue on `s` and return the launch error.
cudaError_t launch_prepass(const LaunchArgs& a, int total_blocks, cudaStream_t s);
// The wide-call kernels (histogram, scan, scatter, sorted records), launched
// after the pre-pass; each returns at once for jobs whose call is not wide.
// sort_blocks / prepass_blocks: the calls' ceil(n / kSortBlock) and
// ceil(n / 256) summed over the jobs.  Adds 4 to the launch count.
cudaError_t launch_wide(const LaunchArgs& a, int sort_blocks, int prepass_blocks, cudaStream_t s);
constexpr int kWideLaunches = 4;
// Sort axis and bucket width of a job (host, at creation).
void wide_geometry(const double* unit_dirs, int n_dir, float tau_fast, double axis[3],
                   double* cone_sin, double* bucket_w);
// Launches the accumulate kernel for ordinary calls and, when a.any_wide is
// set, the one for wide calls after it (one or two launches).
cudaError_t launch_accumulate(int variant, const LaunchArgs& a, int grid, cudaStream_t s);
int accumulate_blocks_per_sm(int variant);
// Per-device caches of launch properties cover device ordinals below this.
constexpr int kMaxDevices = 64;
// The calling thread's current device, or -1 (rad_api.cu).
int current_device();
// Diagnostics to stderr when the environment variable RAD_LOG is set to a
// level >= `level` (1: errors and decisions, 2: also per-job events), printf
// style, one line per call (rad_api.cu).
void rad_log(int level, const char* fmt, ...)
#if defined(__GNUC__)
    __attribute__((format(printf, 2, 3)))
#endif
    ;
size_t accumulate_smem_bytes(int variant);
// Readout of several species accumulated in separate contexts on one grid:
// coherent K0 |sum_s f_s U_s|^2, incoherent K0 sum_s (1 - f_s^2) |V_s|^2.
constexpr int kMaxSpecies = 16;
struct SpeciesArgs {
  int n_species;
  int mixed;                         // 1: FP32 state with compensation, 0: FP64 state
  const float* state[kMaxSpecies];   // mixed
  const double* state64[kMaxSpecies];
  int kind[kMaxSpecies], flags[kMaxSpecies];
  double width[kMaxSpecies];
};
cudaError_t launch_readout_species(const SpeciesArgs& a, int n_omega, int n_bins,
                                   const double* omega, const double* dirs, double* coh,
                                   double* inc, double* tot, cudaStream_t s);
cudaError_t launch_readout(const float* state, int mixed, const double* state64, int n_omega,
                           int n_bins, const double* omega, const double* dirs, rad_ff ff,
                           double* coh, double* inc, double* tot, cudaStream_t s);
cudaError_t launch_fp64(const double* omega, const double* dirs, int n_omega, int n_dir,
                        long long n, const double* r, const double* beta, const double* bdot,
                        const double* w, double t, double dt, double* state64, int* status,
                        cudaStream_t s);
cudaError_t launch_state_add(float* state, const float* other, int n_bins, int n_comps,
                             cudaStream_t s);
cudaError_t launch_state64_add(double* state, const double* other, int n_bins, cudaStream_t s);

void count_launches(int n);

}  // namespace radimpl
