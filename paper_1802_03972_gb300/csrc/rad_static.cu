// rad_accumulate_static: one accumulation step for callers that cannot
// allocate device memory.  All working memory lives in one file-scope device
// array (g_scratch) whose device address is looked up once per device; the
// step then runs the library's usual pre-pass and accumulate kernels on it.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <mutex>

#include "rad.h"
#include "rad_ctx.h"
#include "rad_impl.h"

using namespace radimpl;

namespace {

// Byte offsets inside the scratch array (each 256-byte aligned).
constexpr size_t kOffJob = 0;                                   // JobStatic
constexpr size_t kOffRef = 1024;                                // double[4]
constexpr size_t kOffStatus = kOffRef + 32;                     // int
constexpr size_t kOffCounter = kOffRef + 40;                    // unsigned long long
constexpr size_t kOffOmTab = 1280;                              // float[kOmTab][MAX_OMEGA]
constexpr size_t kOffOmTurns = kOffOmTab + 4 * kOmTab * RAD_STATIC_MAX_OMEGA;  // double[MAX_OMEGA]
constexpr size_t kOffDirTab = kOffOmTurns + 8 * RAD_STATIC_MAX_OMEGA;       // float[12][MAX_DIRS]
constexpr size_t kOffDirs = kOffDirTab + 4 * 12 * RAD_STATIC_MAX_DIRS;      // double[MAX_DIRS][3]
constexpr int kMaxTiles = 8192;
constexpr size_t kOffTileCnt = kOffDirs + 8 * 3 * RAD_STATIC_MAX_DIRS;      // unsigned[kMaxTiles]
constexpr size_t kOffRec = kOffTileCnt + 4 * kMaxTiles;                     // float[MAX_PARTICLES][20]
constexpr int kMaxChunks = 4;
constexpr size_t kOffPart = kOffRec + 4 * (size_t)kRecFields * RAD_STATIC_MAX_PARTICLES;
constexpr size_t kScratchUsed = kOffPart + 4 * (size_t)kMaxChunks * kComps * RAD_STATIC_MAX_BINS;
static_assert(kScratchUsed <= RAD_STATIC_SCRATCH_BYTES, "scratch layout exceeds its size");
static_assert(sizeof(JobStatic) <= kOffRef - kOffJob, "job table does not fit");
static_assert(kOffRef % 256 == 0 && kOffOmTab % 256 == 0 && kOffOmTurns % 256 == 0 &&
                  kOffDirTab % 256 == 0 && kOffDirs % 256 == 0 && kOffTileCnt % 256 == 0 &&
                  kOffRec % 256 == 0 && kOffPart % 256 == 0,
              "scratch offsets must stay 256-byte aligned");

// The scratch array: held by every GPU that loads the library until exit.
static __device__ __align__(256) unsigned char g_scratch[RAD_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_base[kMaxDevices] = {};

// Device address of g_scratch on the current device (looked up once per device).
cudaError_t scratch_base(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_base[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return e;
    g_base[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_base[dev];
  return cudaSuccess;
}

constexpr double kTwoPi = 6.283185307179586476925286766559;

// One block: frequency and direction tables, zeroed counters, the job table.
__global__ void __launch_bounds__(1024) static_setup_kernel(const double* __restrict__ omega,
                                                            const double* __restrict__ dirs,
                                                            JobStatic js, unsigned char* base) {
  __shared__ float s_max[32];
  __shared__ int s_bad;
  if (threadIdx.x == 0) s_bad = 0;
  __syncthreads();
  float* om_tab = reinterpret_cast<float*>(base + kOffOmTab);
  double* om_turns = reinterpret_cast<double*>(base + kOffOmTurns);
  float* dir_tab = reinterpret_cast<float*>(base + kOffDirTab);
  double* nd = reinterpret_cast<double*>(base + kOffDirs);
  unsigned* tile_cnt = reinterpret_cast<unsigned*>(base + kOffTileCnt);
  const int no = js.n_omega, ndir = js.n_dir;
  float mx = 0.0f;
  for (int i = threadIdx.x; i < no; i += blockDim.x) {
    double om = omega[i];
    if (!(om > 0.0) || !isfinite(om)) {
      // invalid: a harmless finite stand-in; the step is skipped (see below)
      s_bad = 1;
      om = 1.0;
    }
    const double turns = om / kTwoPi;
    const float hi = __double2float_rn(turns);
    const float lo = __double2float_rn(turns - (double)hi);
    om_turns[i] = turns;
    om_tab[i] = hi;
    om_tab[no + i] = __double2float_rn(kTwoPi * (double)hi);
    om_tab[2 * no + i] = __double2float_rn(kTwoPi * (double)lo);
    mx = fmaxf(mx, fabsf(hi));
  }
  for (int d = threadIdx.x; d < ndir; d += blockDim.x) {
    double n[3] = {dirs[3 * d], dirs[3 * d + 1], dirs[3 * d + 2]};
    const double len = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    if (!(len > 0.0) || !isfinite(len)) {
      s_bad = 1;
      n[0] = n[1] = 0.0;
      n[2] = 1.0;
    } else {
      for (int i = 0; i < 3; ++i) n[i] /= len;
    }
    int ax = 0;
    if (fabs(n[1]) < fabs(n[ax])) ax = 1;
    if (fabs(n[2]) < fabs(n[ax])) ax = 2;
    double a[3] = {0.0, 0.0, 0.0};
    a[ax] = 1.0;
    const double an = a[0] * n[0] + a[1] * n[1] + a[2] * n[2];
    double e1[3] = {a[0] - an * n[0], a[1] - an * n[1], a[2] - an * n[2]};
    const double l1 = sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
    for (int i = 0; i < 3; ++i) e1[i] /= l1;
    const double e2[3] = {n[1] * e1[2] - n[2] * e1[1], n[2] * e1[0] - n[0] * e1[2],
                          n[0] * e1[1] - n[1] * e1[0]};
    for (int i = 0; i < 3; ++i) {
      nd[3 * d + i] = n[i];
      const float hi = __double2float_rn(n[i]);
      dir_tab[i * ndir + d] = hi;
      dir_tab[(3 + i) * ndir + d] = __double2float_rn(n[i] - (double)hi);
      dir_tab[(6 + i) * ndir + d] = __double2float_rn(e1[i]);
      dir_tab[(9 + i) * ndir + d] = __double2float_rn(e2[i]);
    }
  }
  // Calls share the array: clear what must start at zero.
  for (int i = threadIdx.x; i < js.n_tiles; i += blockDim.x) tile_cnt[i] = 0u;
  for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
  if ((threadIdx.x & 31) == 0) s_max[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    float m = 0.0f;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) m = fmaxf(m, s_max[i]);
    js.tau_fast = (float)(2097152.0 / fmax((double)m, 1e-300));  // 2^21 turns
    // An invalid grid skips the step: every particle then weighs zero, so the
    // caller's accumulators keep their value, and the status word says why.
    js.skip = s_bad;
    *reinterpret_cast<JobStatic*>(base + kOffJob) = js;
    *reinterpret_cast<int*>(base + kOffStatus) = s_bad ? ST_BAD_GRID : 0;
    *reinterpret_cast<unsigned long long*>(base + kOffCounter) = 0ULL;
  }
}

}  // namespace

extern "C" rad_status rad_accumulate_static(const double* omega, int32_t n_omega,
                                            const double* dirs, int32_t n_dir, int64_t n,
                                            const double* r, const double* beta,
                                            const double* beta_dot, const double* w, double t,
                                            double dt, float* state, void* stream) {
  if (!omega || !dirs || !state || n_omega < 1 || n_dir < 1) return RAD_EINVAL;
  if (n_omega > RAD_STATIC_MAX_OMEGA || n_dir > RAD_STATIC_MAX_DIRS ||
      (long long)n_omega * n_dir > RAD_STATIC_MAX_BINS || n < 0 || n > RAD_STATIC_MAX_PARTICLES)
    return RAD_EINVAL;
  if (!isfinite(t) || !isfinite(dt) || !(dt > 0.0)) return RAD_EINVAL;
  if (n > 0 && (!r || !beta || !beta_dot || !w)) return RAD_EINVAL;
  unsigned char* base = nullptr;
  if (scratch_base(&base) != cudaSuccess) return RAD_ECUDA;
  if (n == 0) return RAD_OK;
  cudaStream_t s = (cudaStream_t)stream;

  // Tiling and chunking as a context with the default tile would use, with at
  // most kMaxChunks work-item chunks so the partials fit the array.
  const int variant = 0;
  JobStatic js;
  memset(&js, 0, sizeof(js));
  js.n_omega = n_omega;
  js.n_dir = n_dir;
  js.n_bins = n_omega * n_dir;
  fill_tiles(js, variant, default_omega_tile(variant, n_omega));
  if (js.n_tiles > kMaxTiles) return RAD_EINVAL;
  int ck = auto_chunk_for(variant, n, js.n_tiles, false);  // (no fine-chunked tail here)
  int n_chunks = (int)((n + ck - 1) / ck);
  if (n_chunks > kMaxChunks) {
    long long c2 = (n + kMaxChunks - 1) / kMaxChunks;
    ck = (int)((c2 + kChunkAlign - 1) / kChunkAlign * kChunkAlign);
    n_chunks = (int)((n + ck - 1) / ck);
  }
  js.chunk_cap = kMaxChunks;
  js.n_cap = RAD_STATIC_MAX_PARTICLES;
  js.om_tab = reinterpret_cast<const float*>(base + kOffOmTab);
  js.om_turns = reinterpret_cast<const double*>(base + kOffOmTurns);
  js.omega = omega;
  js.dir_tab = reinterpret_cast<const float*>(base + kOffDirTab);
  js.dirs = reinterpret_cast<const double*>(base + kOffDirs);
  js.state = state;
  js.partials = reinterpret_cast<float*>(base + kOffPart);
  js.tile_cnt = reinterpret_cast<unsigned*>(base + kOffTileCnt);
  js.rec = reinterpret_cast<float*>(base + kOffRec);
  js.ref = reinterpret_cast<double*>(base + kOffRef);
  js.status = reinterpret_cast<int*>(base + kOffStatus);

  static_setup_kernel<<<1, 1024, 0, s>>>(omega, dirs, js, base);
  count_launches(1);
  if (cudaGetLastError() != cudaSuccess) return RAD_ECUDA;

  LaunchArgs a;
  memset(&a, 0, sizeof(a));
  a.js = reinterpret_cast<const JobStatic*>(base + kOffJob);
  a.n_jobs = 1;
  a.use_inline = 1;
  a.n_items = (long long)js.n_tiles * n_chunks;
  a.item_counter = reinterpret_cast<unsigned long long*>(base + kOffCounter);
  JobCall& K = a.inline_call;
  K.n = n;
  K.r = r;
  K.beta = beta;
  K.bdot = beta_dot;
  K.w = w;
  K.t = t;
  K.dt = dt;
  K.ck = ck;
  K.n_chunks = n_chunks;
  if (launch_prepass(a, (int)((n + 255) / 256), s) != cudaSuccess) return RAD_ECUDA;
  const long long grid = std::min<long long>(a.n_items, resident_ctas(variant));
  if (launch_accumulate(variant, a, (int)grid, s) != cudaSuccess) return RAD_ECUDA;
  return RAD_OK;
}

// Status of the latest rad_accumulate_static call on this device: one 4-byte
// read of the status word in the scratch array, in stream order.
extern "C" rad_status rad_static_status(void* stream) {
  unsigned char* base = nullptr;
  if (scratch_base(&base) != cudaSuccess) return RAD_ECUDA;
  cudaStream_t s = (cudaStream_t)stream;
  int st = 0;
  if (cudaMemcpyAsync(&st, base + kOffStatus, sizeof(int), cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return RAD_ECUDA;
  if (st & ST_BOUNDS) {
    rad_log(1, "an index check of the debug build failed in the allocation-free entry (status 0x%x)",
            st);
    return RAD_ECUDA;
  }
  if (st & ST_TIMEOUT) return RAD_ETIMEOUT;
  if (st & ST_BAD_GRID) return RAD_EINVAL;
  if (st & ST_BAD_PARTICLE) return RAD_EDATA;
  return RAD_OK;
}
