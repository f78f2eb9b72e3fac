// C ABI of the radiation library: contexts, accumulate/readout, checkpoint and
// merge, tile configuration, batched persistent launches with CUDA graphs.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>
#include <stdlib.h>
#include <stdio.h>
#include <stdarg.h>

#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <new>
#include <vector>

#include "rad_ctx.h"
#include "rad_impl.h"

using namespace radimpl;

namespace {

constexpr double kTwoPi = 6.283185307179586476925286766559;
constexpr uint32_t kBlobMagic = 0x52414453u;  // "RADS"
constexpr uint32_t kBlobVersion = 1u;

struct BlobHeader {
  uint32_t magic, version;
  int32_t prec, n_omega, n_dir, n_comp;
  int32_t elem_size, reserved;
  uint64_t payload_bytes;
};

bool is_device_ptr(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

int device_sm_count() {
  static std::atomic<int> cached[kMaxDevices];  // per device; 0 = not yet
  const int dev = current_device();
  const bool cache = dev >= 0 && dev < kMaxDevices;
  if (cache) {
    const int c = cached[dev].load(std::memory_order_relaxed);
    if (c > 0) return c;
  }
  int n = 0;
  if (dev < 0 || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) {
    cudaGetLastError();
    return 1;
  }
  if (cache) cached[dev].store(n, std::memory_order_relaxed);
  return n;
}

template <class T>
cudaError_t dmalloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) return cudaSuccess;
  return cudaMalloc((void**)p, count * sizeof(T));
}

}  // namespace

namespace radimpl {

void rad_log(int level, const char* fmt, ...) {
  static const int threshold = [] {
    const char* v = getenv("RAD_LOG");
    return v ? atoi(v) : 0;
  }();
  if (level > threshold) return;
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  fprintf(stderr, "[rad] %s\n", buf);
}

int current_device() {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  return dev;
}

rad_status check_device(rad_ctx* c) {
  const int d = current_device();
  if (d == c->device) return RAD_OK;
  rad_log(1, "a context of device %d was used with device %d current", c->device, d);
  c->last_err = RAD_EINVAL;
  return RAD_EINVAL;
}

rad_status fail(rad_ctx* c, rad_status s) {
  if (c) {
    c->last_err = s;
    if (s == RAD_ECUDA) c->failed = true;
  }
  return s;
}

rad_status cuda_check(rad_ctx* c, cudaError_t e) {
  if (e == cudaSuccess) return RAD_OK;
  rad_log(1, "CUDA error %d (%s)%s", (int)e, cudaGetErrorString(e),
          e == cudaErrorMemoryAllocation ? "" : "; the context is now failed");
  return fail(c, e == cudaErrorMemoryAllocation ? RAD_ENOMEM : RAD_ECUDA);
}

// Valid tile widths for a variant: 32 * W * m with m dividing THREADS / 32.
int default_omega_tile(int variant, int n_omega) {
  const Variant v = variant_info(variant);
  const int wmin = 32 * v.w * v.passes, wmax = v.threads * v.w * v.passes;
  int wt = wmin;
  while (wt < n_omega && wt < wmax) wt *= 2;
  return wt;
}

bool valid_omega_tile(int variant, int wt) {
  const Variant v = variant_info(variant);
  const int unit = 32 * v.w * v.passes;
  if (wt < unit || wt > v.threads * v.w * v.passes) return false;
  if (wt % unit) return false;
  const int m = wt / unit;
  return (v.threads / 32) % m == 0;
}

void fill_tiles(JobStatic& js, int variant, int wt) {
  const Variant v = variant_info(variant);
  js.wt = wt;
  js.nt = v.threads * v.w * v.passes / wt;
  js.tiles_om = (js.n_omega + wt - 1) / wt;
  js.tiles_dir = (js.n_dir + js.nt - 1) / js.nt;
  js.n_tiles = js.tiles_om * js.tiles_dir;
}

int resident_ctas(int variant) {
  return device_sm_count() * accumulate_blocks_per_sm(variant);
}

// Particles per (coarse) work item: kItemsPerCta items per resident CTA in
// total when the job's last tiles are fine-chunked (fine_tail), else
// kItemsPerCtaUniform; items a multiple of the shared-memory tile.  Depends only
// on the job's shape, n and the device, so a job is chunked the same way alone
// and in a batch.
int auto_chunk_for(int variant, long long n, int n_tiles, bool fine_tail) {
  const long long target =
      (long long)(fine_tail ? kItemsPerCta : kItemsPerCtaUniform) * resident_ctas(variant);
  long long chunks = (target + n_tiles - 1) / n_tiles;
  const long long max_chunks = (n + kChunkAlign - 1) / kChunkAlign;
  chunks = std::max(1LL, std::min(chunks, max_chunks));
  long long ck = (n + chunks - 1) / chunks;
  ck = (ck + kChunkAlign - 1) / kChunkAlign * kChunkAlign;
  if (ck < kMinChunk && n > kMinChunk) ck = kMinChunk;
  if (ck > (1LL << 30)) ck = 1LL << 30;
  return (int)ck;
}

int auto_chunk(const rad_ctx* c, int variant, long long n, int n_tiles) {
  if (c->tile.chunk > 0) return c->tile.chunk;
  return auto_chunk_for(variant, n, n_tiles, variant_tensor_core(variant) && !c->h_js.literal);
}

rad_status upload_static(rad_ctx* c) {
  c->generation++;
  return cuda_check(c, cudaMemcpyAsync(c->d_js, &c->h_js, sizeof(JobStatic),
                                       cudaMemcpyHostToDevice, c->stream));
}

rad_status ensure_capacity(rad_ctx* c, long long n, int n_chunks, long long fine_floats) {
  bool changed = false;
  if (n > c->h_js.n_cap) {
    long long cap = std::max(n, c->h_js.n_cap * 3 / 2);
    cap = (cap + 255) / 256 * 256;
    JobStatic& js = c->h_js;
    if (js.rec) cudaStreamSynchronize(c->stream);
    void* old[] = {js.rec, js.perm, js.sort_counts, js.bucket_base, js.gref};
    for (void* p : old)
      if (p) cudaFree(p);
    js.rec = nullptr;
    js.perm = js.sort_counts = js.bucket_base = nullptr;
    js.gref = nullptr;
    // the record buffer, and the sort buffers of wide calls (12 B per particle)
    rad_status s = cuda_check(c, dmalloc(&js.rec, (size_t)cap * kRecFields));
    if (s == RAD_OK && js.wide_flag) {
      s = cuda_check(c, dmalloc(&js.perm, (size_t)cap));
      if (s == RAD_OK)
        s = cuda_check(c, dmalloc(&js.sort_counts,
                                  (size_t)((cap + kSortBlock - 1) / kSortBlock) * kSortBuckets));
      if (s == RAD_OK) s = cuda_check(c, dmalloc(&js.bucket_base, (size_t)kSortBuckets));
      if (s == RAD_OK) s = cuda_check(c, dmalloc(&js.gref, (size_t)3 * ((cap + kGroup - 1) / kGroup)));
    }
    if (s != RAD_OK) {
      js.n_cap = 0;
      return s;
    }
    js.n_cap = cap;
    changed = true;
  }
  if (n_chunks > c->h_js.chunk_cap) {
    const int cap = std::max(n_chunks, c->h_js.chunk_cap * 3 / 2);
    if (c->h_js.partials) {
      cudaStreamSynchronize(c->stream);
      cudaFree(c->h_js.partials);
      c->h_js.partials = nullptr;
    }
    rad_status s = cuda_check(c, dmalloc(&c->h_js.partials, (size_t)cap * kComps * c->n_bins));
    if (s != RAD_OK) {
      c->h_js.chunk_cap = 0;
      return s;
    }
    if (c->h_js.literal) {
      if (c->h_js.partials_p) cudaFree(c->h_js.partials_p);
      s = cuda_check(c, dmalloc(&c->h_js.partials_p, (size_t)cap * 4 * c->n_bins));
      if (s != RAD_OK) {
        c->h_js.chunk_cap = 0;
        return s;
      }
    }
    c->h_js.chunk_cap = cap;
    changed = true;
  }
  if (fine_floats > c->h_js.fine_cap) {
    const long long cap = std::max(fine_floats, c->h_js.fine_cap * 3 / 2);
    if (c->h_js.partials_f) {
      cudaStreamSynchronize(c->stream);
      cudaFree(c->h_js.partials_f);
      c->h_js.partials_f = nullptr;
    }
    rad_status s = cuda_check(c, dmalloc(&c->h_js.partials_f, (size_t)cap));
    if (s != RAD_OK) {
      c->h_js.fine_cap = 0;
      return s;
    }
    c->h_js.fine_cap = cap;
    changed = true;
  }
  return changed ? upload_static(c) : RAD_OK;
}

// Host copy of the amplitude form factor of Table 1 (f(0) = 1), for the
// per-frequency f^2 table of the literal sum.
double host_form_factor(int kind, double width, double omega) {
  const double x = omega * width / (2.0 * 299792458.0);
  const double s = x == 0.0 ? 1.0 : sin(x) / x;
  switch (kind) {
    case RAD_FF_CIC: return s;
    case RAD_FF_TSC: return s * s;
    case RAD_FF_QSC: return s * s * s;
    case RAD_FF_GAUSS: {
      const double g = omega * width / 299792458.0;
      return exp(-0.5 * g * g);
    }
    default: return 1.0;
  }
}

rad_status stage_inputs(rad_ctx* c, long long n, const double*& r, const double*& beta,
                        const double*& bdot, const double*& w) {
  const bool dev = is_device_ptr(r) && is_device_ptr(beta) && is_device_ptr(bdot) &&
                   is_device_ptr(w);
  if (dev) return RAD_OK;
  const size_t need = (size_t)10 * n;
  if (need > c->stage_cap) {
    if (c->d_stage) {
      cudaStreamSynchronize(c->stream);
      cudaFree(c->d_stage);
      c->d_stage = nullptr;
    }
    rad_status s = cuda_check(c, dmalloc(&c->d_stage, need));
    if (s != RAD_OK) {
      c->stage_cap = 0;
      return s;
    }
    c->stage_cap = need;
  }
  const double* src[4] = {r, beta, bdot, w};
  const size_t cnt[4] = {(size_t)3 * n, (size_t)3 * n, (size_t)3 * n, (size_t)n};
  double* dst = c->d_stage;
  const double* out[4];
  for (int i = 0; i < 4; ++i) {
    rad_status s = cuda_check(c, cudaMemcpyAsync(dst, src[i], cnt[i] * sizeof(double),
                                                 cudaMemcpyDefault, c->stream));
    if (s != RAD_OK) return s;
    out[i] = dst;
    dst += cnt[i];
  }
  r = out[0];
  beta = out[1];
  bdot = out[2];
  w = out[3];
  return RAD_OK;
}

rad_status enqueue_accumulate(rad_ctx* c, long long n, const double* r, const double* beta,
                              const double* bdot, const double* w, double t, double dt) {
  if (c->prec == RAD_PREC_FP64) {
    return cuda_check(c, launch_fp64(c->d_omega, c->d_dirs, c->n_omega, c->n_dir, n, r, beta,
                                     bdot, w, t, dt, c->d_state64, c->h_js.status, c->stream));
  }
  const int variant = c->tile.variant;
  const int ck = auto_chunk(c, variant, n, c->h_js.n_tiles);
  const int n_chunks = (int)((n + ck - 1) / ck);
  const TailPlan tail = tail_plan(variant_tensor_core(variant) && !c->h_js.literal, n,
                                  c->h_js.n_tiles, ck, n_chunks, resident_ctas(variant));
  rad_status s = ensure_capacity(c, n, n_chunks, tail.fine_floats(c->h_js.nt * c->h_js.wt));
  if (s != RAD_OK) return s;
  LaunchArgs a;
  memset(&a, 0, sizeof(a));
  a.js = c->d_js;
  a.jc = nullptr;
  a.n_jobs = 1;
  a.use_inline = 1;
  a.n_items = tail.items(c->h_js.n_tiles, n_chunks);
  a.item_counter = c->d_counter;  // [0], [1]: item counters; [2]: the wide flag
  // A call of at most one sorted group is never wide (the pre-pass does not
  // flag it): it needs neither the wide-call kernels nor the second kernel.
  a.any_wide = n > kGroup ? c->h_js.wide_flag : nullptr;
  JobCall& K = a.inline_call;
  K.n = n;
  K.r = r;
  K.beta = beta;
  K.bdot = bdot;
  K.w = w;
  K.t = t;
  K.dt = dt;
  K.ck = ck;
  K.n_chunks = n_chunks;
  set_tail(K, tail);
  K.item_begin = 0;
  K.block_begin = 0;
  s = cuda_check(c, cudaMemsetAsync(c->d_counter, 0, kCounterWords * sizeof(unsigned long long),
                                    c->stream));
  if (s != RAD_OK) return s;
  cudaEvent_t* ev = nullptr;
  if (c->prof_on) {
    if (c->prof_used + 3 > c->prof_ev.size()) {
      for (int i = 0; i < 3; ++i) {
        cudaEvent_t e;
        s = cuda_check(c, cudaEventCreate(&e));
        if (s != RAD_OK) return s;
        c->prof_ev.push_back(e);
      }
    }
    ev = &c->prof_ev[c->prof_used];
    c->prof_used += 3;
    cudaEventRecord(ev[0], c->stream);
    a.prof_clk = c->d_prof_clk;
  }
  s = cuda_check(c, launch_prepass(a, (int)((n + 255) / 256), c->stream));
  if (s == RAD_OK && a.any_wide)
    s = cuda_check(c, launch_wide(a, (int)((n + kSortBlock - 1) / kSortBlock), (int)((n + 255) / 256),
                                  c->stream));
  if (s != RAD_OK) return s;
  if (ev) cudaEventRecord(ev[1], c->stream);
  const long long grid = std::min<long long>(a.n_items, resident_ctas(variant));
  s = cuda_check(c, launch_accumulate(variant, a, (int)grid, c->stream));
  if (ev) cudaEventRecord(ev[2], c->stream);
  return s;
}

}  // namespace radimpl

extern "C" {

const char* rad_status_str(rad_status s) {
  switch (s) {
    case RAD_OK: return "ok";
    case RAD_EINVAL: return "invalid argument";
    case RAD_ENOMEM: return "out of memory";
    case RAD_ECUDA: return "CUDA error";
    case RAD_EDATA: return "invalid particle data";
    case RAD_ETIMEOUT: return "timed out";
    case RAD_EBUSY: return "busy";
    case RAD_ESTATE: return "invalid state";
    default: return "unknown status";
  }
}

rad_status rad_create(const double* omega, int32_t n_omega, const double* dirs, int32_t n_dir,
                      rad_ff ff, int32_t prec, void* stream, rad_ctx** out) {
  if (!out) return RAD_EINVAL;
  *out = nullptr;
  if (!omega || !dirs || n_omega < 1 || n_dir < 1) return RAD_EINVAL;
  if ((long long)n_omega * n_dir > 0x7fffffffLL) return RAD_EINVAL;
  if (prec != RAD_PREC_MIXED && prec != RAD_PREC_FP64) return RAD_EINVAL;
  if (ff.kind < RAD_FF_POINT || ff.kind > RAD_FF_GAUSS || !(ff.width >= 0.0) ||
      !isfinite(ff.width) || (ff.flags & ~(RAD_FF_3D | RAD_FF_LITERAL)) != 0)
    return RAD_EINVAL;
  // The literal sum weighs each particle with f(omega) of Table 1 (Eq. 12): it
  // needs the mixed path and the direction-independent form factor.
  const bool literal = (ff.flags & RAD_FF_LITERAL) != 0;
  if (literal && (prec != RAD_PREC_MIXED || (ff.flags & RAD_FF_3D))) return RAD_EINVAL;
  for (int i = 0; i < n_omega; ++i)
    if (!(omega[i] > 0.0) || !isfinite(omega[i])) return RAD_EINVAL;
  std::vector<double> nd((size_t)3 * n_dir);
  for (int d = 0; d < n_dir; ++d) {
    const double x = dirs[3 * d], y = dirs[3 * d + 1], z = dirs[3 * d + 2];
    const double len = sqrt(x * x + y * y + z * z);
    if (!isfinite(len) || !(len > 0.0)) return RAD_EINVAL;
    nd[3 * d] = x / len;
    nd[3 * d + 1] = y / len;
    nd[3 * d + 2] = z / len;
  }
  rad_ctx* c = new (std::nothrow) rad_ctx();
  if (!c) return RAD_ENOMEM;
  {  // FNV-1a over the grids' bytes: contexts read out together must share them
    uint64_t h = 1469598103934665603ULL;
    auto mix = [&h](const void* p, size_t n) {
      const unsigned char* b = static_cast<const unsigned char*>(p);
      for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * 1099511628211ULL;
    };
    mix(omega, sizeof(double) * (size_t)n_omega);
    mix(nd.data(), sizeof(double) * nd.size());
    c->grid_hash = h;
    c->device = current_device();
  }
  c->n_omega = n_omega;
  c->n_dir = n_dir;
  c->n_bins = n_omega * n_dir;
  c->ff = ff;
  c->prec = prec;
  c->stream = (cudaStream_t)stream;
  c->tile.variant = kDefaultVariant;
  c->tile.omega_tile = default_omega_tile(kDefaultVariant, n_omega);
  c->tile.chunk = 0;

  // Frequency table: omega/2pi split hi/lo; (hi, 2pi hi, 2pi lo) floats.
  std::vector<float> om_tab((size_t)kOmTab * n_omega);
  std::vector<double> om_turns(n_omega);
  double om_hi_max = 0.0;
  for (int i = 0; i < n_omega; ++i) {
    const double turns = omega[i] / kTwoPi;
    const float hi = (float)turns;
    const float lo = (float)(turns - (double)hi);
    om_turns[i] = turns;
    om_tab[i] = hi;
    om_tab[n_omega + i] = (float)(kTwoPi * (double)hi);
    om_tab[2 * n_omega + i] = (float)(kTwoPi * (double)lo);
    om_hi_max = std::max(om_hi_max, (double)fabsf(hi));
  }
  // Direction table: n (hi, lo) and a transverse orthonormal basis (e1, e2).
  std::vector<float> dir_tab((size_t)kDirTab * n_dir);
  for (int d = 0; d < n_dir; ++d) {
    const double* n = &nd[3 * d];
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
      const float hi = (float)n[i];
      dir_tab[(size_t)i * n_dir + d] = hi;
      dir_tab[(size_t)(3 + i) * n_dir + d] = (float)(n[i] - (double)hi);
      dir_tab[(size_t)(6 + i) * n_dir + d] = (float)e1[i];
      dir_tab[(size_t)(9 + i) * n_dir + d] = (float)e2[i];
    }
  }

  JobStatic& js = c->h_js;
  memset(&js, 0, sizeof(js));
  js.n_omega = n_omega;
  js.n_dir = n_dir;
  js.n_bins = c->n_bins;
  fill_tiles(js, c->tile.variant, c->tile.omega_tile);
  js.tau_fast = (float)(2097152.0 / std::max(om_hi_max, 1e-300));  // 2^21 turns
  wide_geometry(nd.data(), n_dir, js.tau_fast, js.axis, &js.cone_sin, &js.bucket_w);

  rad_status s = RAD_OK;
  auto chk = [&](cudaError_t e) {
    if (s == RAD_OK && e != cudaSuccess) s = (e == cudaErrorMemoryAllocation) ? RAD_ENOMEM : RAD_ECUDA;
  };
  chk(dmalloc(&c->d_omega, n_omega));
  chk(dmalloc(&c->d_om_turns, n_omega));
  chk(dmalloc(&c->d_om_tab, om_tab.size()));
  chk(dmalloc(&c->d_dirs, nd.size()));
  chk(dmalloc(&c->d_dir_tab, dir_tab.size()));
  chk(dmalloc(&c->d_ref, 4));
  chk(dmalloc(&c->d_status, 1));
  chk(dmalloc(&c->d_counter, kCounterWords));
  chk(dmalloc(&c->d_js, 1));
  chk(dmalloc(&c->d_spec, (size_t)3 * c->n_bins));
  if (prec == RAD_PREC_MIXED) {
    chk(dmalloc(&c->d_state, (size_t)2 * kComps * c->n_bins));
    // Enough arrival counters for any tiling (frequency tiles are >= 32 wide).
    c->tile_cnt_cap = ((n_omega + 31) / 32) * n_dir + 1;
    chk(dmalloc(&c->d_tile_cnt, (size_t)c->tile_cnt_cap));
    if (literal) {
      chk(dmalloc(&c->d_state_p, (size_t)8 * c->n_bins));
      chk(dmalloc(&c->d_f2, (size_t)n_omega));
    }
  } else {
    chk(dmalloc(&c->d_state64, (size_t)12 * c->n_bins));
  }
  if (s == RAD_OK) {
    chk(cudaMemcpy(c->d_omega, omega, sizeof(double) * n_omega, cudaMemcpyHostToDevice));
    chk(cudaMemcpy(c->d_om_turns, om_turns.data(), sizeof(double) * n_omega, cudaMemcpyHostToDevice));
    chk(cudaMemcpy(c->d_om_tab, om_tab.data(), sizeof(float) * om_tab.size(), cudaMemcpyHostToDevice));
    chk(cudaMemcpy(c->d_dirs, nd.data(), sizeof(double) * nd.size(), cudaMemcpyHostToDevice));
    chk(cudaMemcpy(c->d_dir_tab, dir_tab.data(), sizeof(float) * dir_tab.size(), cudaMemcpyHostToDevice));
    chk(cudaMemset(c->d_status, 0, sizeof(int)));
    chk(cudaMemset(c->d_ref, 0, 4 * sizeof(double)));
    if (prec == RAD_PREC_MIXED) {
      chk(cudaMemset(c->d_state, 0, sizeof(float) * 2 * kComps * c->n_bins));
      chk(cudaMemset(c->d_tile_cnt, 0, sizeof(unsigned) * c->tile_cnt_cap));
      if (literal && s == RAD_OK) {
        std::vector<float> f2(n_omega);
        for (int i = 0; i < n_omega; ++i) {
          const double f = host_form_factor(ff.kind, ff.width, omega[i]);
          f2[i] = (float)(f * f);
        }
        chk(cudaMemset(c->d_state_p, 0, sizeof(float) * 8 * c->n_bins));
        chk(cudaMemcpy(c->d_f2, f2.data(), sizeof(float) * n_omega, cudaMemcpyHostToDevice));
      }
    } else {
      chk(cudaMemset(c->d_state64, 0, sizeof(double) * 12 * c->n_bins));
    }
  }
  js.om_tab = c->d_om_tab;
  js.om_turns = c->d_om_turns;
  js.omega = c->d_omega;
  js.dir_tab = c->d_dir_tab;
  js.dirs = c->d_dirs;
  js.state = c->d_state;
  js.tile_cnt = c->d_tile_cnt;
  js.ref = c->d_ref;
  js.status = c->d_status;
  js.literal = literal ? 1 : 0;
  js.f2_tab = c->d_f2;
  js.state_p = c->d_state_p;
  // the wide flag lives in the counter block, zeroed before every call
  js.wide_flag = c->d_counter ? reinterpret_cast<int*>(c->d_counter + 2) : nullptr;
  if (literal) {
    c->tile.variant = kLiteralVariant;
    c->tile.omega_tile = default_omega_tile(kLiteralVariant, n_omega);
    fill_tiles(js, c->tile.variant, c->tile.omega_tile);
  }
  if (s == RAD_OK) chk(cudaMemcpy(c->d_js, &js, sizeof(JobStatic), cudaMemcpyHostToDevice));
  if (s != RAD_OK) {
    rad_destroy(c);
    return s;
  }
  *out = c;
  return RAD_OK;
}

void rad_destroy(rad_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  void* ptrs[] = {c->d_omega, c->d_om_turns, c->d_om_tab, c->d_dirs, c->d_dir_tab, c->d_ref,
                  c->d_status, c->d_counter, c->d_js, c->d_spec, c->d_state, c->d_state64,
                  c->d_tile_cnt, c->h_js.rec, c->h_js.partials, c->d_stage, c->d_state_p,
                  c->d_f2, c->h_js.partials_p, c->d_push, c->d_push_bdot, c->h_js.perm,
                  c->h_js.sort_counts, c->h_js.bucket_base, c->h_js.gref, c->h_js.partials_f};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  for (cudaEvent_t e : c->prof_ev) cudaEventDestroy(e);
  if (c->d_prof_clk) cudaFree(c->d_prof_clk);
  cudaGetLastError();
  delete c;
}

rad_status rad_accumulate(rad_ctx* c, int64_t n, const double* r, const double* beta,
                          const double* beta_dot, const double* w, double t, double dt) {
  radimpl::TraceRange trace("rad_accumulate");
  if (!c) return RAD_EINVAL;
  if (c->failed) return RAD_ESTATE;
  if (check_device(c) != RAD_OK) return RAD_EINVAL;
  if (n < 0 || !isfinite(t) || !isfinite(dt) || !(dt > 0.0)) return fail(c, RAD_EINVAL);
  if (n == 0) return RAD_OK;
  if (!r || !beta || !beta_dot || !w) return fail(c, RAD_EINVAL);
  if (n > (1LL << 40)) return fail(c, RAD_EINVAL);
  rad_status s = stage_inputs(c, n, r, beta, beta_dot, w);
  if (s != RAD_OK) return s;
  return enqueue_accumulate(c, n, r, beta, beta_dot, w, t, dt);
}

static rad_status check_status_word(rad_ctx* c) {
  int st = 0;
  rad_status s = cuda_check(c, cudaMemcpyAsync(&st, c->d_status, sizeof(int),
                                               cudaMemcpyDeviceToHost, c->stream));
  if (s != RAD_OK) return s;
  s = cuda_check(c, cudaStreamSynchronize(c->stream));
  if (s != RAD_OK) return s;
  if (st & ST_BOUNDS) {
    // A debug build's index check failed: a sizing error inside the library.
    rad_log(1, "an index check of the debug build failed (status 0x%x)", st);
    c->failed = true;
    return fail(c, RAD_ECUDA);
  }
  if (st & ST_TIMEOUT) {
    // A bounded wait in the kernel gave up: the accumulators are incomplete.
    c->failed = true;
    return fail(c, RAD_ETIMEOUT);
  }
  if (st & ST_BAD_PARTICLE) {
    const int keep = st & ~ST_BAD_PARTICLE;
    s = cuda_check(c, cudaMemcpy(c->d_status, &keep, sizeof(int), cudaMemcpyHostToDevice));
    if (s != RAD_OK) return s;
    return fail(c, RAD_EDATA);
  }
  return RAD_OK;
}

rad_status rad_sync(rad_ctx* c) {
  if (!c) return RAD_EINVAL;
  if (c->failed) return RAD_ESTATE;
  if (check_device(c) != RAD_OK) return RAD_EINVAL;
  rad_status s = cuda_check(c, cudaStreamSynchronize(c->stream));
  if (s != RAD_OK) return s;
  return check_status_word(c);
}

rad_status rad_spectrum_ff(rad_ctx* c, rad_ff ff, double* coh, double* inc, double* tot) {
  radimpl::TraceRange trace("rad_spectrum");
  if (!c) return RAD_EINVAL;
  if (c->failed) return RAD_ESTATE;
  if (check_device(c) != RAD_OK) return RAD_EINVAL;
  // RAD_FF_LITERAL only matters at creation; the readout ignores it.
  if (ff.kind < RAD_FF_POINT || ff.kind > RAD_FF_GAUSS || !(ff.width >= 0.0) ||
      !isfinite(ff.width) || (ff.flags & ~(RAD_FF_3D | RAD_FF_LITERAL)) != 0)
    return fail(c, RAD_EINVAL);
  double* outs[3] = {coh, inc, tot};
  double* dev_out[3];
  bool host[3];
  for (int i = 0; i < 3; ++i) {
    host[i] = outs[i] && !is_device_ptr(outs[i]);
    dev_out[i] = outs[i] ? (host[i] ? c->d_spec + (size_t)i * c->n_bins : outs[i]) : nullptr;
  }
  rad_status s = cuda_check(c, launch_readout(c->d_state, c->prec == RAD_PREC_MIXED, c->d_state64,
                                              c->n_omega, c->n_bins, c->d_omega, c->d_dirs, ff,
                                              dev_out[0], dev_out[1], dev_out[2], c->stream));
  if (s != RAD_OK) return s;
  for (int i = 0; i < 3; ++i) {
    if (!host[i]) continue;
    s = cuda_check(c, cudaMemcpyAsync(outs[i], dev_out[i], sizeof(double) * c->n_bins,
                                      cudaMemcpyDeviceToHost, c->stream));
    if (s != RAD_OK) return s;
  }
  return check_status_word(c);
}

rad_status rad_spectrum_species(rad_ctx* const* ctxs, const rad_ff* ffs, int32_t n_species,
                                double* coh, double* inc, double* tot) {
  radimpl::TraceRange trace("rad_spectrum_species");
  if (!ctxs || !ffs || n_species < 1 || n_species > kMaxSpecies) return RAD_EINVAL;
  rad_ctx* c0 = ctxs[0];
  if (!c0) return RAD_EINVAL;
  SpeciesArgs a;
  memset(&a, 0, sizeof(a));
  a.n_species = n_species;
  a.mixed = c0->prec == RAD_PREC_MIXED;
  for (int i = 0; i < n_species; ++i) {
    rad_ctx* c = ctxs[i];
    const rad_ff& ff = ffs[i];
    if (!c) return RAD_EINVAL;
    if (c->failed) return RAD_ESTATE;
  if (check_device(c) != RAD_OK) return RAD_EINVAL;
    if (c->n_omega != c0->n_omega || c->n_dir != c0->n_dir || c->grid_hash != c0->grid_hash ||
        c->prec != c0->prec)
      return fail(c0, RAD_EINVAL);
    if (ff.kind < RAD_FF_POINT || ff.kind > RAD_FF_GAUSS || !(ff.width >= 0.0) ||
        !isfinite(ff.width) || (ff.flags & ~(RAD_FF_3D | RAD_FF_LITERAL)) != 0)
      return fail(c0, RAD_EINVAL);
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == c) return fail(c0, RAD_EINVAL);  // a species counted twice
    a.state[i] = c->d_state;
    a.state64[i] = c->d_state64;
    a.kind[i] = ff.kind;
    a.flags[i] = ff.flags;
    a.width[i] = ff.width;
  }
  // Every species' queued work must be complete before its state is read; a
  // species that saw invalid particles is reported after the spectra are written.
  rad_status data = RAD_OK;
  for (int i = 0; i < n_species; ++i) {
    const rad_status s = check_status_word(ctxs[i]);
    if (s == RAD_EDATA) data = RAD_EDATA;
    else if (s != RAD_OK) return s;
  }
  double* outs[3] = {coh, inc, tot};
  double* dev_out[3];
  bool host[3];
  for (int i = 0; i < 3; ++i) {
    host[i] = outs[i] && !is_device_ptr(outs[i]);
    dev_out[i] = outs[i] ? (host[i] ? c0->d_spec + (size_t)i * c0->n_bins : outs[i]) : nullptr;
  }
  rad_status s = cuda_check(c0, launch_readout_species(a, c0->n_omega, c0->n_bins, c0->d_omega,
                                                       c0->d_dirs, dev_out[0], dev_out[1],
                                                       dev_out[2], c0->stream));
  for (int i = 0; s == RAD_OK && i < 3; ++i) {
    if (!host[i]) continue;
    s = cuda_check(c0, cudaMemcpyAsync(outs[i], dev_out[i], sizeof(double) * c0->n_bins,
                                       cudaMemcpyDeviceToHost, c0->stream));
  }
  if (s == RAD_OK) s = cuda_check(c0, cudaStreamSynchronize(c0->stream));
  if (s != RAD_OK) return s;
  return data;
}

rad_status rad_spectrum(rad_ctx* c, double* coh, double* inc, double* tot) {
  if (!c) return RAD_EINVAL;
  return rad_spectrum_ff(c, c->ff, coh, inc, tot);
}

rad_status rad_reset(rad_ctx* c) {
  if (!c) return RAD_EINVAL;
  if (c->failed) return RAD_ESTATE;
  if (check_device(c) != RAD_OK) return RAD_EINVAL;
  cudaError_t e = (c->prec == RAD_PREC_MIXED)
                      ? cudaMemsetAsync(c->d_state, 0, sizeof(float) * 2 * kComps * c->n_bins, c->stream)
                      : cudaMemsetAsync(c->d_state64, 0, sizeof(double) * 12 * c->n_bins, c->stream);
  rad_status s = cuda_check(c, e);
  if (s != RAD_OK) return s;
  if (c->d_state_p) {
    s = cuda_check(c, cudaMemsetAsync(c->d_state_p, 0, sizeof(float) * 8 * c->n_bins, c->stream));
    if (s != RAD_OK) return s;
  }
  s = cuda_check(c, cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream));
  if (s == RAD_OK) c->last_err = RAD_OK;
  return s;
}

rad_status rad_spectrum_literal(rad_ctx* c, double* out) {
  radimpl::TraceRange trace("rad_spectrum_literal");
  if (!c || !out) return RAD_EINVAL;
  if (c->failed) return RAD_ESTATE;
  if (check_device(c) != RAD_OK) return RAD_EINVAL;
  if (!c->d_state_p) return fail(c, RAD_ESTATE);
  const bool host = !is_device_ptr(out);
  double* dst = host ? c->d_spec : out;
  rad_status s = cuda_check(c, launch_readout_literal(c->d_state_p, c->n_bins, dst, c->stream));
  if (s != RAD_OK) return s;
  if (host) {
    s = cuda_check(c, cudaMemcpyAsync(out, dst, sizeof(double) * c->n_bins, cudaMemcpyDeviceToHost,
                                      c->stream));
    if (s != RAD_OK) return s;
  }
  return check_status_word(c);
}

rad_status rad_last_error(const rad_ctx* c) { return c ? c->last_err : RAD_EINVAL; }

rad_status rad_profile_enable(rad_ctx* c, int32_t on) {
  if (!c) return RAD_EINVAL;
  if (c->failed) return RAD_ESTATE;
  if (check_device(c) != RAD_OK) return RAD_EINVAL;
  if (on && !c->d_prof_clk) {
    rad_status s = cuda_check(c, cudaMalloc(&c->d_prof_clk, 2 * sizeof(unsigned long long)));
    if (s == RAD_OK)
      s = cuda_check(c, cudaMemsetAsync(c->d_prof_clk, 0, 2 * sizeof(unsigned long long), c->stream));
    if (s != RAD_OK) return s;
  }
  c->prof_on = on != 0;
  return RAD_OK;
}

rad_status rad_profile_clock(rad_ctx* c, double* sm_mhz) {
  if (!c || !sm_mhz) return RAD_EINVAL;
  if (c->failed) return RAD_ESTATE;
  if (check_device(c) != RAD_OK) return RAD_EINVAL;
  *sm_mhz = 0.0;
  if (!c->d_prof_clk) return RAD_OK;
  unsigned long long h[2] = {0, 0};
  rad_status s = cuda_check(c, cudaMemcpyAsync(h, c->d_prof_clk, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
  if (s == RAD_OK) s = cuda_check(c, cudaStreamSynchronize(c->stream));
  if (s == RAD_OK)
    s = cuda_check(c, cudaMemsetAsync(c->d_prof_clk, 0, 2 * sizeof(unsigned long long), c->stream));
  if (s != RAD_OK) return s;
  if (h[1] > 0) *sm_mhz = 1e3 * (double)h[0] / (double)h[1];
  return RAD_OK;
}

rad_status rad_profile_read(rad_ctx* c, double* prepass_ms, double* accumulate_ms,
                            int64_t* calls) {
  if (!c) return RAD_EINVAL;
  if (c->failed) return RAD_ESTATE;
  if (check_device(c) != RAD_OK) return RAD_EINVAL;
  rad_status s = cuda_check(c, cudaStreamSynchronize(c->stream));
  if (s != RAD_OK) return s;
  double pp = 0.0, ac = 0.0;
  for (size_t i = 0; i + 3 <= c->prof_used; i += 3) {
    float a = 0.f, b = 0.f;
    cudaEventElapsedTime(&a, c->prof_ev[i], c->prof_ev[i + 1]);
    cudaEventElapsedTime(&b, c->prof_ev[i + 1], c->prof_ev[i + 2]);
    pp += a;
    ac += b;
  }
  if (prepass_ms) *prepass_ms = pp;
  if (accumulate_ms) *accumulate_ms = ac;
  if (calls) *calls = (int64_t)(c->prof_used / 3);
  c->prof_used = 0;
  return RAD_OK;
}

// Mixed: the 16 accumulator floats per bin, then (literal mode) the 8 of P.
static size_t payload_bytes(const rad_ctx* c) {
  if (c->prec != RAD_PREC_MIXED) return sizeof(double) * 12 * (size_t)c->n_bins;
  return sizeof(float) * (2 * kComps + (c->d_state_p ? 8 : 0)) * (size_t)c->n_bins;
}
static size_t main_payload_bytes(const rad_ctx* c) {
  return c->prec == RAD_PREC_MIXED ? sizeof(float) * 2 * kComps * (size_t)c->n_bins
                                   : sizeof(double) * 12 * (size_t)c->n_bins;
}

size_t rad_state_size(const rad_ctx* c) {
  if (!c) return 0;
  return sizeof(BlobHeader) + payload_bytes(c);
}

rad_status rad_state_export(rad_ctx* c, void* buf, size_t n) {
  if (!c || !buf) return RAD_EINVAL;
  if (c->failed) return RAD_ESTATE;
  if (check_device(c) != RAD_OK) return RAD_EINVAL;
  if (n < rad_state_size(c)) return fail(c, RAD_EINVAL);
  BlobHeader h;
  memset(&h, 0, sizeof(h));
  h.magic = kBlobMagic;
  h.version = kBlobVersion;
  h.prec = c->prec;
  h.n_omega = c->n_omega;
  h.n_dir = c->n_dir;
  h.n_comp = c->prec == RAD_PREC_MIXED ? 2 * kComps + (c->d_state_p ? 8 : 0) : 12;
  h.elem_size = c->prec == RAD_PREC_MIXED ? 4 : 8;
  h.payload_bytes = payload_bytes(c);
  memcpy(buf, &h, sizeof(h));
  const void* src = c->prec == RAD_PREC_MIXED ? (const void*)c->d_state : (const void*)c->d_state64;
  rad_status s = cuda_check(c, cudaMemcpyAsync((char*)buf + sizeof(h), src, main_payload_bytes(c),
                                               cudaMemcpyDeviceToHost, c->stream));
  if (s != RAD_OK) return s;
  if (c->d_state_p) {
    s = cuda_check(c, cudaMemcpyAsync((char*)buf + sizeof(h) + main_payload_bytes(c), c->d_state_p,
                                      sizeof(float) * 8 * c->n_bins, cudaMemcpyDeviceToHost,
                                      c->stream));
    if (s != RAD_OK) return s;
  }
  return cuda_check(c, cudaStreamSynchronize(c->stream));
}

static rad_status check_blob(rad_ctx* c, const void* buf, size_t n) {
  if (!c || !buf) return RAD_EINVAL;
  if (n < sizeof(BlobHeader)) return RAD_EINVAL;
  BlobHeader h;
  memcpy(&h, buf, sizeof(h));
  if (h.magic != kBlobMagic || h.version != kBlobVersion || h.prec != c->prec ||
      h.n_omega != c->n_omega || h.n_dir != c->n_dir ||
      h.payload_bytes != payload_bytes(c) || n < sizeof(h) + h.payload_bytes)
    return RAD_EINVAL;
  return RAD_OK;
}

rad_status rad_state_import(rad_ctx* c, const void* buf, size_t n) {
  if (!c) return RAD_EINVAL;
  if (c->failed) return RAD_ESTATE;
  if (check_device(c) != RAD_OK) return RAD_EINVAL;
  if (check_blob(c, buf, n) != RAD_OK) return fail(c, RAD_EINVAL);
  void* dst = c->prec == RAD_PREC_MIXED ? (void*)c->d_state : (void*)c->d_state64;
  rad_status s = cuda_check(c, cudaMemcpyAsync(dst, (const char*)buf + sizeof(BlobHeader),
                                               main_payload_bytes(c), cudaMemcpyHostToDevice,
                                               c->stream));
  if (s != RAD_OK) return s;
  if (c->d_state_p) {
    s = cuda_check(c, cudaMemcpyAsync(c->d_state_p,
                                      (const char*)buf + sizeof(BlobHeader) + main_payload_bytes(c),
                                      sizeof(float) * 8 * c->n_bins, cudaMemcpyHostToDevice,
                                      c->stream));
    if (s != RAD_OK) return s;
  }
  return cuda_check(c, cudaStreamSynchronize(c->stream));
}

rad_status rad_state_merge(rad_ctx* c, const void* buf, size_t n) {
  if (!c) return RAD_EINVAL;
  if (c->failed) return RAD_ESTATE;
  if (check_device(c) != RAD_OK) return RAD_EINVAL;
  if (check_blob(c, buf, n) != RAD_OK) return fail(c, RAD_EINVAL);
  void* tmp = nullptr;
  rad_status s = cuda_check(c, cudaMalloc(&tmp, payload_bytes(c)));
  if (s != RAD_OK) return s;
  s = cuda_check(c, cudaMemcpyAsync(tmp, (const char*)buf + sizeof(BlobHeader), payload_bytes(c),
                                    cudaMemcpyHostToDevice, c->stream));
  if (s == RAD_OK) {
    s = c->prec == RAD_PREC_MIXED
            ? cuda_check(c, launch_state_add(c->d_state, (const float*)tmp, c->n_bins, kComps,
                                             c->stream))
            : cuda_check(c, launch_state64_add(c->d_state64, (const double*)tmp, c->n_bins, c->stream));
  }
  if (s == RAD_OK && c->d_state_p) {
    s = cuda_check(c, launch_state_add(c->d_state_p,
                                       (const float*)((const char*)tmp + main_payload_bytes(c)),
                                       c->n_bins, 4, c->stream));
  }
  if (s == RAD_OK) s = cuda_check(c, cudaStreamSynchronize(c->stream));
  cudaFree(tmp);
  return s;
}

rad_status rad_get_tile(const rad_ctx* c, rad_tile* t) {
  if (!c || !t) return RAD_EINVAL;
  *t = c->tile;
  return RAD_OK;
}

rad_status rad_set_tile(rad_ctx* c, const rad_tile* t) {
  if (!c || !t) return RAD_EINVAL;
  if (c->failed) return RAD_ESTATE;
  if (check_device(c) != RAD_OK) return RAD_EINVAL;
  if (c->prec != RAD_PREC_MIXED) return fail(c, RAD_EINVAL);
  if (t->variant < 0 || t->variant >= kNumVariants) return fail(c, RAD_EINVAL);
  // The literal sum has its own kernel variant, used only by literal contexts.
  if ((t->variant == kLiteralVariant) != (c->h_js.literal != 0)) return fail(c, RAD_EINVAL);
  int wt = t->omega_tile > 0 ? t->omega_tile : default_omega_tile(t->variant, c->n_omega);
  if (!valid_omega_tile(t->variant, wt)) return fail(c, RAD_EINVAL);
  if (t->chunk < 0 || (t->chunk % kChunkAlign) != 0) return fail(c, RAD_EINVAL);
  rad_status s = cuda_check(c, cudaStreamSynchronize(c->stream));
  if (s != RAD_OK) return s;
  JobStatic js = c->h_js;
  fill_tiles(js, t->variant, wt);
  if (js.n_tiles > c->tile_cnt_cap) return fail(c, RAD_EINVAL);
  c->h_js = js;
  c->tile.variant = t->variant;
  c->tile.omega_tile = wt;
  c->tile.chunk = t->chunk;
  return upload_static(c);
}

}  // extern "C"
