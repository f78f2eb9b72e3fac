// Autotuner for the mixed-precision tile configuration: kernel variant
// (threads x frequencies per thread), frequency-tile width and particles per
// work item, timed with CUDA events on synthetic particles, cached per grid
// shape bucket in memory and optionally in the file named by RAD_TUNE_CACHE.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "rad_ctx.h"
#include "rad_impl.h"

using namespace radimpl;

namespace {

using Key = std::tuple<int, int, int>;  // n_omega, n_dir, log2 bucket of n

std::mutex g_mu;
std::map<Key, rad_tile> g_cache;
bool g_loaded = false;

int bucket(long long n) {
  int b = 0;
  while ((1LL << (b + 1)) <= n) ++b;
  return b;
}

void load_cache_locked() {
  if (g_loaded) return;
  g_loaded = true;
  const char* path = getenv("RAD_TUNE_CACHE");
  if (!path || !*path) return;
  FILE* f = fopen(path, "r");
  if (!f) return;
  int no, nd, b, v, wt, ck;
  while (fscanf(f, "%d %d %d %d %d %d", &no, &nd, &b, &v, &wt, &ck) == 6) {
    if (v < 0 || v >= kNumVariants || !valid_omega_tile(v, wt) || ck < 0 || ck % kChunkAlign) continue;
    rad_tile t{v, wt, ck, 0};
    g_cache[Key(no, nd, b)] = t;
  }
  fclose(f);
}

void store_cache_locked(const Key& k, const rad_tile& t) {
  g_cache[k] = t;
  const char* path = getenv("RAD_TUNE_CACHE");
  if (!path || !*path) return;
  FILE* f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "%d %d %d %d %d %d\n", std::get<0>(k), std::get<1>(k), std::get<2>(k), t.variant,
          t.omega_tile, t.chunk);
  fclose(f);
}

// Synthetic relativistic bunch for timing: a counter-based hash gives each
// particle its offsets; the values only need the magnitudes of real inputs.
__device__ __forceinline__ double hash01(unsigned long long x) {
  x += 0x9E3779B97F4A7C15ULL;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ULL;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBULL;
  x ^= x >> 31;
  return (double)(x >> 11) * (1.0 / 9007199254740992.0);
}

__global__ void fill_synthetic(long long n, double* r, double* beta, double* bdot, double* w) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const double u0 = hash01(4 * k), u1 = hash01(4 * k + 1), u2 = hash01(4 * k + 2),
               u3 = hash01(4 * k + 3);
  r[k] = (u0 - 0.5) * 4e-6;
  r[n + k] = (u1 - 0.5) * 4e-6;
  r[2 * n + k] = (u2 - 0.5) * 2e-6;
  const double bx = (u1 - 0.5) * 0.02, by = (u0 - 0.5) * 0.02;
  beta[k] = bx;
  beta[n + k] = by;
  beta[2 * n + k] = sqrt(1.0 - 1.0 / (300.0 * 300.0) - bx * bx - by * by);
  bdot[k] = (u3 - 0.5) * 2e13;
  bdot[n + k] = (u2 - 0.5) * 2e13;
  bdot[2 * n + k] = 0.0;
  w[k] = 1e3 + u3 * 1e4;
}

}  // namespace

extern "C" rad_status rad_tune(rad_ctx* c, int64_t n) {
  if (!c || n < 1) return RAD_EINVAL;
  if (c->failed) return RAD_ESTATE;
  if (check_device(c) != RAD_OK) return RAD_EINVAL;
  if (c->prec != RAD_PREC_MIXED) return RAD_OK;  // the FP64 kernel has no tiles
  if (c->h_js.literal) return RAD_OK;             // the literal sum has one variant
  const Key key(c->n_omega, c->n_dir, bucket(n));
  {
    std::lock_guard<std::mutex> lk(g_mu);
    load_cache_locked();
    auto it = g_cache.find(key);
    if (it != g_cache.end()) return rad_set_tile(c, &it->second);
  }
  // Candidates: every variant, the default and half / double frequency tiles,
  // automatic chunking and half / double of it (see n_ckm below).
  std::vector<rad_tile> cands;
  for (int v = 0; v < kNumVariants; ++v) {
    if (v == kLiteralVariant) continue;
    const int wt0 = default_omega_tile(v, c->n_omega);
    for (int wt : {wt0 / 2, wt0, wt0 * 2}) {
      if (!valid_omega_tile(v, wt)) continue;
      cands.push_back({v, wt, 0, 0});
    }
  }
  // Time on a bounded particle count so a trial costs milliseconds.
  const long long nt = std::min<long long>(n, std::max<long long>(
      4096, (long long)(2.0e9 / ((double)c->n_bins + 1.0))));
  double *r = nullptr, *b = nullptr, *bd = nullptr, *w = nullptr;
  void* saved = nullptr;
  rad_status st = RAD_OK;
  const size_t blob = rad_state_size(c);
  rad_tile orig = c->tile;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaMalloc(&r, sizeof(double) * 3 * nt) != cudaSuccess ||
      cudaMalloc(&b, sizeof(double) * 3 * nt) != cudaSuccess ||
      cudaMalloc(&bd, sizeof(double) * 3 * nt) != cudaSuccess ||
      cudaMalloc(&w, sizeof(double) * nt) != cudaSuccess || !(saved = malloc(blob))) {
    st = RAD_ENOMEM;
  }
  if (st == RAD_OK) st = rad_state_export(c, saved, blob);
  if (st == RAD_OK) {
    fill_synthetic<<<(unsigned)((nt + 255) / 256), 256, 0, c->stream>>>(nt, r, b, bd, w);
    count_launches(1);
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
  }
  rad_tile best = orig;
  float best_ms = 1e30f;
  // Half and double the automatic chunk are tried only when the trial runs the
  // caller's particle count: the best chunk depends on it (the blocks' tail at
  // the end of a launch), so one picked on a smaller trial does not carry over.
  const int n_ckm = nt == n ? 3 : 1;
  for (size_t i = 0; st == RAD_OK && i < cands.size(); ++i) {
    for (int ckm = 0; ckm < n_ckm; ++ckm) {
      rad_tile t = cands[i];
      if (ckm) {
        JobStatic js = c->h_js;
        fill_tiles(js, t.variant, t.omega_tile);
        const int ck = auto_chunk_for(t.variant, nt, js.n_tiles,
                                      variant_tensor_core(t.variant) && !c->h_js.literal);
        int ck2 = ckm == 1 ? ck / 2 : ck * 2;
        ck2 = std::max(kChunkAlign, ck2 / kChunkAlign * kChunkAlign);
        if (ck2 == ck) continue;
        t.chunk = ck2;
      }
      if (rad_set_tile(c, &t) != RAD_OK) continue;
      float ms_sum = 0.f;
      for (int rep = 0; rep < 3 && st == RAD_OK; ++rep) {
        cudaEventRecord(e0, c->stream);
        st = rad_accumulate(c, nt, r, b, bd, w, 1e-15, 1e-16);
        cudaEventRecord(e1, c->stream);
        if (cudaEventSynchronize(e1) != cudaSuccess) st = RAD_ECUDA;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0) ms_sum += ms;  // first repetition is warm-up
      }
      if (st == RAD_OK && ms_sum < best_ms) {
        best_ms = ms_sum;
        best = c->tile;
      }
    }
  }
  if (st == RAD_OK) st = rad_set_tile(c, &best);
  if (st == RAD_OK) st = rad_state_import(c, saved, blob);
  if (st == RAD_OK) {
    rad_sync(c);  // clears status bits raised by the synthetic data, if any
    rad_log(1, "tune: %d omega x %d directions, n ~ %lld: variant %d, omega tile %d, chunk %d (%.3f ms per trial)",
            c->n_omega, c->n_dir, (long long)n, best.variant, best.omega_tile, best.chunk,
            best_ms / 2.0);
    std::lock_guard<std::mutex> lk(g_mu);
    store_cache_locked(key, best);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(r);
  cudaFree(b);
  cudaFree(bd);
  cudaFree(w);
  free(saved);
  return st;
}
