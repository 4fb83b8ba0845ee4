// Tile-width autotuning of the tcgen05 GEMMs. The output tile is 128 rows by
// 256, 128 or 64 columns (gemm_tc.cu); which is fastest depends on the shape:
// wide tiles reuse each A tile over more columns, narrow ones waste less on
// ragged edges (the U(1) sector blocks are often tens of columns wide) and
// quantise less over the 152 SMs. The first product of each size class that
// runs outside stream capture and kernel profiling is timed at every width
// and the choice is kept in the context.
#include <algorithm>
#include <cstring>

#include "common.cuh"

namespace osmps {

TcKey tc_key(int grouped, int kind, int out, int64_t a, int64_t b, int64_t c) {
  TcKey k;
  k.v[0] = grouped;
  k.v[1] = kind;
  k.v[2] = out;
  k.v[3] = a;
  k.v[4] = b;
  k.v[5] = c;
  return k;
}

static bool same_key(const int64_t* a, const int64_t* b) {
  for (int i = 0; i < 6; ++i)
    if (a[i] != b[i]) return false;
  return true;
}

int tc_tuned_width(osmps_ctx* ctx, const TcKey& key) {
  for (const auto& e : ctx->tc_tuned)
    if (same_key(e.key, key.v)) return e.bn;
  return 0;
}

bool tc_may_tune(osmps_ctx* ctx) {
  return ctx->tc_autotune == OSMPS_AUTOTUNE_ON && !ctx->capturing && !ctx->prof_on;
}

osmps_status tc_time_launches(osmps_ctx* ctx, cudaStream_t stream, int reps, float* us,
                              const std::function<osmps_status(cudaStream_t)>& fn) {
  (void)ctx;
  cudaEvent_t a = nullptr, b = nullptr;
  OSMPS_CUDA(cudaEventCreate(&a));
  if (cudaEventCreate(&b) != cudaSuccess) {
    cudaEventDestroy(a);
    return set_error(OSMPS_ECUDA, "autotune: cudaEventCreate failed");
  }
  osmps_status st = OSMPS_OK;
  cudaEventRecord(a, stream);
  for (int r = 0; r < reps && st == OSMPS_OK; ++r) st = fn(stream);
  cudaEventRecord(b, stream);
  const cudaError_t e = cudaEventSynchronize(b);
  float ms = 0.0f;
  if (st == OSMPS_OK && e == cudaSuccess) cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (st != OSMPS_OK) return st;
  if (e != cudaSuccess) return set_error(OSMPS_ECUDA, "autotune: %s", cudaGetErrorString(e));
  *us = 1e3f * ms / (float)std::max(reps, 1);
  return OSMPS_OK;
}

int tc_record_tuning(osmps_ctx* ctx, const TcKey& key, const int* widths, const float* us) {
  int best = 0;
  for (int w = 1; w < 3; ++w)
    if (us[w] < us[best]) best = w;
  osmps_ctx::TcTuned e;
  memcpy(e.key, key.v, sizeof e.key);
  e.bn = widths[best];
  for (int w = 0; w < 3; ++w) e.us[w] = 0.0f;
  for (int w = 0; w < 3; ++w) {  // times stored in the order 256, 128, 64
    const int slot = widths[w] == 256 ? 0 : (widths[w] == 128 ? 1 : 2);
    e.us[slot] = us[w];
  }
  for (auto& x : ctx->tc_tuned)
    if (same_key(x.key, e.key)) {
      x = e;
      return e.bn;
    }
  ctx->tc_tuned.push_back(e);
  return e.bn;
}

}  // namespace osmps

using namespace osmps;

extern "C" osmps_status osmps_ctx_set_autotune(osmps_ctx* ctx, int mode) {
  clear_error();
  if (!ctx) return set_error(OSMPS_EINVAL, "osmps_ctx_set_autotune: null context");
  if (mode != OSMPS_AUTOTUNE_OFF && mode != OSMPS_AUTOTUNE_ON)
    return set_error(OSMPS_EINVAL, "osmps_ctx_set_autotune: mode %d", mode);
  ctx->tc_autotune = mode;
  return OSMPS_OK;
}

extern "C" int64_t osmps_ctx_tuning_count(const osmps_ctx* ctx) {
  return ctx ? (int64_t)ctx->tc_tuned.size() : 0;
}

extern "C" osmps_status osmps_ctx_tuning_entry(const osmps_ctx* ctx, int64_t i, int64_t* key, int* width,
                                               float* us3) {
  clear_error();
  if (!ctx || !key || !width || !us3) return set_error(OSMPS_EINVAL, "osmps_ctx_tuning_entry: null argument");
  if (i < 0 || i >= (int64_t)ctx->tc_tuned.size())
    return set_error(OSMPS_EINVAL, "osmps_ctx_tuning_entry: entry %lld of %lld", (long long)i,
                     (long long)ctx->tc_tuned.size());
  const auto& e = ctx->tc_tuned[(size_t)i];
  memcpy(key, e.key, sizeof e.key);
  *width = e.bn;
  for (int w = 0; w < 3; ++w) us3[w] = e.us[w];
  return OSMPS_OK;
}

extern "C" osmps_status osmps_ctx_set_tuning(osmps_ctx* ctx, const int64_t* key, int width) {
  clear_error();
  if (!ctx || !key) return set_error(OSMPS_EINVAL, "osmps_ctx_set_tuning: null argument");
  if (!tc_tile_width_ok(width)) return set_error(OSMPS_EINVAL, "osmps_ctx_set_tuning: width %d", width);
  TcKey k;
  memcpy(k.v, key, sizeof k.v);
  for (auto& x : ctx->tc_tuned)
    if (same_key(x.key, k.v)) {
      x.bn = width;
      for (int w = 0; w < 3; ++w) x.us[w] = 0.0f;
      return OSMPS_OK;
    }
  osmps_ctx::TcTuned e;
  memcpy(e.key, k.v, sizeof e.key);
  e.bn = width;
  for (int w = 0; w < 3; ++w) e.us[w] = 0.0f;
  ctx->tc_tuned.push_back(e);
  return OSMPS_OK;
}
