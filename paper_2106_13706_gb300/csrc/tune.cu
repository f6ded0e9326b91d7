// tune.cu -- kernel-path selection for a problem shape.
//
// The choice depends only on (d, NP, NT): whether the counts fit in
// registers, in lane-private shared-memory histograms, in a per-warp
// histogram, or need the sort path.  A forced path in the context config wins;
// otherwise a tuned entry (filled by ddks_tune_* and persisted as a small text
// cache keyed by d and the size buckets) wins over the built-in defaults.
// ddks_autotune times every configuration that can take a shape and records
// the fastest.
#include <cstdio>
#include <cstdlib>
#include <string>
#include <vector>

#include "ddks_host.h"
#include "ddks_internal.cuh"

constexpr int64_t kDominanceMinN = 32768;
// Pooled N from which key sorts use the radix sort by default: 32-bit keys
// (float32 inputs, 4 digit passes) and 64-bit keys (8 passes).  Measured on
// GB300 against the chunk sort + merges: 32-bit radix ahead from ~16k keys
// per row, 64-bit from a few hundred thousand.
constexpr int64_t kRadixMinN32 = 16384;
constexpr int64_t kRadixMinN64 = 131072;

bool ddks_use_radix(const ddks_ctx* ctx, int64_t N, int key_bits) {
  const int64_t m = ctx->cfg.radix_min_n;
  if (m < 0) return false;
  if (m > 0) return N >= m;
  return N >= (key_bits <= 32 ? kRadixMinN32 : kRadixMinN64);
}

static std::string tune_key(int64_t NP, int64_t NT, int32_t d) {
  auto bucket = [](int64_t n) {
    int b = 0;
    while (n > 1) { n >>= 1; ++b; }
    return b;
  };
  char buf[64];
  std::snprintf(buf, sizeof buf, "d%d_p%d_t%d_w%d", d, bucket(NP), bucket(NT),
                (NP > 65535 || NT > 65535) ? 1 : 0);
  return buf;
}

static bool plan_ok(const ddks_plan& p, int64_t NP, int64_t NT, int32_t d) {
  switch (p.path) {
    case DDKS_PATH_REGISTER: return ddks_register_supported(d, NP, NT);
    case DDKS_PATH_LANE: return ddks_lane_supported(d, NP, NT, p.threads);
    case DDKS_PATH_WARP: return ddks_warp_supported(d, NP, NT);
    case DDKS_PATH_SORT: return ddks_sort_supported(d, NP + NT);
    case DDKS_PATH_DOMINANCE: return ddks_dominance_supported(d, NP, NT);
    case DDKS_PATH_BYTE: return ddks_byte_supported(d, NP, NT);
    default: return false;
  }
}

static ddks_plan default_plan(int64_t NP, int64_t NT, int32_t d) {
  ddks_plan p;
  // d = 2 with many points: O(N log N) range queries beat the N^2 compares
  if (d == 2 && NP + NT >= kDominanceMinN && ddks_dominance_supported(d, NP, NT)) {
    p.path = DDKS_PATH_DOMINANCE;
    return p;
  }
  if (ddks_register_supported(d, NP, NT)) {
    p.path = DDKS_PATH_REGISTER;
    return p;
  }
  if (d <= 4) { p.path = DDKS_PATH_LANE; p.threads = 256; }
  else if (d <= 6) { p.path = DDKS_PATH_LANE; p.threads = 128; }
  else if (d <= 13) { p.path = DDKS_PATH_WARP; p.warps = 8; }
  else { p.path = DDKS_PATH_SORT; }
  if (p.path == DDKS_PATH_LANE && !ddks_lane_supported(d, NP, NT, p.threads)) {
    p.path = DDKS_PATH_WARP;
  }
  if (p.path == DDKS_PATH_WARP && !ddks_warp_supported(d, NP, NT)) p.path = DDKS_PATH_SORT;
  return p;
}

int ddks_select_path(ddks_ctx* ctx, int64_t NP, int64_t NT, int32_t d, ddks_plan* plan) {
  ddks_plan p = default_plan(NP, NT, d);
  if (ctx->cfg.path != DDKS_PATH_AUTO) {
    const int forced = ctx->cfg.path;
    p.path = forced;
    if (forced == DDKS_PATH_LANE) p.threads = d <= 4 ? 256 : (d <= 6 ? 128 : 64);
    if (forced == DDKS_PATH_REGISTER) {
      const int rv = ctx->cfg.register_variant;
      p.fused = rv >= 2 ? rv - 1 : 0;
    }
    if (!plan_ok(p, NP, NT, d)) return DDKS_EUNSUPPORTED;
    *plan = p;
    return DDKS_OK;
  }
  {
    std::lock_guard<std::mutex> g(ctx->tune_mu);
    auto it = ctx->tune.find(tune_key(NP, NT, d));
    if (it != ctx->tune.end() && plan_ok(it->second, NP, NT, d)) p = it->second;
  }
  if (!plan_ok(p, NP, NT, d)) return DDKS_EUNSUPPORTED;
  *plan = p;
  return DDKS_OK;
}

void ddks_tune_load(ddks_ctx* ctx) {
  if (ctx->tune_cache_path.empty()) return;
  FILE* f = std::fopen(ctx->tune_cache_path.c_str(), "r");
  if (!f) return;
  char key[64];
  ddks_plan p;
  while (std::fscanf(f, "%63s %d %d %d %d %d", key, &p.path, &p.threads, &p.warps, &p.reg_occ, &p.fused) == 6) {
    ctx->tune[key] = p;
  }
  std::fclose(f);
}

static void tune_save(ddks_ctx* ctx) {
  if (ctx->tune_cache_path.empty()) return;
  const std::string tmp = ctx->tune_cache_path + ".tmp";
  FILE* f = std::fopen(tmp.c_str(), "w");
  if (!f) return;
  for (auto& kv : ctx->tune)
    std::fprintf(f, "%s %d %d %d %d %d\n", kv.first.c_str(), kv.second.path, kv.second.threads,
                 kv.second.warps, kv.second.reg_occ, kv.second.fused);
  std::fclose(f);
  std::rename(tmp.c_str(), ctx->tune_cache_path.c_str());
}

int ddks_autotune(ddks_ctx* ctx, const void* P, int64_t NP, const void* T, int64_t NT, int32_t d,
                  int32_t dtype, void* stream, int32_t* chosen_path, float* best_ms) {
  if (!ctx) return DDKS_EINVAL;
  int rc = ddks_check_problem(P, NP, T, NT, d, dtype);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return ctx_cuda_fail(ctx, e, "cudaSetDevice");
  const void *dP, *dT;
  if ((rc = ddks_stage_inputs(ctx, P, NP, T, NT, d, dtype, st, &dP, &dT))) return rc;
  if ((rc = ddks_encode_problem(ctx, dP, NP, dT, NT, d, dtype, st, true))) return rc;
  const int64_t N = NP + NT;
  if ((rc = ctx->best.reserve(ctx, 8 * (size_t)N))) return rc;
  if ((rc = ctx->bestj.reserve(ctx, 4 * (size_t)N))) return rc;
  if ((rc = ctx->out3.reserve(ctx, 64 + ddks_reduce_scratch_bytes()))) return rc;
  std::vector<ddks_plan> cands;
  for (int v : {1, 2, 3}) {
    ddks_plan p; p.path = DDKS_PATH_REGISTER; p.fused = v; cands.push_back(p);
  }
  for (int occ : {4, 6, 8}) {
    ddks_plan p; p.path = DDKS_PATH_REGISTER; p.reg_occ = occ; p.fused = 0; cands.push_back(p);
  }
  for (int th : {64, 128, 256}) {
    ddks_plan p; p.path = DDKS_PATH_LANE; p.threads = th; cands.push_back(p);
  }
  { ddks_plan p; p.path = DDKS_PATH_WARP; p.warps = 8; cands.push_back(p); }
  { ddks_plan p; p.path = DDKS_PATH_SORT; cands.push_back(p); }
  { ddks_plan p; p.path = DDKS_PATH_DOMINANCE; cands.push_back(p); }
  { ddks_plan p; p.path = DDKS_PATH_BYTE; cands.push_back(p); }
  cudaEvent_t a, b;
  if ((e = cudaEventCreate(&a)) != cudaSuccess) return ctx_cuda_fail(ctx, e, "cudaEventCreate");
  if ((e = cudaEventCreate(&b)) != cudaSuccess) { cudaEventDestroy(a); return ctx_cuda_fail(ctx, e, "cudaEventCreate"); }
  float best_t = 1e30f;
  ddks_plan best_p;
  unsigned long long ref = ~0ull;
  int result = DDKS_OK;
  for (const ddks_plan& p : cands) {
    if (!plan_ok(p, NP, NT, d)) continue;
    // the sort path re-sorts per origin: skip it when it is obviously slower
    if (p.path == DDKS_PATH_SORT && d <= 13 && best_t < 1e29f) continue;
    float tmin = 1e30f;
    for (int rep = 0; rep < 3 && result == DDKS_OK; ++rep) {
      cudaEventRecord(a, st);
      rc = ddks_count_origins_plan(ctx, p, NP, NT, d, 0, N, (uint64_t*)ctx->best.ptr,
                                   (int32_t*)ctx->bestj.ptr, st);
      if (rc) { result = rc; break; }
      cudaEventRecord(b, st);
      e = ddks_launch_reduce((const uint64_t*)ctx->best.ptr, (const int32_t*)ctx->bestj.ptr, N, 0,
                             (unsigned long long*)ctx->out3.ptr, (char*)ctx->out3.ptr + 64, st);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(ctx->h_out, ctx->out3.ptr, 8, cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) { result = ctx_cuda_fail(ctx, e, "autotune"); break; }
      float ms = 0;
      cudaEventElapsedTime(&ms, a, b);
      tmin = ms < tmin ? ms : tmin;
      if (ref == ~0ull) ref = ctx->h_out[0];
      else if (ctx->h_out[0] != ref) { result = DDKS_ECUDA; ctx->last_err = "autotune: paths disagree"; break; }
    }
    if (result != DDKS_OK) break;
    if (tmin < best_t) { best_t = tmin; best_p = p; }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (result != DDKS_OK) return result;
  if (best_t >= 1e29f) return DDKS_EUNSUPPORTED;
  {
    std::lock_guard<std::mutex> g(ctx->tune_mu);
    ctx->tune[tune_key(NP, NT, d)] = best_p;
    tune_save(ctx);
  }
  if (chosen_path) *chosen_path = best_p.path;
  if (best_ms) *best_ms = best_t;
  return DDKS_OK;
}
