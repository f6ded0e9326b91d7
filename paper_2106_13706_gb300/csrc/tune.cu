// tune.cu -- kernel-path selection for a problem shape.
//
// The choice depends only on (d, NP, NT): whether the counts fit in
// registers, in lane-private shared-memory histograms, in a per-warp
// histogram, or need the sort path.  A forced path in the context config wins;
// otherwise a tuned entry (filled by ddks_tune_* and persisted as a small text
// cache keyed by d and the size buckets) wins over the built-in defaults.
#include <cstdio>
#include <cstdlib>
#include <string>

#include "ddks_host.h"
#include "ddks_internal.cuh"

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
    default: return false;
  }
}

static ddks_plan default_plan(int64_t NP, int64_t NT, int32_t d) {
  ddks_plan p;
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
  while (std::fscanf(f, "%63s %d %d %d %d", key, &p.path, &p.threads, &p.warps, &p.reg_slices) == 5) {
    ctx->tune[key] = p;
  }
  std::fclose(f);
}
