// api.cu -- host side of the C ABI declared in include/ddks.h: argument
// checks, context-owned device scratch, kernel-path selection and the
// synchronous distance entry points.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>

#include "../../include/ddks.h"
#include "ddks_internal.cuh"
#include "ddks_host.h"

// ------------------------------------------------------------------ helpers

const char* ddks_strerror(int code) {
  switch (code) {
    case DDKS_OK: return "ok";
    case DDKS_PENDING: return "pending";
    case DDKS_EINVAL: return "invalid argument";
    case DDKS_ENAN: return "input contains NaN";
    case DDKS_EOVERFLOW: return "size too large (NP*NT >= 2^62 or beyond index range)";
    case DDKS_ENOMEM: return "out of device memory or over the memory budget";
    case DDKS_ECUDA: return "CUDA runtime error";
    case DDKS_ETIMEOUT: return "bounded wait timed out";
    case DDKS_ENOTFOUND: return "unknown ticket";
    case DDKS_EUNSUPPORTED: return "input not supported by the selected kernel path";
    default: return "unknown error";
  }
}

const char* ddks_version(void) { return "0.1.0"; }

void ddks_config_default(ddks_config* cfg) {
  if (!cfg) return;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->device = -1;
  cfg->path = DDKS_PATH_AUTO;
  cfg->hbm_budget_bytes = 0;
  cfg->max_batch = 0;
  cfg->wait_limit_ms = 0;
  cfg->tune_cache = nullptr;
  cfg->graphs = 1;
}

int ctx_cuda_fail(ddks_ctx* ctx, cudaError_t e, const char* where) {
  cudaGetLastError();  // clear a non-sticky error so later calls start clean
  if (ctx) {
    ctx->last_err = std::string(where) + ": " + cudaGetErrorString(e);
  }
  return e == cudaErrorMemoryAllocation ? DDKS_ENOMEM : DDKS_ECUDA;
}

int ddks_classify_pointer(int32_t memory_type, int32_t pointer_device, int32_t device) {
  switch (memory_type) {
    case cudaMemoryTypeDevice:  // device memory is read in place only on its own device
      return pointer_device == device ? 1 : DDKS_EINVAL;
    case cudaMemoryTypeManaged:
      return 1;
    case cudaMemoryTypeUnregistered:
    case cudaMemoryTypeHost:
      return 0;
    default:
      return DDKS_EINVAL;
  }
}

int ddks_pointer_kind(const void* p, int device) {
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 0;  // not known to CUDA: plain host memory
  }
  return ddks_classify_pointer((int32_t)a.type, (int32_t)a.device, (int32_t)device);
}

cudaError_t ddks_smem_attr_raw(const void* func, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, size_t> cur;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> g(mu);
  size_t& have = cur[std::make_pair(func, dev)];
  if (have >= bytes) return cudaSuccess;
  e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) have = bytes;
  return e;
}

bool ddks_is_pageable(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return true;
  }
  return a.type == cudaMemoryTypeUnregistered;
}

int DevBuf::reserve(ddks_ctx* ctx, size_t n) {
  if (n <= bytes) return DDKS_OK;
  if (ptr) cudaFree(ptr);
  ptr = nullptr;
  bytes = 0;
  ++ctx->buf_gen;  // graphs captured before this point hold the old address
  size_t want = n + n / 4 + 256;
  cudaError_t e = cudaMalloc(&ptr, want);
  if (e != cudaSuccess) {
    cudaGetLastError();
    ptr = nullptr;
    return ctx_cuda_fail(ctx, e, "cudaMalloc");
  }
  bytes = want;
  return DDKS_OK;
}

void DevBuf::release() {
  if (ptr) cudaFree(ptr);
  ptr = nullptr;
  bytes = 0;
}

int ddks_check_problem(const void* P, int64_t NP, const void* T, int64_t NT, int32_t d,
                       int32_t dtype) {
  if (!P || !T || NP < 1 || NT < 1 || d < 1 || d > DDKS_MAX_D) return DDKS_EINVAL;
  if (dtype != DDKS_F32 && dtype != DDKS_F64) return DDKS_EINVAL;
  if ((double)NP * (double)NT >= 4.611686018427387904e18) return DDKS_EOVERFLOW;
  if (NP + NT >= ((int64_t)1 << 31) || (NP + NT) * (int64_t)d >= ((int64_t)1 << 40))
    return DDKS_EOVERFLOW;
  return DDKS_OK;
}

// ------------------------------------------------------------------ context

int ddks_ctx_create(const ddks_config* cfg, ddks_ctx** out) {
  if (!out) return DDKS_EINVAL;
  *out = nullptr;
  ddks_ctx* ctx = new (std::nothrow) ddks_ctx();
  if (!ctx) return DDKS_ENOMEM;
  if (cfg) ctx->cfg = *cfg; else ddks_config_default(&ctx->cfg);
  if (ctx->cfg.path < DDKS_PATH_AUTO || ctx->cfg.path > DDKS_PATH_BYTE) { delete ctx; return DDKS_EINVAL; }
  if (ctx->cfg.register_variant < 0 || ctx->cfg.register_variant > 4) { delete ctx; return DDKS_EINVAL; }
  if (ctx->cfg.rank_kernel < 0 || ctx->cfg.rank_kernel > 2) { delete ctx; return DDKS_EINVAL; }
  if (ctx->cfg.hbm_budget_bytes == 0) ctx->cfg.hbm_budget_bytes = 8ull << 30;
  if (ctx->cfg.max_batch <= 0) ctx->cfg.max_batch = 64;
  if (ctx->cfg.wait_limit_ms > 0)
    ctx->dev_wait_ns = ctx->dev_wait_cfg_ns = (unsigned long long)ctx->cfg.wait_limit_ms * 1000000ull;
  if (ctx->cfg.wait_limit_ms <= 0) ctx->cfg.wait_limit_ms = 10000;
  int dev = ctx->cfg.device;
  cudaError_t e;
  if (dev < 0) {
    e = cudaGetDevice(&dev);
    if (e != cudaSuccess) { int rc = ctx_cuda_fail(ctx, e, "cudaGetDevice"); delete ctx; return rc; }
  }
  ctx->device = dev;
  e = cudaSetDevice(dev);
  if (e != cudaSuccess) { int rc = ctx_cuda_fail(ctx, e, "cudaSetDevice"); delete ctx; return rc; }
  e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) { int rc = ctx_cuda_fail(ctx, e, "cudaDeviceGetAttribute"); delete ctx; return rc; }
  e = cudaMallocHost((void**)&ctx->h_out, 64 * sizeof(unsigned long long));
  if (e != cudaSuccess) { int rc = ctx_cuda_fail(ctx, e, "cudaMallocHost"); delete ctx; return rc; }
  const char* tc = ctx->cfg.tune_cache ? ctx->cfg.tune_cache : std::getenv("DDKS_TUNE_CACHE");
  if (tc) ctx->tune_cache_path = tc;
  ddks_tune_load(ctx);
  *out = ctx;
  return DDKS_OK;
}

int ddks_ctx_destroy(ddks_ctx* ctx) {
  if (!ctx) return DDKS_EINVAL;
  cudaSetDevice(ctx->device);
  ddks_serve_shutdown(ctx);
  cudaDeviceSynchronize();
  ddks_graph_clear(ctx);
  for (DevBuf* b : ctx->all_bufs()) b->release();
  if (ctx->h_out) cudaFreeHost(ctx->h_out);
  if (ctx->h_stage) cudaFreeHost(ctx->h_stage);
  for (auto& e : ctx->ev)
    if (e) cudaEventDestroy(e);
  delete ctx;
  return DDKS_OK;
}

const char* ddks_last_cuda_error(ddks_ctx* ctx) { return ctx ? ctx->last_err.c_str() : ""; }

int ddks_ctx_stats(ddks_ctx* ctx, ddks_stats* out) {
  if (!ctx || !out) return DDKS_EINVAL;
  ddks_serve_fill_stats(ctx, out);
  out->kernel_launches += ctx->launches;
  out->graph_captures = ctx->graph_captures;
  out->graph_replays = ctx->graph_replays;
  return DDKS_OK;
}

int ddks_set_stage_timing(ddks_ctx* ctx, int32_t enable) {
  if (!ctx) return DDKS_EINVAL;
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return ctx_cuda_fail(ctx, e, "cudaSetDevice");
  for (auto& ev : ctx->ev) {
    if (!ev) {
      e = cudaEventCreate(&ev);
      if (e != cudaSuccess) return ctx_cuda_fail(ctx, e, "cudaEventCreate");
    }
  }
  ctx->stage_timing = enable != 0;
  return DDKS_OK;
}

int ddks_stage_times(ddks_ctx* ctx, float* encode_ms, float* count_ms, float* reduce_ms) {
  if (!ctx) return DDKS_EINVAL;
  if (encode_ms) *encode_ms = ctx->stage_ms[0];
  if (count_ms) *count_ms = ctx->stage_ms[1];
  if (reduce_ms) *reduce_ms = ctx->stage_ms[2];
  return DDKS_OK;
}

// Records stage event i on st (stage timing turns graph replay off, so this
// never runs inside a capture).
void ddks_stage_mark(ddks_ctx* ctx, int i, cudaStream_t st) {
  if (ctx->stage_timing) cudaEventRecord(ctx->ev[i], st);
}
static void stage_mark(ddks_ctx* ctx, int i, cudaStream_t st) { ddks_stage_mark(ctx, i, st); }

void ddks_stage_collect(ddks_ctx* ctx) {
  if (!ctx->stage_timing) return;
  for (int i = 0; i < 3; ++i) {
    float ms = 0;
    if (cudaEventElapsedTime(&ms, ctx->ev[i], ctx->ev[i + 1]) != cudaSuccess) {
      cudaGetLastError();
      ms = 0;
    }
    ctx->stage_ms[i] = ms;
  }
}

// ------------------------------------------------------------------ distance

// Stage P and T on the device (in place when they are already device memory).
int ddks_stage_inputs(ddks_ctx* ctx, const void* P, int64_t NP, const void* T, int64_t NT,
                      int32_t d, int32_t dtype, cudaStream_t st, const void** dP,
                      const void** dT) {
  const size_t es = dtype == DDKS_F64 ? 8 : 4;
  const int kP = ddks_pointer_kind(P, ctx->device), kT = ddks_pointer_kind(T, ctx->device);
  if (kP < 0 || kT < 0) return DDKS_EINVAL;  // device memory of another GPU
  const bool devP = kP == 1, devT = kT == 1;
  *dP = P;
  *dT = T;
  if (!devP) {
    int rc = ctx->inP.reserve(ctx, es * (size_t)NP * d);
    if (rc) return rc;
    cudaError_t e = cudaMemcpyAsync(ctx->inP.ptr, P, es * (size_t)NP * d, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return ctx_cuda_fail(ctx, e, "copy P to device");
    *dP = ctx->inP.ptr;
  }
  if (!devT) {
    int rc = ctx->inT.reserve(ctx, es * (size_t)NT * d);
    if (rc) return rc;
    cudaError_t e = cudaMemcpyAsync(ctx->inT.ptr, T, es * (size_t)NT * d, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return ctx_cuda_fail(ctx, e, "copy T to device");
    *dT = ctx->inT.ptr;
  }
  return DDKS_OK;
}

// K0 on device inputs: order keys (NaN flag) and min-ranks [d][N] into ctx->rank.
int ddks_encode_problem(ddks_ctx* ctx, const void* dP, int64_t NP, const void* dT, int64_t NT,
                        int32_t d, int32_t dtype, cudaStream_t st, bool want_sorted0) {
  const int64_t N = NP + NT;
  const size_t npad = ddks_rank_scratch_elems(N);
  int rc;
  // one cluster launch for float32 keys (4 digit passes); float64 keys need 8,
  // where the chunk sorts measured faster (8,192 points: 0.045 vs 0.079 ms)
  const int kb = dtype == DDKS_F64 ? 64 : 32;
  if (((ctx->cfg.rank_kernel == 0 && dtype == DDKS_F32) || ctx->cfg.rank_kernel == 2) &&
      ddks_rank_cluster_supported(N, kb, ctx->device)) {
    // one launch: keys, ranks, every dimension's order, dimension 0's P prefix
    if ((rc = ctx->rank.reserve(ctx, 4 * (size_t)N * d))) return rc;
    if ((rc = ctx->sidx0.reserve(ctx, 4 * (size_t)N))) return rc;
    if ((rc = ctx->pfx0.reserve(ctx, 4 * (size_t)N))) return rc;
    if ((rc = ctx->ti1.reserve(ctx, 4 * (size_t)N * d))) return rc;
    if ((rc = ctx->flags.reserve(ctx, 64))) return rc;
    cudaError_t e = cudaMemsetAsync(ctx->flags.ptr, 0, 4, st);
    if (e == cudaSuccess)
      e = ddks_launch_rank_cluster(dP, dT, NP, NT, d, dtype == DDKS_F64, (uint32_t*)ctx->rank.ptr,
                                   (uint32_t*)ctx->ti1.ptr, (uint32_t*)ctx->sidx0.ptr, (uint32_t*)ctx->pfx0.ptr,
                                   (unsigned*)ctx->flags.ptr, st);
    if (e != cudaSuccess) return ctx_cuda_fail(ctx, e, "rank (cluster)");
    ctx->launches += 1;
    ctx->pfx0_valid = true;
    ctx->sorted_rows = (const uint32_t*)ctx->ti1.ptr;
    return DDKS_OK;
  }
  if ((rc = ctx->keys.reserve(ctx, 8 * (size_t)N * d))) return rc;
  if ((rc = ctx->tk1.reserve(ctx, 8 * npad * d))) return rc;
  if ((rc = ctx->tk2.reserve(ctx, 8 * npad * d))) return rc;
  if ((rc = ctx->ti1.reserve(ctx, 4 * npad * d))) return rc;
  if ((rc = ctx->ti2.reserve(ctx, 4 * npad * d))) return rc;
  if ((rc = ctx->rank.reserve(ctx, 4 * (size_t)N * d))) return rc;
  if ((rc = ctx->sidx0.reserve(ctx, 4 * (size_t)N))) return rc;
  if (want_sorted0 && (rc = ctx->pfx0.reserve(ctx, 4 * ((size_t)N + 2 * ddks_rank_pfx_elems(N))))) return rc;
  const int key_bits = dtype == DDKS_F64 ? 64 : 32;
  const bool radix = ddks_use_radix(ctx, N, key_bits);
  if (radix && (rc = ctx->radix.reserve(ctx, 4 * ddks_radix_scratch_words(N, d, 1)))) return rc;
  if ((rc = ctx->flags.reserve(ctx, 64))) return rc;
  cudaError_t e = cudaMemsetAsync(ctx->flags.ptr, 0, 4, st);
  if (e != cudaSuccess) return ctx_cuda_fail(ctx, e, "memset flags");
  e = ddks_launch_encode(dP, dT, NP, NT, d, dtype == DDKS_F64, (uint64_t*)ctx->keys.ptr,
                         (unsigned*)ctx->flags.ptr, st);
  if (e != cudaSuccess) return ctx_cuda_fail(ctx, e, "encode");
  ctx->launches += 1;
  int n = 0, pfx_done = 0;
  uint32_t* pfx0 = want_sorted0 ? (uint32_t*)ctx->pfx0.ptr : nullptr;
  e = ddks_launch_rank((const uint64_t*)ctx->keys.ptr, N, NP, d, (uint64_t*)ctx->tk1.ptr,
                       (uint32_t*)ctx->ti1.ptr, (uint64_t*)ctx->tk2.ptr, (uint32_t*)ctx->ti2.ptr,
                       (uint32_t*)ctx->rank.ptr, want_sorted0 ? (uint32_t*)ctx->sidx0.ptr : nullptr,
                       pfx0, pfx0 ? pfx0 + N : nullptr, &pfx_done, st, &n, key_bits,
                       radix ? (uint32_t*)ctx->radix.ptr : nullptr, &ctx->sorted_rows);
  ctx->launches += n;
  ctx->pfx0_valid = pfx_done != 0;
  if (e != cudaSuccess) return ctx_cuda_fail(ctx, e, "rank");
  return DDKS_OK;
}

// Counts + per-origin maxima for origins [ob, oe) on the encoded problem.
int ddks_count_origins(ddks_ctx* ctx, int64_t NP, int64_t NT, int32_t d, int64_t ob, int64_t oe,
                       uint64_t* best, int32_t* bestj, cudaStream_t st) {
  ddks_plan plan;
  int rc = ddks_select_path(ctx, NP, NT, d, &plan);
  if (rc) return rc;
  return ddks_count_origins_plan(ctx, plan, NP, NT, d, ob, oe, best, bestj, st);
}

int ddks_count_origins_plan(ddks_ctx* ctx, const ddks_plan& plan, int64_t NP, int64_t NT, int32_t d,
                            int64_t ob, int64_t oe, uint64_t* best, int32_t* bestj, cudaStream_t st,
                            unsigned long long* out3, bool* reduced) {
  if (reduced) *reduced = false;
  const int64_t N = NP + NT;
  const uint32_t* rank = (const uint32_t*)ctx->rank.ptr;
  cudaError_t e = cudaSuccess;
  switch (plan.path) {
    case DDKS_PATH_REGISTER:
      e = ddks_launch_register(ctx, rank, N, NP, NT, d, ob, oe, best, bestj, st, plan, out3, reduced);
      break;
    case DDKS_PATH_LANE:
      e = ddks_launch_lane(rank, N, NP, NT, d, ob, oe, best, bestj, st, plan.threads, ctx->num_sms);
      ctx->launches += 1;
      break;
    case DDKS_PATH_WARP:
      if (ddks_warp16_supported(d, NP, NT)) {
        int n = 0;
        e = ddks_launch_warp16(ctx, rank, N, NP, NT, d, ob, oe, best, bestj, st, &n);
        ctx->launches += n;
      } else {
        e = ddks_launch_warp(rank, N, NP, NT, d, ob, oe, best, bestj, st, plan.warps);
        ctx->launches += 1;
      }
      break;
    case DDKS_PATH_SORT:
      e = ddks_launch_sort(rank, N, NP, NT, d, ob, oe, best, bestj, st);
      ctx->launches += 1;
      break;
    case DDKS_PATH_BYTE: {
      int nl = 0;
      e = ddks_launch_byte(ctx, rank, N, NP, NT, d, ob, oe, best, bestj, st, &nl);
      ctx->launches += nl;
      break;
    }
    case DDKS_PATH_DOMINANCE: {
      if (!ctx->pfx0_valid) return DDKS_EUNSUPPORTED;  // needs K0's dimension-0 order and P prefix
      int n = 0;
      e = ddks_launch_dominance(ctx, rank, N, NP, NT, ob, oe, best, bestj, st, &n);
      ctx->launches += n;
      break;
    }
    default:
      return DDKS_EUNSUPPORTED;
  }
  if (e != cudaSuccess) return ctx_cuda_fail(ctx, e, "count kernel");
  return DDKS_OK;
}

static int distance_impl(ddks_ctx* ctx, const void* P, int64_t NP, const void* T, int64_t NT,
                         int32_t d, int32_t dtype, int64_t ob, int64_t oe, uint64_t* per_origin,
                         void* stream, ddks_result* out) {
  if (!ctx || !out) return DDKS_EINVAL;
  int rc = ddks_check_problem(P, NP, T, NT, d, dtype);
  if (rc) { out->status = rc; return rc; }
  const int64_t N = NP + NT;
  if (ob < 0 || oe > N || ob > oe) { out->status = DDKS_EINVAL; return DDKS_EINVAL; }
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return out->status = ctx_cuda_fail(ctx, e, "cudaSetDevice");
  const void *dP, *dT;
  if ((rc = ddks_stage_inputs(ctx, P, NP, T, NT, d, dtype, st, &dP, &dT))) return out->status = rc;
  ddks_plan plan;
  if ((rc = ddks_select_path(ctx, NP, NT, d, &plan))) return out->status = rc;
  const int64_t no = oe - ob;
  GraphKey key;
  key.add(1).add((uint64_t)NP).add((uint64_t)NT).add((uint64_t)d).add((uint64_t)dtype);
  key.add((uint64_t)ob).add((uint64_t)oe).add((uint64_t)plan.path).add((uint64_t)plan.threads);
  key.add((uint64_t)plan.warps).add((uint64_t)plan.reg_occ).add((uint64_t)plan.fused).add_ptr(dP).add_ptr(dT);
  key.add((uint64_t)ctx->stage_timing);
  rc = ddks_graph_run(ctx, key.h, st, [&](cudaStream_t s) -> int {
    int r;
    stage_mark(ctx, 0, s);
    if ((r = ddks_encode_problem(ctx, dP, NP, dT, NT, d, dtype, s,
                                 plan.path == DDKS_PATH_REGISTER || plan.path == DDKS_PATH_DOMINANCE)))
      return r;
    stage_mark(ctx, 1, s);
    if ((r = ctx->best.reserve(ctx, 8 * (size_t)(no > 0 ? no : 1)))) return r;
    if ((r = ctx->bestj.reserve(ctx, 4 * (size_t)(no > 0 ? no : 1)))) return r;
    if ((r = ctx->out3.reserve(ctx, 64 + ddks_reduce_scratch_bytes()))) return r;
    bool reduced = false;
    if ((r = ddks_count_origins_plan(ctx, plan, NP, NT, d, ob, oe, (uint64_t*)ctx->best.ptr,
                                     (int32_t*)ctx->bestj.ptr, s, (unsigned long long*)ctx->out3.ptr, &reduced)))
      return r;
    stage_mark(ctx, 2, s);
    if (!reduced) {
      cudaError_t ee = ddks_launch_reduce((const uint64_t*)ctx->best.ptr, (const int32_t*)ctx->bestj.ptr, no,
                                          ob, (unsigned long long*)ctx->out3.ptr, (char*)ctx->out3.ptr + 64, s);
      ctx->launches += 2;
      if (ee != cudaSuccess) return ctx_cuda_fail(ctx, ee, "reduce");
    }
    stage_mark(ctx, 3, s);
    return DDKS_OK;
  });
  if (rc) return out->status = rc;
  e = cudaMemcpyAsync(ctx->h_out, ctx->out3.ptr, 3 * sizeof(unsigned long long),
                      cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ctx->h_out + 4, ctx->flags.ptr, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && per_origin && no > 0)
    e = cudaMemcpyAsync(per_origin, ctx->best.ptr, 8 * (size_t)no, cudaMemcpyDefault, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return out->status = ctx_cuda_fail(ctx, e, "result copy");
  ddks_stage_collect(ctx);
  const unsigned flags = (unsigned)(ctx->h_out[4] & 0xFFFFFFFFull);
  if (flags & ddks::kFlagNaN) return out->status = DDKS_ENAN;
  if (flags & ddks::kFlagTimeout) return out->status = DDKS_ETIMEOUT;
  if (flags & ddks::kFlagBounds) {
    ctx->last_err = "a kernel's bounds check failed";
    return out->status = DDKS_ECUDA;
  }
  out->num_max = ctx->h_out[0];
  out->denom = (uint64_t)NP * (uint64_t)NT;
  out->D = (double)out->num_max / (double)out->denom;
  out->argmax_origin = no > 0 ? (int64_t)ctx->h_out[1] : -1;
  out->argmax_orthant = no > 0 ? (int32_t)ctx->h_out[2] : 0;
  out->status = DDKS_OK;
  return DDKS_OK;
}

int ddks_distance(ddks_ctx* ctx, const void* P, int64_t NP, const void* T, int64_t NT, int32_t d,
                  int32_t dtype, void* stream, ddks_result* out) {
  if (NP < 1 || NT < 1) {
    if (out) out->status = DDKS_EINVAL;
    return DDKS_EINVAL;
  }
  return distance_impl(ctx, P, NP, T, NT, d, dtype, 0, NP + NT, nullptr, stream, out);
}

int ddks_distance_range(ddks_ctx* ctx, const void* P, int64_t NP, const void* T, int64_t NT,
                        int32_t d, int32_t dtype, int64_t o_begin, int64_t o_end,
                        uint64_t* per_origin, void* stream, ddks_result* out) {
  return distance_impl(ctx, P, NP, T, NT, d, dtype, o_begin, o_end, per_origin, stream, out);
}
