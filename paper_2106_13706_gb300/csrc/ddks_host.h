// ddks_host.h -- host-side context and helpers shared by the library's .cu files.
#pragma once
#include <condition_variable>
#include <cstdint>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/ddks.h"

struct ddks_ctx;

// A context-owned device buffer that grows on demand (never shrinks).
struct DevBuf {
  void* ptr = nullptr;
  size_t bytes = 0;
  int reserve(ddks_ctx* ctx, size_t n);
  void release();
};

// Kernel configuration chosen for one problem shape.
struct ddks_plan {
  int path = DDKS_PATH_AUTO;
  int threads = 256;  // lane path: threads per CTA (one origin each)
  int warps = 8;      // warp path: warps per CTA (one origin each)
  int reg_occ = 4;    // register path occupancy class: 4, 6, 8 (8, 12, 16 resident 64-thread CTAs per SM)
  int fused = 0;      // register path: 0 = bit planes staged by the pack kernel, 1..3 = built in shared
                      // memory by the count kernel (count_fused.cu, kernel shapes listed there)
};

struct ServeState;  // serve.cu

// A captured CUDA graph for one repeated call (graph.cu).
struct GraphEntry {
  uint64_t key = 0;            // hash of the call's shapes, plan and device addresses
  uint64_t gen = 0;            // ctx->buf_gen when captured
  cudaGraphExec_t exec = nullptr;
  uint64_t kernels = 0;        // kernels one replay launches
  uint64_t last_use = 0;
  bool primed = false;         // a direct run of this key has succeeded
};

struct ddks_ctx {
  ddks_config cfg{};
  int device = 0;
  int num_sms = 152;
  // bound on each device-side wait for an asynchronous copy (ns): the
  // config's wait_limit_ms when given, else 1 s; ddks_set_device_wait_limit
  unsigned long long dev_wait_ns = 1000000000ull;
  unsigned long long dev_wait_cfg_ns = 1000000000ull;  // the value fixed at creation
  std::string last_err;
  uint64_t launches = 0;
  // scratch of the synchronous entry points
  DevBuf inP, inT, keys, tk1, tk2, ti1, ti2, rank, sidx0, best, bestj, out3, flags;
  DevBuf pfx0;         // P points before each dimension-0 sorted position (+ chunk scratch)
  bool pfx0_valid = false;  // pfx0 holds the current problem's prefix
  const uint32_t* sorted_rows = nullptr;  // K0 by radix sort: pooled indices per dimension in sorted order, [d][N]
  DevBuf reg_words, reg_meta;                   // register path
  DevBuf warp_words;                            // warp path: packed rank pairs
  DevBuf perm_keys, perm_labels, perm_best, perm_codes;  // permutation test
  DevBuf sig_cells, sig_logp;                   // significance
  DevBuf batch_desc, batch_work;                // batched launch
  DevBuf apx_small, apx_cnt, apx_U, apx_hist;   // vdKS / rdKS (approx.cu)
  DevBuf rdks_aux;                              // rdKS by histogram: buckets, candidates
  DevBuf dom_work;                              // d = 2 range-query path (dominance.cu)
  DevBuf radix;                                 // radix sort counts / offsets / flags (radix.cu)
  unsigned long long* h_out = nullptr;          // pinned, 64 entries
  void* h_stage = nullptr;                      // pinned staging for uploads
  size_t h_stage_bytes = 0;
  // stage timing (ddks_set_stage_timing)
  bool stage_timing = false;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  float stage_ms[3] = {0, 0, 0};
  // autotuner: key -> plan
  std::string tune_cache_path;
  std::map<std::string, ddks_plan> tune;
  std::mutex tune_mu;
  // batched launch: tile shapes per dimension (origins per work unit, points
  // per staged tile), set by ddks_autotune_batch; per-group kernel times when tuning
  // per dimension: bit-sliced units (127) for 2..6, byte units (127) for 7, 8
  int batch_ot[12] = {64, 64, 127, 127, 127, 127, 127, 127, 127, 64, 64, 64};
  int batch_pt[12] = {512, 512, 512, 512, 512, 512, 512, 512, 512, 512, 512, 512};
  bool batch_timing = false;
  float batch_group_ms[12] = {};
  // serving
  ServeState* serve = nullptr;  // owned; freed by ddks_serve_shutdown
  // graph replay (graph.cu); buf_gen counts scratch reallocations
  uint64_t buf_gen = 0;
  cudaStream_t cap_st = nullptr;
  std::vector<GraphEntry> graphs;
  uint64_t graph_tick = 0, graph_captures = 0, graph_replays = 0;

  std::vector<DevBuf*> all_bufs() {
    return {&inP, &inT, &keys, &tk1, &tk2, &ti1, &ti2, &rank, &sidx0, &pfx0, &best, &bestj, &out3,
            &flags, &reg_words, &reg_meta, &warp_words, &perm_keys, &perm_labels, &perm_best, &perm_codes,
            &sig_cells, &sig_logp, &batch_desc, &batch_work, &apx_small, &apx_cnt, &apx_U, &apx_hist, &dom_work,
            &radix, &rdks_aux};
  }
};

int ctx_cuda_fail(ddks_ctx* ctx, cudaError_t e, const char* where);
// 1: device memory of `device` or managed memory (read in place); 0: host
// memory (copied by the call); DDKS_EINVAL: device memory of another GPU.
int ddks_pointer_kind(const void* p, int device);
// true for host memory CUDA does not know (pageable): a copy from it is staged
// by the driver before the copy call returns
bool ddks_is_pageable(const void* p);
int ddks_check_problem(const void* P, int64_t NP, const void* T, int64_t NT, int32_t d, int32_t dtype);
int ddks_stage_inputs(ddks_ctx* ctx, const void* P, int64_t NP, const void* T, int64_t NT,
                      int32_t d, int32_t dtype, cudaStream_t st, const void** dP, const void** dT);
int ddks_encode_problem(ddks_ctx* ctx, const void* dP, int64_t NP, const void* dT, int64_t NT,
                        int32_t d, int32_t dtype, cudaStream_t st, bool want_sorted0);
void ddks_stage_mark(ddks_ctx* ctx, int i, cudaStream_t st);
bool ddks_use_radix(const ddks_ctx* ctx, int64_t N, int key_bits);  // tune.cu: radix vs chunk sort + merges
void ddks_stage_collect(ddks_ctx* ctx);  // after the stream has synchronised
int ddks_count_origins(ddks_ctx* ctx, int64_t NP, int64_t NT, int32_t d, int64_t ob, int64_t oe,
                       uint64_t* best, int32_t* bestj, cudaStream_t st);
// out3 / reduced as for ddks_launch_register (only the register path reduces)
int ddks_count_origins_plan(ddks_ctx* ctx, const ddks_plan& plan, int64_t NP, int64_t NT, int32_t d,
                            int64_t ob, int64_t oe, uint64_t* best, int32_t* bestj, cudaStream_t st,
                            unsigned long long* out3 = nullptr, bool* reduced = nullptr);

// tune.cu
int ddks_select_path(ddks_ctx* ctx, int64_t NP, int64_t NT, int32_t d, ddks_plan* plan);
void ddks_tune_load(ddks_ctx* ctx);

// count_register.cu
// out3 (optional): the kernel also reduces over origins and writes
// {num_max, arg-max origin, orthant} there; *reduced tells whether it did.
cudaError_t ddks_launch_register(ddks_ctx* ctx, const uint32_t* rank, int64_t N, int64_t NP,
                                 int64_t NT, int d, int64_t ob, int64_t oe, uint64_t* best,
                                 int32_t* bestj, cudaStream_t st, const ddks_plan& plan,
                                 unsigned long long* out3 = nullptr, bool* reduced = nullptr);
bool ddks_register_supported(int d, int64_t NP, int64_t NT);

// rank_cluster.cu: K0 (order keys, min-ranks, dimension-0 order and P
// prefix, every dimension's sorted order) in one launch of d thread-block
// clusters, for samples whose rows fit a cluster's shared memory
bool ddks_rank_cluster_supported(int64_t N, int key_bits, int device);
cudaError_t ddks_launch_rank_cluster(const void* P, const void* T, int64_t NP, int64_t NT, int d, bool f64,
                                     uint32_t* rank, uint32_t* sorted, uint32_t* sidx0, uint32_t* pfx0,
                                     unsigned* flags, cudaStream_t st);

// count_fused.cu: the register path's count with the bit planes built in
// shared memory; the caller has zeroed gcnt, done and packed
bool ddks_fused_supported(int ds, int64_t N, int variant);
size_t ddks_fused_scratch_bytes(int ds, int64_t N, int64_t blocks);
cudaError_t ddks_fused_count(ddks_ctx* ctx, int ds, int variant, const uint32_t* rankL, const uint32_t* orank,
                             const void* meta, int64_t no, int64_t N, int64_t NP, int64_t NT, int64_t NPpad,
                             int64_t Lrow, uint32_t* gcnt, unsigned* done, unsigned long long* packed, uint64_t* best,
                             int32_t* bestj, int64_t ob, unsigned long long* out3, unsigned* flags,
                             void* scratch, cudaStream_t st, int* launches);

// graph.cu: a hash of everything a captured graph depends on
struct GraphKey {
  uint64_t h = 1469598103934665603ull;  // FNV-1a
  GraphKey& add(uint64_t v) {
    for (int i = 0; i < 8; ++i) { h ^= (v >> (8 * i)) & 0xFF; h *= 1099511628211ull; }
    return *this;
  }
  GraphKey& add_ptr(const void* p) { return add((uint64_t)(uintptr_t)p); }
  GraphKey& add_bytes(const void* p, size_t n) {
    const unsigned char* b = (const unsigned char*)p;
    for (size_t i = 0; i < n; ++i) { h ^= b[i]; h *= 1099511628211ull; }
    return *this;
  }
};
// mode 0: run body directly on st; 1: body is being captured on *run_st;
// 2: a captured graph was launched on st
int ddks_graph_begin(ddks_ctx* ctx, uint64_t key, cudaStream_t st, cudaStream_t* run_st, int* mode);
int ddks_graph_end(ddks_ctx* ctx, uint64_t key, cudaStream_t st, int mode, int body_rc, uint64_t l0,
                   uint64_t g0);
void ddks_graph_mark(ddks_ctx* ctx, uint64_t key);
void ddks_graph_clear(ddks_ctx* ctx);

// Run body(stream) directly, or through the graph captured for `key` (the
// graph replay note in ddks.h).  body enqueues work only: no synchronisation,
// no host reads of device results.
template <typename F>
int ddks_graph_run(ddks_ctx* ctx, uint64_t key, cudaStream_t st, F&& body) {
  key = GraphKey().add(key).add(ctx->dev_wait_ns).h;  // the wait bound is a kernel argument too
  cudaStream_t run_st = st;
  int mode = 0;
  int rc = ddks_graph_begin(ctx, key, st, &run_st, &mode);
  if (rc) return rc;
  if (mode == 2) return 0;  // replayed
  const uint64_t l0 = ctx->launches, g0 = ctx->buf_gen;
  const int brc = body(run_st);
  if (mode == 0) {  // direct
    if (brc == 0) ddks_graph_mark(ctx, key);
    return brc;
  }
  rc = ddks_graph_end(ctx, key, st, mode, brc, l0, g0);
  if (rc == 1) return body(st);  // capture dropped: run directly
  return rc;
}

// dominance.cu
bool ddks_dominance_supported(int d, int64_t NP, int64_t NT);
cudaError_t ddks_launch_dominance(ddks_ctx* ctx, const uint32_t* rank, int64_t N, int64_t NP, int64_t NT,
                                  int64_t ob, int64_t oe, uint64_t* best, int32_t* bestj, cudaStream_t st,
                                  int* launches);

// count_byte.cu
bool ddks_byte_supported(int d, int64_t NP, int64_t NT);
cudaError_t ddks_launch_byte(ddks_ctx* ctx, const uint32_t* rank, int64_t N, int64_t NP, int64_t NT, int d,
                             int64_t ob, int64_t oe, uint64_t* best, int32_t* bestj, cudaStream_t st,
                             int* launches);

// count_warp.cu
bool ddks_warp16_supported(int d, int64_t NP, int64_t NT);
cudaError_t ddks_launch_warp16(ddks_ctx* ctx, const uint32_t* rank, int64_t N, int64_t NP, int64_t NT,
                               int d, int64_t o_begin, int64_t o_end, uint64_t* best, int32_t* bestj,
                               cudaStream_t st, int* launches);

// serve.cu
void ddks_serve_shutdown(ddks_ctx* ctx);
void ddks_serve_fill_stats(ddks_ctx* ctx, ddks_stats* out);
