// serve.cu -- continuous batching of two-sample ddKS requests.
//
// ddks_submit copies a request's points into library-owned device memory
// (stream-ordered allocations from the device's memory pool; from pageable
// host memory the worker's stream waits on an event for the copy, otherwise
// submit waits for it) and queues it.  Worker threads (two, each with its own
// internal context and stream) repeatedly admit queued requests in arrival
// order while the sum of the admitted requests' device footprints stays
// within the HBM budget and the batch stays within max_batch, run the admitted
// requests as one batched launch (batch.cu: one persistent launch per
// dimension over all their work units), and publish the results.  Requests
// that arrive while a batch is on the GPU join the next one; with two workers
// two batches overlap on the device.  A request above the batched kernels'
// size (16,384 pooled points) fills the GPU by itself: it runs alone, one at
// a time, through the single-problem path (ddks_distance), and small requests
// behind a waiting large one may go first.  A request whose footprint alone
// exceeds the budget is refused at submit with DDKS_ENOMEM.  ddks_poll reads
// a result, optionally waiting a bounded time.  No device code waits on the
// host: the only waits are host condition variables with timeouts.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "ddks_host.h"
#include "ddks_internal.cuh"

namespace {

struct Request {
  uint64_t ticket = 0;
  void* P = nullptr;  // device copies of the inputs, freed by the worker that served them
  void* T = nullptr;
  int64_t NP = 0, NT = 0;
  int32_t d = 0, dtype = 0;
  uint64_t footprint = 0;
  int status = DDKS_PENDING;
  ddks_result res{};
  cudaEvent_t ready = nullptr;  // input copies still in flight (pageable host inputs)
  bool big = false;             // above the batched kernels' size: runs alone
};

constexpr int64_t kBigN = 16384;  // pooled points above which a request runs alone

constexpr int kWorkers = 2;

}  // namespace

struct ServeState {
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<Request>> pending;
  std::unordered_map<uint64_t, std::shared_ptr<Request>> reqs;
  uint64_t next_ticket = 1;
  uint64_t resident = 0, resident_peak = 0;
  int big_running = 0;  // large requests on the GPU (at most one)
  uint64_t submitted = 0, admitted = 0, completed = 0, rejected = 0, batches = 0;
  bool stop = false;
  std::vector<std::thread> workers;
  std::vector<ddks_ctx*> wctx;
  std::vector<cudaStream_t> streams;
  cudaStream_t sub_st = nullptr;  // input copies of ddks_submit
  std::mutex sub_mu;
};

static uint64_t request_footprint(int64_t NP, int64_t NT, int32_t d, int32_t dtype) {
  const uint64_t N = (uint64_t)(NP + NT);
  const uint64_t es = dtype == DDKS_F64 ? 8 : 4;
  // inputs, ranks, per-origin maxima and arg-maxima, sort and key scratch
  return N * d * (es + 4 + 8 + 24) + N * 12 + 4096;
}

static void worker_loop(ddks_ctx* owner, int w) {
  ServeState* S = owner->serve;
  ddks_ctx* ctx = S->wctx[w];
  cudaStream_t st = S->streams[w];
  cudaSetDevice(ctx->device);
  const uint64_t budget = owner->cfg.hbm_budget_bytes;
  const int max_batch = owner->cfg.max_batch;
  for (;;) {
    std::vector<std::shared_ptr<Request>> batch;
    bool big = false;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      // A large request fills the GPU by itself: it runs alone and one at a
      // time (two at once would each take twice as long); small requests
      // behind a waiting large one may go first.  Otherwise arrival order.
      auto admissible = [&](const std::shared_ptr<Request>& r) {
        return S->resident + r->footprint <= budget && (!r->big || S->big_running == 0);
      };
      S->cv_work.wait(lk, [&] {
        if (S->stop) return true;
        for (auto& r : S->pending)
          if (admissible(r)) return true;
        return false;
      });
      if (S->stop) return;
      for (auto it = S->pending.begin(); it != S->pending.end() && (int)batch.size() < max_batch;) {
        auto r = *it;
        if (r->big) {
          if (batch.empty() && admissible(r)) {  // alone
            it = S->pending.erase(it);
            S->resident += r->footprint;
            S->admitted += 1;
            S->big_running += 1;
            batch.push_back(r);
            big = true;
            break;
          }
          ++it;  // small requests behind it may go first
          continue;
        }
        if (S->resident + r->footprint > budget) break;  // arrival order within the budget
        it = S->pending.erase(it);
        S->resident += r->footprint;
        S->admitted += 1;
        batch.push_back(r);
      }
      if (S->resident > S->resident_peak) S->resident_peak = S->resident;
      S->batches += 1;
    }
    // the batch's input copies, where submit did not wait for them
    for (auto& r : batch)
      if (r->ready) {
        cudaStreamWaitEvent(st, r->ready, 0);
        cudaEventDestroy(r->ready);
        r->ready = nullptr;
      }
    // group by dtype (one batched launch per dtype)
    for (int dt = 0; dt < 2; ++dt) {
      std::vector<const void*> Ps, Ts;
      std::vector<int64_t> NPs, NTs;
      std::vector<int32_t> ds;
      std::vector<std::shared_ptr<Request>> members;
      for (auto& r : batch)
        if (r->dtype == dt) {
          Ps.push_back(r->P);
          Ts.push_back(r->T);
          NPs.push_back(r->NP);
          NTs.push_back(r->NT);
          ds.push_back(r->d);
          members.push_back(r);
        }
      if (members.empty()) continue;
      std::vector<ddks_result> out(members.size());
      // one request: the single-problem path; several: one batched launch
      int rc = members.size() == 1
                   ? ddks_distance(ctx, Ps[0], NPs[0], Ts[0], NTs[0], ds[0], dt, st, out.data())
                   : ddks_batch_distance(ctx, (int32_t)members.size(), Ps.data(), NPs.data(), Ts.data(),
                                         NTs.data(), ds.data(), dt, st, out.data());
      if (rc != DDKS_OK) {
        // find the failing members one by one so one bad request does not fail the rest
        for (size_t i = 0; i < members.size(); ++i) {
          ddks_result one{};
          const int r1 = ddks_distance(ctx, Ps[i], NPs[i], Ts[i], NTs[i], ds[i], dt, st, &one);
          out[i] = one;
          out[i].status = r1;
        }
      }
      // the calls above synchronised st: the inputs can go back to the pool
      for (auto& m : members) {
        cudaFreeAsync(m->P, st);
        cudaFreeAsync(m->T, st);
      }
      std::lock_guard<std::mutex> g(S->mu);
      for (size_t i = 0; i < members.size(); ++i) {
        members[i]->res = out[i];
        members[i]->status = out[i].status;
        members[i]->P = members[i]->T = nullptr;
      }
    }
    {
      std::lock_guard<std::mutex> g(S->mu);
      for (auto& r : batch) {
        S->resident -= r->footprint;
        S->completed += 1;
      }
      if (big) S->big_running -= 1;
    }
    S->cv_done.notify_all();
    S->cv_work.notify_all();
  }
}

static int serve_start(ddks_ctx* ctx) {
  if (ctx->serve) return DDKS_OK;
  ServeState* S = new (std::nothrow) ServeState();
  if (!S) return DDKS_ENOMEM;
  ddks_config cfg = ctx->cfg;
  cfg.device = ctx->device;
  cfg.graphs = 0;  // device batches rarely repeat a membership: capture would not pay
  for (int w = 0; w < kWorkers; ++w) {
    ddks_ctx* c = nullptr;
    int rc = ddks_ctx_create(&cfg, &c);
    cudaStream_t st = nullptr;
    cudaError_t e = rc == DDKS_OK ? cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) : cudaSuccess;
    if (rc != DDKS_OK || e != cudaSuccess) {
      if (c) ddks_ctx_destroy(c);
      for (size_t i = 0; i < S->wctx.size(); ++i) {
        cudaStreamDestroy(S->streams[i]);
        ddks_ctx_destroy(S->wctx[i]);
      }
      delete S;
      return rc != DDKS_OK ? rc : ctx_cuda_fail(ctx, e, "cudaStreamCreate");
    }
    S->wctx.push_back(c);
    S->streams.push_back(st);
  }
  cudaError_t e = cudaStreamCreateWithFlags(&S->sub_st, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    for (size_t i = 0; i < S->wctx.size(); ++i) {
      cudaStreamDestroy(S->streams[i]);
      ddks_ctx_destroy(S->wctx[i]);
    }
    delete S;
    return ctx_cuda_fail(ctx, e, "cudaStreamCreate");
  }
  ctx->serve = S;
  for (int w = 0; w < kWorkers; ++w) S->workers.emplace_back(worker_loop, ctx, w);
  return DDKS_OK;
}

void ddks_serve_shutdown(ddks_ctx* ctx) {
  ServeState* S = ctx->serve;
  if (!S) return;
  {
    std::lock_guard<std::mutex> g(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  S->cv_done.notify_all();
  for (auto& t : S->workers) t.join();
  for (auto& r : S->pending) {  // never admitted: their inputs go back to the pool
    cudaFreeAsync(r->P, S->sub_st);
    cudaFreeAsync(r->T, S->sub_st);
    if (r->ready) cudaEventDestroy(r->ready);
  }
  cudaStreamSynchronize(S->sub_st);
  cudaStreamDestroy(S->sub_st);
  for (size_t i = 0; i < S->wctx.size(); ++i) {
    cudaStreamDestroy(S->streams[i]);
    ddks_ctx_destroy(S->wctx[i]);
  }
  delete S;
  ctx->serve = nullptr;
}

void ddks_serve_fill_stats(ddks_ctx* ctx, ddks_stats* out) {
  std::memset(out, 0, sizeof(*out));
  ServeState* S = ctx->serve;
  if (!S) return;
  std::lock_guard<std::mutex> g(S->mu);
  out->submitted = S->submitted;
  out->admitted = S->admitted;
  out->completed = S->completed;
  out->rejected = S->rejected;
  out->batches = S->batches;
  out->bytes_resident = S->resident;
  out->bytes_resident_peak = S->resident_peak;
  uint64_t k = 0;
  for (auto* c : S->wctx) k += c->launches;
  out->kernel_launches = k;
}

int ddks_submit(ddks_ctx* ctx, const void* P, int64_t NP, const void* T, int64_t NT, int32_t d,
                int32_t dtype, uint64_t* ticket) {
  if (!ctx || !ticket) return DDKS_EINVAL;
  int rc = ddks_check_problem(P, NP, T, NT, d, dtype);
  if (rc) return rc;
  if ((rc = serve_start(ctx))) return rc;
  ServeState* S = ctx->serve;
  auto r = std::make_shared<Request>();
  r->NP = NP;
  r->NT = NT;
  r->d = d;
  r->dtype = dtype;
  r->footprint = request_footprint(NP, NT, d, dtype);
  r->big = NP + NT > kBigN;
  if (r->footprint > ctx->cfg.hbm_budget_bytes) {
    std::lock_guard<std::mutex> g(S->mu);
    S->rejected += 1;
    return DDKS_ENOMEM;
  }
  const size_t es = dtype == DDKS_F64 ? 8 : 4;
  const size_t bP = es * (size_t)NP * d, bT = es * (size_t)NT * d;
  // copy the inputs (host or device) to the device so the caller may free
  // them on return.  From pageable host memory the driver has staged the
  // data by the time the copy call returns, so the worker's stream waits on
  // an event instead; device and page-locked inputs are waited for here.
  {
    std::lock_guard<std::mutex> g(S->sub_mu);
    cudaError_t e = cudaSetDevice(ctx->device);
    const bool pageable = ddks_is_pageable(P) && ddks_is_pageable(T);
    if (e == cudaSuccess) e = cudaMallocAsync(&r->P, bP, S->sub_st);
    if (e == cudaSuccess) e = cudaMallocAsync(&r->T, bT, S->sub_st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(r->P, P, bP, cudaMemcpyDefault, S->sub_st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(r->T, T, bT, cudaMemcpyDefault, S->sub_st);
    if (e == cudaSuccess && pageable) {
      e = cudaEventCreateWithFlags(&r->ready, cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventRecord(r->ready, S->sub_st);
    } else if (e == cudaSuccess) {
      e = cudaStreamSynchronize(S->sub_st);
    }
    if (e != cudaSuccess) {
      if (r->P) cudaFreeAsync(r->P, S->sub_st);
      if (r->T) cudaFreeAsync(r->T, S->sub_st);
      cudaStreamSynchronize(S->sub_st);
      if (r->ready) cudaEventDestroy(r->ready);
      return ctx_cuda_fail(ctx, e, "submit copy");
    }
  }
  {
    std::lock_guard<std::mutex> g(S->mu);
    r->ticket = S->next_ticket++;
    S->reqs[r->ticket] = r;
    S->pending.push_back(r);
    S->submitted += 1;
    *ticket = r->ticket;
  }
  S->cv_work.notify_one();
  return DDKS_OK;
}

int ddks_poll(ddks_ctx* ctx, uint64_t ticket, int32_t timeout_us, ddks_result* out) {
  if (!ctx || !out) return DDKS_EINVAL;
  ServeState* S = ctx->serve;
  if (!S) return DDKS_ENOTFOUND;
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) return DDKS_ENOTFOUND;
  std::shared_ptr<Request> r = it->second;
  if (r->status == DDKS_PENDING && timeout_us > 0) {
    S->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us),
                        [&] { return r->status != DDKS_PENDING || S->stop; });
  }
  if (r->status == DDKS_PENDING) return DDKS_PENDING;
  *out = r->res;
  out->status = r->status;
  S->reqs.erase(it);
  return r->status;
}
