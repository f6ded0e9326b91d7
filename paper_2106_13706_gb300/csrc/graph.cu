// graph.cu -- graph replay of repeated calls.
//
// A call of ddks_distance / ddks_distance_range / ddks_permutation_test /
// ddks_batch_distance enqueues a fixed sequence of kernels and memsets for a
// given problem shape.  When the same shape (and the same device addresses)
// comes again, the sequence is captured into a CUDA graph on a private stream
// and every later repetition launches the graph: one launch instead of ten to
// twenty, which is most of the time of a small problem.  Everything a graph
// bakes in is in its key, except the context's scratch addresses, which
// buf_gen tracks: a reallocation retires every graph captured before it.
#include "ddks_host.h"

namespace {

constexpr size_t kMaxGraphs = 16;

GraphEntry* find(ddks_ctx* ctx, uint64_t key) {
  for (auto& g : ctx->graphs)
    if (g.key == key) return &g;
  return nullptr;
}

void drop_exec(GraphEntry& g) {
  if (g.exec) cudaGraphExecDestroy(g.exec);
  g.exec = nullptr;
}

}  // namespace

int ddks_graph_begin(ddks_ctx* ctx, uint64_t key, cudaStream_t st, cudaStream_t* run_st, int* mode) {
  *mode = 0;
  *run_st = st;
  if (!ctx->cfg.graphs || ctx->stage_timing || ctx->batch_timing) return DDKS_OK;
  const uint64_t tick = ++ctx->graph_tick;
  GraphEntry* g = find(ctx, key);
  if (g && g->exec && g->gen == ctx->buf_gen) {
    g->last_use = tick;
    cudaError_t e = cudaGraphLaunch(g->exec, st);
    if (e != cudaSuccess) return ctx_cuda_fail(ctx, e, "cudaGraphLaunch");
    ctx->launches += g->kernels;
    ++ctx->graph_replays;
    *mode = 2;
    return DDKS_OK;
  }
  if (!g) {  // first occurrence: remember it, run directly
    if (ctx->graphs.size() >= kMaxGraphs) {
      size_t old = 0;
      for (size_t i = 1; i < ctx->graphs.size(); ++i)
        if (ctx->graphs[i].last_use < ctx->graphs[old].last_use) old = i;
      drop_exec(ctx->graphs[old]);
      ctx->graphs.erase(ctx->graphs.begin() + (std::ptrdiff_t)old);
    }
    GraphEntry n;
    n.key = key;
    n.last_use = tick;
    ctx->graphs.push_back(n);
    return DDKS_OK;
  }
  g->last_use = tick;
  if (!g->primed) return DDKS_OK;  // no successful direct run yet: its scratch may still grow
  // seen before (or captured against scratch that has moved since): capture
  drop_exec(*g);
  if (!ctx->cap_st) {
    cudaError_t e = cudaStreamCreateWithFlags(&ctx->cap_st, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      cudaGetLastError();
      ctx->cap_st = nullptr;
      return DDKS_OK;
    }
  }
  if (cudaStreamBeginCapture(ctx->cap_st, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
    cudaGetLastError();
    return DDKS_OK;
  }
  *run_st = ctx->cap_st;
  *mode = 1;
  return DDKS_OK;
}

// Ends a capture.  Returns 1 when the capture is unusable (the body failed, or
// scratch was reallocated while capturing) and the body must run directly.
int ddks_graph_end(ddks_ctx* ctx, uint64_t key, cudaStream_t st, int mode, int body_rc, uint64_t l0,
                   uint64_t g0) {
  if (mode != 1) return body_rc;
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(ctx->cap_st, &graph);
  const uint64_t kernels = ctx->launches - l0;
  ctx->launches = l0;  // nothing ran yet
  if (body_rc != DDKS_OK || e != cudaSuccess || !graph || ctx->buf_gen != g0) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return 1;
  }
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  GraphEntry* g = find(ctx, key);
  if (!g) {  // cannot happen: begin() left the entry in place
    cudaGraphExecDestroy(exec);
    return 1;
  }
  g->exec = exec;
  g->gen = ctx->buf_gen;
  g->kernels = kernels;
  ++ctx->graph_captures;
  e = cudaGraphLaunch(exec, st);
  if (e != cudaSuccess) return ctx_cuda_fail(ctx, e, "cudaGraphLaunch");
  ctx->launches += kernels;
  return DDKS_OK;
}

void ddks_graph_mark(ddks_ctx* ctx, uint64_t key) {
  if (GraphEntry* g = find(ctx, key)) g->primed = true;
}

void ddks_graph_clear(ddks_ctx* ctx) {
  for (auto& g : ctx->graphs) drop_exec(g);
  ctx->graphs.clear();
  if (ctx->cap_st) cudaStreamDestroy(ctx->cap_st);
  ctx->cap_st = nullptr;
}
