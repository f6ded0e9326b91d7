// batch_internal.cuh -- descriptors shared by the batched launch's kernels
// (batch.cu: work units and reduction; batch_rank.cu: K0 of the batch).
#pragma once
#include <cstdint>

#include <cuda_runtime.h>

// One problem of a batch, as the kernels see it.
struct BatchDesc {
  const void* P;
  const void* T;
  int64_t NP, NT;
  int64_t off_pool;  // offset of the problem in best/bestj and the pooled arrays
  int64_t off_rank;  // offset of the problem's [d][N] ranks
  int64_t unit0;     // first work unit of the problem (within its dimension group)
  int32_t d, is_f64;
};

// Layout of the batch's rank buffer (u32): [ranks: sum of N*d][ranks in list
// order: sum of N*d][sorted order: sum of N][lists: sum of N][P prefix: sum of N].
//   rank[m][i]   min-rank of point i in dimension m (x_m >= o_m <=> rank >= rank)
//   rankL[m][p]  rank in dimension m of the point at list position p
//   ord[p]       point at dimension-0 sorted position p
//   lst[p]       P points in dimension-0 order at [0, NP), T points at [NP, N)
//   pfx[p]       P points at dimension-0 sorted positions < p
struct RankAreas {
  uint32_t* rank;
  uint32_t* rankL;
  uint32_t* ord;
  uint32_t* lst;
  uint32_t* pfx;
};

constexpr int kBatchMaxN = 16384;  // pooled points of a batched problem (16-bit list positions)

// K0 of the batch: one CTA per entry (problem, dimension) of dprob/ddim, the
// entries grouped by size class as the host ordered them.  Returns the first
// launch error.
struct BatchRankClass {
  int first, count;  // entries [first, first + count) of dprob/ddim
  int cap;           // largest N of the class
  bool wide;         // 1024 threads (N > 4096) or 256
};
cudaError_t ddks_batch_rank(const BatchDesc* desc, const int* dprob, const int* ddim, const BatchRankClass* cls,
                            int ncls, bool f64, const RankAreas& ra, unsigned* flags, cudaStream_t st);
