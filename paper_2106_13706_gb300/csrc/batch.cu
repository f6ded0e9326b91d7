// batch.cu -- many independent ddKS problems of different N and d in one
// persistent launch (the batched form of Sec. 2.1's statistic).
//
// K0b (k_batch_rank): one CTA per (problem, dimension) maps the coordinates to
//   order-preserving keys, sorts (key, index) in shared memory and writes each
//   point's min-rank, so x_m >= o_m <=> rank_m(x) >= rank_m(o) (Eq. g).
// K5 (k_batch_count): a persistent kernel.  Work units are (problem, tile of
//   64 origins); CTAs take units from a device counter until none are left, so
//   problems of very different sizes share the GPU without a launch each.  A
//   unit with d <= 6 keeps lane-private shared histograms (4 threads per
//   origin), one with 7 <= d <= 11 one shared histogram per warp and origin.
//   Each origin's max |cP*NT - cT*NP| (Eq. d1) and lowest orthant go to the
//   problem's slice of best/bestj.
// K_r (k_batch_reduce): one CTA per problem: max over origins, lowest origin.
#include <algorithm>
#include <cstring>
#include <vector>

#include "ddks_host.h"
#include "ddks_internal.cuh"

struct BatchDesc {
  const void* P;
  const void* T;
  int64_t NP, NT;
  int64_t off_pool;  // offset of the problem in best/bestj (pooled points)
  int64_t off_rank;  // offset of the problem's [d][N] ranks
  int64_t unit0;     // first work unit of the problem
  int32_t d, is_f64;
};

namespace {

constexpr int kMaxBatchN = 16384;   // so NP, NT < 65536: P and T counts share one 32-bit bin
constexpr int kMaxGroups = 16;      // dimensions 1..11 of the batched problems
constexpr int kThreads = 256;
// tile shapes of the batched units, per dimension group (ddks_autotune_batch):
// origins per work unit (32, 64 or 128) and points per staged tile
constexpr int kOT = 64;        // default origins per work unit
constexpr int kTile = 512;     // default points per staged tile

DDKS_DEV bool pair_less(uint64_t ka, uint32_t ia, uint64_t kb, uint32_t ib) {
  return ka < kb || (ka == kb && ia < ib);
}

__global__ void __launch_bounds__(1024)
k_batch_rank(const BatchDesc* __restrict__ desc, const int* __restrict__ cta_prob,
             const int* __restrict__ cta_dim, uint32_t* __restrict__ rank, unsigned* __restrict__ flags) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const BatchDesc D = desc[cta_prob[blockIdx.x]];
  const int m = cta_dim[blockIdx.x];
  const int64_t N = D.NP + D.NT;
  int P2 = 1;
  while (P2 < N) P2 <<= 1;
  uint64_t* sk = reinterpret_cast<uint64_t*>(smraw);
  uint32_t* si = reinterpret_cast<uint32_t*>(sk + P2);
  for (int i = threadIdx.x; i < P2; i += blockDim.x) {
    uint64_t key = ~0ull;
    if (i < N) {
      if (D.is_f64) {
        const double v = i < D.NP ? ((const double*)D.P)[(int64_t)i * D.d + m]
                                  : ((const double*)D.T)[(int64_t)(i - D.NP) * D.d + m];
        if (v != v) atomicOr(flags, ddks::kFlagNaN);
        key = ddks::order_key(v);
      } else {
        const float v = i < D.NP ? ((const float*)D.P)[(int64_t)i * D.d + m]
                                 : ((const float*)D.T)[(int64_t)(i - D.NP) * D.d + m];
        if (v != v) atomicOr(flags, ddks::kFlagNaN);
        key = ddks::order_key(v);
      }
    }
    sk[i] = key;
    si[i] = (uint32_t)i;
  }
  __syncthreads();
  for (int size = 2; size <= P2; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int t = threadIdx.x; t < P2 / 2; t += blockDim.x) {
        const int lo = 2 * t - (t & (stride - 1));
        const int hi = lo + stride;
        const bool asc = ((lo & size) == 0);
        const uint64_t ka = sk[lo], kb = sk[hi];
        const uint32_t ia = si[lo], ib = si[hi];
        const bool swap = asc ? pair_less(kb, ib, ka, ia) : pair_less(ka, ia, kb, ib);
        if (swap) { sk[lo] = kb; sk[hi] = ka; si[lo] = ib; si[hi] = ia; }
      }
      __syncthreads();
    }
  }
  uint32_t* R = rank + D.off_rank + (int64_t)m * N;
  for (int p = threadIdx.x; p < N; p += blockDim.x) {
    const uint64_t key = sk[p];
    int lo = 0, hi = p;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (sk[mid] < key) lo = mid + 1; else hi = mid;
    }
    R[si[p]] = (uint32_t)lo;
  }
}

// The two compare bits of a packed pair difference r (bit 15: low half,
// bit 31: high half) as code bits 2q and 2q + 1: two shifts and one 3-input op.
DDKS_DEV uint32_t pair_bits(uint32_t r, int q) {
  return ((r >> (15 - 2 * q)) & (1u << (2 * q))) | ((r >> (30 - 2 * q)) & (2u << (2 * q)));
}

// lane-private histograms: OT origins x (kThreads / OT) slices of the points
template <int DD>
DDKS_DEV void unit_lane(const BatchDesc& D, const uint32_t* __restrict__ rk, int64_t o0,
                        uint32_t* sm, uint64_t* best, int32_t* bestj, int OT, int PT) {
  constexpr int NB = 1 << DD;
  const int S = kThreads / OT;
  const int64_t N = D.NP + D.NT;
  const int tid = threadIdx.x, ol = tid / S, s = tid - ol * S;
  constexpr int NPR = (DD + 1) / 2;              // dimension pairs
  uint32_t* hist = sm;                          // [NB][kThreads]: P count | T count << 16
  uint32_t* tile = sm + NB * kThreads;          // [NPR][PT] packed 16-bit rank pairs | 0x80008000
  const int64_t k = o0 + ol;
  const bool active = k < N;
  // the origin's ranks as packed pairs (see unit_warp: one subtract, two compares)
  uint32_t op[NPR];
#pragma unroll
  for (int q = 0; q < NPR; ++q) {
    const uint32_t lo = active ? rk[(int64_t)(2 * q) * N + k] : 0u;
    const uint32_t hi = (active && 2 * q + 1 < DD) ? rk[(int64_t)(2 * q + 1) * N + k] : 0u;
    op[q] = lo | (hi << 16);
  }
  for (int j = 0; j < NB; ++j) hist[j * kThreads + tid] = 0;
  for (int64_t base = 0; base < N; base += PT) {
    const int cnt = (int)((N - base) < PT ? (N - base) : PT);
    __syncthreads();
    for (int e = tid; e < NPR * cnt; e += kThreads) {
      const int q = e / cnt, j = e - q * cnt;
      const uint32_t lo = rk[(int64_t)(2 * q) * N + base + j];
      const uint32_t hi = 2 * q + 1 < DD ? rk[(int64_t)(2 * q + 1) * N + base + j] : 0u;
      tile[q * PT + j] = (lo | (hi << 16)) | 0x80008000u;
    }
    __syncthreads();
    int pend = (int)(D.NP - base);
    pend = pend < 0 ? 0 : (pend > cnt ? cnt : pend);
    for (int j = s; j < cnt; j += S) {
      uint32_t c = 0;
#pragma unroll
      for (int q = 0; q < NPR; ++q) c |= pair_bits(tile[q * PT + j] - op[q], q);
      c &= (uint32_t)NB - 1u;  // an odd DD's padding half is dropped
      atomicAdd(&hist[c * kThreads + tid], j < pend ? 1u : (1u << 16));
    }
  }
  __syncthreads();
  uint64_t bv = 0;
  int bj = 0;
  if (active) {
    for (int j = s; j < NB; j += S) {
      uint64_t a = 0, b = 0;
      for (int q = 0; q < S; ++q) {
        const int col = ol * S + q;
        const uint32_t v = hist[j * kThreads + col];
        a += v & 0xFFFFu;
        b += v >> 16;
      }
      const uint64_t num = ddks::numer(a, b, (uint64_t)D.NP, (uint64_t)D.NT);
      if (num > bv) { bv = num; bj = j; }
    }
  }
  for (int off = 1; off < S; off <<= 1) {
    const uint64_t v2 = __shfl_xor_sync(0xffffffffu, bv, off);
    const int j2 = __shfl_xor_sync(0xffffffffu, bj, off);
    if (v2 > bv || (v2 == bv && j2 < bj)) { bv = v2; bj = j2; }
  }
  if (active && s == 0) {
    best[D.off_pool + k] = bv;
    bestj[D.off_pool + k] = bv ? bj : 0;
  }
  __syncthreads();
}

// 7 <= d <= 11: the CTA's 8 warps take one origin each (8 rounds of 8 per
// unit of 64), with one shared histogram per warp (P count | T count << 16).
// Point tiles are staged in shared memory once for the 8 warps, ranks packed
// as 16-bit pairs (N <= 16384): (x | 0x8000) - o keeps each half apart and its
// bit 15 is [x >= o], so one subtract compares two dimensions.
template <int DD>
DDKS_DEV void unit_warp(const BatchDesc& D, const uint32_t* __restrict__ rk, int64_t o0,
                        uint32_t* sm, uint64_t* best, int32_t* bestj, int OT, int PT) {
  constexpr int d = DD, nb = 1 << DD, npair = (DD + 1) >> 1;
  const int64_t N = D.NP + D.NT;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int kW = kThreads / 32;
  // two copies of the warp's histogram (even and odd lanes) halve the
  // same-address collisions of its increments
  uint32_t* hist = sm + (size_t)warp * 2 * nb;          // [kW][2][nb]
  uint32_t* tile = sm + (size_t)kW * 2 * nb;            // [npair][PT] packed pairs
  for (int round = 0; round < OT / kW; ++round) {
    const int64_t k = o0 + round * kW + warp;
    const bool active = k < N;
    // the origin's ranks as packed pairs; an odd last dimension is paired
    // with a high half that every point passes
    uint32_t op[npair];
#pragma unroll
    for (int q = 0; q < npair; ++q) {
      uint32_t lo = 0, hi = 0;
      if (active) {
        lo = rk[(int64_t)(2 * q) * N + k];
        hi = 2 * q + 1 < d ? rk[(int64_t)(2 * q + 1) * N + k] : 0u;
      }
      op[q] = lo | (hi << 16);
    }
    for (int j = lane; j < 2 * nb; j += 32) hist[j] = 0;
    for (int64_t base = 0; base < N; base += PT) {
      const int cnt = (int)((N - base) < PT ? (N - base) : PT);
      __syncthreads();  // the previous tile is consumed (and the histograms are zeroed)
      for (int e = threadIdx.x; e < npair * cnt; e += kThreads) {
        const int q = e / cnt, j = e - q * cnt;
        const uint32_t lo = rk[(int64_t)(2 * q) * N + base + j];
        const uint32_t hi = 2 * q + 1 < d ? rk[(int64_t)(2 * q + 1) * N + base + j] : 0u;
        tile[q * PT + j] = (lo | (hi << 16)) | 0x80008000u;
      }
      __syncthreads();
      if (active) {
        const int pend = (int)(D.NP - base < 0 ? 0 : (D.NP - base > cnt ? cnt : D.NP - base));
        for (int j = lane; j < cnt; j += 32) {
          uint32_t c = 0;
#pragma unroll
          for (int q = 0; q < npair; ++q) c |= pair_bits(tile[q * PT + j] - op[q], q);
          c &= (uint32_t)nb - 1u;  // an odd d's padding half is always >= and is dropped here
          // (warp-aggregated increments by match.any measured slower: 13.1 vs 9.3 ms per batch)
          atomicAdd(&hist[(lane & 1) * nb + c], j < pend ? 1u : (1u << 16));
        }
      }
    }
    __syncwarp();
    if (active) {
      uint64_t bv = 0;
      int bj = 0;
      for (int j = lane; j < nb; j += 32) {
        const uint32_t v0 = hist[j], v1 = hist[nb + j];
        const uint64_t num =
            ddks::numer((v0 & 0xFFFFu) + (v1 & 0xFFFFu), (v0 >> 16) + (v1 >> 16), (uint64_t)D.NP, (uint64_t)D.NT);
        if (num > bv) { bv = num; bj = j; }
      }
      for (int off = 16; off > 0; off >>= 1) {
        const uint64_t v2 = __shfl_down_sync(0xffffffffu, bv, off);
        const int j2 = __shfl_down_sync(0xffffffffu, bj, off);
        if (v2 > bv || (v2 == bv && j2 < bj)) { bv = v2; bj = j2; }
      }
      if (lane == 0) {
        best[D.off_pool + k] = bv;
        bestj[D.off_pool + k] = bv ? bj : 0;
      }
    }
    __syncwarp();
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kThreads)
k_batch_count(const BatchDesc* __restrict__ desc, int count, int64_t total_units,
              const uint32_t* __restrict__ rank, unsigned long long* __restrict__ next_unit,
              uint64_t* __restrict__ best, int32_t* __restrict__ bestj, int OT, int PT) {
  extern __shared__ __align__(16) uint32_t sm[];
  __shared__ long long unit;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) unit = (long long)atomicAdd(next_unit, 1ull);
    __syncthreads();
    const long long u = unit;
    if (u >= total_units) break;
    // problem of this unit: last problem whose unit0 <= u
    int lo = 0, hi = count - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (desc[mid].unit0 <= u) lo = mid; else hi = mid - 1;
    }
    const BatchDesc D = desc[lo];
    const int64_t o0 = (u - D.unit0) * OT;
    const uint32_t* rk = rank + D.off_rank;
    switch (D.d) {
      case 1: unit_lane<1>(D, rk, o0, sm, best, bestj, OT, PT); break;
      case 2: unit_lane<2>(D, rk, o0, sm, best, bestj, OT, PT); break;
      case 3: unit_lane<3>(D, rk, o0, sm, best, bestj, OT, PT); break;
      case 4: unit_lane<4>(D, rk, o0, sm, best, bestj, OT, PT); break;
      case 5: unit_lane<5>(D, rk, o0, sm, best, bestj, OT, PT); break;
      case 6: unit_lane<6>(D, rk, o0, sm, best, bestj, OT, PT); break;
      case 7: unit_warp<7>(D, rk, o0, sm, best, bestj, OT, PT); break;
      case 8: unit_warp<8>(D, rk, o0, sm, best, bestj, OT, PT); break;
      case 9: unit_warp<9>(D, rk, o0, sm, best, bestj, OT, PT); break;
      case 10: unit_warp<10>(D, rk, o0, sm, best, bestj, OT, PT); break;
      default: unit_warp<11>(D, rk, o0, sm, best, bestj, OT, PT); break;
    }
  }
}

__global__ void __launch_bounds__(1024)
k_batch_reduce(const BatchDesc* __restrict__ desc, const uint64_t* __restrict__ best,
               const int32_t* __restrict__ bestj, unsigned long long* __restrict__ out) {
  __shared__ unsigned long long sv[32];
  __shared__ long long si[32];
  const BatchDesc D = desc[blockIdx.x];
  const int64_t no = D.NP + D.NT;
  const uint64_t* b = best + D.off_pool;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned long long v = 0;
  for (int64_t i = threadIdx.x; i < no; i += blockDim.x) v = b[i] > v ? b[i] : v;
  for (int off = 16; off > 0; off >>= 1) {
    const unsigned long long v2 = __shfl_down_sync(0xffffffffu, v, off);
    v = v2 > v ? v2 : v;
  }
  if (lane == 0) sv[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long m = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = sv[w] > m ? sv[w] : m;
    sv[0] = m;
  }
  __syncthreads();
  const unsigned long long vmax = sv[0];
  long long idx = no;
  for (int64_t i = threadIdx.x; i < no; i += blockDim.x)
    if (b[i] == vmax) { idx = i; break; }
  for (int off = 16; off > 0; off >>= 1) {
    const long long i2 = __shfl_down_sync(0xffffffffu, idx, off);
    idx = i2 < idx ? i2 : idx;
  }
  __syncthreads();
  if (lane == 0) si[warp] = idx;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long m = no;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = si[w] < m ? si[w] : m;
    out[3 * blockIdx.x + 0] = vmax;
    out[3 * blockIdx.x + 1] = (unsigned long long)m;
    out[3 * blockIdx.x + 2] = (unsigned long long)(long long)bestj[D.off_pool + m];
  }
}

size_t unit_smem(int d, int PT) {
  if (d <= 6) return (size_t)(1u << d) * kThreads * 4 + (size_t)((d + 1) / 2) * PT * 4;
  return (size_t)(kThreads / 32) * 2 * (1u << d) * 4 + (size_t)((d + 1) / 2) * PT * 4;
}

}  // namespace

// Batched distances for problems that fit the batch kernels (N <= 16384, d <= 11);
// the others go through the single-problem path.  Synchronous.
int ddks_batch_distance(ddks_ctx* ctx, int32_t count, const void* const* P, const int64_t* NP,
                        const void* const* T, const int64_t* NT, const int32_t* d, int32_t dtype,
                        void* stream, ddks_result* out) {
  if (!ctx || count < 0 || (count > 0 && (!P || !NP || !T || !NT || !d || !out))) return DDKS_EINVAL;
  if (count == 0) return DDKS_OK;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return ctx_cuda_fail(ctx, e, "cudaSetDevice");
  const size_t es = dtype == DDKS_F64 ? 8 : 4;
  std::vector<int> batched, single;
  for (int i = 0; i < count; ++i) {
    const int rc = ddks_check_problem(P[i], NP[i], T[i], NT[i], d[i], dtype);
    if (rc) { out[i].status = rc; return rc; }
    if (NP[i] + NT[i] <= kMaxBatchN && d[i] <= 11) batched.push_back(i); else single.push_back(i);
  }
  int rc = DDKS_OK;
  if (!batched.empty()) {
    // problems of one dimension form a group with its own persistent launch,
    // its shared memory sized for that dimension
    std::stable_sort(batched.begin(), batched.end(), [&](int a, int b) { return d[a] < d[b]; });
    const int nb = (int)batched.size();
    // stage host inputs into one device buffer
    size_t host_bytes = 0;
    std::vector<char> is_dev(2 * nb);
    for (int b = 0; b < nb; ++b) {
      const int i = batched[b];
      const int kP = ddks_pointer_kind(P[i], ctx->device), kT = ddks_pointer_kind(T[i], ctx->device);
      if (kP < 0 || kT < 0) { out[i].status = DDKS_EINVAL; return DDKS_EINVAL; }  // another GPU's memory
      is_dev[2 * b] = kP == 1;
      is_dev[2 * b + 1] = kT == 1;
      if (!is_dev[2 * b]) host_bytes += (es * NP[i] * d[i] + 15) & ~(size_t)15;
      if (!is_dev[2 * b + 1]) host_bytes += (es * NT[i] * d[i] + 15) & ~(size_t)15;
    }
    if (host_bytes && (rc = ctx->inP.reserve(ctx, host_bytes))) return rc;
    std::vector<BatchDesc> hd(nb);
    std::vector<int> cta_prob, cta_dim;
    size_t hoff = 0;
    int64_t off_pool = 0, off_rank = 0, units = 0;
    size_t smem_rank = 0, smem_unit = 0;
    struct Group { int d, first, count; int64_t units; double work; };
    std::vector<Group> groups;
    for (int b = 0; b < nb; ++b) {
      const int i = batched[b];
      BatchDesc& D = hd[b];
      D.P = P[i];
      D.T = T[i];
      if (!is_dev[2 * b]) {
        void* dst = (char*)ctx->inP.ptr + hoff;
        e = cudaMemcpyAsync(dst, P[i], es * NP[i] * d[i], cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return ctx_cuda_fail(ctx, e, "batch copy");
        D.P = dst;
        hoff += (es * NP[i] * d[i] + 15) & ~(size_t)15;
      }
      if (!is_dev[2 * b + 1]) {
        void* dst = (char*)ctx->inP.ptr + hoff;
        e = cudaMemcpyAsync(dst, T[i], es * NT[i] * d[i], cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return ctx_cuda_fail(ctx, e, "batch copy");
        D.T = dst;
        hoff += (es * NT[i] * d[i] + 15) & ~(size_t)15;
      }
      D.NP = NP[i];
      D.NT = NT[i];
      D.d = d[i];
      D.is_f64 = dtype == DDKS_F64;
      const int64_t N = NP[i] + NT[i];
      D.off_pool = off_pool;
      D.off_rank = off_rank;
      if (groups.empty() || groups.back().d != d[i]) {
        groups.push_back(Group{d[i], b, 0, 0, 0.0});
        units = 0;  // units are numbered within a group
      }
      D.unit0 = units;
      off_pool += N;
      off_rank += N * d[i];
      const int OT = ctx->batch_ot[d[i]];
      units += (N + OT - 1) / OT;
      groups.back().count += 1;
      groups.back().units = units;
      groups.back().work += (double)N * (double)N * d[i];
      for (int m = 0; m < d[i]; ++m) { cta_prob.push_back(b); cta_dim.push_back(m); }
      int P2 = 1;
      while (P2 < N) P2 <<= 1;
      smem_rank = std::max(smem_rank, (size_t)P2 * 12);
      smem_unit = std::max(smem_unit, unit_smem(d[i], ctx->batch_pt[d[i]]));
    }
    const size_t desc_bytes = sizeof(BatchDesc) * nb + 8 * cta_prob.size() + 64;
    if ((rc = ctx->batch_desc.reserve(ctx, desc_bytes))) return rc;
    if ((rc = ctx->rank.reserve(ctx, 4 * (size_t)off_rank))) return rc;
    if ((rc = ctx->best.reserve(ctx, 8 * (size_t)off_pool))) return rc;
    if ((rc = ctx->bestj.reserve(ctx, 4 * (size_t)off_pool))) return rc;
    if ((rc = ctx->batch_work.reserve(ctx, 8 * (3 * (size_t)nb + 4 + kMaxGroups)))) return rc;
    if ((rc = ctx->flags.reserve(ctx, 64))) return rc;
    char* dd = (char*)ctx->batch_desc.ptr;
    BatchDesc* ddesc = (BatchDesc*)dd;
    int* dprob = (int*)(dd + sizeof(BatchDesc) * nb);
    int* ddim = dprob + cta_prob.size();
    // the descriptor upload goes through pinned staging owned by the context
    const size_t up = sizeof(BatchDesc) * nb + 8 * cta_prob.size();
    if (ctx->h_stage_bytes < up) {
      if (ctx->h_stage) cudaFreeHost(ctx->h_stage);
      ctx->h_stage = nullptr;
      ctx->h_stage_bytes = 0;
      e = cudaMallocHost(&ctx->h_stage, up * 2);
      if (e != cudaSuccess) return ctx_cuda_fail(ctx, e, "cudaMallocHost");
      ctx->h_stage_bytes = up * 2;
    }
    e = cudaStreamSynchronize(st);  // the staging buffer may still feed an earlier copy
    if (e != cudaSuccess) return ctx_cuda_fail(ctx, e, "batch sync");
    char* hs = (char*)ctx->h_stage;
    std::memcpy(hs, hd.data(), sizeof(BatchDesc) * nb);
    std::memcpy(hs + sizeof(BatchDesc) * nb, cta_prob.data(), 4 * cta_prob.size());
    std::memcpy(hs + sizeof(BatchDesc) * nb + 4 * cta_prob.size(), cta_dim.data(), 4 * cta_dim.size());
    e = cudaMemcpyAsync(dd, hs, up, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return ctx_cuda_fail(ctx, e, "batch descriptors");
    unsigned long long* work = (unsigned long long*)ctx->batch_work.ptr;  // [kMaxGroups] unit counters
    unsigned long long* res = work + kMaxGroups;
    // the groups with the most work start first
    std::vector<int> gorder(groups.size());
    for (size_t g = 0; g < groups.size(); ++g) gorder[g] = (int)g;
    std::stable_sort(gorder.begin(), gorder.end(),
                     [&](int a, int b) { return groups[a].work > groups[b].work; });
    // the descriptors hold every shape and input address the kernels see
    GraphKey key;
    key.add(3).add((uint64_t)nb).add((uint64_t)units).add((uint64_t)smem_rank).add((uint64_t)smem_unit);
    key.add_bytes(hs, up).add_bytes(ctx->batch_ot, sizeof ctx->batch_ot).add_bytes(ctx->batch_pt, sizeof ctx->batch_pt);
    if (ctx->batch_timing) key.add(0xB7);  // tuning runs directly (events between the launches)
    rc = ddks_graph_run(ctx, key.h, st, [&](cudaStream_t s) -> int {
      cudaError_t ee = cudaMemsetAsync(work, 0, 8 * kMaxGroups, s);
      if (ee == cudaSuccess) ee = cudaMemsetAsync(ctx->flags.ptr, 0, 4, s);
      if (ee == cudaSuccess)
        ee = cudaFuncSetAttribute(k_batch_rank, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_rank);
      if (ee == cudaSuccess) {
        k_batch_rank<<<(unsigned)cta_prob.size(), 1024, smem_rank, s>>>(
            ddesc, dprob, ddim, (uint32_t*)ctx->rank.ptr, (unsigned*)ctx->flags.ptr);
        ee = cudaGetLastError();
      }
      if (ee == cudaSuccess)
        ee = cudaFuncSetAttribute(k_batch_count, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_unit);
      for (size_t gi = 0; gi < gorder.size() && ee == cudaSuccess; ++gi) {
        const Group& G = groups[gorder[gi]];
        const int OT = ctx->batch_ot[G.d], PT = ctx->batch_pt[G.d];
        const size_t sm_g = unit_smem(G.d, PT);
        cudaEvent_t ev0 = nullptr, ev1 = nullptr;
        if (ctx->batch_timing) {
          cudaEventCreate(&ev0);
          cudaEventCreate(&ev1);
          cudaEventRecord(ev0, s);
        }
        int blocks_per_sm = 1;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, k_batch_count, kThreads, sm_g);
        if (blocks_per_sm < 1) blocks_per_sm = 1;
        int64_t grid = (int64_t)ctx->num_sms * blocks_per_sm;
        if (grid > G.units) grid = G.units;
        k_batch_count<<<(unsigned)grid, kThreads, sm_g, s>>>(
            ddesc + G.first, G.count, G.units, (const uint32_t*)ctx->rank.ptr, work + gorder[gi],
            (uint64_t*)ctx->best.ptr, (int32_t*)ctx->bestj.ptr, OT, PT);
        ee = cudaGetLastError();
        ctx->launches += 1;
        if (ctx->batch_timing) {
          cudaEventRecord(ev1, s);
          cudaEventSynchronize(ev1);
          float ms = 0;
          cudaEventElapsedTime(&ms, ev0, ev1);
          ctx->batch_group_ms[G.d] = ms;
          cudaEventDestroy(ev0);
          cudaEventDestroy(ev1);
        }
      }
      if (ee == cudaSuccess) {
        k_batch_reduce<<<nb, 1024, 0, s>>>(ddesc, (const uint64_t*)ctx->best.ptr,
                                           (const int32_t*)ctx->bestj.ptr, res);
        ee = cudaGetLastError();
      }
      ctx->launches += 2;
      if (ee != cudaSuccess) return ctx_cuda_fail(ctx, ee, "batch");
      return DDKS_OK;
    });
    if (rc) return rc;
    std::vector<unsigned long long> hres(3 * (size_t)nb);
    unsigned hflags = 0;
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(hres.data(), res, 8 * 3 * (size_t)nb, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hflags, ctx->flags.ptr, 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return ctx_cuda_fail(ctx, e, "batch");
    if (hflags & ddks::kFlagNaN) {
      for (int b = 0; b < nb; ++b) out[batched[b]].status = DDKS_ENAN;
      return DDKS_ENAN;
    }
    for (int b = 0; b < nb; ++b) {
      ddks_result& r = out[batched[b]];
      r.num_max = hres[3 * b];
      r.denom = (uint64_t)hd[b].NP * (uint64_t)hd[b].NT;
      r.D = (double)r.num_max / (double)r.denom;
      r.argmax_origin = (int64_t)hres[3 * b + 1];
      r.argmax_orthant = (int32_t)hres[3 * b + 2];
      r.status = DDKS_OK;
    }
  }
  for (int i : single) {
    rc = ddks_distance(ctx, P[i], NP[i], T[i], NT[i], d[i], dtype, stream, &out[i]);
    if (rc) return rc;
  }
  return DDKS_OK;
}

int ddks_set_batch_shape(ddks_ctx* ctx, int32_t d, int32_t origins_per_unit, int32_t points_per_tile) {
  if (!ctx || d < 1 || d > 11) return DDKS_EINVAL;
  if (origins_per_unit != 32 && origins_per_unit != 64 && origins_per_unit != 128) return DDKS_EINVAL;
  if (points_per_tile != 256 && points_per_tile != 512 && points_per_tile != 1024) return DDKS_EINVAL;
  ctx->batch_ot[d] = origins_per_unit;
  ctx->batch_pt[d] = points_per_tile;
  return DDKS_OK;
}

// Times every tile shape on this batch, per dimension group, keeps the fastest
// for each dimension present and checks that every shape gives the same
// results.  shapes (optional): [12][2] (origins per unit, points per tile).
int ddks_autotune_batch(ddks_ctx* ctx, int32_t count, const void* const* P, const int64_t* NP,
                        const void* const* T, const int64_t* NT, const int32_t* d, int32_t dtype, void* stream,
                        int32_t* shapes) {
  if (!ctx || count < 1 || !d) return DDKS_EINVAL;
  int ot0[12], pt0[12];
  std::memcpy(ot0, ctx->batch_ot, sizeof ot0);
  std::memcpy(pt0, ctx->batch_pt, sizeof pt0);
  float best_ms[12];
  int best_ot[12], best_pt[12];
  for (int k = 0; k < 12; ++k) { best_ms[k] = 3.0e38f; best_ot[k] = ot0[k]; best_pt[k] = pt0[k]; }
  std::vector<ddks_result> ref((size_t)count), got((size_t)count);
  bool have_ref = false;
  int rc = DDKS_OK;
  ctx->batch_timing = true;
  for (int ot : {32, 64, 128}) {
    for (int pt : {256, 512, 1024}) {
      for (int k = 1; k < 12; ++k) { ctx->batch_ot[k] = ot; ctx->batch_pt[k] = pt; }
      for (int rep = 0; rep < 2 && rc == DDKS_OK; ++rep)  // the second run is timed warm
        rc = ddks_batch_distance(ctx, count, P, NP, T, NT, d, dtype, stream, got.data());
      if (rc) break;
      if (!have_ref) {
        ref = got;
        have_ref = true;
      } else {
        for (int i = 0; i < count; ++i)
          if (got[i].num_max != ref[i].num_max || got[i].argmax_origin != ref[i].argmax_origin ||
              got[i].argmax_orthant != ref[i].argmax_orthant) {
            ctx->last_err = "batch autotune: tile shapes disagree";
            rc = DDKS_ECUDA;
          }
      }
      if (rc) break;
      for (int k = 1; k < 12; ++k) {
        const float ms = ctx->batch_group_ms[k];
        if (ms > 0.0f && ms < best_ms[k]) { best_ms[k] = ms; best_ot[k] = ot; best_pt[k] = pt; }
        ctx->batch_group_ms[k] = 0.0f;
      }
    }
    if (rc) break;
  }
  ctx->batch_timing = false;
  if (rc) {
    std::memcpy(ctx->batch_ot, ot0, sizeof ot0);
    std::memcpy(ctx->batch_pt, pt0, sizeof pt0);
    return rc;
  }
  std::memcpy(ctx->batch_ot, best_ot, sizeof best_ot);
  std::memcpy(ctx->batch_pt, best_pt, sizeof best_pt);
  if (shapes)
    for (int k = 0; k < 12; ++k) { shapes[2 * k] = ctx->batch_ot[k]; shapes[2 * k + 1] = ctx->batch_pt[k]; }
  return DDKS_OK;
}
