// rank_cluster.cu -- K0 in one launch for pooled samples of up to about 125k
// (float) or 85k (double) points (half that where clusters of 16 CTAs cannot
// be scheduled): order keys, per-dimension min-ranks, every dimension's
// sorted order, the dimension-0 P prefix.
//
// x_m >= o_m <=> rank_m(x) >= rank_m(o) with rank = the number of pooled
// values strictly below (Eq. g only ever compares coordinates with ">="), so
// the count kernels work on ranks.  Here one thread-block cluster of 16 CTAs
// (8 where the GPU does not schedule clusters of 16)
// ranks one dimension: CTA c holds positions [c*S, (c+1)*S) of the row in
// shared memory, and a stable LSD radix sort with 8-bit digits runs entirely
// in the cluster's distributed shared memory -- per pass each CTA ranks its
// elements stably by digit (per-warp digit counters, lanes with equal digits
// found by ballots) and reorders them locally into digit order, the cluster's
// digit counts are read across CTAs to give every (digit, CTA) its first
// output position, and each run of equal digits is copied, consecutive
// threads to consecutive positions, into the shared memory of the CTAs that
// own those positions.  Three buffers rotate (current, staging, destination),
// so one cluster barrier after the counts and one after the copies suffice.
// A pass whose digit is the same for every key is skipped.  After the last pass the
// positions hold the keys in sorted order with ties in pooled-index order;
// the min-rank of a position is its run's first position (a running maximum
// of run heads within the CTA, carried across CTAs), and dimension 0 also
// gets the count of P points (pooled index < NP) before each position.
//
// Replaces the encode kernel, the global radix passes and the rank kernels
// (about a dozen latency-bound launches) by one launch of d clusters.
#include <cooperative_groups.h>

#include <mutex>

#include "ddks_host.h"
#include "ddks_internal.cuh"

namespace cg = cooperative_groups;

namespace {

constexpr int kEMax = 16;        // positions per thread at most (S <= kEMax * kKT)
constexpr int kKT = 512;         // threads per CTA
static_assert(kKT == 512, "the digit-count prefix splits the warps into two halves of 256 threads");
constexpr int kKW = kKT / 32;    // warps per CTA
constexpr size_t kSmemCap = 220u * 1024u;

template <typename V> struct KeyOf;
template <> struct KeyOf<float> { using K = uint32_t; static constexpr int kPasses = 4; };
template <> struct KeyOf<double> { using K = uint64_t; static constexpr int kPasses = 8; };

// shared memory of one CTA for a segment of S positions
template <typename K>
__host__ __device__ constexpr size_t cluster_smem(int64_t S) {
  return (size_t)S * sizeof(K) * 3     // keys: current, staging, destination
         + (size_t)S * 4 * 3           // pooled indices, the same three
         + (size_t)S * 2               // rank of each element among its warp's equal digits
         + (size_t)kKW * 256 * 4       // per-warp digit counters
         + 16;
}

// exclusive prefixes over the CTA's threads (kKT of them) of two values each;
// ws2: 2 * kKW words
DDKS_DEV void cta_exscan2(uint32_t v0, uint32_t v1, uint32_t* ws2, uint32_t& e0, uint32_t& e1) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t a = v0, b = v1;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const uint32_t x = __shfl_up_sync(0xffffffffu, a, off);
    const uint32_t y = __shfl_up_sync(0xffffffffu, b, off);
    if (lane >= off) { a += x; b += y; }
  }
  if (lane == 31) { ws2[warp] = a; ws2[kKW + warp] = b; }
  __syncthreads();
  if (warp == 0) {
    const uint32_t t0 = lane < kKW ? ws2[lane] : 0u, t1 = lane < kKW ? ws2[kKW + lane] : 0u;
    uint32_t p0 = t0, p1 = t1;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const uint32_t x = __shfl_up_sync(0xffffffffu, p0, off);
      const uint32_t y = __shfl_up_sync(0xffffffffu, p1, off);
      if (lane >= off) { p0 += x; p1 += y; }
    }
    if (lane < kKW) { ws2[lane] = p0 - t0; ws2[kKW + lane] = p1 - t1; }
  }
  __syncthreads();
  e0 = ws2[warp] + a - v0;
  e1 = ws2[kKW + warp] + b - v1;
  __syncthreads();
}

// Grid: d clusters of kC CTAs; cluster m ranks dimension m, CTA c of it holds
// positions [c*S, c*S + S).  Outputs: rank[m*N + i] = min-rank of point i;
// sorted[m*N + p] = pooled index at sorted position p; dimension 0 also
// sidx0[p] = sorted[p] and pfx0[p] = P points before position p.
template <typename V, int CL>
__global__ void __launch_bounds__(kKT, 1)
k_rank_cluster(const V* __restrict__ P, const V* __restrict__ T, int64_t NP, int64_t NT, int d, int S,
               uint32_t Smag, uint32_t* __restrict__ rank, uint32_t* __restrict__ sorted, uint32_t* __restrict__ sidx0,
               uint32_t* __restrict__ pfx0, unsigned* __restrict__ flags) {
  using K = typename KeyOf<V>::K;
  constexpr int kPasses = KeyOf<V>::kPasses;
  cg::cluster_group cl = cg::this_cluster();
  const int c = (int)cl.block_rank();
  const int m = (int)(blockIdx.x / CL);
  const int64_t N = NP + NT;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  extern __shared__ __align__(16) unsigned char kraw[];
  // three key / index buffers: current (A), local staging (B), destination (C)
  K* keyA = reinterpret_cast<K*>(kraw);
  K* keyB = keyA + S;
  K* keyC = keyB + S;
  uint32_t* idxA = reinterpret_cast<uint32_t*>(keyC + S);
  uint32_t* idxB = idxA + S;
  uint32_t* idxC = idxB + S;
  uint16_t* rloc = reinterpret_cast<uint16_t*>(idxC + S);
  uint32_t* wcnt = reinterpret_cast<uint32_t*>(rloc + S + (S & 1));  // [kKW][256]
  __shared__ uint32_t hist[256], doff[256], lstart[256], half_tot[256], ws[2 * kKW], whead[kKW], wpc[kKW];
  __shared__ uint32_t s_info[2];  // read by the other CTAs: last run head in the segment, its P points
  __shared__ unsigned long long s_left;
  __shared__ int s_skip;
  const int64_t seg0 = (int64_t)c * S;
  const int cnt = N - seg0 >= S ? S : (N > seg0 ? (int)(N - seg0) : 0);  // positions held
  const int E = (S + kKT - 1) / kKT;  // warp w holds positions [w*32*E, (w+1)*32*E)

  // order keys in pooled order (position = pooled index)
  unsigned nan = 0;
  for (int q = tid; q < cnt; q += kKT) {
    const int64_t i = seg0 + q;
    const V v = i < NP ? P[i * d + m] : T[(i - NP) * d + m];
    nan |= v != v ? 1u : 0u;
    keyA[q] = (K)ddks::order_key(v);
    idxA[q] = (uint32_t)i;
  }
  if (__syncthreads_or(nan) && tid == 0) atomicOr(flags, ddks::kFlagNaN);

  for (int pass = 0; pass < kPasses; ++pass) {
    const int shift = 8 * pass;
    // each warp ranks its positions stably by digit: rloc = rank among the
    // warp's earlier elements of the same digit, wcnt = the warp's counts
    for (int i = tid; i < kKW * 256; i += kKT) wcnt[i] = 0u;
    __syncthreads();
    // Digits and groups of equal digits first (independent iterations), then
    // each group takes its offset with one shared atomic add by its lowest
    // lane: the returned value is the warp's count so far, and the shuffle
    // that hands it to the group waits for it, so a warp's atomics on one
    // address happen in program order (stable ranks).
    uint32_t dgs[kEMax], prs[kEMax];
#pragma unroll
    for (int j = 0; j < kEMax; ++j) {
      dgs[j] = 0u;
      prs[j] = 0u;
      if (j < E) {
        const int q = w * 32 * E + j * 32 + lane;
        const bool v = q < cnt;
        const uint32_t vm = __ballot_sync(0xffffffffu, v);
        if (vm != 0u) {  // warp-uniform
          dgs[j] = v ? (uint32_t)(keyA[q] >> shift) & 255u : 0u;
          const uint32_t pr = ddks::same_digit(dgs[j]) & vm;
          prs[j] = v ? pr : 0u;  // nonzero exactly on the lanes that hold an element
        }
      }
    }
#pragma unroll
    for (int j = 0; j < kEMax; ++j) {
      if (j < E && __any_sync(0xffffffffu, prs[j] != 0u)) {  // warp-uniform
        const int q = w * 32 * E + j * 32 + lane;
        const int leader = __ffs(prs[j]) - 1;  // -1 exactly on lanes past the end
        uint32_t base = 0;
        if (lane == leader) base = atomicAdd(&wcnt[w * 256 + dgs[j]], (uint32_t)__popc(prs[j]));
        base = __shfl_sync(0xffffffffu, base, leader < 0 ? lane : leader);
        if (leader >= 0 && q < cnt) rloc[q] = (uint16_t)(base + (uint32_t)__popc(prs[j] & ((1u << lane) - 1u)));
      }
    }
    __syncthreads();
    {
      // thread (h, t): digit t over warps [h * kKW / 2, (h + 1) * kKW / 2):
      // the warps' offsets within the digit, and the CTA's count of it
      const int t = tid & 255, h = tid >> 8;
      uint32_t s = 0;
#pragma unroll
      for (int q = h * (kKW / 2); q < (h + 1) * (kKW / 2); ++q) {
        const uint32_t x = wcnt[q * 256 + t];
        wcnt[q * 256 + t] = s;
        s += x;
      }
      if (h == 0) half_tot[t] = s;
      __syncthreads();
      if (h == 1) {
        const uint32_t lo = half_tot[t];
#pragma unroll
        for (int q = kKW / 2; q < kKW; ++q) wcnt[q * 256 + t] += lo;
        hist[t] = lo + s;
      }
    }
    if (tid == 0) s_skip = 0;
    cl.sync();  // every CTA's counts are complete
    uint32_t tot = 0, before = 0, mine = 0;
    if (tid < 256) {
#pragma unroll
      for (int r = 0; r < CL; ++r) {
        const uint32_t h = cl.map_shared_rank(hist, (unsigned)r)[tid];
        tot += h;
        before += r < c ? h : 0u;
        mine = r == c ? h : mine;
      }
    }
    uint32_t dbase, lbase;
    cta_exscan2(tid < 256 ? tot : 0u, tid < 256 ? mine : 0u, ws, dbase, lbase);
    if (tid < 256) {
      doff[tid] = dbase + before;  // global position of this CTA's first element with digit tid
      lstart[tid] = lbase;         // its local position in digit order
      if (tot == (uint32_t)N) s_skip = 1;  // every key has this digit: the pass keeps the order
    }
    __syncthreads();
    if (s_skip) {  // CTA- and cluster-uniform (every CTA sees the same totals)
      cl.sync();   // no CTA rewrites its counts while another still reads them
      continue;
    }
    // local reorder into digit order (stable), in the staging buffer
    for (int j = 0; j < E; ++j) {
      const int q = w * 32 * E + j * 32 + lane;
      if (q >= cnt) break;
      const K k = keyA[q];
      const uint32_t dg = (uint32_t)(k >> shift) & 255u;
      const uint32_t lr = lstart[dg] + wcnt[w * 256 + dg] + rloc[q];
      keyB[lr] = k;
      idxB[lr] = idxA[q];
    }
    __syncthreads();
    // runs of equal digits to the CTAs that own their positions: consecutive
    // threads write consecutive positions of the destination buffer
    for (int lr = tid; lr < cnt; lr += kKT) {
      const K k = keyB[lr];
      const uint32_t dg = (uint32_t)(k >> shift) & 255u;
      const uint32_t pos = doff[dg] + ((uint32_t)lr - lstart[dg]);
      // dst = pos / S: Smag = ceil(2^32 / S) for S >= 2 gives the quotient
      // or one more (pos < 2^31); S == 1 passes Smag = 0
      uint32_t dst = S == 1 ? pos : __umulhi(pos, Smag);
      if (dst * (uint32_t)S > pos) --dst;
      const uint32_t li = pos - dst * (uint32_t)S;
      if (pos >= (uint64_t)N || dst >= (uint32_t)CL || li >= (uint32_t)S) {  // never store out of range
        atomicOr(flags, ddks::kFlagBounds);
        continue;
      }
      cl.map_shared_rank(keyC, dst)[li] = k;
      cl.map_shared_rank(idxC, dst)[li] = idxB[lr];
    }
    cl.sync();  // the destination buffers are complete everywhere
    // rotate: the destination becomes current; the old current (last read
    // before this pass's first barrier) becomes the next destination
    K* tk = keyA; keyA = keyC; keyC = tk;
    uint32_t* ti = idxA; idxA = idxC; idxC = ti;
  }

  // run heads and P points, per warp chunk, then carried across the cluster
  if (tid == 0) s_left = (c > 0 && cnt > 0) ? (unsigned long long)cl.map_shared_rank(keyA, (unsigned)(c - 1))[S - 1] : 0ull;
  __syncthreads();
  auto head_at = [&](int q) -> bool {
    if (q >= cnt) return false;
    if (seg0 + q == 0) return true;
    const K left = q > 0 ? keyA[q - 1] : (K)s_left;
    return keyA[q] != left;
  };
  {
    uint32_t lh = 0, pc = 0;
    for (int j = 0; j < E; ++j) {
      const int q = w * 32 * E + j * 32 + lane;
      const uint32_t hm = __ballot_sync(0xffffffffu, head_at(q));
      if (hm) lh = (uint32_t)(seg0 + w * 32 * E + j * 32) + 31u - (uint32_t)__clz(hm);
      pc += (uint32_t)__popc(__ballot_sync(0xffffffffu, q < cnt && idxA[q] < (uint64_t)NP));
    }
    if (lane == 0) { whead[w] = lh; wpc[w] = pc; }
  }
  __syncthreads();
  if (tid == 0) {
    uint32_t lh = 0, pc = 0;
#pragma unroll
    for (int q = 0; q < kKW; ++q) { lh = whead[q] > lh ? whead[q] : lh; pc += wpc[q]; }
    s_info[0] = lh;
    s_info[1] = pc;
  }
  cl.sync();  // every CTA's summary is complete
  // the earlier CTAs' summaries (all loads issued together) and the earlier warps'
  uint32_t carry = 0, pbefore = 0;
#pragma unroll
  for (int r = 0; r < CL; ++r) {
    if (r < c) {
      const uint32_t* o = cl.map_shared_rank(s_info, (unsigned)r);
      const uint32_t h = o[0], pc = o[1];
      carry = h > carry ? h : carry;
      pbefore += pc;
    }
  }
  // the last read of another CTA's shared memory is done: arrive now, wait
  // before exiting (a relaxed arrival, so the stores below need not drain)
  asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
#pragma unroll
  for (int q = 0; q < kKW; ++q) {
    if (q < w) {
      carry = whead[q] > carry ? whead[q] : carry;
      pbefore += wpc[q];
    }
  }
  uint32_t* rk = rank + (int64_t)m * N;
  uint32_t* so = sorted ? sorted + (int64_t)m * N : nullptr;
  for (int j = 0; j < E; ++j) {
    const int q = w * 32 * E + j * 32 + lane;
    const uint32_t g0 = (uint32_t)(seg0 + w * 32 * E + j * 32);
    const bool v = q < cnt;
    const uint32_t hm = __ballot_sync(0xffffffffu, head_at(q));
    const uint32_t upto = hm & (0xffffffffu >> (31 - lane));  // heads at lanes <= this one
    const uint32_t run = upto ? g0 + 31u - (uint32_t)__clz(upto) : carry;
    const uint32_t idx = v ? idxA[q] : 0u;
    const bool isP = v && idx < (uint64_t)NP;
    const uint32_t pm = __ballot_sync(0xffffffffu, isP);
    if (v && idx >= (uint64_t)N) {  // an index that cannot come out of a correct sort: flag, skip
      atomicOr(flags, ddks::kFlagBounds);
    } else if (v) {
      rk[idx] = run;
      if (so) so[g0 + lane] = idx;
      if (m == 0) {
        sidx0[g0 + lane] = idx;
        pfx0[g0 + lane] = pbefore + (uint32_t)__popc(pm & ((1u << lane) - 1u));
      }
    }
    if (hm) carry = g0 + 31u - (uint32_t)__clz(hm);
    pbefore += (uint32_t)__popc(pm);
  }
  asm volatile("barrier.cluster.wait.aligned;" ::: "memory");  // no CTA leaves while another may still read it
}

}  // namespace

namespace {

// Largest cluster size (16, else 8) that the device schedules with the most
// shared memory this kernel asks for; looked up once per device.
std::mutex g_cl_mu;
int g_cl_size[128] = {};

template <typename V>
int cluster_size_for(int dev) {
  std::lock_guard<std::mutex> g(g_cl_mu);
  if (dev < 0 || dev >= 128) return 8;
  if (g_cl_size[dev]) return g_cl_size[dev];
  int best = 8;
  auto kern = k_rank_cluster<V, 16>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess &&
      ddks_smem_attr(kern, kSmemCap) == cudaSuccess) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(16, 1, 1);
    cfg.blockDim = dim3(kKT, 1, 1);
    cfg.dynamicSmemBytes = kSmemCap;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 16;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) == cudaSuccess && n >= 1) best = 16;
  }
  cudaGetLastError();
  g_cl_size[dev] = best;
  return best;
}

}  // namespace

bool ddks_rank_cluster_supported(int64_t N, int key_bits, int device) {
  if (N < 1 || N >= ((int64_t)1 << 31)) return false;
  const int CL = key_bits == 64 ? cluster_size_for<double>(device) : cluster_size_for<float>(device);
  const int64_t S = (N + CL - 1) / CL;
  const size_t smem = key_bits == 64 ? cluster_smem<uint64_t>(S) : cluster_smem<uint32_t>(S);
  return smem <= kSmemCap && S <= (int64_t)kEMax * kKT;
}

cudaError_t ddks_launch_rank_cluster(const void* P, const void* T, int64_t NP, int64_t NT, int d, bool f64,
                                     uint32_t* rank, uint32_t* sorted, uint32_t* sidx0, uint32_t* pfx0,
                                     unsigned* flags, cudaStream_t st) {
  const int64_t N = NP + NT;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (!ddks_rank_cluster_supported(N, f64 ? 64 : 32, dev) || d < 1 || !rank || !sidx0 || !pfx0)
    return cudaErrorInvalidValue;
  const int CL = f64 ? cluster_size_for<double>(dev) : cluster_size_for<float>(dev);
  const int S = (int)((N + CL - 1) / CL);
  // ceil(2^32 / S) fits 32 bits for S >= 2; S == 1 divides by itself
  const uint32_t Smag = S == 1 ? 0u : (uint32_t)((((uint64_t)1 << 32) + (uint64_t)S - 1) / (uint64_t)S);
  auto go = [&](auto kern, size_t smem, auto* p, auto* t) -> cudaError_t {
    cudaError_t r = ddks_smem_attr(kern, (int)smem);
    if (r != cudaSuccess) return r;
    if (CL > 8 && (r = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1)) != cudaSuccess)
      return r;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(CL * d), 1, 1);
    cfg.blockDim = dim3(kKT, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)CL;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, p, t, NP, NT, d, S, Smag, rank, sorted, sidx0, pfx0, flags);
  };
  const double* pd = (const double*)P;
  const double* td = (const double*)T;
  const float* pf = (const float*)P;
  const float* tf = (const float*)T;
  if (f64)
    return CL == 16 ? go(k_rank_cluster<double, 16>, cluster_smem<uint64_t>(S), pd, td)
                    : go(k_rank_cluster<double, 8>, cluster_smem<uint64_t>(S), pd, td);
  return CL == 16 ? go(k_rank_cluster<float, 16>, cluster_smem<uint32_t>(S), pf, tf)
                  : go(k_rank_cluster<float, 8>, cluster_smem<uint32_t>(S), pf, tf);
}
