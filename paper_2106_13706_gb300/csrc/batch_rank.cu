// batch_rank.cu -- K0 of the batched launch (the ranks behind Eq. g for every
// problem of a batch).
//
// x_m >= o_m <=> rank_m(x) >= rank_m(o) with rank = the number of pooled
// values strictly below, so the count kernels work on min-ranks.  One CTA per
// (problem, dimension) sorts that coordinate of the problem's pooled points
// in shared memory: order-preserving integer keys stay in place and a stable
// LSD radix sort with 8-bit digits moves 16-bit point indices between two
// buffers.  Per pass each warp ranks its contiguous chunk of positions
// stably by digit (lanes with equal digits found by ballots, one shared
// atomic per group on the warp's own counters, taken in program order), the
// warps' counts give each (digit, warp) its first output position, and every
// element is written once to its place.  A pass whose digit is the same for
// every key keeps the order and is skipped.  Then the min-rank of a sorted
// position is the first position of its run of equal keys (a running maximum
// of run heads, carried from warp to warp), and the dimension-0 CTA also
// writes the sorted order, the P points before each position and the two
// samples' lists in dimension-0 order.
//
// Problems are launched in two size classes (256 threads up to 4,096
// points, 1,024 above), each with the shared memory its largest member
// needs, so small problems are not held to one CTA per SM by the largest.
#include "batch_internal.cuh"
#include "ddks_internal.cuh"

namespace {

constexpr int kEMax = 16;  // positions per thread at most

template <typename V> struct KeyOf;
template <> struct KeyOf<float> { using K = uint32_t; };
template <> struct KeyOf<double> { using K = uint64_t; };

template <typename V>
__host__ __device__ constexpr size_t radix_smem(int cap, int threads) {
  return (size_t)cap * sizeof(typename KeyOf<V>::K) + (size_t)cap * 2 * 2 + (size_t)(threads / 32) * 256 * 4;
}

template <typename V, int THREADS>
__global__ void __launch_bounds__(THREADS)
k_batch_radix(const BatchDesc* __restrict__ desc, const int* __restrict__ dprob, const int* __restrict__ ddim,
              int cap, const RankAreas ra, unsigned* __restrict__ flags) {
  using K = typename KeyOf<V>::K;
  constexpr int kW = THREADS / 32;
  constexpr int kPasses = (int)sizeof(K);
  static_assert(THREADS >= 256, "one thread per digit in the digit prefix");
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ uint32_t tot[256], dstart[256], wsum[32], wmax[32];
  __shared__ int s_skip;
  const BatchDesc D = desc[dprob[blockIdx.x]];
  const int m = ddim[blockIdx.x];
  const int N = (int)(D.NP + D.NT), NP = (int)D.NP;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  K* key = reinterpret_cast<K*>(smraw);
  uint16_t* ixA = reinterpret_cast<uint16_t*>(key + cap);
  uint16_t* ixB = ixA + cap;
  uint32_t* wcnt = reinterpret_cast<uint32_t*>(ixB + cap);  // [kW][256]
  const int E = (N + THREADS - 1) / THREADS;  // the host keeps N <= cap <= kEMax * THREADS
  if (N > cap || E > kEMax) {
    if (tid == 0) atomicOr(flags, ddks::kFlagBounds);
    return;
  }
  const V* Pv = static_cast<const V*>(D.P);
  const V* Tv = static_cast<const V*>(D.T);
  unsigned nan = 0;
  for (int q = tid; q < N; q += THREADS) {
    const V v = q < NP ? Pv[(int64_t)q * D.d + m] : Tv[(int64_t)(q - NP) * D.d + m];
    nan |= v != v ? 1u : 0u;
    key[q] = (K)ddks::order_key(v);
    ixA[q] = (uint16_t)q;
  }
  if (__syncthreads_or(nan) && tid == 0) atomicOr(flags, ddks::kFlagNaN);

  for (int pass = 0; pass < kPasses; ++pass) {
    const int shift = 8 * pass;
    for (int i = tid; i < kW * 256; i += THREADS) wcnt[i] = 0u;
    __syncthreads();
    // stable rank of each element among its warp's earlier elements of the
    // same digit: rr = digit << 16 | rank
    uint32_t rr[kEMax];
#pragma unroll
    for (int j = 0; j < kEMax; ++j) {
      rr[j] = 0u;
      if (j < E) {  // CTA-uniform
        const int q = (w * E + j) * 32 + lane;
        const bool v = q < N;
        const uint32_t vm = __ballot_sync(0xffffffffu, v);
        if (vm != 0u) {  // warp-uniform
          const uint32_t dg = v ? (uint32_t)(key[ixA[q]] >> shift) & 255u : 0u;
          const uint32_t sd = ddks::same_digit(dg);  // every lane takes part in its ballots
          const uint32_t pr = v ? sd & vm : 0u;
          const int leader = __ffs(pr) - 1;  // -1 exactly on the lanes past the end
          uint32_t base = 0;
          if (lane == leader) base = atomicAdd(&wcnt[w * 256 + dg], (uint32_t)__popc(pr));
          base = __shfl_sync(0xffffffffu, base, leader < 0 ? lane : leader);
          rr[j] = (dg << 16) | (base + (uint32_t)__popc(pr & ((1u << lane) - 1u)));
        }
      }
    }
    __syncthreads();
    if (tid == 0) s_skip = 0;  // read only after the barriers below
    uint32_t x = 0, inc = 0;
    if (tid < 256) {
      // the warps' offsets within digit tid, then the CTA's count of it
      uint32_t s = 0;
      for (int q = 0; q < kW; ++q) {
        const uint32_t c = wcnt[q * 256 + tid];
        wcnt[q * 256 + tid] = s;
        s += c;
      }
      x = s;
      inc = s;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, off);
        if (lane >= off) inc += y;
      }
      if (lane == 31) wsum[w] = inc;
    }
    __syncthreads();
    if (tid < 256) {
      uint32_t add = 0;
      for (int q = 0; q < w; ++q) add += wsum[q];
      dstart[tid] = add + inc - x;
      if (x == (uint32_t)N) s_skip = 1;  // every key has this digit: the pass keeps the order
    }
    __syncthreads();
    if (s_skip) continue;  // CTA-uniform
#pragma unroll
    for (int j = 0; j < kEMax; ++j) {
      if (j < E) {
        const int q = (w * E + j) * 32 + lane;
        if (q < N) {
          const uint32_t dg = rr[j] >> 16;
          const uint32_t pos = dstart[dg] + wcnt[w * 256 + dg] + (rr[j] & 0xFFFFu);
          if (pos < (uint32_t)N) ixB[pos] = ixA[q];
          else atomicOr(flags, ddks::kFlagBounds);  // never stores out of range
        }
      }
    }
    __syncthreads();
    uint16_t* t = ixA;
    ixA = ixB;
    ixB = t;
  }

  // run heads: the last one of each warp's chunk, and each chunk's P points
  auto head = [&](int q) -> bool { return q < N && (q == 0 || key[ixA[q]] != key[ixA[q - 1]]); };
  {
    uint32_t lh = 0, pc = 0;
    for (int j = 0; j < E; ++j) {
      const int q = (w * E + j) * 32 + lane;
      const uint32_t hm = __ballot_sync(0xffffffffu, head(q));
      if (hm) lh = (uint32_t)((w * E + j) * 32) + 31u - (uint32_t)__clz(hm);
      pc += (uint32_t)__popc(__ballot_sync(0xffffffffu, q < N && ixA[q] < NP));
    }
    if (lane == 0) {
      wmax[w] = lh;  // 0 when the chunk has no head (position 0 always is one)
      wsum[w] = pc;
    }
  }
  __syncthreads();
  uint32_t cur = 0, prun = 0;
  for (int q = 0; q < w; ++q) {
    cur = wmax[q] > cur ? wmax[q] : cur;
    prun += wsum[q];
  }
  uint32_t* R = ra.rank + D.off_rank + (int64_t)m * N;
  uint32_t* od = ra.ord + D.off_pool;
  uint32_t* ls = ra.lst + D.off_pool;
  uint32_t* pf = ra.pfx + D.off_pool;
  const uint32_t le_mask = lane == 31 ? 0xffffffffu : ((2u << lane) - 1u);
  for (int j = 0; j < E; ++j) {
    const int base = (w * E + j) * 32;
    const int q = base + lane;
    const uint32_t hm = __ballot_sync(0xffffffffu, head(q));
    const uint32_t le = hm & le_mask;
    const uint32_t lo = le ? (uint32_t)base + 31u - (uint32_t)__clz(le) : cur;
    if (hm) cur = (uint32_t)base + 31u - (uint32_t)__clz(hm);
    const uint32_t i = q < N ? ixA[q] : 0u;
    if (q < N) R[i] = lo;
    if (m == 0) {
      // Points with x_0 < o_0 are exactly the positions < rank_0(o), so a
      // sample's first pfx-many list entries are an origin's phase A.
      const bool isP = q < N && i < (uint32_t)NP;
      const uint32_t pm = __ballot_sync(0xffffffffu, isP);
      const uint32_t p = prun + (uint32_t)__popc(pm & ((1u << lane) - 1u));
      if (q < N) {
        od[q] = i;
        pf[q] = p;
        if (isP) ls[p] = i;
        else ls[NP + q - (int)p] = i;
      }
      prun += (uint32_t)__popc(pm);
    }
  }
}

template <typename V>
cudaError_t launch_class(const BatchDesc* desc, const int* dprob, const int* ddim, const BatchRankClass& c,
                         const RankAreas& ra, unsigned* flags, cudaStream_t st) {
  const int cap = (c.cap + 7) & ~7;
  cudaError_t e;
  if (c.wide) {
    const size_t smem = radix_smem<V>(cap, 1024);
    e = ddks_smem_attr(k_batch_radix<V, 1024>, (int)smem);
    if (e != cudaSuccess) return e;
    k_batch_radix<V, 1024><<<c.count, 1024, smem, st>>>(desc, dprob + c.first, ddim + c.first, cap, ra, flags);
  } else {
    const size_t smem = radix_smem<V>(cap, 256);
    e = ddks_smem_attr(k_batch_radix<V, 256>, (int)smem);
    if (e != cudaSuccess) return e;
    k_batch_radix<V, 256><<<c.count, 256, smem, st>>>(desc, dprob + c.first, ddim + c.first, cap, ra, flags);
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t ddks_batch_rank(const BatchDesc* desc, const int* dprob, const int* ddim, const BatchRankClass* cls,
                            int ncls, bool f64, const RankAreas& ra, unsigned* flags, cudaStream_t st) {
  for (int k = 0; k < ncls; ++k) {
    if (cls[k].count == 0) continue;
    if (cls[k].cap > (cls[k].wide ? 1024 : 256) * kEMax || cls[k].cap > kBatchMaxN) return cudaErrorInvalidValue;
    const cudaError_t e = f64 ? launch_class<double>(desc, dprob, ddim, cls[k], ra, flags, st)
                              : launch_class<float>(desc, dprob, ddim, cls[k], ra, flags, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}
