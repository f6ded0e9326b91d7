// count_sort.cu -- orthant counts for any d by sorting codes (segmented count).
//
// When 2^d bins no longer fit on chip, the counts of one origin o are found by
// sorting: the CTA forms, for every pooled point x, the key
// 2*c(x, o) + [x in T] with c = sum_m [r_m(x) >= r_m(o)] 2^m (Sec. 2.2.1,
// Eq. g), sorts the N keys in shared memory (bitonic), and reads the counts
// off the runs of equal keys: the run of 2c holds cP(o, c), the run of 2c+1
// holds cT(o, c).  Orthants without points contribute 0 and cannot raise the
// maximum.  The CTA then reduces max |cP*NT - cT*NP| (Eq. d1) with the lowest
// orthant reaching it.  Needs N <= 32768 (keys resident in shared memory).
#include "ddks_internal.cuh"

namespace {

constexpr int kThreads = 1024;
constexpr int64_t kMaxSortN = 32768;

DDKS_DEV int lower_bound_u32(const uint32_t* a, int n, uint32_t v) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (a[mid] < v) lo = mid + 1; else hi = mid;
  }
  return lo;
}

__global__ void __launch_bounds__(kThreads)
k_sort(const uint32_t* __restrict__ rank, int64_t N, int64_t NP, int64_t NT, int d,
       int64_t o_begin, int64_t o_end, uint64_t* __restrict__ best, int32_t* __restrict__ bestj) {
  extern __shared__ uint32_t key[];  // [P2]
  __shared__ uint32_t o[ddks::kMaxD];
  __shared__ unsigned long long rv[kThreads / 32];
  __shared__ int rj[kThreads / 32];
  const int n = (int)N;
  int P2 = 1;
  while (P2 < n) P2 <<= 1;
  for (int64_t k = o_begin + blockIdx.x; k < o_end; k += gridDim.x) {
    __syncthreads();
    if (threadIdx.x < d) o[threadIdx.x] = rank[(int64_t)threadIdx.x * N + k];
    __syncthreads();
    for (int i = threadIdx.x; i < P2; i += blockDim.x) {
      if (i < n) {
        uint32_t c = 0;
        for (int m = 0; m < d; ++m) c |= (uint32_t)(rank[(int64_t)m * N + i] >= o[m]) << m;
        key[i] = (c << 1) | (i >= NP ? 1u : 0u);
      } else {
        key[i] = 0xFFFFFFFFu;  // pads sort last and are never a real key (d <= 30)
      }
    }
    __syncthreads();
    for (int size = 2; size <= P2; size <<= 1) {
      for (int stride = size >> 1; stride > 0; stride >>= 1) {
        for (int t = threadIdx.x; t < P2 / 2; t += blockDim.x) {
          const int lo = 2 * t - (t & (stride - 1));
          const int hi = lo + stride;
          const uint32_t a = key[lo], b = key[hi];
          const bool asc = ((lo & size) == 0);
          if (asc ? (b < a) : (a < b)) { key[lo] = b; key[hi] = a; }
        }
        __syncthreads();
      }
    }
    // segmented counts: the thread at the last position of a key run reports it
    uint64_t bv = 0;
    int bj = 0x7FFFFFFF;
    for (int p = threadIdx.x; p < n; p += blockDim.x) {
      const uint32_t v = key[p];
      if (p + 1 < n && key[p + 1] == v) continue;
      const uint32_t code = v >> 1;
      uint64_t cp, ct;
      if (v & 1u) {
        const int sT = lower_bound_u32(key, p + 1, v);
        ct = (uint64_t)(p + 1 - sT);
        const int sP = lower_bound_u32(key, sT, v - 1);
        cp = (uint64_t)(sT - sP);  // zero when no P point has this code
      } else {
        if (p + 1 < n && key[p + 1] == (v | 1u)) continue;  // the T run reports the pair
        const int sP = lower_bound_u32(key, p + 1, v);
        cp = (uint64_t)(p + 1 - sP);
        ct = 0;
      }
      const uint64_t num = ddks::numer(cp, ct, (uint64_t)NP, (uint64_t)NT);
      if (num > bv || (num == bv && (int)code < bj)) { bv = num; bj = (int)code; }
    }
    for (int off = 16; off > 0; off >>= 1) {
      const uint64_t v2 = __shfl_down_sync(0xffffffffu, bv, off);
      const int j2 = __shfl_down_sync(0xffffffffu, bj, off);
      if (v2 > bv || (v2 == bv && j2 < bj)) { bv = v2; bj = j2; }
    }
    if ((threadIdx.x & 31) == 0) { rv[threadIdx.x >> 5] = bv; rj[threadIdx.x >> 5] = bj; }
    __syncthreads();
    if (threadIdx.x == 0) {
      uint64_t b = rv[0];
      int j = rj[0];
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
        if (rv[w] > b || (rv[w] == b && rj[w] < j)) { b = rv[w]; j = rj[w]; }
      best[k - o_begin] = b;
      bestj[k - o_begin] = b ? j : 0;
    }
  }
}

}  // namespace

bool ddks_sort_supported(int d, int64_t N) { return d >= 1 && d <= ddks::kMaxD && N <= kMaxSortN; }

cudaError_t ddks_launch_sort(const uint32_t* rank, int64_t N, int64_t NP, int64_t NT, int d,
                             int64_t o_begin, int64_t o_end, uint64_t* best, int32_t* bestj,
                             cudaStream_t st) {
  if (!ddks_sort_supported(d, N)) return cudaErrorInvalidValue;
  int P2 = 1;
  while (P2 < N) P2 <<= 1;
  const size_t sm = (size_t)P2 * 4u;
  cudaError_t e = ddks_smem_attr(k_sort, (int)sm);
  if (e != cudaSuccess) return e;
  const int64_t no = o_end - o_begin;
  if (no <= 0) return cudaSuccess;
  int grid = (int)(no < 152 * 8 ? no : 152 * 8);
  k_sort<<<grid, kThreads, sm, st>>>(rank, N, NP, NT, d, o_begin, o_end, best, bestj);
  return cudaGetLastError();
}
