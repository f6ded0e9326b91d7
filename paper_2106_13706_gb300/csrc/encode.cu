// encode.cu -- K0: ingest and rank-encode the pooled sample.
//
// The statistic only ever asks whether x_m >= o_m (Sec. 2.2.1, Eq. g), so each
// coordinate can be replaced by any strictly order-preserving integer.  K0 maps
// every coordinate to an order-preserving 64-bit key (NaN raises a flag),
// sorts each dimension's (key, index) pairs, and replaces every coordinate by
// its min-rank  #{j : key_j < key_i}.  Then x_m >= o_m <=> rank(x)_m >= rank(o)_m
// exactly, ties included, and every later kernel compares 32-bit integers
// whatever the input type.
//
// Sort: bitonic sort of 2048-element chunks in shared memory.  With at most 4
// chunks a dimension (N <= 8192) every element then finds its min-rank as
// the sum of one lower_bound per sorted chunk, and its position in the full
// (key, index) order for dimension 0.  Larger inputs merge the chunks in
// passes in which every element finds its output slot by binary search in the
// partner run (pairs are unique because the index breaks ties), then take one
// lower_bound per element in the fully sorted keys.
#include "ddks_internal.cuh"

namespace {

constexpr int kChunk = 2048;
constexpr int kChunkThreads = 1024;
constexpr int64_t kMaxMultiChunks = 4;  // above this (N > 8192), merge passes

template <typename V>
__global__ void k_encode(const V* __restrict__ P, const V* __restrict__ T, int64_t NP, int64_t NT,
                         int d, uint64_t* __restrict__ keys, unsigned* __restrict__ flags) {
  const int64_t N = NP + NT;
  const int64_t total = N * d;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / d;
    const int m = (int)(e - i * d);
    const V v = i < NP ? P[e] : T[e - NP * d];
    if (v != v) atomicOr(flags, ddks::kFlagNaN);
    keys[(int64_t)m * N + i] = ddks::order_key(v);
  }
}

DDKS_DEV bool pair_less(uint64_t ka, uint32_t ia, uint64_t kb, uint32_t ib) {
  return ka < kb || (ka == kb && ia < ib);
}

// grid: (chunks, d).  Sorts chunk blockIdx.x of dimension blockIdx.y.
// With out_p, dimensions m < pfx_dims also write out_p[m * Npad + base + t] =
// #{j < t : sorted element j of the chunk is a P point}.
__global__ void __launch_bounds__(kChunkThreads)
k_chunk_sort(const uint64_t* __restrict__ keys, int64_t N, int64_t Npad, int64_t NP,
             uint64_t* __restrict__ out_k, uint32_t* __restrict__ out_i, uint32_t* __restrict__ out_p,
             int pfx_dims) {
  extern __shared__ __align__(16) unsigned char smraw[];
  uint64_t* sk = reinterpret_cast<uint64_t*>(smraw);   // [kChunk]
  uint32_t* si = reinterpret_cast<uint32_t*>(sk + kChunk);
  const int m = blockIdx.y;
  const int64_t base = (int64_t)blockIdx.x * kChunk;
  for (int t = threadIdx.x; t < kChunk; t += blockDim.x) {
    const int64_t g = base + t;
    if (g < N) {
      sk[t] = keys[(int64_t)m * N + g];
      si[t] = (uint32_t)g;
    } else {
      sk[t] = ~0ull;          // pads sort last; the index keeps pairs unique
      si[t] = (uint32_t)g;
    }
  }
  __syncthreads();
  for (int size = 2; size <= kChunk; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int t = threadIdx.x; t < kChunk / 2; t += blockDim.x) {
        const int lo = 2 * t - (t & (stride - 1));
        const int hi = lo + stride;
        const bool asc = ((lo & size) == 0);
        const uint64_t ka = sk[lo], kb = sk[hi];
        const uint32_t ia = si[lo], ib = si[hi];
        const bool swap = asc ? pair_less(kb, ib, ka, ia) : pair_less(ka, ia, kb, ib);
        if (swap) {
          sk[lo] = kb; sk[hi] = ka;
          si[lo] = ib; si[hi] = ia;
        }
      }
      __syncthreads();
    }
  }
  for (int t = threadIdx.x; t < kChunk; t += blockDim.x) {
    out_k[(int64_t)m * Npad + base + t] = sk[t];
    out_i[(int64_t)m * Npad + base + t] = si[t];
  }
  if (out_p && m < pfx_dims) {
    // exclusive prefix of the P flags of the sorted chunk: thread t owns
    // elements 2t, 2t+1
    __shared__ uint32_t wsum[kChunkThreads / 32 + 1];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const uint32_t f0 = si[2 * t] < (uint64_t)NP ? 1u : 0u, f1 = si[2 * t + 1] < (uint64_t)NP ? 1u : 0u;
    const uint32_t v = f0 + f1;
    uint32_t incl = v;
    for (int off = 1; off < 32; off <<= 1) {
      const uint32_t x = __shfl_up_sync(0xffffffffu, incl, off);
      if (lane >= off) incl += x;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      const uint32_t w = wsum[lane];
      uint32_t wi = w;
      for (int off = 1; off < 32; off <<= 1) {
        const uint32_t x = __shfl_up_sync(0xffffffffu, wi, off);
        if (lane >= off) wi += x;
      }
      wsum[lane] = wi - w;
      if (lane == 31) wsum[32] = wi;
    }
    __syncthreads();
    const uint32_t ex = wsum[warp] + incl - v;
    uint32_t* P = out_p + (int64_t)m * Npad + base;
    P[2 * t] = ex;
    P[2 * t + 1] = ex + f0;
  }
}

// One merge pass over runs of length L (Npad is a multiple of kChunk <= L).
// grid-stride over (d * Npad) elements.  With in_p / out_p, dimensions
// m < pfx_dims also carry each element's count of P points before it within
// its run: after the merge that is its own count plus the partner run's count
// below its slot.
__global__ void k_merge_pass(const uint64_t* __restrict__ in_k, const uint32_t* __restrict__ in_i,
                             uint64_t* __restrict__ out_k, uint32_t* __restrict__ out_i,
                             const uint32_t* __restrict__ in_p, uint32_t* __restrict__ out_p,
                             int64_t Npad, int64_t NP, int d, int64_t L, int pfx_dims) {
  const int64_t total = Npad * d;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t m = e / Npad;
    const int64_t p = e - m * Npad;
    const uint64_t* K = in_k + m * Npad;
    const uint32_t* I = in_i + m * Npad;
    const uint64_t key = K[p];
    const uint32_t idx = I[p];
    const int64_t r = p / L;
    const int64_t a = p - r * L;
    const int64_t ps = (r ^ 1) * L;  // partner run start
    int64_t dst;
    const bool carry = in_p && m < pfx_dims;
    const uint32_t* Pin = carry ? in_p + m * Npad : nullptr;
    uint32_t pc = carry ? Pin[p] : 0u;
    if (ps >= Npad) {
      dst = p;
    } else {
      const int64_t plen = (Npad - ps) < L ? (Npad - ps) : L;
      // number of partner elements strictly below (key, idx)
      int64_t lo = 0, hi = plen;
      while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (pair_less(K[ps + mid], I[ps + mid], key, idx)) lo = mid + 1; else hi = mid;
      }
      const int64_t start = (r < (r ^ 1) ? r : (r ^ 1)) * L;
      dst = start + a + lo;
      if (carry)
        pc += lo < plen ? Pin[ps + lo]
                        : Pin[ps + plen - 1] + (I[ps + plen - 1] < (uint64_t)NP ? 1u : 0u);
    }
    out_k[m * Npad + dst] = key;
    out_i[m * Npad + dst] = idx;
    if (carry) out_p[m * Npad + dst] = pc;
  }
}

// With few sorted chunks: rank[m][i] = sum over chunks of #{keys < key_i}
// (one lower_bound per chunk), and for dimension 0 the position of (key_i, i)
// in the full sorted order, which places i in sorted_idx0.  The searches of up
// to 8 chunks advance together (independent loads in flight).
__global__ void k_rank_multi(const uint64_t* __restrict__ keys, const uint64_t* __restrict__ ck,
                             const uint32_t* __restrict__ ci, const uint32_t* __restrict__ cpfx,
                             int64_t N, int64_t NPc, int64_t Npad, int d, uint32_t* __restrict__ rank,
                             uint32_t* __restrict__ sorted_idx0, uint32_t* __restrict__ pprefix0) {
  constexpr int kG = 8;
  const int64_t total = N * d;
  const int nch = (int)(Npad / kChunk);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t m = e / N;
    const int64_t i = e - m * N;
    const uint64_t key = keys[e];
    const bool want_pos = m == 0 && sorted_idx0;
    uint32_t r = 0, pos = 0, pb = 0;
    for (int c0 = 0; c0 < nch; c0 += kG) {
      int lo[kG], hi[kG];
#pragma unroll
      for (int g = 0; g < kG; ++g) { lo[g] = 0; hi[g] = c0 + g < nch ? kChunk : 0; }
      const uint64_t* K = ck + m * Npad + (int64_t)c0 * kChunk;
      for (int step = 0; step < 12; ++step) {  // 2^11 = kChunk: at most 12 halvings
#pragma unroll
        for (int g = 0; g < kG; ++g) {
          if (lo[g] < hi[g]) {
            const int mid = (lo[g] + hi[g]) >> 1;
            if (K[g * kChunk + mid] < key) lo[g] = mid + 1; else hi[g] = mid;
          }
        }
      }
#pragma unroll
      for (int g = 0; g < kG; ++g) r += (uint32_t)lo[g];
      if (want_pos) {
        // continue past equal keys with a smaller index
        const uint32_t* I = ci + m * Npad + (int64_t)c0 * kChunk;
        int lo2[kG], hi2[kG];
#pragma unroll
        for (int g = 0; g < kG; ++g) { lo2[g] = lo[g]; hi2[g] = c0 + g < nch ? kChunk : 0; }
        for (int step = 0; step < 12; ++step) {
#pragma unroll
          for (int g = 0; g < kG; ++g) {
            if (lo2[g] < hi2[g]) {
              const int mid = (lo2[g] + hi2[g]) >> 1;
              if (K[g * kChunk + mid] == key && I[g * kChunk + mid] < (uint32_t)i) lo2[g] = mid + 1;
              else hi2[g] = mid;
            }
          }
        }
#pragma unroll
        for (int g = 0; g < kG; ++g) {
          pos += (uint32_t)lo2[g];
          if (pprefix0 && c0 + g < nch) {
            const int64_t cb = (int64_t)(c0 + g) * kChunk;  // dimension 0: chunk start
            pb += lo2[g] < kChunk ? cpfx[cb + lo2[g]]
                                  : cpfx[cb + kChunk - 1] + (ci[cb + kChunk - 1] < (uint64_t)NPc ? 1u : 0u);
          }
        }
      }
    }
    rank[e] = r;
    if (want_pos) {
      sorted_idx0[pos] = (uint32_t)i;
      if (pprefix0) pprefix0[pos] = pb;  // P points before position pos
    }
  }
}

// rank[m][i] = #{j : key_j < key_i}, by lower_bound in the sorted keys of m.
__global__ void k_rank(const uint64_t* __restrict__ keys, const uint64_t* __restrict__ sorted_k,
                       int64_t N, int64_t Npad, int d, uint32_t* __restrict__ rank) {
  const int64_t total = N * d;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t m = e / N;
    const uint64_t key = keys[e];
    const uint64_t* S = sorted_k + m * Npad;
    int64_t lo = 0, hi = N;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (S[mid] < key) lo = mid + 1; else hi = mid;
    }
    rank[e] = (uint32_t)lo;
  }
}

__global__ void k_copy_idx(const uint32_t* __restrict__ sorted_i, const uint32_t* __restrict__ sorted_p,
                           int64_t N, uint32_t* __restrict__ out, uint32_t* __restrict__ out_p) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    out[i] = sorted_i[i];
    if (out_p) out_p[i] = sorted_p[i];
  }
}

int grid_for(int64_t work, int threads) {
  int64_t g = (work + threads - 1) / threads;
  if (g > 152 * 64) g = 152 * 64;
  return (int)(g < 1 ? 1 : g);
}

}  // namespace

cudaError_t ddks_launch_encode(const void* P, const void* T, int64_t NP, int64_t NT, int d,
                               int is_f64, uint64_t* keys, unsigned* flags, cudaStream_t st) {
  const int64_t total = (NP + NT) * d;
  const int threads = 256;
  if (is_f64)
    k_encode<double><<<grid_for(total, threads), threads, 0, st>>>(
        (const double*)P, (const double*)T, NP, NT, d, keys, flags);
  else
    k_encode<float><<<grid_for(total, threads), threads, 0, st>>>(
        (const float*)P, (const float*)T, NP, NT, d, keys, flags);
  return cudaGetLastError();
}

size_t ddks_rank_scratch_elems(int64_t N) {
  const int64_t chunks = (N + kChunk - 1) / kChunk;
  return (size_t)(chunks * kChunk);
}

// keys: [d][N].  tmp buffers: d * Npad elements each.  rank: [d][N].
// sorted_idx0 (optional): the pooled indices in increasing (rank_0, index) order.
// pprefix0 (optional, with sorted_idx0; u32 [N] plus 2 * ddks_rank_pfx_elems(N)
// of scratch at cpfx): pprefix0[p] = #{P points among sorted positions < p}.
size_t ddks_rank_pfx_elems(int64_t N) { return ddks_rank_scratch_elems(N); }

cudaError_t ddks_launch_rank(const uint64_t* keys, int64_t N, int64_t NP, int d, uint64_t* tmp_keys,
                             uint32_t* tmp_idx, uint64_t* tmp_keys2, uint32_t* tmp_idx2,
                             uint32_t* rank, uint32_t* sorted_idx0, uint32_t* pprefix0, uint32_t* cpfx,
                             int* pfx_done, cudaStream_t st, int* launches) {
  const int64_t Npad = (int64_t)ddks_rank_scratch_elems(N);
  const int64_t chunks = Npad / kChunk;
  dim3 g((unsigned)chunks, (unsigned)d);
  const size_t smem = (size_t)kChunk * 12;
  const bool pfx = sorted_idx0 && pprefix0 && cpfx;
  if (pfx_done) *pfx_done = pfx ? 1 : 0;
  cudaError_t e = cudaFuncSetAttribute(k_chunk_sort, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  uint32_t* cp = pfx ? cpfx : nullptr;             // [Npad] P prefixes, dimension 0
  uint32_t* cp2 = pfx ? cpfx + Npad : nullptr;     // [Npad] the other merge buffer
  k_chunk_sort<<<g, kChunkThreads, smem, st>>>(keys, N, Npad, NP, tmp_keys, tmp_idx, cp, 1);
  int n = 1;
  if (chunks <= kMaxMultiChunks) {
    k_rank_multi<<<grid_for(N * d, 256), 256, 0, st>>>(keys, tmp_keys, tmp_idx, cp, N, NP, Npad, d, rank,
                                                       sorted_idx0, pfx ? pprefix0 : nullptr);
    if (launches) *launches += 2;
    return cudaGetLastError();
  }
  uint64_t *ck = tmp_keys, *nk = tmp_keys2;
  uint32_t *ci = tmp_idx, *ni = tmp_idx2;
  for (int64_t L = kChunk; L < Npad; L <<= 1) {
    k_merge_pass<<<grid_for(Npad * d, 256), 256, 0, st>>>(ck, ci, nk, ni, cp, cp2, Npad, NP, d, L, 1);
    ++n;
    uint64_t* tk = ck; ck = nk; nk = tk;
    uint32_t* ti = ci; ci = ni; ni = ti;
    uint32_t* tp = cp; cp = cp2; cp2 = tp;
  }
  k_rank<<<grid_for(N * d, 256), 256, 0, st>>>(keys, ck, N, Npad, d, rank);
  ++n;
  if (sorted_idx0) {
    k_copy_idx<<<grid_for(N, 256), 256, 0, st>>>(ci, cp, N, sorted_idx0, pfx ? pprefix0 : nullptr);
    ++n;
  }
  if (launches) *launches += n;
  return cudaGetLastError();
}

// Sort S segments of N keys each ([S][N]; ties broken by the pooled index) and
// carry, for every segment, the count of P points (index < NP) before each
// sorted position.  Buffers hold S * ddks_rank_scratch_elems(N) elements each
// (k1/k2 keys, i1/i2 indices, p1/p2 prefixes); *out_k, *out_i, *out_p point at
// the ones holding the result, laid out [S][Npad] with positions >= N padding.
cudaError_t ddks_launch_sort_segments(const uint64_t* keys, int64_t N, int64_t NP, int S, uint64_t* k1,
                                      uint32_t* i1, uint32_t* p1, uint64_t* k2, uint32_t* i2,
                                      uint32_t* p2, const uint64_t** out_k, const uint32_t** out_i,
                                      const uint32_t** out_p, cudaStream_t st, int* launches) {
  const int64_t Npad = (int64_t)ddks_rank_scratch_elems(N);
  const int64_t chunks = Npad / kChunk;
  const size_t smem = (size_t)kChunk * 12;
  cudaError_t e = cudaFuncSetAttribute(k_chunk_sort, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_chunk_sort<<<dim3((unsigned)chunks, (unsigned)S), kChunkThreads, smem, st>>>(keys, N, Npad, NP, k1, i1,
                                                                                  p1, S);
  int n = 1;
  uint64_t *ck = k1, *nk = k2;
  uint32_t *ci = i1, *ni = i2, *cp = p1, *np = p2;
  for (int64_t L = kChunk; L < Npad; L <<= 1) {
    k_merge_pass<<<grid_for(Npad * S, 256), 256, 0, st>>>(ck, ci, nk, ni, cp, np, Npad, NP, S, L, S);
    ++n;
    uint64_t* tk = ck; ck = nk; nk = tk;
    uint32_t* ti = ci; ci = ni; ni = ti;
    uint32_t* tp = cp; cp = np; np = tp;
  }
  *out_k = ck;
  *out_i = ci;
  *out_p = cp;
  if (launches) *launches += n;
  return cudaGetLastError();
}
