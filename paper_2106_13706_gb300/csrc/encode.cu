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
// passes: each CTA produces 2048 consecutive outputs of a merged pair of runs,
// finding where its output range starts in the two runs by a merge-path
// search (pairs are unique because the index breaks ties), staging both input
// ranges in shared memory and merging them there.  The last pass writes the
// min-ranks (and dimension 0's sorted order) directly instead of the merged
// arrays.
#include "ddks_internal.cuh"

namespace {

constexpr int kChunk = 2048;       // sorted chunks and merge tiles
constexpr int kSortEach = 4;       // sorted positions per thread of k_chunk_sort (4 measured faster than 8)
constexpr int kChunkThreads = kChunk / kSortEach;
constexpr int64_t kMaxMultiChunks = 4;  // above this (N > 8192), merge passes

// One thread per point: its d coordinates (row-major input) to the key rows
// [d][N] (consecutive points of a warp write consecutive keys of each row).
template <typename V>
__global__ void k_encode(const V* __restrict__ P, const V* __restrict__ T, int64_t NP, int64_t NT,
                         int d, uint64_t* __restrict__ keys, unsigned* __restrict__ flags) {
  const int64_t N = NP + NT;
  bool nan = false;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const V* row = i < NP ? P + i * d : T + (i - NP) * d;
    for (int m = 0; m < d; ++m) {
      const V v = row[m];
      nan |= v != v;
      keys[(int64_t)m * N + i] = ddks::order_key(v);
    }
  }
  if (nan) atomicOr(flags, ddks::kFlagNaN);
}

DDKS_DEV bool pair_less(uint64_t ka, uint32_t ia, uint64_t kb, uint32_t ib) {
  return ka < kb || (ka == kb && ia < ib);
}

// grid: (chunks, d).  Sorts chunk blockIdx.x of dimension blockIdx.y by
// (key, index) with a bitonic network.  Thread t holds the E consecutive
// positions E t .. E t + E - 1 in registers: compare-exchange stages of stride
// < E stay inside a thread, strides E .. 16 E pair thread t with
// t ^ (stride / E) of the same warp (shuffles), larger strides go through
// shared memory.
// With out_p, dimensions m < pfx_dims also write out_p[m * Npad + base + p] =
// #{q < p : sorted element q of the chunk is a P point}.
template <int CH, int E>
__global__ void __launch_bounds__(CH / E)
k_chunk_sort(const uint64_t* __restrict__ keys, int64_t N, int64_t Npad, int64_t NP,
             uint64_t* __restrict__ out_k, uint32_t* __restrict__ out_i, uint32_t* __restrict__ out_p,
             int pfx_dims) {
  constexpr int kChunk = CH;  // this kernel's chunk
  constexpr int kChunkThreads = CH / E;
  extern __shared__ __align__(16) unsigned char cs_raw[];
  uint64_t* sk = reinterpret_cast<uint64_t*>(cs_raw);   // [CH]
  uint32_t* si = reinterpret_cast<uint32_t*>(sk + CH);  // [CH]
  __shared__ uint32_t wsum[kChunkThreads / 32 + 1];
  const int m = blockIdx.y;
  const int t = threadIdx.x;
  const int64_t base = (int64_t)blockIdx.x * kChunk;
  const int q0 = t * E;
  uint64_t k[E];
  uint32_t ix[E];
  // coalesced loads through shared memory
  for (int q = t; q < kChunk; q += kChunkThreads) {
    const int64_t g = base + q;
    sk[q] = g < N ? keys[(int64_t)m * N + g] : ~0ull;  // pads sort last; the index keeps pairs unique
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < E; ++j) {
    k[j] = sk[q0 + j];
    ix[j] = (uint32_t)(base + q0 + j);
  }
  __syncthreads();
  for (int size = 2; size <= kChunk; size <<= 1) {
    int stride = size >> 1;
    if (stride >= E * 32) {  // partners in other warps: through shared memory
#pragma unroll
      for (int j = 0; j < E; ++j) { sk[q0 + j] = k[j]; si[q0 + j] = ix[j]; }
      __syncthreads();
      for (; stride >= E * 32; stride >>= 1) {
        for (int pr = t; pr < kChunk / 2; pr += kChunkThreads) {
          const int lo = 2 * pr - (pr & (stride - 1));
          const int hi = lo + stride;
          const bool asc = (lo & size) == 0;
          const uint64_t ka = sk[lo], kb = sk[hi];
          const uint32_t ia = si[lo], ib = si[hi];
          if (asc ? pair_less(kb, ib, ka, ia) : pair_less(ka, ia, kb, ib)) {
            sk[lo] = kb; sk[hi] = ka;
            si[lo] = ib; si[hi] = ia;
          }
        }
        __syncthreads();
      }
#pragma unroll
      for (int j = 0; j < E; ++j) { k[j] = sk[q0 + j]; ix[j] = si[q0 + j]; }
      __syncthreads();  // the next size writes these slots again
    }
    for (; stride >= E; stride >>= 1) {  // partner thread t ^ (stride / E) in this warp
      const int xm = stride / E;
      const bool lower = (t & xm) == 0;
#pragma unroll
      for (int j = 0; j < E; ++j) {
        const uint64_t ok = __shfl_xor_sync(0xffffffffu, k[j], xm);
        const uint32_t oi = __shfl_xor_sync(0xffffffffu, ix[j], xm);
        const bool asc = ((q0 + j) & size) == 0;
        const bool keep_min = lower == asc;
        if (keep_min != pair_less(k[j], ix[j], ok, oi)) { k[j] = ok; ix[j] = oi; }
      }
    }
#pragma unroll
    for (int sd = E / 2; sd >= 1; sd >>= 1) {  // inside the thread (sd <= stride: indices stay static)
      if (sd > stride) continue;
#pragma unroll
      for (int a = 0; a < E; ++a) {
        if (a & sd) continue;
        const int b = a | sd;
        const bool asc = ((q0 + a) & size) == 0;
        if (asc ? pair_less(k[b], ix[b], k[a], ix[a]) : pair_less(k[a], ix[a], k[b], ix[b])) {
          const uint64_t tk = k[a]; k[a] = k[b]; k[b] = tk;
          const uint32_t ti = ix[a]; ix[a] = ix[b]; ix[b] = ti;
        }
      }
    }
  }
  // coalesced stores through shared memory
#pragma unroll
  for (int j = 0; j < E; ++j) { sk[q0 + j] = k[j]; si[q0 + j] = ix[j]; }
  __syncthreads();
  for (int q = t; q < kChunk; q += kChunkThreads) {
    out_k[(int64_t)m * Npad + base + q] = sk[q];
    out_i[(int64_t)m * Npad + base + q] = si[q];
  }
  if (out_p && m < pfx_dims) {
    // exclusive prefix of the P flags over the sorted chunk
    const int lane = t & 31, warp = t >> 5;
    uint32_t f[E], v = 0;
#pragma unroll
    for (int j = 0; j < E; ++j) { f[j] = ix[j] < (uint64_t)NP ? 1u : 0u; v += f[j]; }
    uint32_t incl = v;
    for (int off = 1; off < 32; off <<= 1) {
      const uint32_t x = __shfl_up_sync(0xffffffffu, incl, off);
      if (lane >= off) incl += x;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      const uint32_t w = lane < kChunkThreads / 32 ? wsum[lane] : 0u;
      uint32_t wi = w;
      for (int off = 1; off < 32; off <<= 1) {
        const uint32_t x = __shfl_up_sync(0xffffffffu, wi, off);
        if (lane >= off) wi += x;
      }
      if (lane < kChunkThreads / 32) wsum[lane] = wi - w;
    }
    __syncthreads();
    uint32_t ex = wsum[warp] + incl - v;
#pragma unroll
    for (int j = 0; j < E; ++j) { si[q0 + j] = ex; ex += f[j]; }  // si is free again after the copy above
    __syncthreads();
    uint32_t* Pout = out_p + (int64_t)m * Npad + base;
    for (int q = t; q < kChunk; q += kChunkThreads) Pout[q] = si[q];
  }
}

// One merge pass over runs of length L (a multiple of kChunk; Npad a multiple
// of kChunk): grid (Npad / kChunk, d), CTA (x, m) writes sorted positions
// [x * kChunk, (x + 1) * kChunk) of dimension m.  Its pair of runs A, B; the
// merge-path search gives a0 = the number of A elements among the first D
// outputs of the pair; the CTA stages A[a0, a1) and B[b0, b1) in shared
// memory, then each thread merges kMergeEach outputs from its own merge-path
// split.  With in_p / out_p, dimensions m < pfx_dims also carry each element's
// count of P points (index < NP) before it: preA(i) + preB(j) for the i A and
// j B elements that precede it, preX(p) being X's carried count at p (for p at
// the end of X: the last count plus the last element's flag).
constexpr int kMergeEach = 8;  // outputs per thread

// Outputs per merge CTA: 1024 for small inputs (twice the CTAs, half the
// latency chain each), 2048 otherwise.
int merge_tile_for(int64_t N) { return N <= 131072 ? 1024 : 2048; }

DDKS_DEV int64_t merge_path(const uint64_t* Ak, const uint32_t* Ai, int64_t na, const uint64_t* Bk,
                            const uint32_t* Bi, int64_t nb, int64_t D) {
  int64_t lo = D > nb ? D - nb : 0, hi = D < na ? D : na;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (pair_less(Ak[mid], Ai[mid], Bk[D - 1 - mid], Bi[D - 1 - mid])) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// With rank (the last pass, whose pair of runs is the whole dimension) the
// CTA writes no merged arrays: each output p < N gives rank[m][index] = its
// min-rank (the position of the first equal key: p itself when the key
// differs from the previous output, found for each thread's first output by
// lower_bound in both runs), and for dimension 0 sorted_idx0[p] = index and
// pprefix0[p] = the carried P count.
// The same search by a whole warp: 32 probes per round (the answer a is the
// first index at which A[a] < B[D-1-a] fails), so a run of 2^k elements
// takes about k / 5 rounds of dependent global loads instead of k.
DDKS_DEV int64_t merge_path_warp(const uint64_t* Ak, const uint32_t* Ai, int64_t na, const uint64_t* Bk,
                                 const uint32_t* Bi, int64_t nb, int64_t D) {
  const int lane = threadIdx.x & 31;
  int64_t lo = D > nb ? D - nb : 0, hi = D < na ? D : na;
  while (lo < hi) {
    const int64_t step = (hi - lo) / 32 + 1;
    const int64_t c = lo + lane * step;
    const bool past = c >= hi || !pair_less(Ak[c], Ai[c], Bk[D - 1 - c], Bi[D - 1 - c]);  // answer <= c
    const unsigned bal = __ballot_sync(0xffffffffu, past);
    const int f = __ffs(bal) - 1;
    if (f < 0) {
      lo = lo + 31 * step + 1;
    } else if (f == 0) {
      hi = lo;
    } else {
      const int64_t cf = lo + f * step;
      lo = lo + (f - 1) * step + 1;
      hi = cf < hi ? cf : hi;
    }
  }
  return lo;
}

template <int TILE>
__global__ void __launch_bounds__(TILE / kMergeEach)
k_merge_tile(const uint64_t* __restrict__ in_k, const uint32_t* __restrict__ in_i,
             uint64_t* __restrict__ out_k, uint32_t* __restrict__ out_i,
             const uint32_t* __restrict__ in_p, uint32_t* __restrict__ out_p,
             int64_t Npad, int64_t NP, int64_t L, int pfx_dims, int64_t N, uint32_t* __restrict__ rank,
             uint32_t* __restrict__ sorted_idx0, uint32_t* __restrict__ pprefix0) {
  constexpr int kChunk = TILE;  // outputs of this CTA (runs stay multiples of the 2048-element chunks)
  __shared__ uint64_t sk[kChunk];
  __shared__ uint32_t si[kChunk];
  __shared__ uint32_t sp[kChunk + 2];
  __shared__ int64_t s_a0, s_a1;
  const int64_t m = blockIdx.y;
  const int64_t pos0 = (int64_t)blockIdx.x * kChunk;
  const uint64_t* K = in_k + m * Npad;
  const uint32_t* I = in_i + m * Npad;
  const bool carry = in_p && m < pfx_dims;
  const uint32_t* Pin = carry ? in_p + m * Npad : nullptr;
  const int64_t run0 = (pos0 / (2 * L)) * (2 * L);
  const int64_t na = (Npad - run0) < L ? (Npad - run0) : L;
  const int64_t bS = run0 + L;
  const int64_t nb = bS >= Npad ? 0 : ((Npad - bS) < L ? (Npad - bS) : L);
  if (nb == 0) {  // no partner: the run is already in place
    for (int t = threadIdx.x; t < kChunk; t += blockDim.x) {
      const int64_t p = pos0 + t;
      out_k[m * Npad + p] = K[p];
      out_i[m * Npad + p] = I[p];
      if (carry) out_p[m * Npad + p] = Pin[p];
    }
    return;
  }
  const uint64_t *Ak = K + run0, *Bk = K + bS;
  const uint32_t *Ai = I + run0, *Bi = I + bS;
  const int64_t D0 = pos0 - run0, D1 = D0 + kChunk;  // runs are multiples of kChunk
  if (threadIdx.x < 32) {
    const int64_t a = merge_path_warp(Ak, Ai, na, Bk, Bi, nb, D0);
    if (threadIdx.x == 0) s_a0 = a;
  } else if (threadIdx.x < 64) {
    const int64_t a = merge_path_warp(Ak, Ai, na, Bk, Bi, nb, D1);
    if (threadIdx.x == 32) s_a1 = a;
  }
  __syncthreads();
  const int64_t a0 = s_a0, a1 = s_a1, b0 = D0 - a0, b1 = D1 - a1;
  const int nA = (int)(a1 - a0), nB = (int)(b1 - b0);
  for (int t = threadIdx.x; t < kChunk; t += blockDim.x) {
    if (t < nA) { sk[t] = Ak[a0 + t]; si[t] = Ai[a0 + t]; }
    else { sk[t] = Bk[b0 + t - nA]; si[t] = Bi[b0 + t - nA]; }
  }
  // carried counts: sp[0..nA] = preA(a0 .. a1), sp[nA+1 .. nA+1+nB] = preB(b0 .. b1)
  if (carry) {
    const uint32_t* PA = Pin + run0;
    const uint32_t* PB = Pin + bS;
    for (int t = threadIdx.x; t < kChunk + 2; t += blockDim.x) {
      uint32_t v;
      if (t <= nA) {
        const int64_t p = a0 + t;
        v = p < na ? PA[p] : PA[na - 1] + (Ai[na - 1] < (uint64_t)NP ? 1u : 0u);
      } else {
        const int64_t p = b0 + (t - nA - 1);
        v = p < nb ? PB[p] : PB[nb - 1] + (Bi[nb - 1] < (uint64_t)NP ? 1u : 0u);
      }
      sp[t] = v;
    }
  }
  __syncthreads();
  const uint64_t *sAk = sk, *sBk = sk + nA;
  const uint32_t *sAi = si, *sBi = si + nA;
  const int d0 = threadIdx.x * kMergeEach;
  int i = (int)merge_path(sAk, sAi, nA, sBk, sBi, nB, d0);
  int j = d0 - i;
  // the heads of both runs stay in registers: each output loads only the
  // successor on the side it took; the carried P counts advance by the
  // taken element's flag (preX(p + 1) = preX(p) + [X_p is a P point])
  uint64_t ka = i < nA ? sAk[i] : 0ull, kb = j < nB ? sBk[j] : 0ull;
  uint32_t ia = i < nA ? sAi[i] : 0u, ib = j < nB ? sBi[j] : 0u;
  uint32_t pa = carry ? sp[i] : 0u, pb = carry ? sp[nA + 1 + j] : 0u;
  if (rank) {
    const int64_t p0 = pos0 + d0;
    const uint64_t first = (i < nA && (j >= nB || pair_less(sAk[i], sAi[i], sBk[j], sBi[j]))) ? sAk[i] : sBk[j];
    // #{keys < first} in the two runs: the min-rank of the first output
    int64_t lo = 0, hi = na;
    while (lo < hi) { const int64_t mid = (lo + hi) >> 1; if (Ak[mid] < first) lo = mid + 1; else hi = mid; }
    int64_t r = lo;
    lo = 0; hi = nb;
    while (lo < hi) { const int64_t mid = (lo + hi) >> 1; if (Bk[mid] < first) lo = mid + 1; else hi = mid; }
    r += lo;
    uint64_t prev = first;
    uint32_t* R = rank + m * N;
#pragma unroll
    for (int e = 0; e < kMergeEach; ++e) {
      const int64_t p = p0 + e;
      const bool takeA = j >= nB || (i < nA && pair_less(ka, ia, kb, ib));
      const uint32_t pc = pa + pb;
      const uint64_t key = takeA ? ka : kb;
      const uint32_t idx = takeA ? ia : ib;
      const uint32_t isp = idx < (uint64_t)NP ? 1u : 0u;
      if (takeA) {
        ++i;
        pa += isp;
        if (i < nA) { ka = sAk[i]; ia = sAi[i]; }
      } else {
        ++j;
        pb += isp;
        if (j < nB) { kb = sBk[j]; ib = sBi[j]; }
      }
      if (key != prev) r = p;
      prev = key;
      if (p < N) {
        R[idx] = (uint32_t)r;
        if (m == 0 && sorted_idx0) {
          sorted_idx0[p] = idx;
          if (pprefix0) pprefix0[p] = pc;
        }
      }
    }
    return;
  }
  uint64_t ok[kMergeEach];
  uint32_t oi[kMergeEach], op[kMergeEach];
#pragma unroll
  for (int e = 0; e < kMergeEach; ++e) {
    const bool takeA = j >= nB || (i < nA && pair_less(ka, ia, kb, ib));
    op[e] = pa + pb;
    ok[e] = takeA ? ka : kb;
    oi[e] = takeA ? ia : ib;
    const uint32_t isp = oi[e] < (uint64_t)NP ? 1u : 0u;
    if (takeA) {
      ++i;
      pa += isp;
      if (i < nA) { ka = sAk[i]; ia = sAi[i]; }
    } else {
      ++j;
      pb += isp;
      if (j < nB) { kb = sBk[j]; ib = sBi[j]; }
    }
  }
  // through shared memory, so that the global stores are coalesced
  __syncthreads();
#pragma unroll
  for (int e = 0; e < kMergeEach; ++e) {
    sk[d0 + e] = ok[e];
    si[d0 + e] = oi[e];
    if (carry) sp[d0 + e] = op[e];
  }
  __syncthreads();
  uint64_t* Ok = out_k + m * Npad + pos0;
  uint32_t* Oi = out_i + m * Npad + pos0;
  for (int t = threadIdx.x; t < kChunk; t += blockDim.x) {
    Ok[t] = sk[t];
    Oi[t] = si[t];
    if (carry) out_p[m * Npad + pos0 + t] = sp[t];
  }
}

// With few sorted chunks: rank[m][i] = sum over chunks of #{keys < key_i}
// (one lower_bound per chunk), and for dimension 0 the position of (key_i, i)
// in the full sorted order, which places i in sorted_idx0.  The searches of up
// to 8 chunks advance together (independent loads in flight).
template <int CH>
__global__ void k_rank_multi(const uint64_t* __restrict__ keys, const uint64_t* __restrict__ ck,
                             const uint32_t* __restrict__ ci, const uint32_t* __restrict__ cpfx,
                             int64_t N, int64_t NPc, int64_t Npad, int d, uint32_t* __restrict__ rank,
                             uint32_t* __restrict__ sorted_idx0, uint32_t* __restrict__ pprefix0) {
  constexpr int kG = 8;
  constexpr int kChunk = CH;
  constexpr int kSteps = CH == 2048 ? 12 : 14;  // at most log2(CH) + 1 halvings
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
      for (int step = 0; step < kSteps; ++step) {
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
        for (int step = 0; step < kSteps; ++step) {
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

int grid_for(int64_t work, int threads) {
  int64_t g = (work + threads - 1) / threads;
  if (g > 152 * 64) g = 152 * 64;
  return (int)(g < 1 ? 1 : g);
}

}  // namespace

cudaError_t ddks_launch_encode(const void* P, const void* T, int64_t NP, int64_t NT, int d,
                               int is_f64, uint64_t* keys, unsigned* flags, cudaStream_t st) {
  const int64_t total = NP + NT;  // one thread per point
  const int threads = 256;
  if (is_f64)
    k_encode<double><<<grid_for(total, threads), threads, 0, st>>>(
        (const double*)P, (const double*)T, NP, NT, d, keys, flags);
  else
    k_encode<float><<<grid_for(total, threads), threads, 0, st>>>(
        (const float*)P, (const float*)T, NP, NT, d, keys, flags);
  return cudaGetLastError();
}

namespace {
// 2048-element chunks throughout: 8192-element chunks (one CTA of 1024
// threads each) measured slower on both the mid-size inputs (too few CTAs,
// searches of 14 steps) and the large ones (more sorting work per element).
int64_t chunk_for(int64_t) { return kChunk; }

cudaError_t launch_chunk_sort(int64_t CH, dim3 g, const uint64_t* keys, int64_t N, int64_t Npad, int64_t NP,
                              uint64_t* out_k, uint32_t* out_i, uint32_t* out_p, int pfx_dims, cudaStream_t st) {
  const size_t smem = (size_t)CH * 12;
  k_chunk_sort<kChunk, kSortEach><<<g, kChunk / kSortEach, smem, st>>>(keys, N, Npad, NP, out_k, out_i, out_p,
                                                                       pfx_dims);
  return cudaGetLastError();
}
}  // namespace

size_t ddks_rank_scratch_elems(int64_t N) {
  const int64_t CH = chunk_for(N);
  const int64_t chunks = (N + CH - 1) / CH;
  return (size_t)(chunks * CH);
}

// keys: [d][N].  tmp buffers: d * Npad elements each.  rank: [d][N].
// sorted_idx0 (optional): the pooled indices in increasing (rank_0, index) order.
// pprefix0 (optional, with sorted_idx0; u32 [N] plus 2 * ddks_rank_pfx_elems(N)
// of scratch at cpfx): pprefix0[p] = #{P points among sorted positions < p}.
size_t ddks_rank_pfx_elems(int64_t N) { return ddks_rank_scratch_elems(N); }

// With radix_scratch (ddks_radix_scratch_words(N, d, 1) words): the radix
// sort of radix.cu over the low key_bits of the keys replaces the chunk sort
// and merges; pprefix0 then needs no cpfx scratch, and *sorted_rows (if
// given) points at the pooled indices of every dimension in sorted order,
// [d][N] inside the tmp_idx buffers (nullptr on the merge path).
cudaError_t ddks_launch_rank(const uint64_t* keys, int64_t N, int64_t NP, int d, uint64_t* tmp_keys,
                             uint32_t* tmp_idx, uint64_t* tmp_keys2, uint32_t* tmp_idx2,
                             uint32_t* rank, uint32_t* sorted_idx0, uint32_t* pprefix0, uint32_t* cpfx,
                             int* pfx_done, cudaStream_t st, int* launches, int key_bits,
                             uint32_t* radix_scratch, const uint32_t** sorted_rows) {
  if (sorted_rows) *sorted_rows = nullptr;
  if (radix_scratch) {
    const bool pfx = sorted_idx0 && pprefix0;
    if (pfx_done) *pfx_done = pfx ? 1 : 0;
    const uint64_t* sk;
    const uint32_t* si;
    cudaError_t e = ddks_radix_sort(keys, tmp_keys, tmp_idx, tmp_keys2, tmp_idx2, N, N, d, key_bits, radix_scratch,
                                    &sk, &si, st, launches);
    if (e != cudaSuccess) return e;
    if (sorted_rows) *sorted_rows = si;
    return ddks_radix_ranks(sk, si, N, N, d, NP, rank, pfx ? pprefix0 : nullptr, 1, sorted_idx0, radix_scratch, st,
                            launches);
  }
  const int64_t Npad = (int64_t)ddks_rank_scratch_elems(N);
  const int64_t CH = chunk_for(N);
  const int64_t chunks = Npad / CH;
  const bool pfx = sorted_idx0 && pprefix0 && cpfx;
  if (pfx_done) *pfx_done = pfx ? 1 : 0;
  uint32_t* cp = pfx ? cpfx : nullptr;             // [Npad] P prefixes, dimension 0
  uint32_t* cp2 = pfx ? cpfx + Npad : nullptr;     // [Npad] the other merge buffer
  cudaError_t e = launch_chunk_sort(CH, dim3((unsigned)chunks, (unsigned)d), keys, N, Npad, NP, tmp_keys, tmp_idx,
                                    cp, 1, st);
  if (e != cudaSuccess) return e;
  int n = 1;
  if (chunks <= kMaxMultiChunks) {
    k_rank_multi<kChunk><<<grid_for(N * d, 256), 256, 0, st>>>(keys, tmp_keys, tmp_idx, cp, N, NP, Npad, d, rank,
                                                               sorted_idx0, pfx ? pprefix0 : nullptr);
    if (launches) *launches += 2;
    return cudaGetLastError();
  }
  const int TILE = merge_tile_for(N);
  const int64_t tiles = Npad / TILE;
  uint64_t *ck = tmp_keys, *nk = tmp_keys2;
  uint32_t *ci = tmp_idx, *ni = tmp_idx2;
  for (int64_t L = CH; L < Npad; L <<= 1) {
    const bool last = 2 * L >= Npad;  // the final pass writes ranks instead of merged arrays
    if (TILE == 1024)
      k_merge_tile<1024><<<dim3((unsigned)tiles, (unsigned)d), 1024 / kMergeEach, 0, st>>>(
          ck, ci, nk, ni, cp, cp2, Npad, NP, L, 1, N, last ? rank : nullptr, last ? sorted_idx0 : nullptr,
          last && pfx ? pprefix0 : nullptr);
    else
      k_merge_tile<2048><<<dim3((unsigned)tiles, (unsigned)d), 2048 / kMergeEach, 0, st>>>(
          ck, ci, nk, ni, cp, cp2, Npad, NP, L, 1, N, last ? rank : nullptr, last ? sorted_idx0 : nullptr,
          last && pfx ? pprefix0 : nullptr);
    ++n;
    uint64_t* tk = ck; ck = nk; nk = tk;
    uint32_t* ti = ci; ci = ni; ni = ti;
    uint32_t* tp = cp; cp = cp2; cp2 = tp;
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
  const int64_t CH = chunk_for(N);
  cudaError_t e = launch_chunk_sort(CH, dim3((unsigned)(Npad / CH), (unsigned)S), keys, N, Npad, NP, k1, i1, p1, S,
                                    st);
  if (e != cudaSuccess) return e;
  int n = 1;
  const int TILE = merge_tile_for(N);
  const int64_t tiles = Npad / TILE;
  uint64_t *ck = k1, *nk = k2;
  uint32_t *ci = i1, *ni = i2, *cp = p1, *np = p2;
  for (int64_t L = CH; L < Npad; L <<= 1) {
    if (TILE == 1024)
      k_merge_tile<1024><<<dim3((unsigned)tiles, (unsigned)S), 1024 / kMergeEach, 0, st>>>(
          ck, ci, nk, ni, cp, np, Npad, NP, L, S, N, nullptr, nullptr, nullptr);
    else
      k_merge_tile<2048><<<dim3((unsigned)tiles, (unsigned)S), 2048 / kMergeEach, 0, st>>>(
          ck, ci, nk, ni, cp, np, Npad, NP, L, S, N, nullptr, nullptr, nullptr);
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
