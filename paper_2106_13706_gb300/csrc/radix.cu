// radix.cu -- stable LSD radix sort of rows of 64-bit order keys with their
// positions, and what the exact and rdKS paths need from a sorted row: each
// element's min-rank (the first sorted position of its key) and the count of
// P points (pooled index < NP) before each sorted position.
//
// One pass per 8-bit digit, lowest first: k_radix_hist counts the digits of
// each tile of 2048 consecutive elements; a scan of each digit's counts over
// the tiles plus a scan of the digit totals gives every (digit, tile) pair
// its first output position; k_radix_scatter ranks its tile stably by the digit
// (warp-level match of equal digits, per-warp digit counters in shared
// memory), places the tile in digit order in shared memory and writes each
// digit's run to its output range.  Stable inside tiles and across them, so
// after the last pass every row is sorted by key with ties in input order
// (the pooled index, as the inputs carry their positions).
//
// k_radix_rank_tiles turns sorted rows into min-ranks: a position starts a
// run when its key differs from its left neighbour, and the run start of a
// position is the last run start at or before it (a running maximum), seeded
// per tile by a binary search when the tile opens inside a run.  The P counts
// before each position are per-tile prefixes of ballot counts plus the sum of
// the earlier tiles' totals (k_radix_pfx_carry).
#include <cstdint>

#include "ddks_internal.cuh"

namespace {

constexpr int kRT = 256;             // threads per CTA (8 warps)
constexpr int kRW = kRT / 32;
constexpr int kRI = 8;               // elements per thread of the rank kernel
constexpr int kRTile = kRT * kRI;    // 2048 positions per rank tile
constexpr int64_t kSelfScanTiles = 128;  // up to here the scatter CTAs sum the counts themselves

DDKS_DEV uint32_t digit_of(uint64_t k, int shift) { return (uint32_t)(k >> shift) & 255u; }

// exclusive prefix sum over the CTA's threads; ws: kRW words
DDKS_DEV uint32_t block_exscan(uint32_t v, uint32_t* ws) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t incl = v;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const uint32_t x = __shfl_up_sync(0xffffffffu, incl, off);
    if (lane >= off) incl += x;
  }
  if (lane == 31) ws[warp] = incl;
  __syncthreads();
  uint32_t carry = 0;
  for (int q = 0; q < warp; ++q) carry += ws[q];
  __syncthreads();  // ws is free again on return
  return carry + incl - v;
}

// cnt[(row * 256 + digit) * tiles + tile] = elements of the tile with that
// digit.  Lanes with equal digits add once per group (high key bytes take
// few values, and same-address shared atomics serialise).
template <int RI>
__global__ void __launch_bounds__(kRT)
k_radix_hist(const uint64_t* __restrict__ keys, int64_t n, int64_t stride, int shift, int64_t tiles,
             uint32_t* __restrict__ cnt) {
  constexpr int kTile = kRT * RI;
  __shared__ uint32_t h[256];
  const int64_t row = blockIdx.y, tile = blockIdx.x;
  const int lane = threadIdx.x & 31;
  h[threadIdx.x] = 0;
  __syncthreads();
  const uint64_t* K = keys + row * stride + tile * kTile;
  const int64_t nv = n - tile * kTile;
  uint64_t k[RI];
#pragma unroll
  for (int j = 0; j < RI; ++j) {
    const int64_t e = j * kRT + threadIdx.x;
    k[j] = e < nv ? K[e] : 0ull;
  }
#pragma unroll
  for (int j = 0; j < RI; ++j) {
    const bool v = j * kRT + (int64_t)threadIdx.x < nv;
    const uint32_t dg = digit_of(k[j], shift);
    const uint32_t vary = __reduce_or_sync(0xffffffffu, dg) ^ __reduce_and_sync(0xffffffffu, dg);
    if (__popc(vary) >= 6) {  // many distinct digits in the warp: few collisions, one add per lane
      if (v) atomicAdd(&h[dg], 1u);
    } else {  // few distinct digits: one add per group of equal digits
      const uint32_t vm = __ballot_sync(0xffffffffu, v);
      const uint32_t peers = ddks::same_digit(dg) & vm;
      if (v && (peers >> lane) == 1u) atomicAdd(&h[dg], (uint32_t)__popc(peers));
    }
  }
  __syncthreads();
  cnt[((size_t)row * 256 + threadIdx.x) * tiles + tile] = h[threadIdx.x];
}

// Grid (256, rows): CTA (digit, row) turns the digit's tile counts into
// exclusive prefixes over the tiles (off) and the row's digit total (tot).
__global__ void __launch_bounds__(kRT)
k_radix_tile_scan(const uint32_t* __restrict__ cnt, int64_t tiles, uint32_t* __restrict__ off,
                  uint32_t* __restrict__ tot) {
  __shared__ uint32_t ws[kRW];
  const size_t rd = (size_t)blockIdx.y * 256 + blockIdx.x;
  const uint32_t* C = cnt + rd * tiles;
  uint32_t* O = off + rd * tiles;
  uint32_t carry = 0;
  for (int64_t b0 = 0; b0 < tiles; b0 += 4 * kRT) {
    uint32_t c[4], s = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t q = b0 + 4 * threadIdx.x + j;
      c[j] = q < tiles ? C[q] : 0u;
      s += c[j];
    }
    const uint32_t ex = block_exscan(s, ws);
    uint32_t run = carry + ex;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t q = b0 + 4 * threadIdx.x + j;
      if (q < tiles) O[q] = run;
      run += c[j];
    }
    // the chunk's total: the last thread's exclusive prefix plus its sum
    if (threadIdx.x == kRT - 1) ws[0] = ex + s;
    __syncthreads();
    carry += ws[0];
    __syncthreads();
  }
  if (threadIdx.x == 0) tot[rd] = carry;
}

// One digit pass, in -> out.  in_i == nullptr: the input indices are the
// positions.  off / tot: k_radix_tile_scan of this pass's counts cnt, or
// nullptr to have every CTA sum the counts of its row itself (few tiles).
template <int RI>
__global__ void __launch_bounds__(kRT, 4)
k_radix_scatter(const uint64_t* __restrict__ in_k, const uint32_t* __restrict__ in_i, uint64_t* __restrict__ out_k,
                uint32_t* __restrict__ out_i, int64_t n, int64_t stride, int shift, int64_t tiles,
                const uint32_t* __restrict__ cnt, const uint32_t* __restrict__ off, const uint32_t* __restrict__ tot) {
  constexpr int kTile = kRT * RI;
  __shared__ uint64_t sk[kTile];
  __shared__ uint32_t si[kTile];
  __shared__ uint32_t wcnt[kRW][256];
  __shared__ uint32_t soff[256], sbeg[256];
  __shared__ uint32_t ws[kRW];
  const int64_t row = blockIdx.y, tile = blockIdx.x;
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int64_t base = tile * kTile;
  const int nvalid = (int)(n - base < kTile ? n - base : kTile);
  const uint64_t* K = in_k + row * stride + base;
  const uint32_t* I = in_i ? in_i + row * stride + base : nullptr;
  uint32_t gpre = 0, gtot = 0;  // digit t before this tile / in the whole row
  if (off) {
    gpre = off[((size_t)row * 256 + t) * tiles + tile];
    gtot = tot[(size_t)row * 256 + t];
  } else {
    const uint32_t* C = cnt + ((size_t)row * 256 + t) * tiles;
#pragma unroll 8
    for (int64_t q = 0; q < tiles; ++q) {
      const uint32_t c = C[q];
      gpre += q < tile ? c : 0u;
      gtot += c;
    }
  }
#pragma unroll
  for (int q = 0; q < kRW; ++q) wcnt[q][t] = 0;
  // Warp-striped positions: element j of lane l in warp w sits at
  // w*32*RI + j*32 + l, so ranking in (j, lane) order within a warp and the
  // warps in order is stable.  Positions past the row's end take the largest
  // key (digit 255, ranked after every element of the tile).
  uint64_t k[RI];
  uint32_t ix[RI], r[RI];
#pragma unroll
  for (int j = 0; j < RI; ++j) {
    const int q = w * (RI * 32) + j * 32 + lane;
    const bool v = q < nvalid;
    k[j] = v ? K[q] : ~0ull;
    ix[j] = v ? (I ? I[q] : (uint32_t)(base + q)) : 0u;
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < RI; ++j) {
    const uint32_t dg = digit_of(k[j], shift);
    const uint32_t peers = ddks::same_digit(dg);
    r[j] = wcnt[w][dg] + (uint32_t)__popc(peers & ((1u << lane) - 1u));
    __syncwarp();
    if ((peers >> lane) == 1u) wcnt[w][dg] += (uint32_t)__popc(peers);  // the group's highest lane
    __syncwarp();
  }
  __syncthreads();
  // thread t owns digit t: first the warps' offsets inside the digit, then
  // the digit's offset inside the tile
  uint32_t dsum = 0;
#pragma unroll
  for (int q = 0; q < kRW; ++q) {
    const uint32_t c = wcnt[q][t];
    wcnt[q][t] = dsum;
    dsum += c;
  }
  const uint32_t dbeg = block_exscan(dsum, ws);
  sbeg[t] = dbeg;
  soff[t] = block_exscan(gtot, ws) + gpre;
#pragma unroll
  for (int q = 0; q < kRW; ++q) wcnt[q][t] += dbeg;
  __syncthreads();
#pragma unroll
  for (int j = 0; j < RI; ++j) {
    const uint32_t lr = wcnt[w][digit_of(k[j], shift)] + r[j];
    sk[lr] = k[j];
    si[lr] = ix[j];
  }
  __syncthreads();
  uint64_t* OK = out_k + row * stride;
  uint32_t* OI = out_i + row * stride;
  for (int q = t; q < nvalid; q += kRT) {
    const uint64_t kk = sk[q];
    const uint32_t dg = digit_of(kk, shift);
    const uint32_t dst = soff[dg] + (uint32_t)q - sbeg[dg];
    OK[dst] = kk;
    OI[dst] = si[q];
  }
}

// Min-ranks from sorted rows: rank[row][idx(p)] = first position of key(p)
// (rank may be nullptr); rows below pfx_rows also get pfx[row][p] = P points
// (idx < NP) before position p within the tile and tp[row][tile] = the
// tile's P points (k_radix_pfx_carry adds the earlier tiles' counts); with
// sorted_idx0, row 0 gets sorted_idx0[p] = idx(p).  Positions are visited
// warp-coalesced: segment s = j * 8 + warp covers the 32 positions
// s * 32 + lane of the tile, in increasing order of s.
__global__ void __launch_bounds__(kRT)
k_radix_rank_tiles(const uint64_t* __restrict__ sk, const uint32_t* __restrict__ si, int64_t n, int64_t stride,
                   int64_t NP, uint32_t* __restrict__ rank, uint32_t* __restrict__ pfx, uint32_t* __restrict__ tp,
                   int64_t pfx_rows, uint32_t* __restrict__ sorted_idx0) {
  constexpr int kSeg = kRI * kRW;      // 64 segments of 32 positions
  __shared__ uint64_t kt[kRTile + 1];  // kt[q + 1] = key at base + q, kt[0] = key at base - 1
  __shared__ uint32_t seg_pre[kSeg];   // last run start up to the end of each segment
  __shared__ uint32_t seg_p[kSeg];     // P points before each segment (within the tile)
  __shared__ uint32_t seed_s;
  const int64_t row = blockIdx.y, tile = blockIdx.x;
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int64_t base = tile * kRTile;
  const int nvalid = (int)(n - base < kRTile ? n - base : kRTile);
  const uint64_t* K = sk + row * stride;
  const uint32_t* I = si + row * stride;
  const bool want_rank = rank != nullptr;  // without ranks the keys are not read
  if (want_rank)
    for (int q = t; q < nvalid; q += kRT) kt[q + 1] = K[base + q];
  if (t == 0 && want_rank) {
    // the run start of the tile's first key: base unless the run began before
    int64_t lo = base;
    if (base > 0) {
      const uint64_t key = K[base], left = K[base - 1];
      kt[0] = left;
      if (left == key) {
        int64_t hi = base - 1;  // K[hi] == key: the lower bound lies in [0, hi]
        lo = 0;
        while (lo < hi) {
          const int64_t mid = (lo + hi) >> 1;
          if (K[mid] < key) lo = mid + 1; else hi = mid;
        }
      }
    }
    seed_s = (uint32_t)lo;
  }
  __syncthreads();
  uint32_t hm[kRI];  // run-start lanes of segment j * 8 + w
#pragma unroll
  for (int j = 0; j < kRI; ++j) {
    const int q = j * kRT + t;
    const bool head = want_rank && q < nvalid && (base + q == 0 || kt[q + 1] != kt[q]);
    hm[j] = __ballot_sync(0xffffffffu, head);
    if (lane == 0) seg_pre[j * kRW + w] = hm[j] ? (uint32_t)(base + j * kRT + w * 32 + 31 - __clz(hm[j])) : 0u;
  }
  __syncthreads();
  if (w == 0 && want_rank) {  // running maximum over the 64 segments, seeded
    uint32_t a = seg_pre[2 * lane], b = seg_pre[2 * lane + 1];
    a = a > seed_s ? a : seed_s;
    b = b > a ? b : a;
    uint32_t incl = b;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const uint32_t x = __shfl_up_sync(0xffffffffu, incl, off);
      if (lane >= off) incl = x > incl ? x : incl;
    }
    const uint32_t ex = __shfl_up_sync(0xffffffffu, incl, 1);
    const uint32_t before = lane ? (ex > seed_s ? ex : seed_s) : seed_s;
    seg_pre[2 * lane] = a > before ? a : before;
    seg_pre[2 * lane + 1] = incl;
  }
  __syncthreads();
  const uint32_t lt = lane == 31 ? 0xffffffffu : ((2u << lane) - 1u);  // lanes <= this one
  const bool pf = row < pfx_rows;
  const bool s0 = row == 0 && sorted_idx0 != nullptr;
  uint32_t ix[kRI], pm[kRI];
#pragma unroll
  for (int j = 0; j < kRI; ++j) {
    const int q = j * kRT + t;
    ix[j] = q < nvalid ? I[base + q] : 0u;
    pm[j] = __ballot_sync(0xffffffffu, q < nvalid && (uint64_t)ix[j] < (uint64_t)NP);
    if (pf && lane == 0) seg_p[j * kRW + w] = (uint32_t)__popc(pm[j]);
  }
  if (pf) {
    __syncthreads();
    if (w == 0) {  // exclusive sums over the 64 segments; the tile's total to tp
      const uint32_t a = seg_p[2 * lane], b = seg_p[2 * lane + 1];
      uint32_t incl = a + b;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const uint32_t x = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += x;
      }
      const uint32_t ex = incl - a - b;
      seg_p[2 * lane] = ex;
      seg_p[2 * lane + 1] = ex + a;
      if (lane == 31) tp[row * gridDim.x + tile] = incl;
    }
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < kRI; ++j) {
    const int q = j * kRT + t;
    if (q < nvalid) {
      const int sg = j * kRW + w;
      const uint32_t m = hm[j] & lt;
      const uint32_t rs = m ? (uint32_t)(base + j * kRT + w * 32 + 31 - __clz(m))
                            : (sg ? seg_pre[sg - 1] : seed_s);
      const uint32_t i = ix[j];
      if (rank) rank[row * n + i] = rs;
      if (pf) pfx[row * n + base + q] = seg_p[sg] + (uint32_t)__popc(pm[j] & (lt >> 1));
      if (s0) sorted_idx0[base + q] = i;
    }
  }
}

// Grid (tiles, pfx_rows): adds the P points of the row's earlier tiles to the
// tile's in-tile prefixes.
__global__ void __launch_bounds__(kRT)
k_radix_pfx_carry(uint32_t* __restrict__ pfx, const uint32_t* __restrict__ tp, int64_t n) {
  __shared__ uint32_t ws[kRW];
  const int64_t row = blockIdx.y, tile = blockIdx.x;
  if (tile == 0) return;
  const uint32_t* TP = tp + row * gridDim.x;
  uint32_t c = 0;
  for (int64_t q = threadIdx.x; q < tile; q += kRT) c += TP[q];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) c += __shfl_xor_sync(0xffffffffu, c, off);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = c;
  __syncthreads();
  uint32_t carry = 0;
#pragma unroll
  for (int q = 0; q < kRW; ++q) carry += ws[q];
  const int64_t base = tile * kRTile;
  const int nvalid = (int)(n - base < kRTile ? n - base : kRTile);
  uint32_t* Pr = pfx + row * n + base;
  for (int q = threadIdx.x; q < nvalid; q += kRT) Pr[q] += carry;
}

}  // namespace

namespace {
// Elements per thread of the sort passes: 8 (2048-element tiles), or 2 for
// sorts of under about 38 such tiles, which then spread over more SMs.
// (4-element tiles measured slower than 8 for 40k-200k keys per row: the
// per-CTA fixed work outweighs the extra parallelism.)
int sort_ri(int64_t n, int64_t rows) {
  const int64_t t8 = rows * ((n + 2047) / 2048);
  return t8 >= 38 ? 8 : 2;
}
}  // namespace

size_t ddks_radix_scratch_words(int64_t n, int64_t rows, int64_t pfx_rows) {
  const int64_t tiles = (n + kRT * 2 - 1) / (kRT * 2);  // the smallest sort tile
  const size_t cnt = (size_t)rows * 256 * (size_t)tiles;
  const size_t a = 2 * cnt + (size_t)rows * 256;
  const size_t b = (size_t)pfx_rows * (size_t)((n + kRTile - 1) / kRTile);
  return a > b ? a : b;
}

// Sorts rows of n keys (row r at keys + r * stride) by their low nbits (a
// multiple of 8, at most 64), each key carrying its position in the row.
// Passes alternate between (ka, ia) and (kb, ib), [rows][stride] each, and
// *out_k / *out_i point at the pair holding the result.  scratch:
// ddks_radix_scratch_words(n, rows, .) words.
cudaError_t ddks_radix_sort(const uint64_t* keys, uint64_t* ka, uint32_t* ia, uint64_t* kb, uint32_t* ib, int64_t n,
                            int64_t stride, int64_t rows, int nbits, uint32_t* scratch, const uint64_t** out_k,
                            const uint32_t** out_i, cudaStream_t st, int* launches) {
  if (n <= 0 || rows <= 0 || rows > 65535 || nbits <= 0 || nbits > 64 || nbits % 8 || n > 0xFFFFFFFFll)
    return cudaErrorInvalidValue;
  const int RI = sort_ri(n, rows);
  const int64_t tiles = (n + kRT * RI - 1) / (kRT * RI);
  const size_t ncnt = (size_t)rows * 256 * (size_t)tiles;
  uint32_t* cnt = scratch;
  uint32_t* off = scratch + ncnt;
  uint32_t* tot = off + ncnt;
  const dim3 g((unsigned)tiles, (unsigned)rows);
  const bool self_scan = tiles <= kSelfScanTiles;
  const uint64_t* ck = keys;
  const uint32_t* ci = nullptr;
  uint64_t* dk = ka;
  uint32_t* di = ia;
  int nl = 0;
  for (int shift = 0; shift < nbits; shift += 8) {
    if (RI == 8) k_radix_hist<8><<<g, kRT, 0, st>>>(ck, n, stride, shift, tiles, cnt);
    else k_radix_hist<2><<<g, kRT, 0, st>>>(ck, n, stride, shift, tiles, cnt);
    if (!self_scan) {
      k_radix_tile_scan<<<dim3(256, (unsigned)rows), kRT, 0, st>>>(cnt, tiles, off, tot);
      ++nl;
    }
    const uint32_t* o = self_scan ? nullptr : off;
    if (RI == 8) k_radix_scatter<8><<<g, kRT, 0, st>>>(ck, ci, dk, di, n, stride, shift, tiles, cnt, o, tot);
    else k_radix_scatter<2><<<g, kRT, 0, st>>>(ck, ci, dk, di, n, stride, shift, tiles, cnt, o, tot);
    nl += 2;
    ck = dk;
    ci = di;
    dk = dk == ka ? kb : ka;
    di = di == ia ? ib : ia;
  }
  *out_k = ck;
  *out_i = ci;
  if (launches) *launches += nl;
  return cudaGetLastError();
}

// From sorted rows (sk, si; [rows][stride]): rank[row][i] = min-rank of
// element i, [rows][n] (rank may be nullptr); pfx[row][p] = P points (index
// < NP) before sorted position p for rows [0, pfx_rows), [pfx_rows][n] (pfx
// may be nullptr); sorted_idx0[p] = the index at sorted position p of row 0
// (may be nullptr).  scratch as for the sort, with pfx_rows.
cudaError_t ddks_radix_ranks(const uint64_t* sk, const uint32_t* si, int64_t n, int64_t stride, int64_t rows,
                             int64_t NP, uint32_t* rank, uint32_t* pfx, int64_t pfx_rows, uint32_t* sorted_idx0,
                             uint32_t* scratch, cudaStream_t st, int* launches) {
  if (n <= 0 || rows <= 0 || rows > 65535) return cudaErrorInvalidValue;
  const int64_t tiles = (n + kRTile - 1) / kRTile;
  if (!pfx) pfx_rows = 0;
  uint32_t* tp = scratch;  // [pfx_rows][tiles] P points per tile
  k_radix_rank_tiles<<<dim3((unsigned)tiles, (unsigned)rows), kRT, 0, st>>>(sk, si, n, stride, NP, rank, pfx, tp,
                                                                             pfx_rows, sorted_idx0);
  int nl = 1;
  if (pfx_rows > 0 && tiles > 1) {
    k_radix_pfx_carry<<<dim3((unsigned)tiles, (unsigned)pfx_rows), kRT, 0, st>>>(pfx, tp, n);
    ++nl;
  }
  if (launches) *launches += nl;
  return cudaGetLastError();
}
