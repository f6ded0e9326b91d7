// dominance.cu -- exact ddKS for d = 2 in O(N log N) work (DDKS_PATH_DOMINANCE).
//
// Not in the paper: a sub-quadratic restatement of the same statistic
// (Eq. ddks_tensor_definition with the ">=" split of Eq. g) that skips the
// pairwise compares.  With min-ranks (K0), a point x is on the upper side of
// origin o in dimension m iff rank_m(x) >= rank_m(o).  In the order of
// dimension 0 (K0's sorted_idx0), the points with x_0 >= o_0 are exactly the
// positions >= rank_0(o), so the upper-upper count of a sample is a range
// query: #{positions k >= rank_0(o) : y(k) >= rank_1(o)}, y(k) the
// dimension-1 rank of the point at position k.  The other three quadrants
// follow from the marginals: #{x_0 >= o_0} = N - rank_0(o) (its P part from
// K0's P prefix at that position), #{x_1 >= o_1} = N - rank_1(o) (its P part
// from a histogram of the P points' y ranks).
//
// The range queries run on two wavelet matrices (the wavelet tree variant of
// Information Systems 47, 2015) over a 4-letter alphabet: one over the y
// ranks of all points in dimension-0 order, one over the P points only.
// Level l of a matrix holds the 2-bit symbol (bits 2(LL-1-l) and up) of
// every position as two bit planes, per 32 positions the counts of symbols
// >= 1, >= 2, >= 3 before them, and the next level's order: a stable
// partition by symbol.  A query walks the LL = ceil(L/2) levels with two
// record lookups each (16 bytes: both planes and three 16-bit counts
// relative to a superblock of 65,536 positions, whose bases sit in shared
// memory), half the levels of the binary matrix.  Build: per level a bit
// kernel (warp ballots; counts within 8,192-position chunks), a scan of the
// chunk totals and a scatter kernel; a finalize pass makes the counts
// superblock-relative; query: one thread per origin.
#include <cstring>

#include "../../include/ddks.h"
#include "ddks_host.h"
#include "ddks_internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kScanThreads = 1024;
constexpr int kMaxLevels = 16;         // 2-bit levels: ranks below 2^32
constexpr int kChunkWords = 256;       // words per chunk (8192 positions), one CTA of k_quad_bits
constexpr int kChunkShift = 13;
constexpr int kSBChunks = 8;           // chunks per superblock (65536 positions)
constexpr int kSBShift = 16;
constexpr int kSmemBases = 2048;       // superblock bases held in shared memory by the query (uint4 each)

// Ranks at position k from record r (word k / 32) and superblock base s:
// g[c] = #{positions < k with symbol >= c}, c = 0..4 (g[0] = k, g[4] = 0).
struct Ge {
  uint32_t g1, g2, g3;
};
DDKS_DEV Ge ranks_at(uint4 r, uint4 s, uint32_t k) {
  const uint32_t b = k & 31;
  const uint32_t below = b ? ((1u << b) - 1u) : 0u;
  Ge o;
  o.g1 = s.x + (r.z & 0xFFFFu) + (uint32_t)__popc((r.x | r.y) & below);
  o.g2 = s.y + (r.z >> 16) + (uint32_t)__popc(r.y & below);
  o.g3 = s.z + r.w + (uint32_t)__popc((r.x & r.y) & below);
  return o;
}
DDKS_DEV uint32_t ge_pick(const Ge& g, uint32_t k, uint32_t c) {
  return c == 0 ? k : c == 1 ? g.g1 : c == 2 ? g.g2 : c == 3 ? g.g3 : 0u;
}

// One finalized matrix for the queries: level lv's records at rec + lv *
// stride, its superblock bases at sb + lv * sbstride, its bucket starts
// (first position of each symbol in the next order) at st + lv * 4.
struct QView {
  const uint4* rec;
  const uint4* sb;
  const uint32_t* st;
  uint32_t stride, sbstride;
  int LL;
};

// The two counts one query step needs at position k: x = #{< k with symbol
// >= c}, y = #{< k with symbol >= c + 1} (two popcounts: the masks, counts
// and bases of classes c and c + 1 are selected first).
DDKS_DEV void ranks_c(uint4 r, uint4 s, uint32_t k, uint32_t c, uint32_t& x, uint32_t& y) {
  const uint32_t b = k & 31;
  const uint32_t below = b ? ((1u << b) - 1u) : 0u;
  const uint32_t m1 = r.x | r.y, m2 = r.y, m3 = r.x & r.y;
  const uint32_t q1 = s.x + (r.z & 0xFFFFu), q2 = s.y + (r.z >> 16), q3 = s.z + r.w;
  // class c (c >= 1) and class c + 1 (c + 1 <= 3)
  const uint32_t mc = c == 1 ? m1 : c == 2 ? m2 : m3, qc = c == 1 ? q1 : c == 2 ? q2 : q3;
  const uint32_t mu = c == 0 ? m1 : c == 1 ? m2 : m3, qu = c == 0 ? q1 : c == 1 ? q2 : q3;
  x = c == 0 ? k : qc + (uint32_t)__popc(mc & below);
  y = c == 3 ? 0u : qu + (uint32_t)__popc(mu & below);
}

// #{k in [la, ha) : value(k) >= v} in the all-points matrix and
// #{k in [lp, hp) : value(k) >= v} in the P matrix, both walks at once (v's
// symbol at each level picks the bucket; the symbols above it count as
// greater): the two dependent chains of record loads
// advance together, so their latencies overlap.  A walk whose range is empty
// keeps looking up its (equal) ends and adds nothing.
DDKS_DEV void count_ge4_pair(const QView& qa, const QView& qp, uint32_t la, uint32_t ha, uint32_t lp, uint32_t hp,
                             uint32_t v, uint32_t& ga, uint32_t& gp) {
  ga = 0;
  gp = 0;
  for (int lv = 0; lv < qa.LL && (la < ha || lp < hp); ++lv) {
    const uint32_t c = (v >> (2 * (qa.LL - 1 - lv))) & 3u;
    const uint4* Ra = qa.rec + (size_t)lv * qa.stride;
    const uint4* Sa = qa.sb + (size_t)lv * qa.sbstride;
    const uint4* Rp = qp.rec + (size_t)lv * qp.stride;
    const uint4* Sp = qp.sb + (size_t)lv * qp.sbstride;
    const uint4 ra0 = Ra[la >> 5], ra1 = Ra[ha >> 5], rp0 = Rp[lp >> 5], rp1 = Rp[hp >> 5];
    uint32_t ax, ay, bx, by, cx, cy, dx, dy;
    ranks_c(ra0, Sa[la >> kSBShift], la, c, ax, ay);
    ranks_c(ra1, Sa[ha >> kSBShift], ha, c, bx, by);
    ranks_c(rp0, Sp[lp >> kSBShift], lp, c, cx, cy);
    ranks_c(rp1, Sp[hp >> kSBShift], hp, c, dx, dy);
    ga += by - ay;
    gp += dy - cy;
    const uint32_t sa = qa.st[lv * 4 + c], sp = qp.st[lv * 4 + c];
    la = sa + ax - ay;
    ha = sa + bx - by;
    lp = sp + cx - cy;
    hp = sp + dx - dy;
  }
  ga += ha > la ? ha - la : 0u;
  gp += hp > lp ? hp - lp : 0u;
}


// Level-0 values: y ranks in dimension-0 order, for all points (matrix 0) and
// for the P points (matrix 1, positions = P points before the position);
// hy[y] counts the P points of each y rank.
__global__ void __launch_bounds__(kThreads)
k_dom_init(const uint32_t* __restrict__ rank, const uint32_t* __restrict__ sorted_idx0,
           const uint32_t* __restrict__ pprefix0, int64_t N, int64_t NP, uint32_t* __restrict__ v_all,
           uint32_t* __restrict__ v_p, uint32_t* __restrict__ hy) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t i = sorted_idx0[k];
    const uint32_t y = rank[N + i];
    v_all[k] = y;
    if (i < (uint64_t)NP) {
      v_p[pprefix0[k]] = y;
      atomicAdd(&hy[y], 1u);
    }
  }
}

// Symbol planes of one level: CTA (x, matrix) covers chunk x (kChunkWords
// words).  Record w = {plane 0, plane 1, counts of symbols >= 1 and >= 2
// before the word within the chunk (16 bits each), of >= 3}; the chunk's
// three totals go to ctot[(matrix * nchunks + x) * 4 + c - 1].
__global__ void __launch_bounds__(kChunkWords)
k_quad_bits(const uint32_t* __restrict__ vals, uint32_t n0, uint32_t n1, uint32_t nmax, uint32_t recw,
            uint32_t nchunks, int shift, uint4* __restrict__ rec, uint32_t* __restrict__ ctot) {
  __shared__ uint32_t cw0[kChunkWords], cw1[kChunkWords];
  __shared__ unsigned long long ws[kChunkWords / 32];
  const int mtx = blockIdx.y;
  const uint32_t n = mtx ? n1 : n0;
  const uint32_t* v = vals + (size_t)mtx * nmax;
  uint4* R = rec + (size_t)mtx * recw;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t w0 = blockIdx.x * kChunkWords;
  // warp `warp` builds words w0 + warp + 8 q, q < 32: all loads first, then the ballots
  constexpr int kPerWarp = kChunkWords / (kChunkWords / 32);
  uint32_t x[kPerWarp];
#pragma unroll
  for (int q = 0; q < kPerWarp; ++q) {
    const uint32_t k = (w0 + warp + 8 * q) * 32 + lane;
    x[q] = k < n ? v[k] : 0u;
  }
#pragma unroll
  for (int q = 0; q < kPerWarp; ++q) {
    const uint32_t k = (w0 + warp + 8 * q) * 32 + lane;
    const uint32_t sym = k < n ? (x[q] >> shift) & 3u : 0u;
    const uint32_t b0 = __ballot_sync(0xffffffffu, sym & 1u);
    const uint32_t b1 = __ballot_sync(0xffffffffu, (sym >> 1) & 1u);
    if (lane == 0) {
      cw0[warp + 8 * q] = b0;
      cw1[warp + 8 * q] = b1;
    }
  }
  __syncthreads();
  const uint32_t p0 = cw0[threadIdx.x], p1 = cw1[threadIdx.x];
  // the three counts packed 21 bits apart (a chunk holds at most 8192 of each)
  const unsigned long long c = (unsigned long long)__popc(p0 | p1) | ((unsigned long long)__popc(p1) << 21) |
                               ((unsigned long long)__popc(p0 & p1) << 42);
  unsigned long long incl = c;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const unsigned long long y = __shfl_up_sync(0xffffffffu, incl, off);
    if (lane >= off) incl += y;
  }
  if (lane == 31) ws[warp] = incl;
  __syncthreads();
  unsigned long long before = 0;
  for (int q = 0; q < warp; ++q) before += ws[q];
  const unsigned long long ex = before + incl - c;
  const uint32_t e1 = (uint32_t)(ex & 0x1FFFFFu), e2 = (uint32_t)((ex >> 21) & 0x1FFFFFu),
                 e3 = (uint32_t)(ex >> 42);
  const uint32_t w = w0 + threadIdx.x;
  if (w < recw) R[w] = make_uint4(p0, p1, e1 | (e2 << 16), e3);
  if (threadIdx.x == kChunkWords - 1) {
    const unsigned long long t = before + incl;
    uint32_t* T = ctot + ((size_t)mtx * nchunks + blockIdx.x) * 4;
    T[0] = (uint32_t)(t & 0x1FFFFFu);
    T[1] = (uint32_t)((t >> 21) & 0x1FFFFFu);
    T[2] = (uint32_t)(t >> 42);
  }
}

// One CTA per matrix: exclusive prefixes of the chunk totals into cpre
// (nchunks + 1 entries of 4 words, the last the level's totals) and the
// level's bucket starts st[matrix][lv][c] = #{symbols < c}.
__global__ void __launch_bounds__(kScanThreads)
k_quad_cscan(const uint32_t* __restrict__ ctot, uint32_t* __restrict__ cpre, uint32_t n0, uint32_t n1,
             uint32_t nchunks, size_t cpre_mstride, int lv, uint32_t* __restrict__ st) {
  __shared__ uint32_t ws[3][kScanThreads / 32];
  __shared__ uint32_t carry[3];
  const int mtx = blockIdx.x;
  const uint32_t n = mtx ? n1 : n0;
  const uint32_t* C = ctot + (size_t)mtx * nchunks * 4;
  uint32_t* P = cpre + (size_t)mtx * cpre_mstride;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x < 3) carry[threadIdx.x] = 0;
  __syncthreads();
  for (uint32_t t0 = 0; t0 < nchunks + 1; t0 += kScanThreads) {
    const uint32_t i = t0 + threadIdx.x;
    uint32_t ex[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const uint32_t v = i < nchunks ? C[(size_t)i * 4 + c] : 0u;
      uint32_t incl = v;
      for (int off = 1; off < 32; off <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += y;
      }
      if (lane == 31) ws[c][warp] = incl;
      __syncthreads();
      uint32_t before = carry[c];
      for (int q = 0; q < warp; ++q) before += ws[c][q];
      ex[c] = before + incl - v;
      __syncthreads();
      if (threadIdx.x == kScanThreads - 1) carry[c] = ex[c] + v;
      __syncthreads();
    }
    if (i <= nchunks) {
      P[(size_t)i * 4 + 0] = ex[0];
      P[(size_t)i * 4 + 1] = ex[1];
      P[(size_t)i * 4 + 2] = ex[2];
      P[(size_t)i * 4 + 3] = 0u;
    }
    if (i == nchunks) {  // ex = the level's totals of symbols >= 1, 2, 3
      uint32_t* S = st + ((size_t)mtx * kMaxLevels + lv) * 4;
      S[0] = 0u;
      S[1] = n - ex[0];
      S[2] = n - ex[1];
      S[3] = n - ex[2];
    }
  }
}

// Stable partition of one level by symbol into the next level's order.
__global__ void __launch_bounds__(kThreads)
k_quad_scatter(const uint32_t* __restrict__ vin, uint32_t* __restrict__ vout, uint32_t n0, uint32_t n1,
               uint32_t nmax, uint32_t recw, size_t cpre_mstride, int shift, int lv, const uint4* __restrict__ rec,
               const uint32_t* __restrict__ cpre, const uint32_t* __restrict__ st) {
  const int mtx = blockIdx.y;
  const uint32_t n = mtx ? n1 : n0;
  const uint32_t* v = vin + (size_t)mtx * nmax;
  uint32_t* o = vout + (size_t)mtx * nmax;
  const uint4* R = rec + (size_t)mtx * recw;
  const uint4* P = reinterpret_cast<const uint4*>(cpre + (size_t)mtx * cpre_mstride);
  const uint32_t* S = st + ((size_t)mtx * kMaxLevels + lv) * 4;
  const uint32_t s1 = S[1], s2 = S[2], s3 = S[3];
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const uint32_t y = v[k];
    const uint32_t c = (y >> shift) & 3u;
    const Ge g = ranks_at(R[k >> 5], P[k >> kChunkShift], k);  // chunk-relative records + chunk prefix
    const uint32_t eq = ge_pick(g, k, c) - ge_pick(g, k, c + 1);
    const uint32_t s0 = c == 0 ? 0u : c == 1 ? s1 : c == 2 ? s2 : s3;
    o[s0 + eq] = y;
  }
}

// Makes the records superblock-relative (absolute count = chunk prefix +
// record, minus the superblock's base) and writes the superblock bases
// sb[row][j] = cpre[row][j * kSBChunks] (row = level * 2 + matrix).
__global__ void __launch_bounds__(kThreads)
k_quad_finalize(uint4* __restrict__ rec, const uint32_t* __restrict__ cpre, uint4* __restrict__ sb, uint64_t recs,
                uint32_t recw, size_t cpre_mstride, uint32_t nsb) {
  for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < recs;
       t += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t row = t / recw;
    const uint32_t w = (uint32_t)(t - row * recw);
    const uint32_t chunk = w / kChunkWords, sbi = chunk / kSBChunks;
    const uint4* P = reinterpret_cast<const uint4*>(cpre + row * cpre_mstride);
    const uint4 pc = P[chunk], pb = P[sbi * kSBChunks];
    uint4 r = rec[t];
    const uint32_t a1 = pc.x + (r.z & 0xFFFFu) - pb.x, a2 = pc.y + (r.z >> 16) - pb.y, a3 = pc.z + r.w - pb.z;
    r.z = a1 | (a2 << 16);
    r.w = a3;
    rec[t] = r;
    if (w == sbi * kSBChunks * kChunkWords) sb[row * nsb + sbi] = make_uint4(pb.x, pb.y, pb.z, 0u);
  }
}

// Per origin: the four quadrant counts of each sample and the best orthant.
// hyx[v] = P points with y rank < v.  order (optional, with [ob, oe) the
// whole pooled range): the origins in dimension-1 order.  Neighbouring
// threads then share the high bits of their y ranks, so the upper ends of
// their query ranges (N and NP at level 0, then fixed by those symbols)
// follow the same positions and their record loads coincide.  Superblock
// bases (sbwords uint4 for both matrices and every level) are staged in
// shared memory when they fit.
__global__ void __launch_bounds__(kThreads)
k_dom_query(const uint32_t* __restrict__ rank, const uint32_t* __restrict__ pprefix0,
            const uint32_t* __restrict__ hyx, int64_t N, int64_t NP, int64_t NT, int64_t ob, int64_t oe,
            QView wa, QView wp, uint32_t sbwords, const uint32_t* __restrict__ order, uint64_t* __restrict__ best,
            int32_t* __restrict__ bestj) {
  extern __shared__ uint4 ssb[];  // sbwords entries when they fit, else unused
  __shared__ uint32_t sst[2 * kMaxLevels * 4];
  if (sbwords <= kSmemBases) {  // wa.sb .. wa.sb + sbwords holds both matrices' bases
    for (uint32_t i = threadIdx.x; i < sbwords; i += blockDim.x) ssb[i] = wa.sb[i];
    wp.sb = ssb + (wp.sb - wa.sb);
    wa.sb = ssb;
  }
  for (int i = threadIdx.x; i < 2 * kMaxLevels * 4; i += blockDim.x) sst[i] = wa.st[i];
  __syncthreads();
  wp.st = sst + (wp.st - wa.st);
  wa.st = sst;
  for (int64_t k = ob + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < oe;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t o = order ? (int64_t)order[k] : k;
    const uint32_t rx = rank[o], ry = rank[N + o];
    const uint32_t lxp = rx < (uint64_t)N ? pprefix0[rx] : (uint32_t)NP;  // P points with x_0 < o_0
    uint32_t ga, gp;
    count_ge4_pair(wa, wp, rx, (uint32_t)N, lxp, (uint32_t)NP, ry, ga, gp);
    const uint64_t a3 = ga;  // both >=, all points
    const uint64_t p3 = gp;  // both >=, P
    const uint64_t pyu = (uint64_t)NP - hyx[ry];                          // P with x_1 >= o_1
    const uint64_t axu = (uint64_t)N - rx, pxu = (uint64_t)NP - lxp;      // x_0 >= o_0
    const uint64_t ayu = (uint64_t)N - ry;                                // x_1 >= o_1
    uint64_t cp[4], ca[4];
    cp[3] = p3;
    cp[1] = pxu - p3;  // code 1: x_0 >= o_0, x_1 < o_1
    cp[2] = pyu - p3;  // code 2: x_0 < o_0, x_1 >= o_1
    cp[0] = (uint64_t)NP - cp[1] - cp[2] - cp[3];
    ca[3] = a3;
    ca[1] = axu - a3;
    ca[2] = ayu - a3;
    ca[0] = (uint64_t)N - ca[1] - ca[2] - ca[3];
    uint64_t b = 0;
    int bj = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const uint64_t v = ddks::numer(cp[j], ca[j] - cp[j], (uint64_t)NP, (uint64_t)NT);
      if (v > b) { b = v; bj = j; }
    }
    best[o - ob] = b;
    bestj[o - ob] = bj;
  }
}

int grid_for(int64_t work, int threads, int cap) {
  int64_t g = (work + threads - 1) / threads;
  if (g > cap) g = cap;
  return (int)(g < 1 ? 1 : g);
}

}  // namespace

bool ddks_dominance_supported(int d, int64_t NP, int64_t NT) {
  return d == 2 && NP + NT < ((int64_t)1 << 31) && NP >= 1 && NT >= 1;
}

// Requires K0 with sorted_idx0 and its P prefix (ctx->pfx0_valid).
cudaError_t ddks_launch_dominance(ddks_ctx* ctx, const uint32_t* rank, int64_t N, int64_t NP, int64_t NT,
                                  int64_t ob, int64_t oe, uint64_t* best, int32_t* bestj, cudaStream_t st,
                                  int* launches) {
  int n = 0;
  int L = 1;
  while (((int64_t)1 << L) < N) ++L;  // values (ranks) < N <= 2^L
  const int LL = (L + 1) / 2;         // 2-bit levels
  if (LL > kMaxLevels) return cudaErrorInvalidValue;
  const uint32_t n0 = (uint32_t)N, n1 = (uint32_t)NP, nmax = n0;
  // records per matrix and level: whole chunks covering position nmax (a
  // lookup may read word nmax / 32); superblock bases per matrix and level
  const uint32_t nchunks = nmax / (32 * kChunkWords) + 1;
  const uint32_t recw = nchunks * kChunkWords;
  const uint32_t nsb = (nchunks + kSBChunks - 1) / kSBChunks;
  const size_t cpre_mstride = (size_t)(nchunks + 1) * 4;  // words per matrix and level
  // scratch (u32 words): values [2 bufs][2 matrices][nmax]; records
  // [LL][2][recw] uint4; chunk prefixes [LL][2][nchunks + 1][4]; superblock
  // bases [LL][2][nsb] uint4; chunk totals [2][nchunks][4]; bucket starts
  // [2][kMaxLevels][4]; P counts per y rank [N + 1] and their prefix [N + 1]
  const size_t recwords = (size_t)LL * 2 * recw * 4;
  const size_t prewords = (size_t)LL * 2 * cpre_mstride;
  const size_t sbwords = (size_t)LL * 2 * nsb * 4;
  const size_t scan_tmp = ddks_scan_tmp_elems(1, N + 1);
  const size_t words = (size_t)4 * nmax + recwords + prewords + sbwords + (size_t)2 * nchunks * 4 +
                       2 * kMaxLevels * 4 + 2 * (size_t)(N + 1) + scan_tmp + 8;
  int rc = ctx->dom_work.reserve(ctx, 4 * words);
  if (rc) return cudaErrorMemoryAllocation;
  uint32_t* base = (uint32_t*)ctx->dom_work.ptr;
  uint32_t* vbuf[2] = {base, base + 2 * (size_t)nmax};
  uint4* rec = reinterpret_cast<uint4*>(base + 4 * (size_t)nmax);  // 16-byte aligned: 4 nmax words
  uint32_t* cpre = base + 4 * (size_t)nmax + recwords;
  uint4* sbb = reinterpret_cast<uint4*>(cpre + prewords);  // prewords is a multiple of 4
  uint32_t* ctot = reinterpret_cast<uint32_t*>(sbb) + sbwords;
  uint32_t* stg = ctot + (size_t)2 * nchunks * 4;
  uint32_t* hy = stg + 2 * kMaxLevels * 4;
  uint32_t* hyx = hy + (N + 1);
  uint32_t* tmp = hyx + (N + 1);
  const uint32_t* sorted_idx0 = (const uint32_t*)ctx->sidx0.ptr;
  const uint32_t* pprefix0 = (const uint32_t*)ctx->pfx0.ptr;
  cudaError_t e = cudaMemsetAsync(hy, 0, 4 * (size_t)(N + 1), st);
  if (e != cudaSuccess) return e;
  k_dom_init<<<grid_for(N, kThreads, ctx->num_sms * 8), kThreads, 0, st>>>(rank, sorted_idx0, pprefix0, N, NP,
                                                                         vbuf[0], vbuf[0] + nmax, hy);
  ++n;
  int sl = 0;
  e = ddks_scan_rows(hy, hyx, 1, N + 1, true, tmp, st, &sl);
  if (e != cudaSuccess) return e;
  n += sl;
  const dim3 gs((unsigned)grid_for(nmax, kThreads, ctx->num_sms * 8), 2);
  for (int lv = 0; lv < LL; ++lv) {
    const int shift = 2 * (LL - 1 - lv);
    uint4* rl = rec + (size_t)lv * 2 * recw;
    uint32_t* pl = cpre + (size_t)lv * 2 * cpre_mstride;
    k_quad_bits<<<dim3(nchunks, 2), kChunkWords, 0, st>>>(vbuf[lv & 1], n0, n1, nmax, recw, nchunks, shift, rl, ctot);
    k_quad_cscan<<<2, kScanThreads, 0, st>>>(ctot, pl, n0, n1, nchunks, cpre_mstride, lv, stg);
    n += 2;
    if (lv + 1 < LL) {
      k_quad_scatter<<<gs, kThreads, 0, st>>>(vbuf[lv & 1], vbuf[(lv + 1) & 1], n0, n1, nmax, recw, cpre_mstride,
                                              shift, lv, rl, pl, stg);
      ++n;
    }
  }
  k_quad_finalize<<<grid_for((int64_t)LL * 2 * recw, kThreads, ctx->num_sms * 8), kThreads, 0, st>>>(
      rec, cpre, sbb, (uint64_t)LL * 2 * recw, recw, cpre_mstride, nsb);
  ++n;
  // query views: levels are [lv][matrix][recw records], [lv][matrix][nsb bases]
  const QView wa{rec, sbb, stg, 2 * recw, 2 * nsb, LL};
  const QView wp{rec + recw, sbb + nsb, stg + kMaxLevels * 4, 2 * recw, 2 * nsb, LL};
  const int64_t no = oe - ob;
  if (no > 0) {
    const uint32_t* order = (ob == 0 && oe == N && ctx->sorted_rows) ? ctx->sorted_rows + N : nullptr;
    const uint32_t nbases = (uint32_t)(LL * 2 * nsb);
    const size_t qsmem = nbases <= (uint32_t)kSmemBases ? 16 * (size_t)nbases : 0;
    k_dom_query<<<grid_for(no, kThreads, ctx->num_sms * 16), kThreads, qsmem, st>>>(
        rank, pprefix0, hyx, N, NP, NT, ob, oe, wa, wp, nbases, order, best, bestj);
    ++n;
  }
  if (launches) *launches += n;
  return cudaGetLastError();
}
