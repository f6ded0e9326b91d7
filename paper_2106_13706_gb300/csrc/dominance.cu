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
// by a second query over the whole range).
//
// The range queries run on two wavelet matrices (the wavelet tree variant of
// Information Systems 47, 2015): one over the y ranks of all points in
// dimension-0 order, one
// over the P points only.  Level l of a matrix holds one bit per position
// (bit L-1-l of the value), a per-word prefix count of ones, and the next
// level's order: a stable partition, zeros first.  A query walks the L levels
// with two rank lookups each (an 8-byte word record plus a superblock
// prefix).  Build: per level a bit kernel (warp ballots; prefixes within
// superblocks of 256 words), a scan of the superblock totals and a scatter
// kernel; query: one thread per origin.
#include <cstring>

#include "../../include/ddks.h"
#include "ddks_host.h"
#include "ddks_internal.cuh"

namespace {

constexpr int kThreads = 256;

constexpr int kScanThreads = 1024;
constexpr int kMaxLevels = 32;
constexpr int kSBWords = 256;  // words per superblock (8192 positions), one CTA of k_dom_bits

// One wavelet matrix in device memory for the queries.  Level lv: records at
// rec + lv * stride, record w = {ones before word w, bit word w}.  (While a
// level is built its records count only the ones within their superblock of
// kSBWords words, with the superblock prefixes beside them; k_dom_finalize
// adds those in once every level exists.)
struct WMView {
  const uint2* rec;
  uint32_t stride;
  int L;
};

DDKS_DEV uint32_t rank1(const uint2* rec, const uint32_t* sb, uint32_t k) {
  const uint2 r = rec[k >> 5];
  const uint32_t b = k & 31;
  return sb[k >> 13] + r.x + (b ? (uint32_t)__popc(r.y & ((1u << b) - 1u)) : 0u);
}

// After k_dom_finalize the records hold absolute prefixes: one load per rank.
DDKS_DEV uint32_t rank1_abs(const uint2* rec, uint32_t k) {
  const uint2 r = rec[k >> 5];
  const uint32_t b = k & 31;
  return r.x + (b ? (uint32_t)__popc(r.y & ((1u << b) - 1u)) : 0u);
}

// #{k in [l, r) : value(k) >= v}; Z[lv] = zeros of level lv (finalized records)
DDKS_DEV uint32_t count_ge(const WMView& wm, const uint32_t* Z, uint32_t l, uint32_t r, uint32_t v) {
  const uint32_t len = r - l;
  uint32_t less = 0;
  for (int lv = 0; lv < wm.L && l < r; ++lv) {
    const uint2* rec = wm.rec + (size_t)lv * wm.stride;
    const uint32_t ol = rank1_abs(rec, l), orr = rank1_abs(rec, r);
    if ((v >> (wm.L - 1 - lv)) & 1u) {
      less += (r - l) - (orr - ol);  // the zeros of this level are smaller
      l = Z[lv] + ol;
      r = Z[lv] + orr;
    } else {
      l -= ol;
      r -= orr;
    }
  }
  return len - less;
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

// Bit words of one level: CTA (x, matrix) covers superblock x (kSBWords
// words).  Writes each word's bits and its prefix within the superblock into
// the records, and the superblock's total into sbcnt.
__global__ void __launch_bounds__(kSBWords)
k_dom_bits(const uint32_t* __restrict__ vals, uint32_t n0, uint32_t n1, uint32_t nmax, uint32_t recw,
           uint32_t nsb, int bit, uint2* __restrict__ rec, uint32_t* __restrict__ sbcnt) {
  __shared__ uint32_t cw[kSBWords];
  __shared__ uint32_t ws[kSBWords / 32];
  const int mtx = blockIdx.y;
  const uint32_t n = mtx ? n1 : n0;
  const uint32_t* v = vals + (size_t)mtx * nmax;
  uint2* R = rec + (size_t)mtx * recw;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t w0 = blockIdx.x * kSBWords;
  // warp `warp` builds words w0 + warp + 8 q, q < 32: all loads first, then
  // the ballots
  constexpr int kPerWarp = kSBWords / (kSBWords / 32);
  uint32_t x[kPerWarp];
#pragma unroll
  for (int q = 0; q < kPerWarp; ++q) {
    const uint32_t k = (w0 + warp + 8 * q) * 32 + lane;
    x[q] = k < n ? v[k] : 0u;
  }
#pragma unroll
  for (int q = 0; q < kPerWarp; ++q) {
    const uint32_t k = (w0 + warp + 8 * q) * 32 + lane;
    const uint32_t word = __ballot_sync(0xffffffffu, k < n && ((x[q] >> bit) & 1u));
    if (lane == 0) cw[warp + 8 * q] = word;
  }
  __syncthreads();
  const uint32_t word = cw[threadIdx.x];
  const uint32_t c = (uint32_t)__popc(word);
  uint32_t incl = c;
  for (int off = 1; off < 32; off <<= 1) {
    const uint32_t x = __shfl_up_sync(0xffffffffu, incl, off);
    if (lane >= off) incl += x;
  }
  if (lane == 31) ws[warp] = incl;
  __syncthreads();
  uint32_t before = 0;
  for (int q = 0; q < warp; ++q) before += ws[q];
  const uint32_t w = w0 + threadIdx.x;
  if (w < recw) R[w] = make_uint2(before + incl - c, word);
  if (threadIdx.x == kSBWords - 1) sbcnt[(size_t)mtx * nsb + blockIdx.x] = before + incl;
}

// One CTA per matrix: exclusive prefix of the superblock totals into sb (nsb
// + 1 entries, the last the level's ones); Z[matrix * kMaxLevels + lv] =
// zeros of the level.
__global__ void __launch_bounds__(kScanThreads)
k_dom_sbscan(const uint32_t* __restrict__ sbcnt, uint32_t* __restrict__ sb, uint32_t n0, uint32_t n1, uint32_t nsb,
             uint32_t sbw, int lv, uint32_t* __restrict__ Z) {
  __shared__ uint32_t ws[kScanThreads / 32];
  __shared__ uint32_t carry;
  const int mtx = blockIdx.x;
  const uint32_t n = mtx ? n1 : n0;
  const uint32_t* C = sbcnt + (size_t)mtx * nsb;
  uint32_t* S = sb + (size_t)mtx * sbw;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (uint32_t t0 = 0; t0 < nsb + 1; t0 += kScanThreads) {  // tiles of coalesced entries
    const uint32_t i = t0 + threadIdx.x;
    const uint32_t c = i < nsb ? C[i] : 0u;
    uint32_t incl = c;
    for (int off = 1; off < 32; off <<= 1) {
      const uint32_t x = __shfl_up_sync(0xffffffffu, incl, off);
      if (lane >= off) incl += x;
    }
    if (lane == 31) ws[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      const uint32_t t = ws[lane];
      uint32_t ti = t;
      for (int off = 1; off < 32; off <<= 1) {
        const uint32_t x = __shfl_up_sync(0xffffffffu, ti, off);
        if (lane >= off) ti += x;
      }
      ws[lane] = ti - t;
    }
    __syncthreads();
    const uint32_t ex = carry + ws[warp] + incl - c;
    if (i <= nsb) S[i] = ex;
    if (i == nsb) Z[mtx * kMaxLevels + lv] = n - ex;  // ex = all ones of the level
    __syncthreads();
    if (threadIdx.x == kScanThreads - 1) carry = ex + c;
    __syncthreads();
  }
}

// Adds the superblock prefixes into the records of every level and matrix
// (recs records of recw per matrix and level), for the queries.
__global__ void __launch_bounds__(kThreads)
k_dom_finalize(uint2* __restrict__ rec, const uint32_t* __restrict__ sb, uint64_t recs, uint32_t recw,
               uint32_t sbw) {
  for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < recs;
       t += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t row = t / recw;  // level * 2 + matrix
    const uint32_t w = (uint32_t)(t - row * recw);
    rec[t].x += sb[row * sbw + (w / kSBWords)];
  }
}

// Stable partition of one level (zeros first) into the next level's order.
__global__ void __launch_bounds__(kThreads)
k_dom_scatter(const uint32_t* __restrict__ vin, uint32_t* __restrict__ vout, uint32_t n0, uint32_t n1,
              uint32_t nmax, uint32_t recw, uint32_t sbw, int bit, int lv, const uint2* __restrict__ rec,
              const uint32_t* __restrict__ sb, const uint32_t* __restrict__ Z) {
  const int mtx = blockIdx.y;
  const uint32_t n = mtx ? n1 : n0;
  const uint32_t* v = vin + (size_t)mtx * nmax;
  uint32_t* o = vout + (size_t)mtx * nmax;
  const uint2* R = rec + (size_t)mtx * recw;
  const uint32_t* S = sb + (size_t)mtx * sbw;
  const uint32_t z = Z[mtx * kMaxLevels + lv];
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const uint32_t x = v[k];
    const uint32_t ones = rank1(R, S, k);
    o[((x >> bit) & 1u) ? z + ones : k - ones] = x;
  }
}

// The same with the superblock scan folded in (nsb + 1 <= kFusedSB): every
// CTA scans the level's superblock totals into shared memory itself; CTA 0
// of each matrix also stores the prefixes (for k_dom_finalize) and the
// level's zeros Z (for the queries).  Saves the scan kernel per level.
constexpr uint32_t kFusedSB = 8192;
__global__ void __launch_bounds__(kThreads)
k_dom_scatter_fused(const uint32_t* __restrict__ vin, uint32_t* __restrict__ vout, uint32_t n0, uint32_t n1,
                    uint32_t nmax, uint32_t recw, uint32_t nsb, uint32_t sbw, int bit, int lv,
                    const uint2* __restrict__ rec, const uint32_t* __restrict__ sbcnt, uint32_t* __restrict__ sb,
                    uint32_t* __restrict__ Zg) {
  extern __shared__ uint32_t ssb[];  // nsb + 1 prefixes
  __shared__ uint32_t ws[kThreads / 32];
  __shared__ uint32_t carry;
  const int mtx = blockIdx.y;
  const uint32_t n = mtx ? n1 : n0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t* C = sbcnt + (size_t)mtx * nsb;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (uint32_t t0 = 0; t0 < nsb + 1; t0 += kThreads) {
    const uint32_t i = t0 + threadIdx.x;
    const uint32_t c = i < nsb ? C[i] : 0u;
    uint32_t incl = c;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const uint32_t x = __shfl_up_sync(0xffffffffu, incl, off);
      if (lane >= off) incl += x;
    }
    if (lane == 31) ws[warp] = incl;
    __syncthreads();
    uint32_t before = carry;
    for (int q = 0; q < warp; ++q) before += ws[q];
    const uint32_t ex = before + incl - c;
    if (i <= nsb) ssb[i] = ex;
    __syncthreads();
    if (threadIdx.x == kThreads - 1) carry = ex + c;
    __syncthreads();
  }
  const uint32_t z = n - ssb[nsb];  // ssb[nsb] = the level's ones
  if (blockIdx.x == 0) {
    uint32_t* S = sb + (size_t)mtx * sbw;
    for (uint32_t i = threadIdx.x; i <= nsb; i += kThreads) S[i] = ssb[i];
    if (threadIdx.x == 0) Zg[mtx * kMaxLevels + lv] = z;
  }
  const uint32_t* v = vin + (size_t)mtx * nmax;
  uint32_t* o = vout + (size_t)mtx * nmax;
  const uint2* R = rec + (size_t)mtx * recw;
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const uint32_t x = v[k];
    const uint2 r = R[k >> 5];
    const uint32_t b = k & 31;
    const uint32_t ones = ssb[k >> 13] + r.x + (b ? (uint32_t)__popc(r.y & ((1u << b) - 1u)) : 0u);
    o[((x >> bit) & 1u) ? z + ones : k - ones] = x;
  }
}

// Per origin: the four quadrant counts of each sample and the best orthant.
// hyx[v] = P points with y rank < v.  order (optional, with [ob, oe) the
// whole pooled range): the origins in dimension-1 order.  Neighbouring
// threads then share the high bits of their y ranks, so the upper ends of
// their query ranges (N and NP at level 0, then fixed by those bits) follow
// the same positions and their record loads coincide.
__global__ void __launch_bounds__(kThreads)
k_dom_query(const uint32_t* __restrict__ rank, const uint32_t* __restrict__ pprefix0,
            const uint32_t* __restrict__ hyx, int64_t N, int64_t NP, int64_t NT, int64_t ob, int64_t oe,
            WMView wa, WMView wp, const uint32_t* __restrict__ Zg, const uint32_t* __restrict__ order,
            uint64_t* __restrict__ best, int32_t* __restrict__ bestj) {
  __shared__ uint32_t Z[2 * kMaxLevels];
  if (threadIdx.x < 2 * kMaxLevels) Z[threadIdx.x] = Zg[threadIdx.x];
  __syncthreads();
  for (int64_t k = ob + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < oe;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t o = order ? (int64_t)order[k] : k;
    const uint32_t rx = rank[o], ry = rank[N + o];
    const uint32_t lxp = rx < (uint64_t)N ? pprefix0[rx] : (uint32_t)NP;  // P points with x_0 < o_0
    const uint64_t a3 = count_ge(wa, Z, rx, (uint32_t)N, ry);             // both >=, all points
    const uint64_t p3 = count_ge(wp, Z + kMaxLevels, lxp, (uint32_t)NP, ry);  // both >=, P
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
  if (L > kMaxLevels) return cudaErrorInvalidValue;
  const uint32_t n0 = (uint32_t)N, n1 = (uint32_t)NP, nmax = n0;
  // records per matrix and level: whole superblocks covering position nmax
  // (rank1 may look at word nmax / 32)
  const uint32_t nsb = nmax / (32 * kSBWords) + 1;
  const uint32_t recw = nsb * kSBWords;
  const uint32_t sbw = nsb + 1;
  // scratch (u32 words): values [2 bufs][2 matrices][nmax]; records
  // [L][2][recw] (2 words each); superblock prefixes [L][2][sbw]; superblock
  // totals [2][nsb]; Z [2][kMaxLevels]; P counts per y rank [N + 1] and their
  // prefix [N + 1]
  const size_t recwords = (size_t)L * 2 * recw * 2;
  const size_t scan_tmp = ddks_scan_tmp_elems(1, N + 1);
  const size_t words = (size_t)4 * nmax + recwords + (size_t)L * 2 * sbw + 2 * (size_t)nsb + 2 * kMaxLevels +
                       2 * (size_t)(N + 1) + scan_tmp + 4;
  int rc = ctx->dom_work.reserve(ctx, 4 * words);
  if (rc) return cudaErrorMemoryAllocation;
  uint32_t* base = (uint32_t*)ctx->dom_work.ptr;
  uint32_t* vbuf[2] = {base, base + 2 * (size_t)nmax};
  uint2* rec = reinterpret_cast<uint2*>(base + 4 * (size_t)nmax);  // 8-byte aligned: 4 nmax words
  uint32_t* sbp = base + 4 * (size_t)nmax + recwords;
  uint32_t* sbcnt = sbp + (size_t)L * 2 * sbw;
  uint32_t* Zg = sbcnt + 2 * (size_t)nsb;
  uint32_t* hy = Zg + 2 * kMaxLevels;
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
  for (int lv = 0; lv < L; ++lv) {
    const int bit = L - 1 - lv;
    uint2* rl = rec + (size_t)lv * 2 * recw;
    uint32_t* sl_ = sbp + (size_t)lv * 2 * sbw;
    k_dom_bits<<<dim3(nsb, 2), kSBWords, 0, st>>>(vbuf[lv & 1], n0, n1, nmax, recw, nsb, bit, rl, sbcnt);
    ++n;
    if (lv + 1 < L && nsb + 1 <= kFusedSB) {
      k_dom_scatter_fused<<<gs, kThreads, 4 * (nsb + 1), st>>>(vbuf[lv & 1], vbuf[(lv + 1) & 1], n0, n1, nmax, recw, nsb, sbw,
                                                   bit, lv, rl, sbcnt, sl_, Zg);
      ++n;
      continue;
    }
    k_dom_sbscan<<<2, kScanThreads, 0, st>>>(sbcnt, sl_, n0, n1, nsb, sbw, lv, Zg);
    ++n;
    if (lv + 1 < L) {
      k_dom_scatter<<<gs, kThreads, 0, st>>>(vbuf[lv & 1], vbuf[(lv + 1) & 1], n0, n1, nmax, recw, sbw, bit, lv, rl,
                                             sl_, Zg);
      ++n;
    }
  }
  k_dom_finalize<<<grid_for((int64_t)L * 2 * recw, kThreads, ctx->num_sms * 8), kThreads, 0, st>>>(
      rec, sbp, (uint64_t)L * 2 * recw, recw, sbw);
  ++n;
  // query views: levels are [lv][matrix][recw records], [lv][matrix][sbw prefixes]
  const WMView wa{rec, 2 * recw, L};
  const WMView wp{rec + recw, 2 * recw, L};
  const int64_t no = oe - ob;
  if (no > 0) {
    const uint32_t* order = (ob == 0 && oe == N && ctx->sorted_rows) ? ctx->sorted_rows + N : nullptr;
    k_dom_query<<<grid_for(no, kThreads, ctx->num_sms * 16), kThreads, 0, st>>>(rank, pprefix0, hyx, N, NP, NT, ob,
                                                                              oe, wa, wp, Zg, order, best, bestj);
    ++n;
  }
  if (launches) *launches += n;
  return cudaGetLastError();
}
