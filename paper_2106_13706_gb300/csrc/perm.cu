// perm.cu -- A7/A8: the permutation test (Sec. 4.2) as one batched launch.
//
// Relabelling b of the pooled sample puts into P the NP pooled points with the
// smallest (key, index), key(b, i) = word (i mod 4) of Philox4x64-10 (Salmon,
// Moraes, Dror, Shaw, SC 2011) with counter (i / 4, b, 0, 0) and key (seed, 0).
//
// K3 (k_perm_labels_warp): one warp per relabelling draws the N keys, selects
//   the NP smallest (key, index) pairs by radix selection and sets bit b of
//   their label words: labels[i][b / 32] bit (b % 32) = [i in permuted P].
// K4 (k_perm_count): the orthant code c(o, x) of a pair does not depend on the
//   labels, so each CTA takes an origin, computes the N codes once into shared
//   memory together with n(c) = #{x : c(o, x) = c}, and then counts, for every
//   relabelling b, cP_b(c) = #{x in permuted P : c(o, x) = c} in lane-private
//   shared histograms of 16-bit counters (N <= 16384; warp w of a chunk owns
//   32 consecutive relabellings, so
//   one label word per point serves the whole warp).  With cT_b = n - cP_b the
//   numerator is |cP_b*NT - cT_b*NP| = |cP_b*N - n*NP|; each thread keeps the
//   running maximum of its relabellings and finishes with one atomicMax.
// K_pv (k_perm_pvalue): #{b : num_b >= num_obs}.
#include "ddks_host.h"
#include "ddks_internal.cuh"

namespace {

constexpr int kMaxPermN = 16384;
constexpr int kLabWarps = 8;     // relabellings per CTA (one per warp)
constexpr int kLabCand = 256;    // largest bucket ranked by brute force
constexpr int kCountThreads = 256;
constexpr int kPtsTile = 64;

DDKS_DEV void philox4x64_10(uint64_t c[4], uint64_t k0, uint64_t k1) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += W0; k1 += W1; }
    const uint64_t hi0 = __umul64hi(M0, c[0]), lo0 = M0 * c[0];
    const uint64_t hi1 = __umul64hi(M1, c[2]), lo1 = M1 * c[2];
    const uint64_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
  }
}


// K3, one warp per relabelling: the N Philox keys go to warp-private shared
// memory, a most-significant-digit radix selection (eight 8-bit digits) finds
// the NP-th smallest key K* and how many keys equal to K* belong to P, and
// the points with key < K*, plus the lowest-index ones with key == K*, get
// bit b.  Same labels as sorting the (key, index) pairs.
// K3, one warp per relabelling, without storing the keys: the warp regenerates
// the relabelling's N Philox keys in each pass.  Most-significant-digit radix
// selection (8-bit digits, histograms in warp-private shared memory) narrows
// the NP-th smallest key to one bucket of at most kLabCand keys (usually one
// histogram pass); the bucket's (key, index) pairs are collected and ranked
// by brute force, which gives the threshold pair (K*, i*); a last pass sets
// bit b for every point with (key, i) <= (K*, i*) -- exactly the NP smallest
// (key, index) pairs, as sorting them would.
__global__ void __launch_bounds__(kLabWarps * 32)
k_perm_labels_warp(int64_t N, int64_t NP, int B, const unsigned long long* __restrict__ seedp, int G,
                   uint32_t* __restrict__ labels, unsigned* __restrict__ flags) {
  __shared__ uint32_t hist_all[kLabWarps][256];
  __shared__ unsigned long long ck_all[kLabWarps][kLabCand];
  __shared__ uint32_t ci_all[kLabWarps][kLabCand];
  // seed and the index of the first relabelling, from device memory so a
  // captured graph serves every seed and every range of relabellings
  const uint64_t seed = seedp[0], b_off = seedp[1];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint32_t* hist = hist_all[warp];
  unsigned long long* ck = ck_all[warp];
  uint32_t* ci = ci_all[warp];
  const int n = (int)N;
  const int nc = (n + 3) / 4;  // Philox calls per relabelling
  for (int b = blockIdx.x * kLabWarps + warp; b < B; b += gridDim.x * kLabWarps) {
    uint64_t prefix = 0, pmask = 0;
    uint32_t target = (uint32_t)(NP - 1);  // 0-based rank of the last P point
    uint32_t bucket = (uint32_t)n;
    for (int dg = 7; dg >= 0 && bucket > (uint32_t)kLabCand; --dg) {
      for (int v = lane; v < 256; v += 32) hist[v] = 0;
      __syncwarp();
      for (int c = lane; c < nc; c += 32) {
        uint64_t ctr[4] = {(uint64_t)c, b_off + (uint64_t)b, 0ull, 0ull};
        philox4x64_10(ctr, seed, 0ull);
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (4 * c + q < n && (ctr[q] & pmask) == prefix) atomicAdd(&hist[(ctr[q] >> (8 * dg)) & 255u], 1u);
      }
      __syncwarp();
      // lane l owns digits 8l..8l+7: find the digit holding rank `target`
      uint32_t h[8], loc = 0;
#pragma unroll
      for (int q = 0; q < 8; ++q) { h[q] = hist[8 * lane + q]; loc += h[q]; }
      uint32_t incl = loc;
      for (int off = 1; off < 32; off <<= 1) {
        const uint32_t a = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += a;
      }
      const uint32_t excl = incl - loc;
      const bool mine = target >= excl && target < incl;
      const unsigned owner = __ffs(__ballot_sync(0xffffffffu, mine)) - 1;
      uint32_t digit = 0, below = 0, size = 0;
      if (mine) {
        uint32_t run = excl;
        bool found = false;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          if (!found && target < run + h[q]) {
            digit = 8 * lane + q;
            below = run;
            size = h[q];
            found = true;
          }
          run += h[q];
        }
      }
      digit = __shfl_sync(0xffffffffu, digit, owner);
      below = __shfl_sync(0xffffffffu, below, owner);
      bucket = __shfl_sync(0xffffffffu, size, owner);
      target -= below;
      prefix |= (uint64_t)digit << (8 * dg);
      pmask |= (uint64_t)255 << (8 * dg);
      __syncwarp();
    }
    // collect the bucket (keys matching the prefix), then rank it by brute force
    uint32_t cnt = 0;
    for (int c0 = 0; c0 < nc; c0 += 32) {
      const int c = c0 + lane;
      uint64_t ctr[4] = {(uint64_t)c, b_off + (uint64_t)b, 0ull, 0ull};
      if (c < nc) philox4x64_10(ctr, seed, 0ull);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const bool in = c < nc && 4 * c + q < n && (ctr[q] & pmask) == prefix;
        const unsigned m = __ballot_sync(0xffffffffu, in);
        if (in) {
          const uint32_t pos = cnt + __popc(m & ((1u << lane) - 1u));
          if (pos < (uint32_t)kLabCand) { ck[pos] = ctr[q]; ci[pos] = (uint32_t)(4 * c + q); }
        }
        cnt += __popc(m);
      }
    }
    __syncwarp();
    const int nb = (int)(cnt < (uint32_t)kLabCand ? cnt : (uint32_t)kLabCand);
    if (cnt > (uint32_t)kLabCand && lane == 0) atomicOr(flags, ddks::kFlagBounds);  // > 256 equal keys
    unsigned long long tk = 0;
    uint32_t ti = 0;
    bool found = false;
    for (int j = lane; j < nb; j += 32) {
      const unsigned long long kj = ck[j];
      const uint32_t ij = ci[j];
      uint32_t r = 0;
      for (int t = 0; t < nb; ++t) {
        const unsigned long long kt = ck[t];
        r += (kt < kj || (kt == kj && ci[t] < ij)) ? 1u : 0u;
      }
      if (r == target) { tk = kj; ti = ij; found = true; }
    }
    const unsigned own = __ballot_sync(0xffffffffu, found);
    const int src = own ? __ffs(own) - 1 : 0;
    tk = __shfl_sync(0xffffffffu, tk, src);
    ti = __shfl_sync(0xffffffffu, ti, src);
    // the NP smallest (key, index) pairs: (key, i) <= (tk, ti)
    for (int c = lane; c < nc; c += 32) {
      uint64_t ctr[4] = {(uint64_t)c, b_off + (uint64_t)b, 0ull, 0ull};
      philox4x64_10(ctr, seed, 0ull);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int i = 4 * c + q;
        if (i < n && (ctr[q] < tk || (ctr[q] == tk && (uint32_t)i <= ti)))
          atomicOr(&labels[(int64_t)i * G + (b >> 5)], 1u << (b & 31));
      }
    }
    __syncwarp();
  }
}

// codes in shared memory: u8 for d <= 8
template <int D>
__global__ void __launch_bounds__(kCountThreads)
k_perm_count(const uint32_t* __restrict__ rank, int64_t N, int64_t NP, int B, int G,
             const uint32_t* __restrict__ labels, int R, unsigned long long* __restrict__ perm_best) {
  extern __shared__ __align__(16) unsigned char smraw[];
  constexpr int NB = 1 << D;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int WARPS = kCountThreads / 32;
  uint32_t* nbin = reinterpret_cast<uint32_t*>(smraw);            // [NB]
  constexpr int NW = (NB + 1) / 2;                                 // two 16-bit counters per word
  uint32_t* hist = nbin + NB;                                      // [R][NW][kCountThreads]
  uint32_t* ltile = hist + (size_t)R * NW * kCountThreads;         // [kPtsTile][WARPS * R]
  uint8_t* codes = reinterpret_cast<uint8_t*>(ltile + kPtsTile * WARPS * R);  // [N]
  __shared__ uint32_t o[D];
  const int chunk = kCountThreads * R;            // relabellings per pass
  const int nchunks = (B + chunk - 1) / chunk;
  const int wpc = WARPS * R;                      // label words per point per pass
  for (int64_t k = blockIdx.x; k < N; k += gridDim.x) {
    __syncthreads();
    if (tid < D) o[tid] = rank[(int64_t)tid * N + k];
    for (int j = tid; j < NB; j += kCountThreads) nbin[j] = 0;
    __syncthreads();
    for (int64_t i = tid; i < N; i += kCountThreads) {
      uint32_t c = 0;
#pragma unroll
      for (int m = 0; m < D; ++m) c |= (uint32_t)(rank[(int64_t)m * N + i] >= o[m]) << m;
      codes[i] = (uint8_t)c;
      atomicAdd(&nbin[c], 1u);
    }
    for (int ch = 0; ch < nchunks; ++ch) {
      const int b0 = ch * chunk;
      for (int e = tid; e < R * NW * kCountThreads; e += kCountThreads) hist[e] = 0;
      for (int64_t base = 0; base < N; base += kPtsTile) {
        const int cnt = (int)((N - base) < kPtsTile ? (N - base) : kPtsTile);
        __syncthreads();
        // label words of this chunk's groups for the tile's points
        for (int e = tid; e < cnt * wpc; e += kCountThreads) {
          const int p = e / wpc, w = e - p * wpc;
          const int grp = (b0 >> 5) + w;
          ltile[e] = grp < G ? labels[(base + p) * G + grp] : 0u;
        }
        __syncthreads();
        for (int p = 0; p < cnt; ++p) {
          const uint32_t c = codes[base + p];
#pragma unroll 4
          for (int r = 0; r < R; ++r) {
            // relabelling b = b0 + r*kCountThreads + tid: group (b0>>5) + r*WARPS + warp, bit lane
            const uint32_t w = ltile[p * wpc + r * WARPS + warp];
            const uint32_t bit = (w >> lane) & 1u;
            if (bit) atomicAdd(&hist[((size_t)r * NW + (c >> 1)) * kCountThreads + tid], 1u << (16 * (c & 1)));
          }
        }
      }
      __syncthreads();
      for (int r = 0; r < R; ++r) {
        const int b = b0 + r * kCountThreads + tid;
        if (b >= B) continue;
        uint64_t bv = 0;
        for (int j = 0; j < NB; ++j) {
          const uint64_t cp = (hist[((size_t)r * NW + (j >> 1)) * kCountThreads + tid] >> (16 * (j & 1))) & 0xFFFFu;
          const uint64_t n = nbin[j];
          const uint64_t x = cp * (uint64_t)N, y = n * (uint64_t)NP;
          const uint64_t num = x > y ? x - y : y - x;
          bv = num > bv ? num : bv;
        }
        atomicMax(&perm_best[b], (unsigned long long)bv);
      }
    }
  }
}

// ---------------------------------------------------------------- bit-sliced K4
//
// For N <= 4096 and d <= 5 the relabellings are counted 32 at a time in bit
// slices.  First every origin's points are bucketed by orthant code (one
// counting sort per origin, kept in global memory for all passes).  A pass
// takes 256 relabellings: each CTA stages their label words (8 per point) in
// shared memory, and a warp takes an origin and walks its buckets: lane
// (gg, sub) adds the label words of word gg for a quarter of the bucket's
// points into a bit-sliced counter (Harley-Seal carry-save adders over 16
// words at a time, higher planes by ripple), so one 32-bit operation counts
// 32 relabellings.  The four quarters are summed with shuffles, each lane
// extracts the counts of 8 relabellings, and keeps their running maximum of
// |cP*N - n*NP| (n = bucket size).  The pass ends with a shared then a global
// atomicMax per relabelling.
constexpr int kBitsMaxN = 4096;
constexpr int kSortWarps = 8;
constexpr int kBits2Threads = 1024;
constexpr int kPassWords = 8;                 // label words per point per pass
constexpr int kPassPerms = 32 * kPassWords;   // 256 relabellings per pass
constexpr int kHiPlanes = 8;                  // planes of weight 16..2048 (counts < 4096)

DDKS_DEV void csa(uint32_t& h, uint32_t& l, uint32_t a, uint32_t b, uint32_t c) {
  const uint32_t u = a ^ b;
  h = (a & b) | (u & c);
  l = u ^ c;
}

struct Slices {
  uint32_t ones, twos, fours, eights;
  uint32_t hi[kHiPlanes];
};

DDKS_DEV void slices_zero(Slices& z) {
  z.ones = z.twos = z.fours = z.eights = 0;
#pragma unroll
  for (int k = 0; k < kHiPlanes; ++k) z.hi[k] = 0;
}

// add a weight-16 word into the high planes
DDKS_DEV void add16(Slices& z, uint32_t w) {
#pragma unroll
  for (int k = 0; k < kHiPlanes; ++k) {
    const uint32_t t = z.hi[k] & w;
    z.hi[k] ^= w;
    w = t;
  }
}

// plane k of the counter (weights 1, 2, 4, 8, 16, ..., 2048)
DDKS_DEV uint32_t plane(const Slices& z, int k) {
  return k == 0 ? z.ones : k == 1 ? z.twos : k == 2 ? z.fours : k == 3 ? z.eights : z.hi[k - 4];
}

// z += the counter held by lane (lane ^ off): bit-sliced ripple addition
DDKS_DEV void add_partner(Slices& z, int off) {
  constexpr int K = 4 + kHiPlanes;
  uint32_t carry = 0;
  uint32_t out[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const uint32_t a = plane(z, k);
    const uint32_t b = __shfl_xor_sync(0xffffffffu, a, off);
    const uint32_t u = a ^ b;
    out[k] = u ^ carry;
    carry = (a & b) | (u & carry);
  }
  z.ones = out[0]; z.twos = out[1]; z.fours = out[2]; z.eights = out[3];
#pragma unroll
  for (int k = 0; k < kHiPlanes; ++k) z.hi[k] = out[4 + k];
}

// Bucket sort of every origin's points by orthant code, done once for all
// passes: sidx[o][.] lists the pooled points in code order, boff[o][c] is
// where code c starts (boff[o][NB] = N).  One warp per origin; the codes go
// through warp-private shared memory.
template <int D>
__global__ void __launch_bounds__(kSortWarps * 32)
k_perm_sort(const uint32_t* __restrict__ rank, int N, uint16_t* __restrict__ sidx,
            uint16_t* __restrict__ boff) {
  extern __shared__ __align__(16) unsigned char smb[];
  constexpr int NB = 1 << D;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint32_t* cur = reinterpret_cast<uint32_t*>(smb) + warp * NB;               // [warps][NB]
  uint8_t* wc = smb + kSortWarps * NB * 4 + (size_t)warp * ((N + 15) & ~15);  // [warps][N]
  for (int o = blockIdx.x * kSortWarps + warp; o < N; o += gridDim.x * kSortWarps) {
    uint32_t orank[D];
#pragma unroll
    for (int m = 0; m < D; ++m) orank[m] = rank[(int64_t)m * N + o];
    if (lane < NB) cur[lane] = 0;
    __syncwarp();
    for (int i = lane; i < N; i += 32) {
      uint32_t c = 0;
#pragma unroll
      for (int m = 0; m < D; ++m) c |= (uint32_t)(rank[(int64_t)m * N + i] >= orank[m]) << m;
      wc[i] = (uint8_t)c;
      atomicAdd(&cur[c], 1u);
    }
    __syncwarp();
    {
      const uint32_t v = lane < NB ? cur[lane] : 0u;
      uint32_t incl = v;
      for (int off = 1; off < 32; off <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += t;
      }
      if (lane < NB) {
        cur[lane] = incl - v;
        boff[(size_t)o * (NB + 1) + lane] = (uint16_t)(incl - v);
      }
      if (lane == 0) boff[(size_t)o * (NB + 1) + NB] = (uint16_t)N;
    }
    __syncwarp();
    uint16_t* out = sidx + (size_t)o * N;
    for (int i = lane; i < N; i += 32) out[atomicAdd(&cur[wc[i]], 1u)] = (uint16_t)i;
    __syncwarp();
  }
}

// One pass of 256 relabellings: the CTA stages their label words (8 per
// point), each warp takes origins and walks their code buckets.
template <int D>
__global__ void __launch_bounds__(kBits2Threads, 1)
k_perm_bits(const uint16_t* __restrict__ sidx, const uint16_t* __restrict__ boff, int N, int NP, int B,
            int G, int pass, const uint32_t* __restrict__ labels, unsigned long long* __restrict__ perm_best) {
  extern __shared__ __align__(16) uint32_t sm[];
  constexpr int NB = 1 << D;
  uint32_t* lab = sm;                                         // [N][8]
  uint32_t* cmax = lab + (size_t)N * kPassWords;              // [256] per-CTA maxima
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int W = blockDim.x >> 5;
  const int gg = lane & 7, sub = lane >> 3;
  for (int e = threadIdx.x; e < N * kPassWords; e += blockDim.x) {
    const int p = e / kPassWords, w = e - p * kPassWords;
    const int grp = pass * kPassWords + w;
    lab[e] = grp < G ? labels[(int64_t)p * G + grp] : 0u;
  }
  for (int t = threadIdx.x; t < kPassPerms; t += blockDim.x) cmax[t] = 0;
  __syncthreads();
  uint32_t mx[8];
#pragma unroll
  for (int t = 0; t < 8; ++t) mx[t] = 0;
  for (int o = blockIdx.x * W + warp; o < N; o += gridDim.x * W) {
    const uint16_t* si = sidx + (size_t)o * N;
    const uint16_t* bo = boff + (size_t)o * (NB + 1);
    for (int j = 0; j < NB; ++j) {
      const int start = bo[j];
      const int cnt = (int)bo[j + 1] - start;
      if (cnt == 0) continue;
      // quarter of the bucket for this sub-lane: [qa, qb)
      const int q = (cnt + 3) >> 2;
      const int qa = start + sub * q;
      int qb = qa + q;
      if (qb > start + cnt) qb = start + cnt;
      Slices z;
      slices_zero(z);
      for (int b0 = qa; b0 < qb; b0 += 16) {
        uint32_t w[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) w[u] = (b0 + u < qb) ? lab[(int)si[b0 + u] * kPassWords + gg] : 0u;
        uint32_t tA, tB, fA, fB, eA, eB, s16;
        csa(tA, z.ones, z.ones, w[0], w[1]);
        csa(tB, z.ones, z.ones, w[2], w[3]);
        csa(fA, z.twos, z.twos, tA, tB);
        csa(tA, z.ones, z.ones, w[4], w[5]);
        csa(tB, z.ones, z.ones, w[6], w[7]);
        csa(fB, z.twos, z.twos, tA, tB);
        csa(eA, z.fours, z.fours, fA, fB);
        csa(tA, z.ones, z.ones, w[8], w[9]);
        csa(tB, z.ones, z.ones, w[10], w[11]);
        csa(fA, z.twos, z.twos, tA, tB);
        csa(tA, z.ones, z.ones, w[12], w[13]);
        csa(tB, z.ones, z.ones, w[14], w[15]);
        csa(fB, z.twos, z.twos, tA, tB);
        csa(eB, z.fours, z.fours, fA, fB);
        csa(s16, z.eights, z.eights, eA, eB);
        add16(z, s16);
      }
      // sum the four quarters (lanes gg, gg+8, gg+16, gg+24)
      add_partner(z, 8);
      add_partner(z, 16);
      const uint64_t nb = (uint64_t)cnt * (uint64_t)NP;
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const int b = sub * 8 + t;
        uint32_t c = 0;
#pragma unroll
        for (int kk = 0; kk < 4 + kHiPlanes; ++kk) c |= ((plane(z, kk) >> b) & 1u) << kk;
        const uint64_t x = (uint64_t)c * (uint64_t)N;
        const uint64_t num = x > nb ? x - nb : nb - x;
        mx[t] = num > mx[t] ? (uint32_t)num : mx[t];
      }
    }
  }
  // relabelling gg * 32 + sub * 8 + t of this pass: CTA maximum, then global
#pragma unroll
  for (int t = 0; t < 8; ++t)
    if (mx[t]) atomicMax(&cmax[gg * 32 + sub * 8 + t], mx[t]);
  __syncthreads();
  for (int t = threadIdx.x; t < kPassPerms; t += blockDim.x) {
    const int b = pass * kPassPerms + t;
    if (b < B && cmax[t]) atomicMax(&perm_best[b], (unsigned long long)cmax[t]);
  }
}

__global__ void k_perm_pvalue(const unsigned long long* __restrict__ perm_best, int B,
                              const unsigned long long* __restrict__ obs,
                              unsigned long long* __restrict__ count) {
  unsigned long long c = 0;
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < B; b += gridDim.x * blockDim.x)
    c += perm_best[b] >= obs[0] ? 1ull : 0ull;
  for (int off = 16; off > 0; off >>= 1) c += __shfl_down_sync(0xffffffffu, c, off);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

template <int D>
cudaError_t launch_count(const uint32_t* rank, int64_t N, int64_t NP, int B, int G,
                         const uint32_t* labels, unsigned long long* perm_best, cudaStream_t st,
                         int num_sms) {
  constexpr int NB = 1 << D;
  constexpr int WARPS = kCountThreads / 32;
  // relabellings per pass: R per thread, as many as fit 96 KB of histograms
  // (16-bit counters, N <= 16384)
  constexpr int NW = (NB + 1) / 2;
  int R = (96 * 1024) / (NW * kCountThreads * 4);
  if (R < 1) R = 1;
  const int need = (B + kCountThreads - 1) / kCountThreads;
  if (R > need) R = need;
  if (R > 16) R = 16;
  const size_t smem = (size_t)NB * 4 + (size_t)R * NW * kCountThreads * 4 +
                      (size_t)kPtsTile * WARPS * R * 4 + (size_t)N;
  cudaError_t e = ddks_smem_attr(k_perm_count<D>, (int)smem);
  if (e != cudaSuccess) return e;
  int grid = (int)(N < (int64_t)num_sms * 4 ? N : (int64_t)num_sms * 4);
  k_perm_count<D><<<grid, kCountThreads, smem, st>>>(rank, N, NP, B, G, labels, R, perm_best);
  return cudaGetLastError();
}

}  // namespace

// Relabellings b_off .. b_off + B - 1; count_ge = #{b : num_b >= num_obs}.
static int perm_impl(ddks_ctx* ctx, const void* P, int64_t NP, const void* T, int64_t NT, int32_t d,
                     int32_t dtype, uint64_t b_off, int32_t B, uint64_t seed, void* stream, ddks_result* observed,
                     uint64_t* perm_num_max, uint64_t* count_ge, double* p_value) {
  if (!ctx || !observed) return DDKS_EINVAL;
  int rc = ddks_check_problem(P, NP, T, NT, d, dtype);
  if (rc) return observed->status = rc;
  if (B < 0 || B > (1 << 20) || b_off > ((uint64_t)1 << 40)) return observed->status = DDKS_EINVAL;
  const int64_t N = NP + NT;
  if (N > kMaxPermN || d > 8) return observed->status = DDKS_EUNSUPPORTED;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return observed->status = ctx_cuda_fail(ctx, e, "cudaSetDevice");
  const void *dP, *dT;
  if ((rc = ddks_stage_inputs(ctx, P, NP, T, NT, d, dtype, st, &dP, &dT))) return observed->status = rc;
  ddks_plan plan;
  if ((rc = ddks_select_path(ctx, NP, NT, d, &plan))) return observed->status = rc;
  if ((rc = ctx->out3.reserve(ctx, 64 + ddks_reduce_scratch_bytes()))) return observed->status = rc;
  unsigned long long* out3 = (unsigned long long*)ctx->out3.ptr;
  // out3: [0..2] observed result, [4] #{b : num_b >= num_obs}, [6] seed, [7] first relabelling
  ctx->h_out[16] = seed;
  ctx->h_out[17] = b_off;
  e = cudaMemcpyAsync(out3 + 6, ctx->h_out + 16, 16, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return observed->status = ctx_cuda_fail(ctx, e, "seed upload");
  const int G = (B + 31) / 32;
  const int Bc = B > 0 ? B : 1;
  GraphKey key;
  key.add(2).add((uint64_t)NP).add((uint64_t)NT).add((uint64_t)d).add((uint64_t)dtype).add((uint64_t)B);
  key.add((uint64_t)plan.path).add((uint64_t)plan.threads).add((uint64_t)plan.warps);
  key.add((uint64_t)plan.reg_occ).add((uint64_t)plan.fused).add_ptr(dP).add_ptr(dT).add((uint64_t)ctx->stage_timing);
  rc = ddks_graph_run(ctx, key.h, st, [&](cudaStream_t s) -> int {
    int r;
    if ((r = ddks_encode_problem(ctx, dP, NP, dT, NT, d, dtype, s, plan.path == DDKS_PATH_REGISTER))) return r;
    // observed statistic
    if ((r = ctx->best.reserve(ctx, 8 * (size_t)N))) return r;
    if ((r = ctx->bestj.reserve(ctx, 4 * (size_t)N))) return r;
    bool reduced = false;
    if ((r = ddks_count_origins_plan(ctx, plan, NP, NT, d, 0, N, (uint64_t*)ctx->best.ptr,
                                     (int32_t*)ctx->bestj.ptr, s, out3, &reduced)))
      return r;
    cudaError_t ee = cudaSuccess;
    if (!reduced) {
      ee = ddks_launch_reduce((const uint64_t*)ctx->best.ptr, (const int32_t*)ctx->bestj.ptr, N, 0, out3,
                              (char*)ctx->out3.ptr + 64, s);
      ctx->launches += 2;
      if (ee != cudaSuccess) return ctx_cuda_fail(ctx, ee, "reduce");
    }
    if ((r = ctx->perm_labels.reserve(ctx, 4 * (size_t)N * (G > 0 ? G : 1)))) return r;
    if ((r = ctx->perm_best.reserve(ctx, 8 * (size_t)Bc))) return r;
    unsigned long long* pbest = (unsigned long long*)ctx->perm_best.ptr;
    ee = cudaMemsetAsync(out3 + 4, 0, 8, s);  // p-value count
    if (ee == cudaSuccess && B > 0) {
      ee = cudaMemsetAsync(ctx->perm_labels.ptr, 0, 4 * (size_t)N * G, s);
      if (ee == cudaSuccess) ee = cudaMemsetAsync(pbest, 0, 8 * (size_t)B, s);
      if (ee == cudaSuccess) {
        int grid = (B + kLabWarps - 1) / kLabWarps;
        if (grid > ctx->num_sms * 8) grid = ctx->num_sms * 8;
        k_perm_labels_warp<<<grid, kLabWarps * 32, 0, s>>>(N, NP, B, out3 + 6, G, (uint32_t*)ctx->perm_labels.ptr,
                                                           (unsigned*)ctx->flags.ptr);
        ee = cudaGetLastError();
        ctx->launches += 1;
      }
      if (ee == cudaSuccess) {
        const uint32_t* rank = (const uint32_t*)ctx->rank.ptr;
        const uint32_t* lab = (const uint32_t*)ctx->perm_labels.ptr;
        const size_t smem2 = (size_t)N * kPassWords * 4 + (size_t)kPassPerms * 4;
        if (N <= kBitsMaxN && d <= 5 && smem2 <= 227u * 1024u) {
          const int nb1 = (1 << d) + 1;
          ee = ctx->perm_codes.reserve(ctx, (size_t)N * N * 2 + (size_t)N * nb1 * 2 + 64) ? cudaErrorMemoryAllocation
                                                                                            : cudaSuccess;
          uint16_t* sidx = (uint16_t*)ctx->perm_codes.ptr;
          uint16_t* boff = sidx + (size_t)N * N;
          const size_t smem1 = (size_t)kSortWarps * (1 << d) * 4 + (size_t)kSortWarps * ((N + 15) & ~15);
          auto go = [&](auto sortk, auto bitsk) -> cudaError_t {
            cudaError_t q = ddks_smem_attr(sortk, (int)smem1);
            if (q != cudaSuccess) return q;
            int g1 = (int)((N + kSortWarps - 1) / kSortWarps);
            sortk<<<g1, kSortWarps * 32, smem1, s>>>(rank, (int)N, sidx, boff);
            q = ddks_smem_attr(bitsk, (int)smem2);
            if (q != cudaSuccess) return q;
            const int npass = (B + kPassPerms - 1) / kPassPerms;
            for (int pass = 0; pass < npass && q == cudaSuccess; ++pass) {
              bitsk<<<ctx->num_sms, kBits2Threads, smem2, s>>>(sidx, boff, (int)N, (int)NP, B, G, pass, lab, pbest);
              q = cudaGetLastError();
            }
            ctx->launches += npass;  // plus the sort, counted below
            return q;
          };
          if (ee == cudaSuccess) switch (d) {
            case 1: ee = go(k_perm_sort<1>, k_perm_bits<1>); break;
            case 2: ee = go(k_perm_sort<2>, k_perm_bits<2>); break;
            case 3: ee = go(k_perm_sort<3>, k_perm_bits<3>); break;
            case 4: ee = go(k_perm_sort<4>, k_perm_bits<4>); break;
            default: ee = go(k_perm_sort<5>, k_perm_bits<5>); break;
          }
        } else switch (d) {
          case 1: ee = launch_count<1>(rank, N, NP, B, G, lab, pbest, s, ctx->num_sms); break;
          case 2: ee = launch_count<2>(rank, N, NP, B, G, lab, pbest, s, ctx->num_sms); break;
          case 3: ee = launch_count<3>(rank, N, NP, B, G, lab, pbest, s, ctx->num_sms); break;
          case 4: ee = launch_count<4>(rank, N, NP, B, G, lab, pbest, s, ctx->num_sms); break;
          case 5: ee = launch_count<5>(rank, N, NP, B, G, lab, pbest, s, ctx->num_sms); break;
          case 6: ee = launch_count<6>(rank, N, NP, B, G, lab, pbest, s, ctx->num_sms); break;
          case 7: ee = launch_count<7>(rank, N, NP, B, G, lab, pbest, s, ctx->num_sms); break;
          default: ee = launch_count<8>(rank, N, NP, B, G, lab, pbest, s, ctx->num_sms); break;
        }
        ctx->launches += 1;
      }
      if (ee == cudaSuccess) {
        k_perm_pvalue<<<(B + 255) / 256 < 64 ? (B + 255) / 256 : 64, 256, 0, s>>>(pbest, B, out3, out3 + 4);
        ee = cudaGetLastError();
        ctx->launches += 1;
      }
    }
    if (ee != cudaSuccess) return ctx_cuda_fail(ctx, ee, "permutation test");
    return DDKS_OK;
  });
  if (rc) return observed->status = rc;
  unsigned long long* pbest = (unsigned long long*)ctx->perm_best.ptr;
  e = cudaMemcpyAsync(ctx->h_out, out3, 5 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ctx->h_out + 8, ctx->flags.ptr, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && perm_num_max && B > 0)
    e = cudaMemcpyAsync(perm_num_max, pbest, 8 * (size_t)B, cudaMemcpyDefault, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return observed->status = ctx_cuda_fail(ctx, e, "permutation test");
  if ((unsigned)(ctx->h_out[8] & 0xFFFFFFFFull) & ddks::kFlagNaN) return observed->status = DDKS_ENAN;
  if ((unsigned)(ctx->h_out[8] & 0xFFFFFFFFull) & ddks::kFlagTimeout) return observed->status = DDKS_ETIMEOUT;
  if ((unsigned)(ctx->h_out[8] & 0xFFFFFFFFull) & ddks::kFlagBounds) return observed->status = DDKS_EUNSUPPORTED;
  observed->num_max = ctx->h_out[0];
  observed->denom = (uint64_t)NP * (uint64_t)NT;
  observed->D = (double)observed->num_max / (double)observed->denom;
  observed->argmax_origin = (int64_t)ctx->h_out[1];
  observed->argmax_orthant = (int32_t)ctx->h_out[2];
  observed->status = DDKS_OK;
  const unsigned long long ge = B > 0 ? ctx->h_out[4] : 0ull;
  if (count_ge) *count_ge = ge;
  if (p_value) *p_value = (double)(1 + ge) / (double)(1 + (int64_t)B);
  return DDKS_OK;
}

int ddks_permutation_test(ddks_ctx* ctx, const void* P, int64_t NP, const void* T, int64_t NT,
                          int32_t d, int32_t dtype, int32_t B, uint64_t seed, void* stream,
                          ddks_result* observed, uint64_t* perm_num_max, double* p_value) {
  return perm_impl(ctx, P, NP, T, NT, d, dtype, 0, B, seed, stream, observed, perm_num_max, nullptr, p_value);
}

int ddks_permutation_test_range(ddks_ctx* ctx, const void* P, int64_t NP, const void* T, int64_t NT, int32_t d,
                                int32_t dtype, int64_t b_begin, int64_t b_end, uint64_t seed, void* stream,
                                ddks_result* observed, uint64_t* perm_num_max, uint64_t* count_ge) {
  if (!observed) return DDKS_EINVAL;
  if (b_begin < 0 || b_end < b_begin || b_end - b_begin > (1 << 20)) return observed->status = DDKS_EINVAL;
  return perm_impl(ctx, P, NP, T, NT, d, dtype, (uint64_t)b_begin, (int32_t)(b_end - b_begin), seed, stream,
                   observed, perm_num_max, count_ge, nullptr);
}
