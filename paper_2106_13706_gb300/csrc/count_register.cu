// count_register.cu -- K1: orthant counts in registers for d = 2, 3, 4.
//
// Same statistic as every other path (Sec. 2.1, Eq. ddks_tensor_definition;
// the ">=" split of Sec. 2.2.1, Eq. g; max |cP*NT - cT*NP| of Eq. d1 with the
// normalisation of Eq. abs_difference), computed with three devices that keep
// the per-pair work at one subtract per point and origin plus a few bit ops:
//
// 1. Dimension 0 by order.  Each sample's points are sorted by rank in
//    dimension 0.  For an origin o, the points with x_0 < o_0 are exactly a
//    prefix of that order, of length split(o) = #{x : rank_0(x) < rank_0(o)};
//    the loop over a sample therefore knows bit 0 of every code from the
//    position alone (phase A: bit 0 = 0 before split(o), phase B: bit 0 = 1
//    from split(o) on).  Origins are processed in the same order, so the R
//    origins of a thread have nearby splits and only a short window needs a
//    per-pair phase choice.
// 2. SWAR compares for dimensions 1..d-1.  Coordinates are re-ranked into 15
//    bits relative to the origins of a tile of at most 32767 origins
//    (x' = #{tile origins o' : rank(o') <= rank(x)}, which preserves x >= o for
//    every tile origin o) and packed two per 32-bit word with a guard bit on
//    top of each 16-bit field.  One 32-bit subtract of the origin's word then
//    yields the two ">=" results in bits 15 and 31; a byte permute with
//    sign replication turns them into 0x00/0xFF bytes and a 4-way byte dot
//    product turns those into 4 * (orthant index over dims 1..d-1).
// 3. Packed counters.  1 << (4 * index) is added to a word of eight 4-bit
//    counters (one per orthant of dims 1..d-1).  Every 15 points the nibbles
//    are spread into two words of 8-bit counters, and those are added into
//    per-origin shared-memory counts before they can overflow.
//
// Counts land in cnt[origin][sample][phase][bin]; the orthant code of bin b
// in phase p is p | (b << 1).
#include "ddks_host.h"
#include "ddks_internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kR = 4;          // origins per thread
constexpr int kTP = 2048;      // points per shared-memory tile
constexpr int kTileMax = 32767;  // origins per re-rank tile (15-bit fields)

struct OriginMeta {
  uint32_t oA, oB;  // packed re-ranked coordinates of the origin (no guard bits)
  uint32_t sP, sT;  // splits in list coordinates: P part [0,NP), T part [NP,N)
  uint32_t k;       // pooled index
  uint32_t pad;
};

// ------------------------------------------------------------------ preparation

// Flags over the dimension-0 sorted order: row 0 [p] = (sorted point p is in P),
// row 1 [p] = (its pooled index is an origin of [ob, oe)).
__global__ void k_reg_flags(const uint32_t* __restrict__ sidx0, int64_t N, int64_t NP, int64_t ob,
                            int64_t oe, uint32_t* __restrict__ fP, uint32_t* __restrict__ fO) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < N;
       p += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t i = sidx0[p];
    fP[p] = i < (uint64_t)NP ? 1u : 0u;
    fO[p] = (i >= (uint64_t)ob && i < (uint64_t)oe) ? 1u : 0u;
  }
}

// After exclusive scans of the flags:
//   listpos[p]  position of sorted point p in the list (P points in order, then T)
//   pprefix[r]  number of P points among sorted positions [0, r)
//   olist[q]    pooled index of the q-th origin in [ob, oe), in sorted order
__global__ void k_reg_lists(const uint32_t* __restrict__ sidx0, int64_t N, int64_t NP, int64_t ob,
                            int64_t oe, const uint32_t* __restrict__ pprefix,
                            const uint32_t* __restrict__ exO, uint32_t* __restrict__ listpos,
                            uint32_t* __restrict__ olist) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < N;
       p += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t i = sidx0[p];
    const uint32_t pp = pprefix[p];
    listpos[p] = i < (uint64_t)NP ? pp : (uint32_t)(NP + (p - pp));
    if (i >= (uint64_t)ob && i < (uint64_t)oe) olist[exO[p]] = i;
  }
}

// LUT counts: cnt[t][m'][r] += 1 for every origin q of tile t (m' = m - 1).
__global__ void k_reg_lut_count(const uint32_t* __restrict__ rank, const uint32_t* __restrict__ olist,
                                int64_t N, int64_t no, int ds, int TS, uint32_t* __restrict__ lut) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < no * ds;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = e / ds;
    const int mm = (int)(e - q * ds);
    const int64_t t = q / TS;
    const uint32_t r = rank[(int64_t)(mm + 1) * N + olist[q]];
    atomicAdd(&lut[(t * ds + mm) * N + r], 1u);
  }
}

DDKS_DEV uint32_t rerank(const uint32_t* __restrict__ rank, const uint32_t* __restrict__ lut,
                         int64_t N, int ds, int64_t t, int mm, uint32_t i, bool direct) {
  const uint32_t r = rank[(int64_t)(mm + 1) * N + i];
  return direct ? r : lut[(t * ds + mm) * N + r];
}

// Point words of every tile, in list order: words[t][listpos] (uint2: A, B).
__global__ void k_reg_words(const uint32_t* __restrict__ rank, const uint32_t* __restrict__ lut,
                            const uint32_t* __restrict__ sidx0, const uint32_t* __restrict__ listpos,
                            int64_t N, int ds, int64_t ntiles, bool direct, uint2* __restrict__ words) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ntiles * N;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = e / N;
    const int64_t p = e - t * N;
    const uint32_t i = sidx0[p];
    uint32_t A = 0, B = 0;
    A = rerank(rank, lut, N, ds, t, 0, i, direct) | 0x8000u;
    if (ds >= 2) A |= (rerank(rank, lut, N, ds, t, 1, i, direct) | 0x8000u) << 16;
    if (ds >= 3) B = rerank(rank, lut, N, ds, t, 2, i, direct) | 0x8000u;
    words[t * N + listpos[p]] = make_uint2(A, B);
  }
}

__global__ void k_reg_meta(const uint32_t* __restrict__ rank, const uint32_t* __restrict__ lut,
                           const uint32_t* __restrict__ olist, const uint32_t* __restrict__ pprefix,
                           int64_t N, int64_t NP, int64_t no, int ds, int TS, bool direct,
                           OriginMeta* __restrict__ meta) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < no;
       q += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t k = olist[q];
    const int64_t t = q / TS;
    OriginMeta m;
    m.oA = rerank(rank, lut, N, ds, t, 0, k, direct);
    if (ds >= 2) m.oA |= rerank(rank, lut, N, ds, t, 1, k, direct) << 16;
    m.oB = ds >= 3 ? rerank(rank, lut, N, ds, t, 2, k, direct) : 0u;
    const uint32_t r0 = rank[k];
    const uint32_t sp = pprefix[r0];
    m.sP = sp;
    m.sT = (uint32_t)NP + (r0 - sp);
    m.k = k;
    m.pad = 0;
    meta[q] = m;
  }
}

// ------------------------------------------------------------------ main kernel

template <int DS>
struct Swar {
  // sign bytes of the field results: byte 1 of A (dim 1), byte 3 of A (dim 2),
  // byte 1 of B (dim 3); bit 3 of a selector nibble replicates the byte's msb
  static constexpr uint32_t kSel = DS == 3 ? 0x0DB9u : (DS == 2 ? 0x00B9u : 0x0009u);
  // signed byte weights -4, -8, -16: 0xFF bytes become 4 * index
  static constexpr int kW = DS == 3 ? 0x00F0F8FC : (DS == 2 ? 0x0000F8FC : 0x000000FC);
};

template <int DS>
DDKS_DEV uint32_t one_hot(uint32_t xA, uint32_t xB, uint32_t oA, uint32_t oB) {
  const uint32_t dA = xA - oA;
  const uint32_t dB = DS == 3 ? xB - oB : 0u;
  uint32_t sg;
  asm("prmt.b32 %0, %1, %2, %3;" : "=r"(sg) : "r"(dA), "r"(dB), "r"(Swar<DS>::kSel));
  const int sh = __dp4a((int)sg, Swar<DS>::kW, 0);
  uint32_t inc;
  asm("shf.l.wrap.b32 %0, %1, %2, %3;" : "=r"(inc) : "r"(0u), "r"(1u), "r"(sh));
  return inc;
}

struct Acc {
  uint32_t nibA, nibB;            // 4-bit counters, phase A / B
  uint32_t loA, hiA, loB, hiB;    // 8-bit counters (even / odd bins)
};

template <int MODE>  // 0: phase A only, 1: phase B only, 2: both
DDKS_DEV void nib_flush(Acc& a) {
  if (MODE != 1) {
    a.loA += a.nibA & 0x0F0F0F0Fu;
    a.hiA += (a.nibA >> 4) & 0x0F0F0F0Fu;
    a.nibA = 0;
  }
  if (MODE != 0) {
    a.loB += a.nibB & 0x0F0F0F0Fu;
    a.hiB += (a.nibB >> 4) & 0x0F0F0F0Fu;
    a.nibB = 0;
  }
}

// add the 8-bit counters into shared counts c[phase][bin] and clear them
DDKS_DEV void byte_flush(Acc& a, uint32_t* c) {
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const uint32_t la = (a.loA >> (8 * q)) & 0xFFu, ha = (a.hiA >> (8 * q)) & 0xFFu;
    const uint32_t lb = (a.loB >> (8 * q)) & 0xFFu, hb = (a.hiB >> (8 * q)) & 0xFFu;
    if (la) atomicAdd(&c[2 * q], la);
    if (ha) atomicAdd(&c[2 * q + 1], ha);
    if (lb) atomicAdd(&c[8 + 2 * q], lb);
    if (hb) atomicAdd(&c[8 + 2 * q + 1], hb);
  }
  a.loA = a.hiA = a.loB = a.hiB = 0;
}

template <int DS, int MODE>
DDKS_DEV void add_point(const uint2 w, int j, const uint32_t (&oA)[kR], const uint32_t (&oB)[kR],
                        const int (&spl)[kR], Acc (&acc)[kR]) {
#pragma unroll
  for (int r = 0; r < kR; ++r) {
    const uint32_t inc = one_hot<DS>(w.x, w.y, oA[r], oB[r]);
    if (MODE == 0) acc[r].nibA += inc;
    else if (MODE == 1) acc[r].nibB += inc;
    else if (j < spl[r]) acc[r].nibA += inc;
    else acc[r].nibB += inc;
  }
}

template <int DS, int MODE>
DDKS_DEV void chunk15(const uint2* __restrict__ tw, int j, const uint32_t (&oA)[kR],
                      const uint32_t (&oB)[kR], const int (&spl)[kR], Acc (&acc)[kR]) {
#pragma unroll
  for (int u = 0; u < 15; ++u) add_point<DS, MODE>(tw[j + u], j + u, oA, oB, spl, acc);
#pragma unroll
  for (int r = 0; r < kR; ++r) nib_flush<MODE>(acc[r]);
}

// Positions [a, b) of one sample in the tile.  Chunks of 15 points: a chunk
// wholly before every split runs in phase A, one wholly at or after every
// split in phase B, the rest choose per pair.  The nibbles are spread after
// every chunk; the bytes go to the shared counts every 17 chunks (255 points).
template <int DS>
DDKS_DEV void run_points(const uint2* __restrict__ tw, int a, int b, int lo, int hi,
                         const uint32_t (&oA)[kR], const uint32_t (&oB)[kR], const int (&spl)[kR],
                         Acc (&acc)[kR], int& since_flush, uint32_t* cnt_sample) {
  int j = a;
  while (j < b) {
    if (b - j >= 15) {
      if (j + 15 <= lo) chunk15<DS, 0>(tw, j, oA, oB, spl, acc);
      else if (j >= hi) chunk15<DS, 1>(tw, j, oA, oB, spl, acc);
      else chunk15<DS, 2>(tw, j, oA, oB, spl, acc);
      j += 15;
    } else {
      for (; j < b; ++j) add_point<DS, 2>(tw[j], j, oA, oB, spl, acc);
#pragma unroll
      for (int r = 0; r < kR; ++r) nib_flush<2>(acc[r]);
    }
    if (++since_flush == 17) {
#pragma unroll
      for (int r = 0; r < kR; ++r) byte_flush(acc[r], cnt_sample + r * 32);
      since_flush = 0;
    }
  }
}

// Work unit u = (origin block u / C, point chunk u % C): OC origins against the
// list positions [chunk * CL, (chunk + 1) * CL).  Counts are added into the
// global gcnt[q][sample][phase][bin] when the unit ends.
template <int DS>
__global__ void __launch_bounds__(kThreads, 2)
k_register(const uint2* __restrict__ words, const OriginMeta* __restrict__ meta, int64_t no,
           int64_t N, int64_t NP, int S, int TS, int C, int64_t CL,
           uint32_t* __restrict__ gcnt) {
  extern __shared__ __align__(16) uint32_t sm[];
  const int G = kThreads / S;          // origin groups per CTA
  const int OC = G * kR;               // origins per CTA
  uint2* tile = reinterpret_cast<uint2*>(sm);                 // [kTP]
  uint32_t* cnt = sm + 2 * kTP;                               // [OC][2 samples][2 phases][8 bins]
  const int tid = threadIdx.x;
  const int g = tid / S, s = tid - g * S;
  const int64_t blk = blockIdx.x / C;
  const int64_t c0 = (int64_t)(blockIdx.x % C) * CL;
  const int64_t c1 = (c0 + CL) < N ? (c0 + CL) : N;
  const int64_t q0 = blk * OC;
  const int64_t t = q0 / TS;           // re-rank tile (every block lies inside one)
  const uint2* tw_all = words + t * N;
  for (int i = tid; i < OC * 32; i += kThreads) cnt[i] = 0;
  uint32_t oA[kR], oB[kR], sP[kR], sT[kR];
#pragma unroll
  for (int r = 0; r < kR; ++r) {
    const int64_t q = q0 + g * kR + r;
    if (q < no) {
      const OriginMeta m = meta[q];
      oA[r] = m.oA; oB[r] = m.oB; sP[r] = m.sP; sT[r] = m.sT;
    } else {
      // padding origin: counts are discarded; any values keep the loops valid
      oA[r] = 0; oB[r] = 0; sP[r] = 0; sT[r] = (uint32_t)NP;
    }
  }
  Acc acc[kR];
#pragma unroll
  for (int r = 0; r < kR; ++r) acc[r] = Acc{0, 0, 0, 0, 0, 0};
  uint32_t* mycnt = cnt + (g * kR) * 32;  // origin r of this thread: mycnt + r*32 (+16 for T)
  int cur = -1;      // sample whose counts the byte counters hold
  int since = 0;     // chunks since the last byte flush
  for (int64_t base = c0; base < c1; base += kTP) {
    const int cntp = (int)((c1 - base) < kTP ? (c1 - base) : kTP);
    __syncthreads();
    for (int i = tid; i < cntp; i += kThreads) tile[i] = tw_all[base + i];
    __syncthreads();
    // an odd stride between the slices' ranges keeps their loads in distinct banks
    const int64_t per = ((cntp + S - 1) / S) | 1;
    int64_t a = base + s * per;
    int64_t b = a + per;
    if (b > base + cntp) b = base + cntp;
    if (a > b) a = b;
    for (int part = 0; part < 2; ++part) {
      const int64_t pa = part == 0 ? a : (a > NP ? a : NP);
      const int64_t pb = part == 0 ? (b < NP ? b : NP) : b;
      if (pa >= pb) continue;
      if (part != cur) {
        if (cur >= 0) {
#pragma unroll
          for (int r = 0; r < kR; ++r) byte_flush(acc[r], mycnt + cur * 16 + r * 32);
        }
        cur = part;
        since = 0;
      }
      // splits relative to the tile, clamped to [-1, kTP + 1]
      int spl[kR];
      int lo = kTP + 1, hi = -1;
#pragma unroll
      for (int r = 0; r < kR; ++r) {
        int64_t v = (int64_t)(part == 0 ? sP[r] : sT[r]) - base;
        v = v < -1 ? -1 : (v > kTP + 1 ? kTP + 1 : v);
        spl[r] = (int)v;
        lo = spl[r] < lo ? spl[r] : lo;
        hi = spl[r] > hi ? spl[r] : hi;
      }
      run_points<DS>(tile, (int)(pa - base), (int)(pb - base), lo, hi, oA, oB, spl, acc, since,
                     mycnt + part * 16);
    }
  }
  if (cur >= 0) {
#pragma unroll
    for (int r = 0; r < kR; ++r) byte_flush(acc[r], mycnt + cur * 16 + r * 32);
  }
  __syncthreads();
  for (int i = tid; i < OC * 32; i += kThreads) {
    const int64_t q = q0 + i / 32;
    const uint32_t v = cnt[i];
    if (q < no && v) atomicAdd(&gcnt[q * 32 + (i & 31)], v);
  }
}

// one thread per origin: its 2 * 2^DS orthants from gcnt[q][sample][phase][bin]
__global__ void k_reg_final(const uint32_t* __restrict__ gcnt, const OriginMeta* __restrict__ meta,
                                 int64_t no, int64_t NP, int64_t NT, int64_t ob, int ds,
                                 uint64_t* __restrict__ best, int32_t* __restrict__ bestj) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < no;
       q += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t* c = gcnt + q * 32;
    uint64_t bv = 0;
    int bj = 0;
    const int nbin = 1 << ds;
    for (int code = 0; code < 2 * nbin; ++code) {
      const int ph = code & 1, bin = code >> 1;
      const uint64_t cp = c[ph * 8 + bin], ct = c[16 + ph * 8 + bin];
      const uint64_t num = ddks::numer(cp, ct, (uint64_t)NP, (uint64_t)NT);
      if (num > bv) { bv = num; bj = code; }
    }
    const uint32_t k = meta[q].k;
    best[k - ob] = bv;
    bestj[k - ob] = bj;
  }
}

int64_t tile_size(int S) {
  const int OC = (kThreads / S) * kR;
  return (kTileMax / OC) * OC;
}

}  // namespace

bool ddks_register_supported(int d, int64_t NP, int64_t NT) {
  return d >= 2 && d <= 4 && NP + NT < ((int64_t)1 << 31);
}

cudaError_t ddks_launch_register(ddks_ctx* ctx, const uint32_t* rank, int64_t N, int64_t NP,
                                 int64_t NT, int d, int64_t ob, int64_t oe, uint64_t* best,
                                 int32_t* bestj, cudaStream_t st, const ddks_plan& plan) {
  if (!ddks_register_supported(d, NP, NT)) return cudaErrorInvalidValue;
  const int ds = d - 1;
  const int64_t no = oe - ob;
  if (no <= 0) return cudaSuccess;
  // threads sharing one origin group (point slices inside a CTA tile)
  int S = 8;
  if (plan.reg_slices > 0 && plan.reg_slices <= 16 && (plan.reg_slices & (plan.reg_slices - 1)) == 0)
    S = plan.reg_slices;  // tuned choice
  const int64_t TS = tile_size(S);
  const bool direct = N <= 32768;  // min-ranks already fit 15 bits
  const int64_t ntiles = direct ? 1 : (no + TS - 1) / TS;
  // scratch: listpos N, pprefix N+1, olist no, lut ntiles*ds*N (if !direct), words ntiles*N uint2,
  // meta no
  const int64_t lut_rows = direct ? 0 : ntiles * ds;
  const size_t scan_tmp = ddks_scan_tmp_elems(lut_rows > 2 ? lut_rows : 2, N);
  const size_t n_u32 = (size_t)N + (size_t)N + 1 + (size_t)N + (size_t)no + (size_t)no * 32 +
                       (size_t)lut_rows * N + scan_tmp;
  int rc = ctx->reg_meta.reserve(ctx, n_u32 * 4 + (size_t)no * sizeof(OriginMeta) + 64);
  if (rc) return cudaErrorMemoryAllocation;
  rc = ctx->reg_words.reserve(ctx, (size_t)ntiles * N * sizeof(uint2));
  if (rc) return cudaErrorMemoryAllocation;
  uint32_t* listpos = (uint32_t*)ctx->reg_meta.ptr;
  uint32_t* pprefix = listpos + N;
  uint32_t* exO = pprefix + N + 1;
  uint32_t* olist = exO + N;
  uint32_t* gcnt = olist + no;
  uint32_t* lut = gcnt + no * 32;
  uint32_t* stmp = lut + lut_rows * N;
  OriginMeta* meta = reinterpret_cast<OriginMeta*>(
      (reinterpret_cast<uintptr_t>(stmp + scan_tmp) + 15) & ~(uintptr_t)15);
  uint2* words = (uint2*)ctx->reg_words.ptr;
  const uint32_t* sidx0 = (const uint32_t*)ctx->sidx0.ptr;

  auto grid = [](int64_t w) { int64_t g = (w + 255) / 256; return (int)(g > 152 * 32 ? 152 * 32 : (g < 1 ? 1 : g)); };
  int n = 0;
  k_reg_flags<<<grid(N), 256, 0, st>>>(sidx0, N, NP, ob, oe, pprefix, exO);
  ++n;
  // pprefix and exO are adjacent rows of N + 1 and N entries: scan them separately
  cudaError_t e0 = ddks_scan_rows(pprefix, pprefix, 1, N, true, stmp, st, &n);
  if (e0 == cudaSuccess) e0 = ddks_scan_rows(exO, exO, 1, N, true, stmp, st, &n);
  if (e0 != cudaSuccess) return e0;
  k_reg_lists<<<grid(N), 256, 0, st>>>(sidx0, N, NP, ob, oe, pprefix, exO, listpos, olist);
  ++n;
  if (!direct) {
    cudaError_t e = cudaMemsetAsync(lut, 0, (size_t)lut_rows * N * 4, st);
    if (e != cudaSuccess) return e;
    k_reg_lut_count<<<grid(no * ds), 256, 0, st>>>(rank, olist, N, no, ds, (int)TS, lut);
    ++n;
    e = ddks_scan_rows(lut, lut, lut_rows, N, false, stmp, st, &n);
    if (e != cudaSuccess) return e;
  }
  k_reg_words<<<grid(ntiles * N), 256, 0, st>>>(rank, lut, sidx0, listpos, N, ds, ntiles, direct, words);
  k_reg_meta<<<grid(no), 256, 0, st>>>(rank, lut, olist, pprefix, N, NP, no, ds, (int)TS, direct, meta);
  n += 2;
  const int OC = (kThreads / S) * kR;
  const size_t smem = (size_t)kTP * sizeof(uint2) + (size_t)OC * 32 * 4;
  const int64_t blocks = (no + OC - 1) / OC;
  // point chunks per origin block: about 8 waves of 2 resident CTAs per SM,
  // chunks of at least 2 tiles
  const int64_t slots = (int64_t)ctx->num_sms * 2;
  int64_t C = (8 * slots + blocks - 1) / blocks;
  const int64_t cmax = (N + 2 * kTP - 1) / (2 * kTP);
  if (C > cmax) C = cmax;
  if (C < 1) C = 1;
  const int64_t CL = (N + C - 1) / C;
  C = (N + CL - 1) / CL;
  cudaError_t e = cudaMemsetAsync(gcnt, 0, (size_t)no * 32 * 4, st);
  if (e != cudaSuccess) return e;
  const unsigned ctas = (unsigned)(blocks * C);
  // stage timing: the count stage starts here (the preparation above counts as encoding)
  if (ctx->stage_timing) cudaEventRecord(ctx->ev[1], st);
  switch (ds) {
    case 1:
      e = cudaFuncSetAttribute(k_register<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e == cudaSuccess)
        k_register<1><<<ctas, kThreads, smem, st>>>(words, meta, no, N, NP, S, (int)TS, (int)C, CL, gcnt);
      break;
    case 2:
      e = cudaFuncSetAttribute(k_register<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e == cudaSuccess)
        k_register<2><<<ctas, kThreads, smem, st>>>(words, meta, no, N, NP, S, (int)TS, (int)C, CL, gcnt);
      break;
    default:
      e = cudaFuncSetAttribute(k_register<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e == cudaSuccess)
        k_register<3><<<ctas, kThreads, smem, st>>>(words, meta, no, N, NP, S, (int)TS, (int)C, CL, gcnt);
      break;
  }
  if (e != cudaSuccess) return e;
  k_reg_final<<<grid(no), 256, 0, st>>>(gcnt, meta, no, NP, NT, ob, ds, best, bestj);
  n += 2;
  ctx->launches += n;
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}
