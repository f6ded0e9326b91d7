// count_register.cu -- K1: orthant counts in registers for d = 2, 3, 4.
//
// Same statistic as every other path (Sec. 2.1, Eq. ddks_tensor_definition;
// the ">=" split of Sec. 2.2.1, Eq. g; max |cP*NT - cT*NP| of Eq. d1 with the
// normalisation of Eq. abs_difference), computed with three devices that keep
// the per-pair work at one subtract per point and origin plus a few bit ops:
//
// 1. Dimension 0 by order.  Each sample's points are listed in increasing rank
//    in dimension 0 (the P list, then the T list).  For an origin o, the points
//    of a sample with x_0 < o_0 are exactly a prefix of its list, of length
//    split(o) = #{x : rank_0(x) < rank_0(o)}: bit 0 of a code is known from
//    the position alone (phase A before the split, phase B from it on).
//    Origins are processed in the same order, so the origins of a warp have
//    nearby splits and only a short window needs a per-pair phase choice.
// 2. SWAR compares for dimensions 1..d-1.  A CTA owns 128 origins.  For each of
//    those dimensions it builds, in shared memory, a bitmap over the global
//    ranks of its origins' values and per-word prefix counts, and re-ranks
//    every point as x' = #{distinct origin values <= x} (at most 128).  This
//    keeps x >= o <=> x' >= o' for every origin of the CTA.  The re-ranked
//    values go into 9-bit fields of one 32-bit word (guard bits 8, 17, 26);
//    one 32-bit subtract of the origin's word yields all d-1 ">=" results in
//    the guard bits, a mask keeps them, and a byte dot product (dp4a) turns
//    them into 4 * (orthant index over dims 1..d-1).
// 3. Packed counters.  1 << (4 * index) is added to a word of eight 4-bit
//    counters (two points' one-hots per 3-input add).  After every chunk of
//    12 points the nibbles are spread into two words of 8-bit counters, and
//    every 21 chunks those are added into per-origin shared counts, which go
//    to global counts when the work unit ends.
//
// Work units: (block of 128 origins) x (chunk of one sample's list); a CTA
// works on one unit.  Within a staged tile of points the 8 threads that share
// an origin group take interleaved 12-point chunks, so a warp's lanes read
// distinct banks and move through the tile together.
#include "ddks_host.h"
#include "ddks_internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kR = 4;              // origins per thread
constexpr int kS = 8;              // threads sharing one origin group
constexpr int kG = kThreads / kS;  // origin groups per CTA
constexpr int kOC = kG * kR;       // origins per CTA (128: re-ranked values fit 8 bits)
constexpr int kCh = 12;            // points per chunk (<= 15 for 4-bit counters)
constexpr int kTP = kCh * kS * 22; // points per staged tile (2112)
constexpr int64_t kMaxRegN = 200000;
constexpr int kSlot = 17;          // shared counter words per origin (16 + 1 pad: no bank aliasing)

struct OriginMeta {
  uint32_t sP, sT;  // splits in list coordinates: P part [0, NP), T part [NP, N)
  uint32_t k;       // pooled index
  uint32_t pad;
};

// ------------------------------------------------------------------ preparation

// Flags over the dimension-0 sorted order: fP[p] = (sorted point p is in P),
// fO[p] = (its pooled index is an origin of [ob, oe)).
__global__ void k_reg_flags(const uint32_t* __restrict__ sidx0, int64_t N, int64_t NP, int64_t ob,
                            int64_t oe, uint32_t* __restrict__ fP, uint32_t* __restrict__ fO) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < N;
       p += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t i = sidx0[p];
    fP[p] = i < (uint64_t)NP ? 1u : 0u;
    fO[p] = (i >= (uint64_t)ob && i < (uint64_t)oe) ? 1u : 0u;
  }
}

// After exclusive scans of the flags (pprefix, exO):
//   rankL[m'][l]  rank in dimension m'+1 of the point at list position l
//                 (list = P points by increasing rank_0, then T points)
//   olist[q]      pooled index of the q-th origin of [ob, oe), in sorted order
__global__ void k_reg_lists(const uint32_t* __restrict__ sidx0, const uint32_t* __restrict__ rank,
                            int64_t N, int64_t NP, int ds, int64_t ob, int64_t oe,
                            const uint32_t* __restrict__ pprefix, const uint32_t* __restrict__ exO,
                            uint32_t* __restrict__ rankL, uint32_t* __restrict__ olist) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < N;
       p += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t i = sidx0[p];
    const uint32_t pp = pprefix[p];
    const int64_t l = i < (uint64_t)NP ? (int64_t)pp : NP + (p - pp);
    for (int m = 0; m < ds; ++m) rankL[(int64_t)m * N + l] = rank[(int64_t)(m + 1) * N + i];
    if (i >= (uint64_t)ob && i < (uint64_t)oe) olist[exO[p]] = i;
  }
}

__global__ void k_reg_meta(const uint32_t* __restrict__ rank, const uint32_t* __restrict__ olist,
                           const uint32_t* __restrict__ pprefix, int64_t NP, int64_t no,
                           OriginMeta* __restrict__ meta) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < no;
       q += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t k = olist[q];
    const uint32_t r0 = rank[k];       // dimension 0
    const uint32_t sp = pprefix[r0];   // P points with a smaller dimension-0 value
    OriginMeta m;
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
  // guard bits of the 9-bit fields: 8, 17, 26
  static constexpr uint32_t kGuard = DS == 3 ? 0x04020100u : (DS == 2 ? 0x00020100u : 0x00000100u);
  // after masking, byte 1 holds b1, byte 2 holds 2*b2, byte 3 holds 4*b3;
  // weights 4 give 4*b1 + 8*b2 + 16*b3 = 4 * index
  static constexpr uint32_t kW = 0x04040400u;
};

// a * b + c on the FMA pipe: b is the kernel argument `one` (= 1), which the
// compiler cannot fold, so the add is not moved onto the ALU pipe that the
// mask and shift already load
DDKS_DEV uint32_t mad(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t r;
  asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
  return r;
}

// on = -o (the origin's word negated): x - o = x + on
template <int DS>
DDKS_DEV uint32_t one_hot(uint32_t x, uint32_t on, uint32_t one) {
  const uint32_t g = mad(on, one, x) & Swar<DS>::kGuard;
  const uint32_t sh = __dp4a(g, Swar<DS>::kW, 0u);
  uint32_t inc;
  asm("shf.l.wrap.b32 %0, %1, %2, %3;" : "=r"(inc) : "r"(0u), "r"(1u), "r"(sh));
  return inc;
}

struct Acc {
  uint32_t nibA, nibB;            // 4-bit counters, phase A / B
  uint32_t loA, hiA, loB, hiB;    // 8-bit counters (even / odd bins)
};

template <int MODE>  // 0: phase A only, 1: phase B only, 2: both
DDKS_DEV void nib_flush(Acc& a, uint32_t one) {
  if (MODE != 1) {
    a.loA = mad(a.nibA & 0x0F0F0F0Fu, one, a.loA);
    a.hiA = mad((a.nibA >> 4) & 0x0F0F0F0Fu, one, a.hiA);
    a.nibA = 0;
  }
  if (MODE != 0) {
    a.loB = mad(a.nibB & 0x0F0F0F0Fu, one, a.loB);
    a.hiB = mad((a.nibB >> 4) & 0x0F0F0F0Fu, one, a.hiB);
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

// two points at once: their one-hots are added with one 3-input add
template <int DS, int MODE>
DDKS_DEV void add_two(uint32_t x0, uint32_t x1, int j, const uint32_t (&ow)[kR],
                      const int (&spl)[kR], Acc (&acc)[kR], uint32_t one) {
#pragma unroll
  for (int r = 0; r < kR; ++r) {
    const uint32_t i0 = one_hot<DS>(x0, ow[r], one);
    const uint32_t i1 = one_hot<DS>(x1, ow[r], one);
    if (MODE == 0) {
      acc[r].nibA = acc[r].nibA + i0 + i1;
    } else if (MODE == 1) {
      acc[r].nibB = acc[r].nibB + i0 + i1;
    } else {
      if (j < spl[r]) acc[r].nibA += i0; else acc[r].nibB += i0;
      if (j + 1 < spl[r]) acc[r].nibA += i1; else acc[r].nibB += i1;
    }
  }
}

template <int DS, int MODE>
DDKS_DEV void chunk12(const uint32_t* __restrict__ tile, int j, const uint32_t (&ow)[kR],
                      const int (&spl)[kR], Acc (&acc)[kR], uint32_t one) {
  const uint4* p = reinterpret_cast<const uint4*>(tile + j);
#pragma unroll
  for (int v = 0; v < 3; ++v) {
    const uint4 w = p[v];
    add_two<DS, MODE>(w.x, w.y, j + 4 * v, ow, spl, acc, one);
    add_two<DS, MODE>(w.z, w.w, j + 4 * v + 2, ow, spl, acc, one);
  }
#pragma unroll
  for (int r = 0; r < kR; ++r) nib_flush<MODE>(acc[r], one);
}

template <int DS>
DDKS_DEV void chunk_partial(const uint32_t* __restrict__ tile, int j, int n,
                            const uint32_t (&ow)[kR], const int (&spl)[kR], Acc (&acc)[kR],
                            uint32_t one) {
  for (int u = 0; u < n; ++u) {
    const uint32_t x = tile[j + u];
#pragma unroll
    for (int r = 0; r < kR; ++r) {
      const uint32_t inc = one_hot<DS>(x, ow[r], one);
      if (j + u < spl[r]) acc[r].nibA += inc; else acc[r].nibB += inc;
    }
  }
#pragma unroll
  for (int r = 0; r < kR; ++r) nib_flush<2>(acc[r], one);
}

// Unit u: origin block u / C, chunk u % C of the lists, where chunks
// [0, CP) cover the P list [0, NP) in pieces of CLP and chunks [CP, C) the
// T list [NP, N) in pieces of CLT.
template <int DS, int OCC>
__global__ void __launch_bounds__(kThreads, OCC)
k_register(const uint32_t* __restrict__ rankL, const uint32_t* __restrict__ rank,
           const OriginMeta* __restrict__ meta, int64_t no, int64_t N, int64_t NP, int C, int CP,
           int64_t CLP, int64_t CLT, int NW, uint32_t one, uint32_t* __restrict__ gcnt) {
  extern __shared__ __align__(16) uint32_t sm[];
  uint32_t* tile = sm;                                        // [kTP] packed words
  uint32_t* raw = tile + kTP;                                 // [DS][kTP] next tile's ranks
  uint32_t* cnt = raw + DS * kTP;                             // [kOC][17]: [2 phases][8 bins] + pad
  uint32_t* bits = cnt + kOC * kSlot;                         // [DS][NW] bitmaps over ranks
  uint8_t* pre = reinterpret_cast<uint8_t*>(bits + DS * NW);  // [DS][NW] word prefix counts
  const int tid = threadIdx.x;
  const int g = tid / kS, s = tid - g * kS;
  const int64_t blk = blockIdx.x / C;
  const int ci = blockIdx.x % C;
  const int sample = ci < CP ? 0 : 1;
  int64_t c0, c1;
  if (sample == 0) {
    c0 = (int64_t)ci * CLP;
    c1 = c0 + CLP < NP ? c0 + CLP : NP;
  } else {
    c0 = NP + (int64_t)(ci - CP) * CLT;
    c1 = c0 + CLT < N ? c0 + CLT : N;
  }
  const int64_t q0 = blk * kOC;
  const int nq = (int)((no - q0) < kOC ? (no - q0) : kOC);

  // re-rank tables of this CTA's origins
  for (int i = tid; i < kOC * kSlot; i += kThreads) cnt[i] = 0;
  for (int i = tid; i < DS * NW; i += kThreads) bits[i] = 0;
  __syncthreads();
  for (int i = tid; i < nq * DS; i += kThreads) {
    const int qq = i / DS, m = i - qq * DS;
    const uint32_t r = rank[(int64_t)(m + 1) * N + meta[q0 + qq].k];
    atomicOr(&bits[m * NW + (r >> 5)], 1u << (r & 31));
  }
  __syncthreads();
  {  // exclusive prefix of the popcounts, per dimension: each warp scans one
     // contiguous segment of every dimension, segment totals combine in cnt
    const int warp = tid >> 5, lane = tid & 31;
    constexpr int W = kThreads / 32;
    const int seg = (NW + W - 1) / W;
    uint32_t* segsum = cnt;  // [DS][W], cleared again below
    for (int m = 0; m < DS; ++m) {
      const int a = warp * seg, b = a + seg < NW ? a + seg : NW;
      uint32_t carry = 0;
      for (int base = a; base < b; base += 32) {
        const int w = base + lane;
        const uint32_t c = w < b ? (uint32_t)__popc(bits[m * NW + w]) : 0u;
        uint32_t incl = c;
        for (int off = 1; off < 32; off <<= 1) {
          const uint32_t x = __shfl_up_sync(0xffffffffu, incl, off);
          if (lane >= off) incl += x;
        }
        if (w < b) pre[m * NW + w] = (uint8_t)(carry + incl - c);
        carry += __shfl_sync(0xffffffffu, incl, 31);
      }
      if (lane == 0) segsum[m * W + warp] = carry;
    }
    __syncthreads();
    for (int m = 0; m < DS; ++m) {
      uint32_t off = 0;
      for (int w = 0; w < warp; ++w) off += segsum[m * W + w];
      const int a = warp * seg, b = a + seg < NW ? a + seg : NW;
      for (int w = a + lane; w < b; w += 32) pre[m * NW + w] = (uint8_t)(pre[m * NW + w] + off);
    }
    __syncthreads();
    for (int i = tid; i < DS * W; i += kThreads) segsum[i] = 0;
  }
  __syncthreads();
  // x' = #{distinct origin values whose rank <= r}
  auto rerank = [&](int m, uint32_t r) -> uint32_t {
    const uint32_t w = bits[m * NW + (r >> 5)];
    return (uint32_t)pre[m * NW + (r >> 5)] + (uint32_t)__popc(w & (0xFFFFFFFFu >> (31 - (r & 31))));
  };

  uint32_t ow[kR];
  int sa[kR];  // this sample's split, list coordinates
#pragma unroll
  for (int r = 0; r < kR; ++r) {
    const int64_t q = q0 + g * kR + r;
    if (q < no) {
      const OriginMeta m = meta[q];
      uint32_t w = 0;
#pragma unroll
      for (int mm = 0; mm < DS; ++mm) w |= rerank(mm, rank[(int64_t)(mm + 1) * N + m.k]) << (9 * mm);
      ow[r] = 0u - w;  // negated: the subtract becomes a multiply-add
      sa[r] = (int)(sample == 0 ? m.sP : m.sT);
    } else {
      ow[r] = 0;  // padding origin: its counts are discarded
      sa[r] = 0;
    }
  }
  Acc acc[kR];
#pragma unroll
  for (int r = 0; r < kR; ++r) acc[r] = Acc{0, 0, 0, 0, 0, 0};
  uint32_t* mycnt = cnt + (g * kR) * kSlot;  // origin r of this thread: mycnt + r * kSlot
  int since = 0;  // chunk iterations since the last byte flush (uniform across the CTA)
  // raw ranks of a tile are copied asynchronously while the previous tile is counted
  auto prefetch = [&](int64_t base) {
    const int cntp = (int)((c1 - base) < kTP ? (c1 - base) : kTP);
#pragma unroll
    for (int mm = 0; mm < DS; ++mm) {
      const uint32_t* src = rankL + (int64_t)mm * N + base;
      const unsigned dst = (unsigned)__cvta_generic_to_shared(raw + mm * kTP);
      for (int i = tid; i < cntp; i += kThreads)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst + 4u * i), "l"(src + i) : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  prefetch(c0);
  for (int64_t base = c0; base < c1; base += kTP) {
    const int cntp = (int)((c1 - base) < kTP ? (c1 - base) : kTP);
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    for (int i = tid; i < cntp; i += kThreads) {
      uint32_t w = 0;
#pragma unroll
      for (int mm = 0; mm < DS; ++mm) w |= (rerank(mm, raw[mm * kTP + i]) | 0x100u) << (9 * mm);
      tile[i] = w;
    }
    __syncthreads();
    if (base + kTP < c1) prefetch(base + kTP);
    // splits relative to the tile, clamped to [-1, kTP + 1]
    int spl[kR];
    int lo = kTP + 1, hi = -1;
#pragma unroll
    for (int r = 0; r < kR; ++r) {
      int64_t v = (int64_t)sa[r] - base;
      v = v < -1 ? -1 : (v > kTP + 1 ? kTP + 1 : v);
      spl[r] = (int)v;
      lo = spl[r] < lo ? spl[r] : lo;
      hi = spl[r] > hi ? spl[r] : hi;
    }
    const int iters = (cntp + kS * kCh - 1) / (kS * kCh);
    for (int it = 0; it < iters; ++it) {
      const int j = (it * kS + s) * kCh;
      if (j < cntp) {
        const int n = cntp - j < kCh ? cntp - j : kCh;
        if (n == kCh) {
          if (j + kCh <= lo) chunk12<DS, 0>(tile, j, ow, spl, acc, one);
          else if (j >= hi) chunk12<DS, 1>(tile, j, ow, spl, acc, one);
          else chunk12<DS, 2>(tile, j, ow, spl, acc, one);
        } else {
          chunk_partial<DS>(tile, j, n, ow, spl, acc, one);
        }
      }
      if (++since == 21) {
#pragma unroll
        for (int r = 0; r < kR; ++r) byte_flush(acc[r], mycnt + r * kSlot);
        since = 0;
      }
    }
  }
#pragma unroll
  for (int r = 0; r < kR; ++r) byte_flush(acc[r], mycnt + r * kSlot);
  __syncthreads();
  for (int i = tid; i < nq * 16; i += kThreads) {
    const uint32_t v = cnt[(i >> 4) * kSlot + (i & 15)];
    if (v) atomicAdd(&gcnt[(q0 + (i >> 4)) * 32 + sample * 16 + (i & 15)], v);
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

size_t reg_smem(int ds, int NW) {
  return (size_t)kTP * 4 * (1 + ds) + (size_t)kOC * kSlot * 4 + (size_t)ds * NW * 4 + (size_t)ds * NW + 16;
}

}  // namespace

bool ddks_register_supported(int d, int64_t NP, int64_t NT) {
  const int64_t N = NP + NT;
  if (d < 2 || d > 4 || N > kMaxRegN) return false;
  return reg_smem(d - 1, (int)((N + 31) / 32)) <= 200u * 1024u;
}

cudaError_t ddks_launch_register(ddks_ctx* ctx, const uint32_t* rank, int64_t N, int64_t NP,
                                 int64_t NT, int d, int64_t ob, int64_t oe, uint64_t* best,
                                 int32_t* bestj, cudaStream_t st, const ddks_plan& plan) {
  if (!ddks_register_supported(d, NP, NT)) return cudaErrorInvalidValue;
  const int ds = d - 1;
  const int64_t no = oe - ob;
  if (no <= 0) return cudaSuccess;
  const int NW = (int)((N + 31) / 32);
  // scratch (u32): pprefix N, exO N, olist no, gcnt no*32, rankL ds*N, scan tmp; then meta
  const size_t scan_tmp = ddks_scan_tmp_elems(1, N);
  const size_t n_u32 = (size_t)N * 2 + (size_t)no + (size_t)no * 32 + (size_t)ds * N + scan_tmp;
  int rc = ctx->reg_meta.reserve(ctx, n_u32 * 4 + (size_t)no * sizeof(OriginMeta) + 64);
  if (rc) return cudaErrorMemoryAllocation;
  uint32_t* pprefix = (uint32_t*)ctx->reg_meta.ptr;
  uint32_t* exO = pprefix + N;
  uint32_t* olist = exO + N;
  uint32_t* gcnt = olist + no;
  uint32_t* rankL = gcnt + no * 32;
  uint32_t* stmp = rankL + (size_t)ds * N;
  OriginMeta* meta = reinterpret_cast<OriginMeta*>(
      (reinterpret_cast<uintptr_t>(stmp + scan_tmp) + 15) & ~(uintptr_t)15);
  const uint32_t* sidx0 = (const uint32_t*)ctx->sidx0.ptr;

  auto grid = [](int64_t w) { int64_t g = (w + 255) / 256; return (int)(g > 152 * 32 ? 152 * 32 : (g < 1 ? 1 : g)); };
  int n = 0;
  k_reg_flags<<<grid(N), 256, 0, st>>>(sidx0, N, NP, ob, oe, pprefix, exO);
  ++n;
  cudaError_t e = ddks_scan_rows(pprefix, pprefix, 1, N, true, stmp, st, &n);
  if (e == cudaSuccess) e = ddks_scan_rows(exO, exO, 1, N, true, stmp, st, &n);
  if (e != cudaSuccess) return e;
  k_reg_lists<<<grid(N), 256, 0, st>>>(sidx0, rank, N, NP, ds, ob, oe, pprefix, exO, rankL, olist);
  k_reg_meta<<<grid(no), 256, 0, st>>>(rank, olist, pprefix, NP, no, meta);
  n += 2;
  const int64_t blocks = (no + kOC - 1) / kOC;
  // chunks of the lists per origin block: about 3 waves of the resident CTAs
  const int64_t slots = (int64_t)ctx->num_sms * 3;
  int64_t want = (3 * slots + blocks - 1) / blocks;  // chunks per block
  if (want < 2) want = 2;
  int64_t CL = (N + want - 1) / want;
  if (CL < 2 * kTP) CL = 2 * kTP;
  const int64_t CP = (NP + CL - 1) / CL, CT = (NT + CL - 1) / CL;
  const int64_t CLP = (NP + CP - 1) / CP, CLT = (NT + CT - 1) / CT;
  const int64_t C = CP + CT;
  e = cudaMemsetAsync(gcnt, 0, (size_t)no * 32 * 4, st);
  if (e != cudaSuccess) return e;
  const size_t smem = reg_smem(ds, NW);
  const unsigned ctas = (unsigned)(blocks * C);
  // stage timing: the count stage starts here (the preparation above counts as encoding)
  ddks_stage_mark(ctx, 1, st);
  int occ = plan.reg_occ == 2 || plan.reg_occ == 3 ? plan.reg_occ : 4;
  while (occ > 2 && (size_t)occ * (smem + 1024) > 227u * 1024u) --occ;  // shared memory bound
  auto go = [&](auto kern) -> cudaError_t {
    cudaError_t r = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (r != cudaSuccess) return r;
    kern<<<ctas, kThreads, smem, st>>>(rankL, rank, meta, no, N, NP, (int)C, (int)CP, CLP, CLT, NW, 1u, gcnt);
    return cudaGetLastError();
  };
  if (ds == 1) e = occ == 2 ? go(k_register<1, 2>) : occ == 3 ? go(k_register<1, 3>) : go(k_register<1, 4>);
  else if (ds == 2) e = occ == 2 ? go(k_register<2, 2>) : occ == 3 ? go(k_register<2, 3>) : go(k_register<2, 4>);
  else e = occ == 2 ? go(k_register<3, 2>) : occ == 3 ? go(k_register<3, 3>) : go(k_register<3, 4>);
  if (e != cudaSuccess) return e;
  k_reg_final<<<grid(no), 256, 0, st>>>(gcnt, meta, no, NP, NT, ob, ds, best, bestj);
  n += 2;
  ctx->launches += n;
  return cudaGetLastError();
}
