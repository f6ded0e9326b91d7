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
// 2. SWAR compares for dimensions 1..d-1.  Origins form blocks of 128.  For
//    each block and each of those dimensions, every point is re-ranked as
//    x' = #{distinct values of the block's origins <= x} (at most 128), which
//    keeps x >= o <=> x' >= o' for every origin of the block.  A pack kernel,
//    one CTA per (block, dimension), writes these values once as byte planes.
//    The counting kernel streams the planes and assembles, per tile, 9-bit
//    fields of one 32-bit word per point (guard bits 8, 17, 26); one 32-bit
//    subtract of the origin's word yields all d-1 ">=" results in the guard
//    bits, a mask keeps them, and a byte dot product (dp4a) turns them into
//    4 * (orthant index over dims 1..d-1).
// 3. Packed counters.  1 << (4 * index) is added to a word of eight 4-bit
//    counters (two points' one-hots per 3-input add).  After every chunk of
//    12 points the nibbles are spread into two words of 8-bit counters, and
//    every 21 chunks those are added into per-origin shared counts, which go
//    to global counts when the work unit ends.
//
// Work units: (block of 128 origins) x (chunk of one sample's list); a CTA
// works on one unit.  Tiles of a unit's byte planes arrive in shared memory by
// bulk asynchronous copies (the TMA engine) into a two-stage ring, completion
// on an mbarrier.  Within a tile the 8 threads that share an origin group take
// interleaved 12-point chunks, so a warp's lanes read distinct banks and move
// through the tile together.
#include "ddks_host.h"
#include "ddks_internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kR = 4;              // origins per thread
constexpr int kS = 8;              // threads sharing one origin group
constexpr int kG = kThreads / kS;  // origin groups per CTA
constexpr int kOC = kG * kR;       // origins per block (128: re-ranked values fit 8 bits)
constexpr int kCh = 12;            // points per chunk (<= 15 for 4-bit counters)
constexpr int kTP = kCh * kS * 22; // points per staged tile (2112, a multiple of 16)
constexpr int64_t kMaxRegN = 200000;
constexpr int kSlot = 9;           // shared counter words per origin (8 + 1 pad: no bank aliasing)
constexpr int64_t kMaxChunk = 65520; // list chunk of a unit: its counts fit 16 bits
constexpr int kPackThreads = 256;
constexpr int kPack4Threads = 1024;
constexpr unsigned long long kWaitNs = 1000000000ull;  // bound on one tile wait (1 s)

struct OriginMeta {
  uint32_t sP, sT;  // splits, sample-local: P points / T points with a smaller dimension-0 rank
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
//   rankL[m'][pos]  rank in dimension m'+1 of the point at list position pos
//                   (P points by increasing rank_0 at [0, NP), T points at
//                   [NPpad, NPpad + NT); the padding positions hold rank 0)
//   olist[q]        pooled index of the q-th origin of [ob, oe), in sorted order
//                   (exO = nullptr: every point is an origin, q = p)
__global__ void k_reg_lists(const uint32_t* __restrict__ sidx0, const uint32_t* __restrict__ rank,
                            int64_t N, int64_t NP, int64_t NPpad, int64_t Lrow, int ds, int64_t ob,
                            int64_t oe, const uint32_t* __restrict__ pprefix,
                            const uint32_t* __restrict__ exO, uint32_t* __restrict__ rankL,
                            uint32_t* __restrict__ olist) {
  const int64_t NT = N - NP;
  if (blockIdx.x == 0 && threadIdx.x < 16) {
    for (int m = 0; m < ds; ++m) {
      if (NP + threadIdx.x < NPpad) rankL[(int64_t)m * Lrow + NP + threadIdx.x] = 0;
      if (NPpad + NT + threadIdx.x < Lrow) rankL[(int64_t)m * Lrow + NPpad + NT + threadIdx.x] = 0;
    }
  }
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < N;
       p += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t i = sidx0[p];
    const uint32_t pp = pprefix[p];
    const int64_t pos = i < (uint64_t)NP ? (int64_t)pp : NPpad + (p - pp);
    for (int m = 0; m < ds; ++m) rankL[(int64_t)m * Lrow + pos] = rank[(int64_t)(m + 1) * N + i];
    if (i >= (uint64_t)ob && i < (uint64_t)oe) olist[exO ? exO[p] : (uint32_t)p] = i;
  }
}

// meta[q] for the q-th origin, and orank[m'][q] = its rank in dimension m'+1
__global__ void k_reg_meta(const uint32_t* __restrict__ rank, const uint32_t* __restrict__ olist,
                           const uint32_t* __restrict__ pprefix, int64_t N, int64_t no, int ds,
                           OriginMeta* __restrict__ meta, uint32_t* __restrict__ orank) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < no;
       q += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t k = olist[q];
    const uint32_t r0 = rank[k];       // dimension 0
    const uint32_t sp = pprefix[r0];   // P points with a smaller dimension-0 value
    OriginMeta m;
    m.sP = sp;
    m.sT = r0 - sp;
    m.k = k;
    m.pad = 0;
    meta[q] = m;
    for (int mm = 0; mm < ds; ++mm) orank[(int64_t)mm * no + q] = rank[(int64_t)(mm + 1) * N + k];
  }
}

// Block-wide exclusive scan of one value per thread (THREADS threads, a
// multiple of 32 up to 1024).
template <int THREADS>
DDKS_DEV uint32_t block_exscan(uint32_t v, uint32_t* tmp /* >= 33 words */) {
  constexpr int kWarps = THREADS / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t incl = v;
  for (int off = 1; off < 32; off <<= 1) {
    const uint32_t x = __shfl_up_sync(0xffffffffu, incl, off);
    if (lane >= off) incl += x;
  }
  if (lane == 31) tmp[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const uint32_t w = lane < kWarps ? tmp[lane] : 0u;
    uint32_t wi = w;
    for (int off = 1; off < 32; off <<= 1) {
      const uint32_t x = __shfl_up_sync(0xffffffffu, wi, off);
      if (lane >= off) wi += x;
    }
    if (lane < kWarps) tmp[lane] = wi - w;
  }
  __syncthreads();
  const uint32_t r = tmp[warp] + incl - v;
  __syncthreads();
  return r;
}

// Pack kernel: one CTA per (origin block, dimension m = 1 + blockIdx.y, slice
// blockIdx.z of the list positions).  It marks the block's origin values in a
// bitmap over the global ranks, turns the bitmap into a byte table
// x'(r) = #{marked ranks <= r} (prefix counts of the words, then 4 table bytes
// per nibble of a word by multiplies), and writes its slice of the plane of
// re-ranked values, planes[blk][m-1][pos]; the slice-0 CTA also writes the
// block's origins, oplanes[blk][m-1][slot].
__global__ void __launch_bounds__(kPackThreads, 4)
k_reg_pack(const uint32_t* __restrict__ rankL, const uint32_t* __restrict__ orank, int64_t no,
           int64_t Lrow, int NW, int ds, uint8_t* __restrict__ planes, uint8_t* __restrict__ oplanes) {
  extern __shared__ __align__(16) uint32_t sm[];
  uint32_t* bits = sm;                  // [NW]
  uint32_t* tmp = bits + NW;            // [40] scan scratch
  uint8_t* tab = reinterpret_cast<uint8_t*>(tmp + 40);  // [NW * 32]
  const int tid = threadIdx.x;
  const int blk = blockIdx.x;
  const int mm = blockIdx.y;  // dimension - 1
  const int64_t q0 = (int64_t)blk * kOC;
  const int nq = (int)((no - q0) < kOC ? (no - q0) : kOC);
  const uint32_t* ork = orank + (int64_t)mm * no + q0;
  for (int i = tid; i < NW; i += kPackThreads) bits[i] = 0;
  __syncthreads();
  uint32_t myr = 0;
  if (tid < nq) {
    myr = ork[tid];
    atomicOr(&bits[myr >> 5], 1u << (myr & 31));
  }
  __syncthreads();
  // exclusive prefix of the popcounts over the words; thread t owns the
  // contiguous words [t * seg, (t + 1) * seg)
  const int seg = (NW + kPackThreads - 1) / kPackThreads;
  const int wa = tid * seg < NW ? tid * seg : NW;
  const int wb = wa + seg < NW ? wa + seg : NW;
  uint32_t c = 0;
  for (int w = wa; w < wb; ++w) c += (uint32_t)__popc(bits[w]);
  uint32_t run = block_exscan<kPackThreads>(c, tmp);
  for (int w = wa; w < wb; ++w) {
    const uint32_t bw = bits[w];
    // 32 table bytes of this word, 4 at a time: the nibble's bits spread to
    // bytes (bit i -> byte i) and are prefix-summed across bytes by multiplies
    uint32_t* out = reinterpret_cast<uint32_t*>(tab + (size_t)w * 32);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const uint32_t nib = (bw >> (4 * q)) & 15u;
      const uint32_t spread = (nib * 0x00204081u) & 0x01010101u;
      const uint32_t v = spread * 0x01010101u + run * 0x01010101u;
      out[q] = v;
      run = v >> 24;
    }
  }
  __syncthreads();
  // this CTA's slice of the positions, 4 per step: one 16-byte load of ranks,
  // one 4-byte store of re-ranked bytes
  const int n4 = (int)(Lrow >> 2);
  const int per = (n4 + gridDim.z - 1) / gridDim.z;
  const int i_beg = blockIdx.z * per;
  const int i_end = i_beg + per < n4 ? i_beg + per : n4;
  const uint4* rl = reinterpret_cast<const uint4*>(rankL + (int64_t)mm * Lrow);
  uint32_t* out = reinterpret_cast<uint32_t*>(planes + ((size_t)blk * ds + mm) * Lrow);
  constexpr int kU = 4;  // loads in flight per thread
  for (int i0 = i_beg + tid; i0 < i_end; i0 += kU * kPackThreads) {
    uint4 r[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int i = i0 + u * kPackThreads;
      r[u] = i < i_end ? rl[i] : make_uint4(0, 0, 0, 0);
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int i = i0 + u * kPackThreads;
      if (i < i_end)
        out[i] = (uint32_t)tab[r[u].x] | ((uint32_t)tab[r[u].y] << 8) | ((uint32_t)tab[r[u].z] << 16) |
                 ((uint32_t)tab[r[u].w] << 24);
    }
  }
  if (blockIdx.z == 0 && tid < kOC)
    oplanes[((size_t)blk * ds + mm) * kOC + tid] = tid < nq ? tab[myr] : (uint8_t)0;
}

// 4x4 byte transpose: out[k] byte g = in[g] byte k
DDKS_DEV void transpose4(uint32_t v0, uint32_t v1, uint32_t v2, uint32_t v3, uint32_t (&o)[4]) {
  const uint32_t a_lo = __byte_perm(v0, v1, 0x5140), a_hi = __byte_perm(v0, v1, 0x7362);
  const uint32_t b_lo = __byte_perm(v2, v3, 0x5140), b_hi = __byte_perm(v2, v3, 0x7362);
  o[0] = __byte_perm(a_lo, b_lo, 0x5410);
  o[1] = __byte_perm(a_lo, b_lo, 0x7632);
  o[2] = __byte_perm(a_hi, b_hi, 0x5410);
  o[3] = __byte_perm(a_hi, b_hi, 0x7632);
}

// The pack kernel for four origin blocks at once (N up to ~51k): one CTA per
// (group of 4 blocks, dimension m = 1 + blockIdx.y).  The four re-rank tables
// are interleaved, tab4[r] byte g = x'_g(r), so one rank load and one shared
// load serve four blocks, and a 4x4 byte transpose turns four looked-up words
// into one word of each block's plane.  The exclusive prefix counts of the
// four bitmaps are scanned together, one byte each (a block has at most 128
// distinct values, so no byte carries).
__global__ void __launch_bounds__(kPack4Threads)
k_reg_pack4(const uint32_t* __restrict__ rankL, const uint32_t* __restrict__ orank, int64_t no,
            int64_t blocks, int64_t Lrow, int NW, int ds, uint8_t* __restrict__ planes,
            uint8_t* __restrict__ oplanes) {
  extern __shared__ __align__(16) uint32_t sm[];
  uint32_t* tab4 = sm;                  // [NW * 32]
  uint32_t* bits = tab4 + NW * 32;      // [4][NW]
  uint32_t* tmp = bits + 4 * NW;        // [40] scan scratch
  const int tid = threadIdx.x;
  const int64_t b0 = (int64_t)blockIdx.x * 4;
  const int mm = blockIdx.y;  // dimension - 1
  for (int i = tid; i < 4 * NW; i += kPack4Threads) bits[i] = 0;
  __syncthreads();
  for (int i = tid; i < 4 * kOC; i += kPack4Threads) {
    const int g = i / kOC, slot = i - g * kOC;
    const int64_t q = (b0 + g) * kOC + slot;
    if (b0 + g < blocks && q < no) {
      const uint32_t r = orank[(int64_t)mm * no + q];
      atomicOr(&bits[g * NW + (r >> 5)], 1u << (r & 31));
    }
  }
  __syncthreads();
  const int seg = (NW + kPack4Threads - 1) / kPack4Threads;
  const int wa = tid * seg < NW ? tid * seg : NW;
  const int wb = wa + seg < NW ? wa + seg : NW;
  uint32_t c = 0;
  for (int w = wa; w < wb; ++w)
#pragma unroll
    for (int g = 0; g < 4; ++g) c += (uint32_t)__popc(bits[g * NW + w]) << (8 * g);
  const uint32_t run4 = block_exscan<kPack4Threads>(c, tmp);
  uint32_t run[4];
#pragma unroll
  for (int g = 0; g < 4; ++g) run[g] = (run4 >> (8 * g)) & 0xFFu;
  for (int w = wa; w < wb; ++w) {
    uint32_t bw[4];
#pragma unroll
    for (int g = 0; g < 4; ++g) bw[g] = bits[g * NW + w];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      uint32_t v[4];
#pragma unroll
      for (int g = 0; g < 4; ++g) {
        const uint32_t nib = (bw[g] >> (4 * q)) & 15u;
        v[g] = ((nib * 0x00204081u) & 0x01010101u) * 0x01010101u + run[g] * 0x01010101u;
        run[g] = v[g] >> 24;
      }
      uint32_t e[4];
      transpose4(v[0], v[1], v[2], v[3], e);
      reinterpret_cast<uint4*>(tab4)[w * 8 + q] = make_uint4(e[0], e[1], e[2], e[3]);
    }
  }
  __syncthreads();
  const int n4 = (int)(Lrow >> 2);
  const uint4* rl = reinterpret_cast<const uint4*>(rankL + (int64_t)mm * Lrow);
  const int ng = (int)((blocks - b0) < 4 ? (blocks - b0) : 4);
  uint32_t* out[4];
#pragma unroll
  for (int g = 0; g < 4; ++g)
    out[g] = reinterpret_cast<uint32_t*>(planes + ((size_t)(b0 + (g < ng ? g : 0)) * ds + mm) * Lrow);
  for (int i = tid; i < n4; i += kPack4Threads) {
    const uint4 r = rl[i];
    uint32_t o[4];
    transpose4(tab4[r.x], tab4[r.y], tab4[r.z], tab4[r.w], o);
#pragma unroll
    for (int g = 0; g < 4; ++g)
      if (g < ng) out[g][i] = o[g];
  }
  for (int i = tid; i < 4 * kOC; i += kPack4Threads) {
    const int g = i / kOC, slot = i - g * kOC;
    const int64_t q = (b0 + g) * kOC + slot;
    if (g < ng)
      oplanes[((size_t)(b0 + g) * ds + mm) * kOC + slot] =
          q < no ? (uint8_t)(tab4[orank[(int64_t)mm * no + q]] >> (8 * g)) : (uint8_t)0;
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

// add the 8-bit counters into the origin's shared counters and clear them.
// c[4 * phase + w] holds two 16-bit counts: w = 0: bins 0, 4; 1: bins 2, 6;
// 2: bins 1, 5; 3: bins 3, 7 (low half, high half) -- exactly the byte pairs
// 0 and 2 / 1 and 3 of the even-bin and odd-bin byte words.  A unit adds at
// most its chunk length (< 2^16) to a count.
DDKS_DEV void byte_flush(Acc& a, uint32_t* c) {
  if (a.loA | a.hiA) {
    atomicAdd(&c[0], a.loA & 0x00FF00FFu);
    atomicAdd(&c[1], (a.loA >> 8) & 0x00FF00FFu);
    atomicAdd(&c[2], a.hiA & 0x00FF00FFu);
    atomicAdd(&c[3], (a.hiA >> 8) & 0x00FF00FFu);
  }
  if (a.loB | a.hiB) {
    atomicAdd(&c[4], a.loB & 0x00FF00FFu);
    atomicAdd(&c[5], (a.loB >> 8) & 0x00FF00FFu);
    atomicAdd(&c[6], a.hiB & 0x00FF00FFu);
    atomicAdd(&c[7], (a.hiB >> 8) & 0x00FF00FFu);
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

DDKS_DEV void origin_best(const uint32_t* __restrict__ gcnt, int64_t q, int ds, int64_t NP, int64_t NT,
                          uint64_t& bv, int& bj);

// Fused final step (out3 != nullptr): per-origin maxima into best/bestj at
// pooled index - ob, and the result {num_max, arg-max origin, orthant} into
// out3.  done: [blocks + 1] zeroed tickets; packed: one zeroed word holding
// max over origins of (num << kPackShift) | (kPackMask - position).
struct OriginMetaFinal {
  unsigned long long* out3;
  unsigned* done;
  unsigned long long* packed;
  uint64_t* best;
  int32_t* bestj;
  int64_t ob;
  int blocks;
};
constexpr int kPackShift = 26;                       // positions < 2^26; numerators < 2^38
constexpr unsigned long long kPackMask = (1ull << kPackShift) - 1;

// ---- bulk asynchronous copies with mbarrier completion

DDKS_DEV void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

// expect `bytes` more transaction bytes on the current phase of `bar`
DDKS_DEV void mbar_expect(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// global -> shared bulk copy of `bytes` (a multiple of 16, both addresses
// 16-byte aligned), counted on `bar`
DDKS_DEV void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(dst), "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

DDKS_DEV unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Waits for phase `parity` of `bar` to complete; false after kWaitNs.
DDKS_DEV bool mbar_wait(uint32_t bar, uint32_t parity) {
  unsigned long long t0 = 0;
  for (int it = 0;; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if (it == 0) t0 = global_ns();
    else if (global_ns() - t0 > kWaitNs) return false;
  }
}

// Unit u: origin block u / C, chunk u % C of the lists, where chunks [0, CP)
// cover the P list [0, NP) in pieces of CLP and chunks [CP, C) the T list
// [0, NT) in pieces of CLT (sample-local positions; CLP, CLT multiples of 16).
template <int DS, int OCC>
__global__ void __launch_bounds__(kThreads, OCC)
k_register(const uint8_t* __restrict__ planes, const uint8_t* __restrict__ oplanes,
           const OriginMeta* __restrict__ meta, int64_t no, int64_t NP, int64_t NT, int64_t NPpad,
           int64_t Lrow, int C, int CP, int64_t CLP, int64_t CLT, uint32_t one,
           uint32_t* __restrict__ gcnt, unsigned* __restrict__ flags, const OriginMetaFinal fin) {
  extern __shared__ __align__(16) uint32_t sm[];
  uint32_t* tile = sm;                                            // [kTP] assembled words
  uint8_t* raw = reinterpret_cast<uint8_t*>(tile + kTP);          // [2][DS][kTP] plane ring
  uint32_t* cnt = reinterpret_cast<uint32_t*>(raw + 2 * DS * kTP); // [kOC][9]: 8 words of 16-bit pairs + pad
  uint64_t* bars = reinterpret_cast<uint64_t*>(cnt + kOC * kSlot);  // [2]
  const int tid = threadIdx.x;
  const int g = tid / kS, s = tid - g * kS;
  // block and position indices fit 32 bits (N <= kMaxRegN)
  const int blk = (int)(blockIdx.x / C);
  const int ci = (int)(blockIdx.x % C);
  const int sample = ci < CP ? 0 : 1;
  int c0, c1;
  if (sample == 0) {
    c0 = (int)(ci * CLP);
    c1 = (int)(c0 + CLP < NP ? c0 + CLP : NP);
  } else {
    c0 = (int)((ci - CP) * CLT);
    c1 = (int)(c0 + CLT < NT ? c0 + CLT : NT);
  }
  const uint32_t raw_s = (uint32_t)__cvta_generic_to_shared(raw);
  const uint32_t bar_s = (uint32_t)__cvta_generic_to_shared(bars);
  const int ntiles = c1 > c0 ? (c1 - c0 + kTP - 1) / kTP : 0;
  auto issue = [&](int t) {  // thread 0: the DS planes of tile t into stage t & 1
    const int base = c0 + t * kTP;
    const int n = (c1 - base) < kTP ? (c1 - base) : kTP;
    const uint32_t bytes = (uint32_t)((n + 15) & ~15);
    const uint32_t bar = bar_s + 8u * (t & 1);
    const uint8_t* src = planes + (size_t)blk * DS * Lrow + (sample ? NPpad : 0) + base;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect(bar, bytes * DS);
#pragma unroll
    for (int m = 0; m < DS; ++m)
      bulk_load(raw_s + (uint32_t)(((t & 1) * DS + m) * kTP), src + (size_t)m * Lrow, bytes, bar);
  };
  if (tid == 0) {
    mbar_init(bar_s, 1);
    mbar_init(bar_s + 8, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int i = tid; i < kOC * kSlot; i += kThreads) cnt[i] = 0;
  __syncthreads();
  if (tid == 0 && ntiles > 0) issue(0);

  uint32_t ow[kR];
  int sa[kR];  // this sample's split, sample-local positions
#pragma unroll
  for (int r = 0; r < kR; ++r) {
    const int slot = g * kR + r;
    const int64_t q = (int64_t)blk * kOC + slot;
    if (q < no) {
      uint32_t w = 0;
#pragma unroll
      for (int m = 0; m < DS; ++m) w |= (uint32_t)oplanes[((size_t)blk * DS + m) * kOC + slot] << (9 * m);
      ow[r] = 0u - w;  // negated: the subtract becomes a multiply-add
      const OriginMeta mt = meta[q];
      sa[r] = (int)(sample == 0 ? mt.sP : mt.sT);
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
  for (int t = 0; t < ntiles; ++t) {
    const int base = c0 + t * kTP;
    const int cntp = (c1 - base) < kTP ? (c1 - base) : kTP;
    // stage (t + 1) & 1 was released by the barrier after tile t - 1's assembly
    if (tid == 0 && t + 1 < ntiles) issue(t + 1);
    const bool ok = mbar_wait(bar_s + 8u * (t & 1), (uint32_t)((t >> 1) & 1));
    if (ok) {
      // assemble 4 points per step: byte k of plane word m is field m of point k
      const uint32_t* pl = reinterpret_cast<const uint32_t*>(raw + (t & 1) * DS * kTP);
      for (int i = tid; 4 * i < cntp; i += kThreads) {
        uint32_t p[DS];
#pragma unroll
        for (int m = 0; m < DS; ++m) p[m] = pl[m * (kTP / 4) + i];
        uint4 w;
        uint32_t* wv = reinterpret_cast<uint32_t*>(&w);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          uint32_t x = Swar<DS>::kGuard;
#pragma unroll
          for (int m = 0; m < DS; ++m) x |= ((p[m] >> (8 * k)) & 0xFFu) << (9 * m);
          wv[k] = x;
        }
        reinterpret_cast<uint4*>(tile)[i] = w;
      }
    }
    // the tile is assembled and stage t & 1 may be refilled; a timed-out wait
    // ends the unit
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        atomicOr(flags, ddks::kFlagTimeout);
        // the copy of tile t + 1 may still be in flight: give it a bounded wait
        if (t + 1 < ntiles) mbar_wait(bar_s + 8u * ((t + 1) & 1), (uint32_t)(((t + 1) >> 1) & 1));
      }
      return;
    }
    {
      // splits relative to the tile, clamped to [-1, kTP + 1]
      int spl[kR];
      int lo = kTP + 1, hi = -1;
#pragma unroll
      for (int r = 0; r < kR; ++r) {
        int v = sa[r] - base;
        v = v < -1 ? -1 : (v > kTP + 1 ? kTP + 1 : v);
        spl[r] = v;
        lo = spl[r] < lo ? spl[r] : lo;
        hi = spl[r] > hi ? spl[r] : hi;
      }
      // iterations in which every slice has a whole chunk, then at most one
      // ragged iteration
      const int full = cntp / (kS * kCh);
      const int iters = (cntp + kS * kCh - 1) / (kS * kCh);
      int j = s * kCh;
      for (int it = 0; it < full; ++it, j += kS * kCh) {
        if (j + kCh <= lo) chunk12<DS, 0>(tile, j, ow, spl, acc, one);
        else if (j >= hi) chunk12<DS, 1>(tile, j, ow, spl, acc, one);
        else chunk12<DS, 2>(tile, j, ow, spl, acc, one);
        if (++since == 21) {
#pragma unroll
          for (int r = 0; r < kR; ++r) byte_flush(acc[r], mycnt + r * kSlot);
          since = 0;
        }
      }
      if (full < iters) {
        if (j < cntp) {
          const int n = cntp - j < kCh ? cntp - j : kCh;
          if (n == kCh) chunk12<DS, 2>(tile, j, ow, spl, acc, one);
          else chunk_partial<DS>(tile, j, n, ow, spl, acc, one);
        }
        if (++since == 21) {
#pragma unroll
          for (int r = 0; r < kR; ++r) byte_flush(acc[r], mycnt + r * kSlot);
          since = 0;
        }
      }
    }
    __syncthreads();  // every thread is done with the tile words
  }
#pragma unroll
  for (int r = 0; r < kR; ++r) byte_flush(acc[r], mycnt + r * kSlot);
  __syncthreads();
  const int64_t q0 = (int64_t)blk * kOC;
  const int nq = (int)((no - q0) < kOC ? (no - q0) : kOC);
  for (int i = tid; i < nq * 16; i += kThreads) {
    const int ph = (i >> 3) & 1, b = i & 7;  // i & 15 = phase * 8 + bin
    const uint32_t w = cnt[(i >> 4) * kSlot + ph * 4 + ((b & 1) << 1) + ((b >> 1) & 1)];
    const uint32_t v = (b & 4) ? (w >> 16) : (w & 0xFFFFu);
    if (v) atomicAdd(&gcnt[(q0 + (i >> 4)) * 32 + sample * 16 + (i & 15)], v);
  }
  if (!fin.out3) return;
  // The last unit of an origin block to finish turns the block's counts into
  // per-origin maxima and a packed (num, origin) candidate for the global
  // maximum; the last block to finish writes the result.  Tickets only: no
  // CTA waits for another.
  __shared__ unsigned ticket;
  __threadfence();
  __syncthreads();
  if (tid == 0) ticket = atomicAdd(&fin.done[blk], 1u);
  __syncthreads();
  if (ticket != (unsigned)(C - 1)) return;
  __threadfence();
  for (int q = tid; q < nq; q += kThreads) {
    uint64_t bv;
    int bj;
    origin_best(gcnt, q0 + q, DS, NP, NT, bv, bj);
    const uint32_t k = meta[q0 + q].k;
    const int64_t pos = (int64_t)k - fin.ob;
    fin.best[pos] = bv;
    fin.bestj[pos] = bj;
    // larger numerator first, then the lower origin
    atomicMax(fin.packed, (bv << kPackShift) | (kPackMask - (unsigned long long)pos));
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) ticket = atomicAdd(&fin.done[fin.blocks], 1u);
  __syncthreads();
  if (ticket != (unsigned)(fin.blocks - 1) || tid != 0) return;
  __threadfence();
  const unsigned long long pk = atomicAdd(fin.packed, 0ull);
  const int64_t pos = (int64_t)(kPackMask - (pk & kPackMask));
  fin.out3[0] = pk >> kPackShift;
  fin.out3[1] = (unsigned long long)(fin.ob + pos);
  fin.out3[2] = (unsigned long long)(long long)__ldcg(&fin.bestj[pos]);
}

// The best orthant of origin q from its counts gcnt[q][sample][phase][bin]
// (the code's bit 0 is the phase, i.e. dimension 0).  Reads through L2: the
// counts were added by other CTAs.
DDKS_DEV void origin_best(const uint32_t* __restrict__ gcnt, int64_t q, int ds, int64_t NP, int64_t NT,
                          uint64_t& bv, int& bj) {
  const uint32_t* c = gcnt + q * 32;
  bv = 0;
  bj = 0;
  const int nbin = 1 << ds;
  for (int code = 0; code < 2 * nbin; ++code) {
    const int ph = code & 1, bin = code >> 1;
    const uint64_t cp = __ldcg(&c[ph * 8 + bin]), ct = __ldcg(&c[16 + ph * 8 + bin]);
    const uint64_t num = ddks::numer(cp, ct, (uint64_t)NP, (uint64_t)NT);
    if (num > bv) { bv = num; bj = code; }
  }
}

// one thread per origin: its 2 * 2^DS orthants from gcnt[q][sample][phase][bin]
__global__ void k_reg_final(const uint32_t* __restrict__ gcnt, const OriginMeta* __restrict__ meta,
                            int64_t no, int64_t NP, int64_t NT, int64_t ob, int ds,
                            uint64_t* __restrict__ best, int32_t* __restrict__ bestj) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < no;
       q += (int64_t)gridDim.x * blockDim.x) {
    uint64_t bv;
    int bj;
    origin_best(gcnt, q, ds, NP, NT, bv, bj);
    const uint32_t k = meta[q].k;
    best[k - ob] = bv;
    bestj[k - ob] = bj;
  }
}

size_t reg_smem(int ds) {
  return (size_t)kTP * 4 + (size_t)2 * ds * kTP + (size_t)kOC * kSlot * 4 + 16;
}

size_t pack_smem(int NW) { return (size_t)NW * 4 + 40 * 4 + (size_t)NW * 32; }
size_t pack4_smem(int NW) { return (size_t)NW * 128 + (size_t)NW * 16 + 40 * 4; }

constexpr size_t kPackSmemMax = 227u * 1024u;

}  // namespace

bool ddks_register_supported(int d, int64_t NP, int64_t NT) {
  const int64_t N = NP + NT;
  if (d < 2 || d > 4 || N > kMaxRegN) return false;
  return pack_smem((int)((N + 31) / 32)) <= kPackSmemMax;
}

cudaError_t ddks_launch_register(ddks_ctx* ctx, const uint32_t* rank, int64_t N, int64_t NP,
                                 int64_t NT, int d, int64_t ob, int64_t oe, uint64_t* best,
                                 int32_t* bestj, cudaStream_t st, const ddks_plan& plan,
                                 unsigned long long* out3, bool* reduced) {
  if (reduced) *reduced = false;
  if (!ddks_register_supported(d, NP, NT)) return cudaErrorInvalidValue;
  const int ds = d - 1;
  const int64_t no = oe - ob;
  if (no <= 0) return cudaSuccess;
  const int NW = (int)((N + 31) / 32);
  const int64_t blocks = (no + kOC - 1) / kOC;
  const int64_t NPpad = (NP + 15) & ~(int64_t)15, NTpad = (NT + 15) & ~(int64_t)15;
  const int64_t Lrow = NPpad + NTpad;
  // scratch (u32): pprefix N, exO N, olist no, gcnt no*32 + tickets (blocks + 1) + packed (2),
  // rankL ds*Lrow, orank ds*no, scan tmp; then meta
  const size_t scan_tmp = ddks_scan_tmp_elems(1, N);
  const size_t n_fin = (size_t)blocks + 1 + 4;
  const size_t n_u32 = (size_t)N * 2 + (size_t)no + (size_t)no * 32 + n_fin + (size_t)ds * Lrow +
                       (size_t)ds * no + scan_tmp;
  int rc = ctx->reg_meta.reserve(ctx, n_u32 * 4 + (size_t)no * sizeof(OriginMeta) + 64);
  if (rc) return cudaErrorMemoryAllocation;
  // byte planes [blocks][ds][Lrow] and origin planes [blocks][ds][128]
  rc = ctx->reg_words.reserve(ctx, (size_t)blocks * ds * Lrow + (size_t)blocks * ds * kOC);
  if (rc) return cudaErrorMemoryAllocation;
  uint32_t* pprefix = (uint32_t*)ctx->reg_meta.ptr;
  uint32_t* exO = pprefix + N;
  uint32_t* olist = exO + N;
  uint32_t* gcnt = olist + no;
  unsigned* done = gcnt + no * 32;  // [blocks + 1] tickets, then the packed maximum (8-byte aligned)
  unsigned long long* packed = reinterpret_cast<unsigned long long*>(
      (reinterpret_cast<uintptr_t>(done + blocks + 1) + 7) & ~(uintptr_t)7);
  // rankL must be 16-byte aligned for the pack kernel's vector loads
  uint32_t* rankL = reinterpret_cast<uint32_t*>((reinterpret_cast<uintptr_t>(gcnt + no * 32 + n_fin) + 15) &
                                                ~(uintptr_t)15);
  uint32_t* orank = rankL + (size_t)ds * Lrow;
  uint32_t* stmp = orank + (size_t)ds * no;
  OriginMeta* meta = reinterpret_cast<OriginMeta*>(
      (reinterpret_cast<uintptr_t>(stmp + scan_tmp) + 15) & ~(uintptr_t)15);
  uint8_t* planes = (uint8_t*)ctx->reg_words.ptr;
  uint8_t* oplanes = planes + (size_t)blocks * ds * Lrow;
  const uint32_t* sidx0 = (const uint32_t*)ctx->sidx0.ptr;
  unsigned* flags = (unsigned*)ctx->flags.ptr;

  auto grid = [](int64_t w) { int64_t g = (w + 255) / 256; return (int)(g > 152 * 32 ? 152 * 32 : (g < 1 ? 1 : g)); };
  int n = 0;
  cudaError_t e = cudaSuccess;
  if (ob == 0 && oe == N && ctx->pfx0_valid) {
    // the rank kernel already produced the P prefix over the sorted order, and
    // with every point an origin the origin prefix is the position itself
    pprefix = (uint32_t*)ctx->pfx0.ptr;
    exO = nullptr;
  } else {
    k_reg_flags<<<grid(N), 256, 0, st>>>(sidx0, N, NP, ob, oe, pprefix, exO);
    ++n;
    e = ddks_scan_rows(pprefix, pprefix, 1, N, true, stmp, st, &n);
    if (e == cudaSuccess) e = ddks_scan_rows(exO, exO, 1, N, true, stmp, st, &n);
    if (e != cudaSuccess) return e;
  }
  k_reg_lists<<<grid(N), 256, 0, st>>>(sidx0, rank, N, NP, NPpad, Lrow, ds, ob, oe, pprefix, exO, rankL,
                                       olist);
  k_reg_meta<<<grid(no), 256, 0, st>>>(rank, olist, pprefix, N, no, ds, meta, orank);
  n += 2;
  // stage timing: the count stage (re-rank packing included) starts here
  ddks_stage_mark(ctx, 1, st);
  if (pack4_smem(NW) <= kPackSmemMax) {
    // four blocks per CTA, interleaved tables
    const size_t psmem = pack4_smem(NW);
    e = cudaFuncSetAttribute(k_reg_pack4, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psmem);
    if (e != cudaSuccess) return e;
    k_reg_pack4<<<dim3((unsigned)((blocks + 3) / 4), (unsigned)ds), kPack4Threads, psmem, st>>>(
        rankL, orank, no, blocks, Lrow, NW, ds, planes, oplanes);
  } else {
    const size_t psmem = pack_smem(NW);
    e = cudaFuncSetAttribute(k_reg_pack, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psmem);
    if (e != cudaSuccess) return e;
    // position slices per (block, dimension): enough CTAs for a few waves
    int slices = (int)((ctx->num_sms * 12 + blocks * ds - 1) / (blocks * ds));
    if (slices > 8) slices = 8;
    if (slices < 1) slices = 1;
    k_reg_pack<<<dim3((unsigned)blocks, (unsigned)ds, (unsigned)slices), kPackThreads, psmem, st>>>(
        rankL, orank, no, Lrow, NW, ds, planes, oplanes);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  ++n;
  // chunks of the lists per origin block: about 3 waves of the resident CTAs
  const int64_t slots = (int64_t)ctx->num_sms * 3;
  int64_t want = (3 * slots + blocks - 1) / blocks;  // chunks per block
  if (want < 2) want = 2;
  int64_t CL = (N + want - 1) / want;
  if (CL < 2 * kTP) CL = 2 * kTP;
  if (CL > kMaxChunk - 16) CL = kMaxChunk - 16;  // rounded up to 16 below: <= kMaxChunk
  const int64_t CP = (NP + CL - 1) / CL, CT = (NT + CL - 1) / CL;
  const int64_t CLP = (((NP + CP - 1) / CP) + 15) & ~(int64_t)15;
  const int64_t CLT = (((NT + CT - 1) / CT) + 15) & ~(int64_t)15;
  const int64_t C = CP + CT;
  e = cudaMemsetAsync(gcnt, 0, ((size_t)no * 32 + n_fin) * 4, st);
  if (e != cudaSuccess) return e;
  const size_t smem = reg_smem(ds);
  const unsigned ctas = (unsigned)(blocks * C);
  const int occ = plan.reg_occ == 2 || plan.reg_occ == 3 ? plan.reg_occ : 4;
  OriginMetaFinal fin{out3, done, packed, best, bestj, ob, (int)blocks};
  auto go = [&](auto kern) -> cudaError_t {
    cudaError_t r = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (r != cudaSuccess) return r;
    kern<<<ctas, kThreads, smem, st>>>(planes, oplanes, meta, no, NP, NT, NPpad, Lrow, (int)C, (int)CP, CLP,
                                        CLT, 1u, gcnt, flags, fin);
    return cudaGetLastError();
  };
  if (ds == 1) e = occ == 2 ? go(k_register<1, 2>) : occ == 3 ? go(k_register<1, 3>) : go(k_register<1, 4>);
  else if (ds == 2) e = occ == 2 ? go(k_register<2, 2>) : occ == 3 ? go(k_register<2, 3>) : go(k_register<2, 4>);
  else e = occ == 2 ? go(k_register<3, 2>) : occ == 3 ? go(k_register<3, 3>) : go(k_register<3, 4>);
  if (e != cudaSuccess) return e;
  ++n;
  if (out3) {
    if (reduced) *reduced = true;
  } else {
    k_reg_final<<<grid(no), 256, 0, st>>>(gcnt, meta, no, NP, NT, ob, ds, best, bestj);
    ++n;
  }
  ctx->launches += n;
  return cudaGetLastError();
}
