// count_register.cu -- K1: orthant counts for d = 2, 3, 4, bit-sliced.
//
// Same statistic as every other path (Sec. 2.1, Eq. ddks_tensor_definition;
// the ">=" split of Sec. 2.2.1, Eq. g; max |cP*NT - cT*NP| of Eq. d1 with the
// normalisation of Eq. abs_difference).  Every origin-point pair is compared
// in every dimension; the compares of 32 points run in parallel in the bits
// of 32-bit words:
//
// 1. Dimension 0 by order.  Each sample's points are listed in increasing rank
//    in dimension 0.  For an origin o, the points of a sample with x_0 < o_0
//    are exactly a prefix of its list, of length split(o) = #{x : rank_0(x) <
//    rank_0(o)}: bit 0 of a code is known from the position alone (phase A
//    before the split, phase B from it on).
// 2. Re-ranking.  Origins form blocks of 127.  For each block and each of the
//    dimensions 1..d-1, every point is re-ranked as x' = #{distinct values of
//    the block's origins <= x} (at most 127, 7 bits), which keeps
//    x >= o <=> x' >= o' for every origin of the block.
// 3. Bit slices.  A pack kernel stores, for every group of 32 consecutive list
//    positions and every dimension, the 7 bit planes of x' (bit j of plane k
//    = bit k of point j's x').  A lane holding origin o compares a group in
//    dimension m with one 3-input logic op per bit, from the least significant
//    bit up: r = o'_k ? (plane_k & r) : (plane_k | r), r = all ones at the
//    start, which leaves G_m = the 32 bits [x'_m >= o'_m].
// 4. Counting by subsets.  For every non-empty set S of dimensions the lane
//    adds popcount(AND of G_m over m in S) to a counter (per phase); the
//    orthant counts follow at the end by inclusion-exclusion,
//    count(exactly the dims in B) = sum over S >= B of (-1)^|S \ B| n_S,
//    with n_{} = the phase's number of points.
//
// Work units: (block of 127 origins, one per lane of a 128-thread CTA) x
// (chunk of one sample's groups); a CTA works on one unit.  Tiles of group
// records (7 planes per dimension) arrive in shared memory by bulk
// asynchronous copies (the TMA engine) into a two-stage ring, completion on
// an mbarrier, and every lane reads the same record (broadcast loads).  The
// last unit of a block turns the block's counters into per-origin maxima and
// the last block writes the result.
#include <type_traits>

#include "bulk_copy.cuh"
#include "count_register.cuh"
#include "ddks_host.h"
#include "ddks_internal.cuh"

namespace {

namespace bk = ddks::bulk;

using namespace ddks_reg;

constexpr int kThreads = 64;          // threads per CTA of the count kernel
constexpr int kOPL = 2;               // origin slots per thread
static_assert(kThreads * kOPL == kOC, "one origin block per CTA");
constexpr int kTG = 64;
// ring stages of the count kernel (any occupancy class): two; four stages at
// 8 CTAs per SM measured slower on 2 x 20,000 points (count 0.251 vs 0.205 ms)
__host__ __device__ constexpr int reg_stages(int) { return 2; }               // groups (of 32 points) per staged tile
constexpr int64_t kMaxRegN = 200000;
constexpr int kPackThreads = 512;     // one origin block per CTA
constexpr int kPack4Threads = 1024;   // four origin blocks per CTA

// record of one group: per dimension 8 words (7 planes + 1 pad), 16-byte aligned
template <int DS>
struct Rec {
  static constexpr int kWords = 8 * DS;
  static constexpr int kNS = (1 << DS) - 1;  // non-empty subsets of the DS dimensions
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
//                   [NPpad, NPpad + NT), NPpad and the row length multiples of
//                   32; the padding positions hold rank 0)
//   olist[q]        pooled index of the q-th origin of [ob, oe), in sorted order
//                   (exO = nullptr: every point is an origin, q = p)
__global__ void k_reg_lists(const uint32_t* __restrict__ sidx0, const uint32_t* __restrict__ rank,
                            int64_t N, int64_t NP, int64_t NPpad, int64_t Lrow, int ds, int64_t ob,
                            int64_t oe, const uint32_t* __restrict__ pprefix,
                            const uint32_t* __restrict__ exO, uint32_t* __restrict__ rankL,
                            uint32_t* __restrict__ olist) {
  const int64_t NT = N - NP;
  if (blockIdx.x == 0 && threadIdx.x < 32) {  // at most 31 padding positions per sample
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

// Both of the above in one pass when every point is an origin (the q-th
// origin is the point at sorted position q): list-ordered ranks, meta and
// orank.
__global__ void k_reg_lists_meta(const uint32_t* __restrict__ sidx0, const uint32_t* __restrict__ rank,
                                 int64_t N, int64_t NP, int64_t NPpad, int64_t Lrow, int ds,
                                 const uint32_t* __restrict__ pprefix, uint32_t* __restrict__ rankL,
                                 OriginMeta* __restrict__ meta, uint32_t* __restrict__ orank) {
  const int64_t NT = N - NP;
  if (blockIdx.x == 0 && threadIdx.x < 32) {  // at most 31 padding positions per sample
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
    const uint32_t r0 = rank[i];
    const uint32_t sp = pprefix[r0];  // P points with a smaller dimension-0 value
    OriginMeta mt;
    mt.sP = sp;
    mt.sT = r0 - sp;
    mt.k = i;
    mt.pad = 0;
    meta[p] = mt;
    for (int m = 0; m < ds; ++m) {
      const uint32_t r = rank[(int64_t)(m + 1) * N + i];
      rankL[(int64_t)m * Lrow + pos] = r;
      orank[(int64_t)m * N + p] = r;
    }
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

// 4x4 byte transpose: out[k] byte g = in[g] byte k
DDKS_DEV void transpose4(uint32_t v0, uint32_t v1, uint32_t v2, uint32_t v3, uint32_t (&o)[4]) {
  const uint32_t a_lo = __byte_perm(v0, v1, 0x5140), a_hi = __byte_perm(v0, v1, 0x7362);
  const uint32_t b_lo = __byte_perm(v2, v3, 0x5140), b_hi = __byte_perm(v2, v3, 0x7362);
  o[0] = __byte_perm(a_lo, b_lo, 0x5410);
  o[1] = __byte_perm(a_lo, b_lo, 0x7632);
  o[2] = __byte_perm(a_hi, b_hi, 0x5410);
  o[3] = __byte_perm(a_hi, b_hi, 0x7632);
}

// Pack kernel: one CTA per (group of G origin blocks, dimension m =
// 1 + blockIdx.y).  It marks each block's origin values in a bitmap over the
// global ranks and turns the bitmaps into interleaved re-rank tables,
// tab[r] byte g = x'_g(r) = #{marked ranks of block g <= r} (prefix counts of
// the words, then 4 table bytes per nibble by multiplies; with G = 4 the four
// tables are byte-transposed into one word per rank).  The exclusive prefix
// counts of the G bitmaps are scanned together, one byte each (a block has at
// most 127 distinct values, so no byte carries).  Then each warp takes groups
// of 32 list positions, looks the points up (lane j = point j) and turns bit k
// of every block's x' into plane k with a warp ballot; positions past a
// sample's end get no bits.  Records: rec[blk][group][m-1][8] words.  The
// block's origins go to oplanes[blk][m-1][slot] (x', bytes).
template <int G, int THREADS>
__global__ void __launch_bounds__(THREADS)
k_reg_pack(const uint32_t* __restrict__ rankL, const uint32_t* __restrict__ orank, int64_t no,
           int64_t blocks, int64_t NP, int64_t NT, int64_t NPpad, int64_t Lrow, int NW, int ds,
           uint32_t* __restrict__ rec, uint8_t* __restrict__ oplanes) {
  extern __shared__ __align__(16) uint32_t sm[];
  uint8_t* tabb = reinterpret_cast<uint8_t*>(sm);   // [NW * 32][G] bytes
  uint32_t* bits = sm + NW * 8 * G;                  // [G][NW]
  uint32_t* tmp = bits + G * NW;                     // [40] scan scratch
  const int tid = threadIdx.x;
  const int64_t b0 = (int64_t)blockIdx.x * G;
  const int mm = blockIdx.y;  // dimension - 1
  for (int i = tid; i < G * NW; i += THREADS) bits[i] = 0;
  __syncthreads();
  for (int i = tid; i < G * kOB; i += THREADS) {
    const int g = i / kOB, slot = i - g * kOB;
    const int64_t q = (b0 + g) * kOB + slot;
    if (b0 + g < blocks && q < no) {
      const uint32_t r = orank[(int64_t)mm * no + q];
      atomicOr(&bits[g * NW + (r >> 5)], 1u << (r & 31));
    }
  }
  __syncthreads();
  const int seg = (NW + THREADS - 1) / THREADS;
  const int wa = tid * seg < NW ? tid * seg : NW;
  const int wb = wa + seg < NW ? wa + seg : NW;
  uint32_t c = 0;
  for (int w = wa; w < wb; ++w)
#pragma unroll
    for (int g = 0; g < G; ++g) c += (uint32_t)__popc(bits[g * NW + w]) << (8 * g);
  const uint32_t run4 = block_exscan<THREADS>(c, tmp);
  uint32_t run[G];
#pragma unroll
  for (int g = 0; g < G; ++g) run[g] = (run4 >> (8 * g)) & 0xFFu;
  for (int w = wa; w < wb; ++w) {
    uint32_t bw[G];
#pragma unroll
    for (int g = 0; g < G; ++g) bw[g] = bits[g * NW + w];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      uint32_t v[4] = {0u, 0u, 0u, 0u};
#pragma unroll
      for (int g = 0; g < G; ++g) {
        const uint32_t nib = (bw[g] >> (4 * q)) & 15u;
        v[g] = ((nib * 0x00204081u) & 0x01010101u) * 0x01010101u + run[g] * 0x01010101u;
        run[g] = v[g] >> 24;
      }
      if (G == 4) {
        uint32_t e[4];
        transpose4(v[0], v[1], v[2], v[3], e);
        reinterpret_cast<uint4*>(sm)[w * 8 + q] = make_uint4(e[0], e[1], e[2], e[3]);
      } else {
        sm[w * 8 + q] = v[0];
      }
    }
  }
  __syncthreads();
  const int lane = tid & 31, warp = tid >> 5;
  const int ng = (int)((blocks - b0) < G ? (blocks - b0) : G);
  const uint32_t* rl = rankL + (int64_t)mm * Lrow;
  const int64_t ngroups = Lrow >> 5;
  // 32 x 32 bit transpose across the warp (lane i holds word X_i; afterwards
  // lane j holds the word whose bit i is bit j of X_i): five rounds of
  // exchanging half blocks with the partner lane; keep[j] masks the bits a
  // lane keeps in the round of width j
  uint32_t keep[5];
  transpose_masks(lane, keep);
  constexpr int kU = 4;  // groups in flight per warp
  constexpr int kW = THREADS / 32;
  const int g = lane >> 3, k = lane & 7;
  for (int64_t gb = warp; gb < ngroups; gb += (int64_t)kW * kU) {
    uint32_t x[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int64_t gi = gb + (int64_t)u * kW;
      const int64_t pos = gi * 32 + lane;
      const bool valid = gi < ngroups && (pos < NP || (pos >= NPpad && pos < NPpad + NT));
      const uint32_t r = valid ? rl[pos] : 0u;
      uint32_t v = G == 4 ? reinterpret_cast<const uint32_t*>(tabb)[r] : (uint32_t)tabb[r];
      x[u] = valid ? v : 0u;  // G bytes of x', byte g = block g
    }
#pragma unroll
    for (int rd = 0, j = 16; rd < 5; ++rd, j >>= 1) {
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const uint32_t y = __shfl_xor_sync(0xffffffffu, x[u], j);
        const uint32_t a = (lane & j) ? (y >> j) : (y << j);
        x[u] = (x[u] & keep[rd]) | (a & ~keep[rd]);
      }
    }
    // lane g*8 + k now holds plane k of block g
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int64_t gi = gb + (int64_t)u * kW;
      if (gi < ngroups && g < ng && k < kBits) rec[(((b0 + g) * ngroups + gi) * ds + mm) * 8 + k] = x[u];
    }
  }
  for (int i = tid; i < G * kOC; i += THREADS) {
    const int g = i / kOC, slot = i - g * kOC;
    const int64_t q = (b0 + g) * kOB + slot;
    if (g < ng) {
      uint8_t v = 0;
      if (slot < kOB && q < no) {
        const uint32_t r = orank[(int64_t)mm * no + q];
        v = G == 4 ? (uint8_t)(reinterpret_cast<const uint32_t*>(tabb)[r] >> (8 * g)) : tabb[r];
      }
      oplanes[((size_t)(b0 + g) * ds + mm) * kOC + slot] = v;
    }
  }
}

// ------------------------------------------------------------------ main kernel

// Unit u: origin block u / C, chunk u % C of the groups, where chunks [0, CP)
// cover the P list's groups [0, GP) in pieces of CGP and chunks [CP, C) the T
// list's groups [GP, GP + GT) in pieces of CGT.  Thread t holds origin slots
// t and t + kThreads of the block (kOPL = 2 origins per lane share every
// broadcast load of a group record).
template <int DS, int OCC>
__global__ void __launch_bounds__(kThreads, OCC)
k_register(const uint32_t* __restrict__ rec, const uint8_t* __restrict__ oplanes,
           const OriginMeta* __restrict__ meta, int64_t no, int64_t NP, int64_t NT, int64_t ngroups,
           int C, int CP, int GP, int GT, int CGP, int CGT, uint32_t* __restrict__ gcnt,
           unsigned* __restrict__ flags, const Final fin, unsigned long long wait_ns) {
  constexpr int RW = Rec<DS>::kWords;
  constexpr int NS = Rec<DS>::kNS;
  extern __shared__ __align__(16) uint32_t sm[];
  constexpr int NST = reg_stages(OCC);                                   // ring stages
  uint32_t* tiles = sm;                                                  // [NST][kTG][RW]
  uint64_t* bars = reinterpret_cast<uint64_t*>(tiles + NST * kTG * RW);  // [NST]
  const int tid = threadIdx.x;
  const int blk = (int)(blockIdx.x / C);
  const int ci = (int)(blockIdx.x % C);
  const int sample = ci < CP ? 0 : 1;
  int g0, g1;  // groups [g0, g1) of the block's record array
  if (sample == 0) {
    g0 = ci * CGP;
    g1 = g0 + CGP < GP ? g0 + CGP : GP;
  } else {
    g0 = GP + (ci - CP) * CGT;
    g1 = g0 + CGT < GP + GT ? g0 + CGT : GP + GT;
  }
  const int gbase = sample == 0 ? 0 : GP;  // first group of the sample
  const uint32_t tiles_s = (uint32_t)__cvta_generic_to_shared(tiles);
  const uint32_t bar_s = (uint32_t)__cvta_generic_to_shared(bars);
  const int ntiles = g1 > g0 ? (g1 - g0 + kTG - 1) / kTG : 0;
  auto issue = [&](int t) {  // thread 0: tile t into stage t % NST
    const int base = g0 + t * kTG;
    const int n = (g1 - base) < kTG ? (g1 - base) : kTG;
    const uint32_t bytes = (uint32_t)(n * RW * 4);
    const uint32_t st = (uint32_t)(t % NST);
    const uint32_t bar = bar_s + 8u * st;
    bk::fence_async();
    bk::mbar_expect(bar, bytes);
    bk::load(tiles_s + st * (uint32_t)(kTG * RW * 4), rec + ((size_t)blk * ngroups + base) * RW, bytes, bar);
  };
  if (tid == 0) {
    for (int k = 0; k < NST; ++k) bk::mbar_init(bar_s + 8u * k, 1);
    bk::mbar_init_fence();
  }
  __syncthreads();
  if (tid == 0)
    for (int t = 0; t < NST - 1 && t < ntiles; ++t) issue(t);

  // this lane's origins: comparison masks s[o][m][k] = all ones where bit k
  // of o'_m is set, and the split (sample-local)
  bool real[kOPL];
  int64_t q[kOPL];
  uint32_t s[kOPL][DS][kBits];
  int split[kOPL];
#pragma unroll
  for (int o = 0; o < kOPL; ++o) {
    const int slot = tid + o * kThreads;
    q[o] = (int64_t)blk * kOB + slot;
    real[o] = slot < kOB && q[o] < no;
#pragma unroll
    for (int m = 0; m < DS; ++m) {
      const uint32_t v = real[o] ? (uint32_t)oplanes[((size_t)blk * DS + m) * kOC + slot] : 0u;
#pragma unroll
      for (int k = 0; k < kBits; ++k) s[o][m][k] = 0u - ((v >> k) & 1u);
    }
    split[o] = 0;
    if (real[o]) {
      const OriginMeta mt = meta[q[o]];
      split[o] = (int)(sample == 0 ? mt.sP : mt.sT);
    }
  }
  // acc[S]: points so far in all dimensions of S; snap[S]: acc at the origin's
  // split (phase A part); the phase-B part is acc - snap
  uint32_t acc[kOPL][NS], snap[kOPL][NS];
  bool crossed[kOPL];
#pragma unroll
  for (int o = 0; o < kOPL; ++o) {
    crossed[o] = (g0 - gbase) * 32 >= split[o];  // the unit starts in phase B
#pragma unroll
    for (int S = 0; S < NS; ++S) acc[o][S] = snap[o][S] = 0;
  }
  // The block's origins are consecutive in dimension-0 order, so their splits
  // lie between those of its first and last origin: only sample-local groups
  // [wlo, whi) can hold a split (a split at 32k falls in group k).  Outside
  // that window no origin changes phase (a warp-uniform test per group).
  int wlo, whi;
  {
    const int64_t q0 = (int64_t)blk * kOB;
    const int64_t qL = ((int64_t)(blk + 1) * kOB < no ? (int64_t)(blk + 1) * kOB : no) - 1;
    const OriginMeta m0 = meta[q0], mL = meta[qL];
    wlo = (int)((sample == 0 ? m0.sP : m0.sT) >> 5);
    whi = (int)((sample == 0 ? mL.sP : mL.sT) >> 5) + 1;
  }
  // one group of 32 points against both origins; CHECK: the group lies in
  // the window, so an origin may pass its split here
  auto group = [&](const uint4* __restrict__ tile, int gi, int gidx, auto check) {
    constexpr bool CHECK = decltype(check)::value;
    // compare the group's 32 points with both origins, dimension by dimension
    uint32_t G[kOPL][DS];
#pragma unroll
    for (int m = 0; m < DS; ++m) {
      const uint4 a = tile[(gi * RW + m * 8) / 4];
      const uint4 b = tile[(gi * RW + m * 8) / 4 + 1];
      const uint32_t pl[kBits] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z};
#pragma unroll
      for (int o = 0; o < kOPL; ++o) {
        uint32_t r = 0xFFFFFFFFu;
#pragma unroll
        for (int k = 0; k < kBits; ++k) r = cmp_step(s[o][m][k], pl[k], r);
        G[o][m] = r;
      }
    }
#pragma unroll
    for (int o = 0; o < kOPL; ++o) {
      uint32_t M[NS + 1];
      M[0] = 0xFFFFFFFFu;
#pragma unroll
      for (int S = 1; S <= NS; ++S) {
        // G of the lowest dimension in S; every index folds in the unrolled loop
        const uint32_t gl = (S & 1) ? G[o][0] : ((S & 2) ? G[o][DS > 1 ? 1 : 0] : G[o][DS > 2 ? 2 : 0]);
        M[S] = M[S & (S - 1)] & gl;
      }
      if (CHECK) {
        const int pos0 = gidx * 32;  // sample-local position of bit 0
        if (!crossed[o] && pos0 + 32 > split[o]) {
          // the group holds the origin's split, or begins phase B
          const uint32_t pa = pos0 < split[o] ? ~(0xFFFFFFFFu << (split[o] - pos0)) : 0u;  // phase-A points
#pragma unroll
          for (int S = 1; S <= NS; ++S) snap[o][S - 1] = acc[o][S - 1] + (uint32_t)__popc(M[S] & pa);
          crossed[o] = true;
        }
      }
#pragma unroll
      for (int S = 1; S <= NS; ++S) acc[o][S - 1] += (uint32_t)__popc(M[S]);
    }
  };
  for (int t = 0; t < ntiles; ++t) {
    const int base = g0 + t * kTG;
    const int n = (g1 - base) < kTG ? (g1 - base) : kTG;
    // stage (t - 1) % NST was released by the barrier that ended tile t - 1
    if (tid == 0 && t + NST - 1 < ntiles) issue(t + NST - 1);
    const bool ok = bk::wait(bar_s + 8u * (uint32_t)(t % NST), (uint32_t)((t / NST) & 1), wait_ns);
    if (ok) {
      const uint4* tile = reinterpret_cast<const uint4*>(tiles + (t % NST) * kTG * RW);
      // tile-local groups [wa, wb) lie in the window; before it no split is
      // reached, after it every split is behind
      const int off = base - gbase;  // sample-local group of gi = 0
      const int wa = wlo - off < 0 ? 0 : (wlo - off > n ? n : wlo - off);
      const int wb = whi - off < wa ? wa : (whi - off > n ? n : whi - off);
#pragma unroll 2
      for (int gi = 0; gi < wa; ++gi) group(tile, gi, off + gi, std::false_type{});
      for (int gi = wa; gi < wb; ++gi) group(tile, gi, off + gi, std::true_type{});
#pragma unroll 2
      for (int gi = wb; gi < n; ++gi) group(tile, gi, off + gi, std::false_type{});
    }
    // every thread is done with stage t % NST; a timed-out wait ends the unit
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        atomicOr(flags, ddks::kFlagTimeout);
        // the copies of tiles t .. t + NST - 2 may still be in flight: wait
        // for them (bounded) so that none lands after the CTA has exited
        for (int k = t; k < t + NST - 1 && k < ntiles; ++k)
          bk::wait(bar_s + 8u * (uint32_t)(k % NST), (uint32_t)((k / NST) & 1), bk::kDrainNs);
      }
      return;
    }
  }
#pragma unroll
  for (int o = 0; o < kOPL; ++o) {
    if (!real[o]) continue;
    uint32_t* c = gcnt + q[o] * kCnt;
#pragma unroll
    for (int S = 0; S < NS; ++S) {
      const uint32_t all = acc[o][S];
      const uint32_t b = crossed[o] ? all - snap[o][S] : 0u;
      if (all) atomicAdd(&c[(sample * 2 + 0) * NS + S], all);
      if (b) atomicAdd(&c[(sample * 2 + 1) * NS + S], b);
    }
  }
  // The last unit of an origin block to finish turns the block's counters
  // into per-origin maxima and a packed (num, origin) candidate for the
  // global maximum; the last block to finish writes the result.  Tickets
  // only: no CTA waits for another.
  __shared__ unsigned ticket;
  __threadfence();
  __syncthreads();
  if (tid == 0) ticket = atomicAdd(&fin.done[blk], 1u);
  __syncthreads();
  if (ticket != (unsigned)(C - 1)) return;
  __threadfence();
#pragma unroll
  for (int o = 0; o < kOPL; ++o) {
    if (!real[o]) continue;
    uint64_t bv;
    int bj;
    const OriginMeta mt = meta[q[o]];
    origin_best<DS, false>(gcnt, mt, q[o], NP, NT, bv, bj);
    const int64_t pos = (int64_t)mt.k - fin.ob;
    fin.best[pos] = bv;
    fin.bestj[pos] = bj;
    // larger numerator first, then the lower origin
    atomicMax(fin.packed, (bv << kPackShift) | (kPackMask - (unsigned long long)pos));
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) ticket = atomicAdd(&fin.done[fin.blocks], 1u);
  __syncthreads();
  if (ticket != (unsigned)(fin.blocks - 1) || tid != 0 || !fin.out3) return;
  __threadfence();
  const unsigned long long pk = atomicAdd(fin.packed, 0ull);
  const int64_t pos = (int64_t)(kPackMask - (pk & kPackMask));
  fin.out3[0] = pk >> kPackShift;
  fin.out3[1] = (unsigned long long)(fin.ob + pos);
  fin.out3[2] = (unsigned long long)(long long)__ldcg(&fin.bestj[pos]);
}

size_t reg_smem(int ds, int occ) { return (size_t)reg_stages(occ) * kTG * 8 * ds * 4 + 8 * 4 + 16; }
size_t pack_smem(int NW, int G) { return (size_t)NW * 32 * G + (size_t)G * NW * 4 + 40 * 4; }
constexpr size_t kPackSmemMax = 227u * 1024u;

}  // namespace

bool ddks_register_supported(int d, int64_t NP, int64_t NT) {
  const int64_t N = NP + NT;
  if (d < 2 || d > 4 || N > kMaxRegN) return false;
  return pack_smem((int)((N + 31) / 32), 1) <= kPackSmemMax;
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
  const int64_t blocks = (no + kOB - 1) / kOB;
  // each sample's part of the list is padded to whole groups of 32
  const int64_t NPpad = (NP + 31) & ~(int64_t)31, NTpad = (NT + 31) & ~(int64_t)31;
  const int64_t Lrow = NPpad + NTpad;
  const int64_t ngroups = Lrow / 32;
  const int GP = (int)(NPpad / 32), GT = (int)(NTpad / 32);
  // scratch (u32): pprefix N, exO N, olist no, gcnt no*32 + tickets (blocks + 1) + packed,
  // rankL ds*Lrow, orank ds*no, scan tmp; then meta
  const size_t scan_tmp = ddks_scan_tmp_elems(1, N);
  const size_t n_fin = (size_t)blocks + 1 + 4;
  const size_t n_u32 = (size_t)N * 2 + (size_t)no + (size_t)no * kCnt + n_fin + (size_t)ds * Lrow +
                       (size_t)ds * no + scan_tmp;
  int rc = ctx->reg_meta.reserve(ctx, n_u32 * 4 + (size_t)no * sizeof(OriginMeta) + 64);
  if (rc) return cudaErrorMemoryAllocation;
  // group records [blocks][ngroups][ds][8] u32 and origin values [blocks][ds][128] u8
  const bool fused = plan.fused && ddks_fused_supported(ds, N, plan.fused);
  const size_t rec_words = fused ? 0 : (size_t)blocks * ngroups * ds * 8;
  rc = ctx->reg_words.reserve(ctx, fused ? ddks_fused_scratch_bytes(ds, N, blocks)
                                         : rec_words * 4 + (size_t)blocks * ds * kOC);
  if (rc) return cudaErrorMemoryAllocation;
  uint32_t* pprefix = (uint32_t*)ctx->reg_meta.ptr;
  uint32_t* exO = pprefix + N;
  uint32_t* olist = exO + N;
  uint32_t* gcnt = olist + no;
  unsigned* done = gcnt + no * kCnt;  // [blocks + 1] tickets, then the packed maximum (8-byte aligned)
  unsigned long long* packed = reinterpret_cast<unsigned long long*>(
      (reinterpret_cast<uintptr_t>(done + blocks + 1) + 7) & ~(uintptr_t)7);
  uint32_t* rankL = reinterpret_cast<uint32_t*>((reinterpret_cast<uintptr_t>(gcnt + no * kCnt + n_fin) + 15) &
                                                ~(uintptr_t)15);
  uint32_t* orank = rankL + (size_t)ds * Lrow;
  uint32_t* stmp = orank + (size_t)ds * no;
  OriginMeta* meta = reinterpret_cast<OriginMeta*>(
      (reinterpret_cast<uintptr_t>(stmp + scan_tmp) + 15) & ~(uintptr_t)15);
  uint32_t* rec = (uint32_t*)ctx->reg_words.ptr;
  uint8_t* oplanes = reinterpret_cast<uint8_t*>(rec + rec_words);
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
  if (exO == nullptr) {  // every point an origin, q = sorted position
    k_reg_lists_meta<<<grid(N), 256, 0, st>>>(sidx0, rank, N, NP, NPpad, Lrow, ds, pprefix, rankL, meta, orank);
    n += 1;
  } else {
    k_reg_lists<<<grid(N), 256, 0, st>>>(sidx0, rank, N, NP, NPpad, Lrow, ds, ob, oe, pprefix, exO, rankL,
                                         olist);
    k_reg_meta<<<grid(no), 256, 0, st>>>(rank, olist, pprefix, N, no, ds, meta, orank);
    n += 2;
  }
  // stage timing: the count stage (re-rank packing included) starts here
  ddks_stage_mark(ctx, 1, st);
  if (fused) {
    e = cudaMemsetAsync(gcnt, 0, ((size_t)no * kCnt + n_fin) * 4, st);
    if (e == cudaSuccess)
      e = ddks_fused_count(ctx, ds, plan.fused, rankL, orank, meta, no, N, NP, NT, NPpad, Lrow, gcnt, done, packed, best, bestj,
                           ob, out3, flags, ctx->reg_words.ptr, st, &n);
    if (e != cudaSuccess) return e;
    if (reduced) *reduced = out3 != nullptr;
    ctx->launches += n;
    return cudaSuccess;
  }
  if (pack_smem(NW, 4) <= kPackSmemMax) {
    const size_t psmem = pack_smem(NW, 4);
    e = ddks_smem_attr(k_reg_pack<4, kPack4Threads>, (int)psmem);
    if (e != cudaSuccess) return e;
    k_reg_pack<4, kPack4Threads><<<dim3((unsigned)((blocks + 3) / 4), (unsigned)ds), kPack4Threads, psmem, st>>>(
        rankL, orank, no, blocks, NP, NT, NPpad, Lrow, NW, ds, rec, oplanes);
  } else {
    const size_t psmem = pack_smem(NW, 1);
    e = ddks_smem_attr(k_reg_pack<1, kPackThreads>, (int)psmem);
    if (e != cudaSuccess) return e;
    k_reg_pack<1, kPackThreads><<<dim3((unsigned)blocks, (unsigned)ds), kPackThreads, psmem, st>>>(
        rankL, orank, no, blocks, NP, NT, NPpad, Lrow, NW, ds, rec, oplanes);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  ++n;
  // chunks of the groups per origin block: about 3 waves of the resident CTAs
  const int64_t slots = (int64_t)ctx->num_sms * 12;
  int64_t want = (3 * slots + blocks - 1) / blocks;  // chunks per block
  if (want < 2) want = 2;
  int64_t CG = (ngroups + want - 1) / want;
  if (CG < 2) CG = 2;
  const int64_t CP = (GP + CG - 1) / CG, CT = (GT + CG - 1) / CG;
  const int CGP = (int)((GP + CP - 1) / CP), CGT = (int)((GT + CT - 1) / CT);
  const int64_t C = CP + CT;
  e = cudaMemsetAsync(gcnt, 0, ((size_t)no * kCnt + n_fin) * 4, st);
  if (e != cudaSuccess) return e;
  const unsigned ctas = (unsigned)(blocks * C);
  // resident 64-thread CTAs per SM the kernel is built for: 8, 12 or 16
  const int occ = plan.reg_occ == 4 ? 8 : plan.reg_occ == 8 ? 16 : 12;
  const size_t smem = reg_smem(ds, occ);
  Final fin{out3, done, packed, best, bestj, ob, (int)blocks};
  auto go = [&](auto kern) -> cudaError_t {
    cudaError_t r = ddks_smem_attr(kern, (int)smem);
    if (r != cudaSuccess) return r;
    kern<<<ctas, kThreads, smem, st>>>(rec, oplanes, meta, no, NP, NT, ngroups, (int)C, (int)CP, GP, GT, CGP,
                                        CGT, gcnt, flags, fin, ctx->dev_wait_ns);
    return cudaGetLastError();
  };
  if (ds == 1) e = occ == 8 ? go(k_register<1, 8>) : occ == 12 ? go(k_register<1, 12>) : go(k_register<1, 16>);
  else if (ds == 2) e = occ == 8 ? go(k_register<2, 8>) : occ == 12 ? go(k_register<2, 12>) : go(k_register<2, 16>);
  else e = occ == 8 ? go(k_register<3, 8>) : occ == 12 ? go(k_register<3, 12>) : go(k_register<3, 16>);
  if (e != cudaSuccess) return e;
  ++n;
  if (reduced) *reduced = out3 != nullptr;
  ctx->launches += n;
  return cudaGetLastError();
}
