// count_register.cuh -- pieces shared by the two bit-sliced count kernels of
// the register path (count_register.cu: bit planes staged in global memory by
// a pack kernel; count_fused.cu: bit planes built in shared memory by the
// count kernel itself).
//
// Both compute, for origin blocks of kOB origins (consecutive in dimension-0
// order), the orthant counts of Eq. membership by subsets: for every
// non-empty set S of the dimensions 1..d-1 and every phase (points before the
// origin's dimension-0 split, A, and from it on, B), the number of points of a
// sample that are >= the origin in every dimension of S.  Inclusion-exclusion
// turns them into orthant counts; the maximum of |cP*NT - cT*NP| (Eq. d1 with
// the normalisation of Eq. abs_difference) follows per origin.
#pragma once
#include <cstdint>

#include "ddks_internal.cuh"

namespace ddks_reg {

constexpr int kOC = 128;      // origin slots per block
constexpr int kOB = kOC - 1;  // origins per block (re-ranked values <= 127 fit 7 bits)
constexpr int kBits = 7;      // bit planes per dimension
constexpr int kCnt = 32;      // counters per origin: [sample][phase][subset] (<= 2*2*7 used)

struct OriginMeta {
  uint32_t sP, sT;  // splits, sample-local: P points / T points with a smaller dimension-0 rank
  uint32_t k;       // pooled index
  uint32_t pad;
};

// The fused final step: per-origin maxima into best/bestj at pooled index -
// ob and (out3 != nullptr) the result {num_max, arg-max origin, orthant}.
// done: [blocks + 1] zeroed tickets; packed: one zeroed word holding the
// maximum over origins of (num << kPackShift) | (kPackMask - position).
struct Final {
  unsigned long long* out3;
  unsigned* done;
  unsigned long long* packed;
  uint64_t* best;
  int32_t* bestj;
  int64_t ob;
  int blocks;
};
constexpr int kPackShift = 26;  // positions < 2^26; numerators < 2^38
constexpr unsigned long long kPackMask = (1ull << kPackShift) - 1;

// One bit of the bit-sliced comparison, from the least significant bit up:
// r = s ? (pl & r) : (pl | r), s = all ones where the origin's bit is set --
// one 3-input logic op (truth table 0x8E for operands s, pl, r).
DDKS_DEV uint32_t cmp_step(uint32_t s, uint32_t pl, uint32_t r) {
  uint32_t d;
  asm("lop3.b32 %0, %1, %2, %3, 0x8E;" : "=r"(d) : "r"(s), "r"(pl), "r"(r));
  return d;
}

// The orthant counts of one origin, sample and phase from its subset
// counters: n[0] = all points of the phase, n[S] = points >= the origin in
// every dimension of S.  count(exactly the dims in B) = sum over S >= B of
// (-1)^|S \ B| n[S].
template <int DS>
DDKS_DEV void orthants(const uint32_t (&n)[1 << DS], uint32_t (&cnt)[1 << DS]) {
#pragma unroll
  for (int B = 0; B < (1 << DS); ++B) {
    int64_t v = 0;
#pragma unroll
    for (int S = 0; S < (1 << DS); ++S)
      if ((S & B) == B) v += (__popc(S ^ B) & 1) ? -(int64_t)n[S] : (int64_t)n[S];
    cnt[B] = (uint32_t)v;
  }
}

// The best code of origin q.  Counters c[sample][phase][S - 1] hold, for
// AB = true, the phase-A and phase-B counts; for AB = false, the counts over
// all points and over phase B.
template <int DS, bool AB>
DDKS_DEV void origin_best(const uint32_t* __restrict__ gcnt, const OriginMeta& mt, int64_t q, int64_t NP,
                          int64_t NT, uint64_t& bv, int& bj) {
  constexpr int NS = (1 << DS) - 1;
  const uint32_t* c = gcnt + q * kCnt;
  uint32_t cnt[2][2][1 << DS];  // [sample][phase A, B][bin]
#pragma unroll
  for (int smp = 0; smp < 2; ++smp) {
    const uint32_t size = smp == 0 ? (uint32_t)NP : (uint32_t)NT;
    const uint32_t split = smp == 0 ? mt.sP : mt.sT;
    uint32_t nA[1 << DS], nB[1 << DS];
    nA[0] = split;
    nB[0] = size - split;
#pragma unroll
    for (int S = 1; S <= NS; ++S) {
      const uint32_t x = __ldcg(&c[(smp * 2 + 0) * NS + S - 1]);
      const uint32_t b = __ldcg(&c[(smp * 2 + 1) * NS + S - 1]);
      nA[S] = AB ? x : x - b;
      nB[S] = b;
    }
    orthants<DS>(nA, cnt[smp][0]);
    orthants<DS>(nB, cnt[smp][1]);
  }
  bv = 0;
  bj = 0;
  // code = bin << 1 | phase (bit 0 is dimension 0), lowest code first
#pragma unroll
  for (int code = 0; code < (2 << DS); ++code) {
    const int ph = code & 1, bin = code >> 1;
    const uint64_t num = ddks::numer(cnt[0][ph][bin], cnt[1][ph][bin], (uint64_t)NP, (uint64_t)NT);
    if (num > bv) { bv = num; bj = code; }
  }
}

// Per-origin maxima of block blk (threads [0, nthreads) of the CTA, one origin
// each) and its candidate for the global maximum; then, by ticket, the last
// block writes the result.  Called by every thread of the CTA that completed
// the block's counters, after a fence and a CTA barrier.
template <int DS, bool AB>
DDKS_DEV void finish_block(const uint32_t* __restrict__ gcnt, const OriginMeta* __restrict__ meta, int64_t no,
                           int64_t NP, int64_t NT, int blk, const Final& fin, unsigned* s_ticket) {
  const int tid = threadIdx.x, nthreads = blockDim.x;
  for (int slot = tid; slot < kOB; slot += nthreads) {
    const int64_t q = (int64_t)blk * kOB + slot;
    if (q >= no) break;
    uint64_t bv;
    int bj;
    const OriginMeta mt = meta[q];
    origin_best<DS, AB>(gcnt, mt, q, NP, NT, bv, bj);
    const int64_t pos = (int64_t)mt.k - fin.ob;
    fin.best[pos] = bv;
    fin.bestj[pos] = bj;
    // larger numerator first, then the lower origin
    atomicMax(fin.packed, (bv << kPackShift) | (kPackMask - (unsigned long long)pos));
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) *s_ticket = atomicAdd(&fin.done[fin.blocks], 1u);
  __syncthreads();
  if (*s_ticket != (unsigned)(fin.blocks - 1) || tid != 0 || !fin.out3) return;
  __threadfence();
  const unsigned long long pk = atomicAdd(fin.packed, 0ull);
  const int64_t pos = (int64_t)(kPackMask - (pk & kPackMask));
  fin.out3[0] = pk >> kPackShift;
  fin.out3[1] = (unsigned long long)(fin.ob + pos);
  fin.out3[2] = (unsigned long long)(long long)__ldcg(&fin.bestj[pos]);
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

// Masks of the 32 x 32 bit transpose across a warp (lane i holds word X_i;
// afterwards lane j holds the word whose bit i is bit j of X_i): five rounds
// of exchanging half blocks with the partner lane; keep[rd] masks the bits a
// lane keeps in the round of width 16 >> rd.
DDKS_DEV void transpose_masks(int lane, uint32_t (&keep)[5]) {
  uint32_t m = 0xFFFF0000u;
#pragma unroll
  for (int rd = 0, j = 16; rd < 5; ++rd, j >>= 1) {
    keep[rd] = (lane & j) ? ~(m >> j) : ~m;
    m ^= m >> (j >> 1);
  }
}

DDKS_DEV uint32_t transpose32(uint32_t x, int lane, const uint32_t (&keep)[5]) {
#pragma unroll
  for (int rd = 0, j = 16; rd < 5; ++rd, j >>= 1) {
    const uint32_t y = __shfl_xor_sync(0xffffffffu, x, j);
    const uint32_t a = (lane & j) ? (y >> j) : (y << j);
    x = (x & keep[rd]) | (a & ~keep[rd]);
  }
  return x;
}

}  // namespace ddks_reg
