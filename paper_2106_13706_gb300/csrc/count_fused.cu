// count_fused.cu -- K1f: the register path's bit-sliced orthant counts for
// d = 2, 3, 4 with the bit planes built in shared memory by the count kernel.
//
// The statistic and the counting are those of count_register.cu (Sec. 2.1,
// Eq. ddks_tensor_definition; the ">=" split of Sec. 2.2.1, Eq. g; Eq.
// membership by subsets and inclusion-exclusion; max |cP*NT - cT*NP| of Eq. d1
// with the normalisation of Eq. abs_difference): dimension 0 by the position
// in dimension-0 order (phase A before the origin's split, phase B from it
// on), dimensions 1..d-1 by bit-sliced compares of values re-ranked against
// the origin block (x' = #distinct origin values of the block <= x, 7 bits).
//
// What differs is where the bit planes come from.  A prep kernel writes, once
// per origin block and dimension, the re-rank table over the global ranks as
// a bitmap of the block's origin ranks with per-word prefix counts:
//   x'(r) = pf[r >> 5] + popc(bm[r >> 5] << (31 - (r & 31))).
// The count kernel is persistent: CTA i takes a contiguous range of the
// (origin block, group of 32 list positions) units.  At each block it loads
// the block's table into shared memory with one bulk copy; its four warp
// pairs then take batches of 16 groups in turn: the ranks of a batch arrive
// by bulk asynchronous copies (the TMA engine, mbarrier completion, bounded
// waits), each warp of the pair looks up x' for 8 groups and turns the 32
// points' x' into bit planes with a 32 x 32 warp transpose, and after a pair
// barrier both warps compare their 2 x 32 origins with every group of the
// batch.  The planes never leave shared memory.
//
// Counters per origin and sample are kept separately for phase A and phase B;
// the origins of a block are consecutive in dimension-0 order, so all but a
// few groups per sample lie wholly before or wholly after every origin's
// split, and only those few need per-origin phase masks.  At the end of a
// (block, sample) piece the pairs' counters are summed in shared memory and
// added to global counters; the CTA that completes a block's groups (ticket)
// computes the block's per-origin maxima, and the last block the result.
#include "bulk_copy.cuh"
#include "count_register.cuh"
#include "ddks_host.h"
#include "ddks_internal.cuh"

namespace {

using namespace ddks_reg;
namespace bk = ddks::bulk;

constexpr int kBG = 16;                 // groups per batch (each warp of a pair builds 8)
constexpr int kPrepThreads = 256;

// uint2 words of one block's table: DS rows of W words, padded to 16 bytes
__host__ __device__ constexpr int64_t tab_stride(int ds, int W) { return ((int64_t)ds * W + 1) & ~(int64_t)1; }

// Dynamic shared memory of the count kernel, in this order:
//   stab  uint2 [DS][W] (padded to 16 bytes)   the current block's table
//   acc   u32 [kOC][2][NS]                    a piece's counters, summed over the pairs
//   per warp pair (NPR of them): rbuf u32 [2][DS][kBG * 32] ranks of a batch (two stages)
//                  pbuf u32 [2][kBG][DS][8]   bit planes of a batch (two stages)
template <int DS, int NPR>
struct FusedSmem {
  static constexpr int NS = (1 << DS) - 1;
  static constexpr size_t acc_bytes = (size_t)kOC * 2 * NS * 4;
  static constexpr size_t rbuf_bytes = (size_t)2 * DS * kBG * 32 * 4;
  static constexpr size_t pbuf_bytes = (size_t)2 * kBG * DS * 8 * 4;
  static constexpr size_t pair_bytes = rbuf_bytes + pbuf_bytes;
  __host__ __device__ static constexpr size_t tab_bytes(int W) { return (size_t)tab_stride(DS, W) * 8; }
  __host__ __device__ static constexpr size_t total(int W) { return tab_bytes(W) + acc_bytes + NPR * pair_bytes; }
};

// ------------------------------------------------------------------ prep

// One CTA per origin block: bitmap of the block's origin ranks per dimension
// (dimensions 1..DS), the exclusive prefix counts of its words, and the
// origins' own re-ranked values.
//   tab[blk][m][w] = {bitmap word w, #set bits in words < w}
//   oval[blk][m][slot] = x' of the slot's origin (0 for the pad slot and past no)
template <int DS>
__global__ void __launch_bounds__(kPrepThreads)
k_fused_tables(const uint32_t* __restrict__ orank, int64_t no, int W, uint2* __restrict__ tab,
               uint8_t* __restrict__ oval) {
  extern __shared__ __align__(16) uint32_t fsm[];
  uint32_t* bits = fsm;                                    // [DS][W]
  uint8_t* pf = reinterpret_cast<uint8_t*>(fsm + DS * W);  // [DS][W]
  __shared__ uint32_t tmp[40];
  const int tid = threadIdx.x;
  const int blk = blockIdx.x;
  for (int i = tid; i < DS * W; i += kPrepThreads) bits[i] = 0u;
  __syncthreads();
  for (int i = tid; i < DS * kOB; i += kPrepThreads) {
    const int m = i / kOB, slot = i - m * kOB;
    const int64_t q = (int64_t)blk * kOB + slot;
    if (q < no) {
      const uint32_t r = orank[(int64_t)m * no + q];
      atomicOr(&bits[m * W + (r >> 5)], 1u << (r & 31));
    }
  }
  __syncthreads();
  // prefix counts of all DS rows at once, one byte each (a block has at most
  // 127 distinct values per dimension, so no byte carries into the next)
  const int seg = (W + kPrepThreads - 1) / kPrepThreads;
  const int wa = tid * seg < W ? tid * seg : W;
  const int wb = wa + seg < W ? wa + seg : W;
  uint32_t c = 0;
  for (int w = wa; w < wb; ++w)
#pragma unroll
    for (int m = 0; m < DS; ++m) c += (uint32_t)__popc(bits[m * W + w]) << (8 * m);
  uint32_t run = block_exscan<kPrepThreads>(c, tmp);
  for (int w = wa; w < wb; ++w) {
#pragma unroll
    for (int m = 0; m < DS; ++m) {
      const uint32_t bw = bits[m * W + w];
      pf[m * W + w] = (uint8_t)((run >> (8 * m)) & 0xFFu);
      run += (uint32_t)__popc(bw) << (8 * m);
    }
  }
  __syncthreads();
  uint2* out = tab + (int64_t)blk * tab_stride(DS, W);
  for (int i = tid; i < DS * W; i += kPrepThreads) out[i] = make_uint2(bits[i], pf[i]);
  for (int i = tid; i < DS * kOC; i += kPrepThreads) {
    const int m = i / kOC, slot = i - m * kOC;
    const int64_t q = (int64_t)blk * kOB + slot;
    uint32_t v = 0;
    if (slot < kOB && q < no) {
      const uint32_t r = orank[(int64_t)m * no + q];
      v = pf[m * W + (r >> 5)] + (uint32_t)__popc(bits[m * W + (r >> 5)] << (31 - (r & 31)));
    }
    oval[((int64_t)blk * DS + m) * kOC + slot] = (uint8_t)v;
  }
}

// ------------------------------------------------------------------ count

// barrier of the 64 threads of a warp pair that also ORs a flag over them
DDKS_DEV bool pair_or(int id, bool v) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 q, %1, 0;\n bar.red.or.pred p, %2, 64, q;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(r)
      : "r"((uint32_t)v), "r"(id)
      : "memory");
  return r != 0;
}

// x' of global rank r from the block's table row (shared memory)
DDKS_DEV uint32_t rerank(const uint2* __restrict__ row, uint32_t r) {
  const uint2 t = row[r >> 5];
  return t.y + (uint32_t)__popc(t.x << (~r & 31u));
}

// Persistent count kernel: CTA b takes units [units * b / grid, units * (b + 1)
// / grid) of the (origin block, group) sequence, block-major, within a block
// the P list's GP groups then the T list's GT groups.
// NPR warp pairs per CTA; MINB resident CTAs per SM the registers are budgeted
// for; UNR the unroll of the group loop.
template <int DS, int NPR, int MINB, int UNR>
__global__ void __launch_bounds__(64 * NPR, MINB)
k_fused(const uint32_t* __restrict__ rankL, const uint2* __restrict__ tab, const uint8_t* __restrict__ oval,
        const OriginMeta* __restrict__ meta, int64_t no, int64_t NP, int64_t NT, int64_t NPpad, int64_t Lrow,
        int W, int GP, int GT, int64_t units, uint32_t* __restrict__ gcnt, unsigned* __restrict__ flags,
        const Final fin, unsigned long long wait_ns) {
  using SM = FusedSmem<DS, NPR>;
  constexpr int kPairs = NPR, kFThreads = 64 * NPR;
  constexpr int NS = SM::NS;
  extern __shared__ __align__(16) unsigned char fraw[];
  __shared__ __align__(8) unsigned long long bars[1 + 2 * kPairs];
  __shared__ unsigned s_abort, s_last, s_ticket;
  uint2* stab = reinterpret_cast<uint2*>(fraw);
  uint32_t* acc = reinterpret_cast<uint32_t*>(fraw + SM::tab_bytes(W));
  const int tid = threadIdx.x, lane = tid & 31;
  const int pair = tid >> 6, tp = tid & 63, half = tp >> 5;
  const int pair_bar = 1 + pair;  // named barrier of the pair (0 is the CTA barrier)
  unsigned char* pbase = fraw + SM::tab_bytes(W) + SM::acc_bytes + (size_t)pair * SM::pair_bytes;
  uint32_t* rbuf = reinterpret_cast<uint32_t*>(pbase);
  uint32_t* pbuf = reinterpret_cast<uint32_t*>(pbase + SM::rbuf_bytes);
  const uint32_t bar0 = (uint32_t)__cvta_generic_to_shared(bars);  // the table's barrier
  const uint32_t rbar = bar0 + 8u * (uint32_t)(1 + 2 * pair);      // this pair's two rank stages
  const uint32_t rbuf_s = (uint32_t)__cvta_generic_to_shared(rbuf);
  const uint32_t stab_s = (uint32_t)__cvta_generic_to_shared(stab);
  if (tid == 0) {
    for (int i = 0; i < 1 + 2 * kPairs; ++i) bk::mbar_init(bar0 + 8u * i, 1);
    bk::mbar_init_fence();
    s_abort = 0;
  }
  for (int i = tid; i < kOC * 2 * NS; i += kFThreads) acc[i] = 0u;
  __syncthreads();
  const int64_t per = (int64_t)GP + GT;
  const int64_t u0 = units * blockIdx.x / gridDim.x, u1 = units * (blockIdx.x + 1) / gridDim.x;
  uint32_t visits = 0;  // table loads so far (the phase of bars[0])
  uint32_t jj = 0;      // batches of this pair so far: stage jj & 1, phase (jj >> 1) & 1
  for (int64_t u = u0; u < u1;) {
    const int blk = (int)(u / per);
    const int64_t bend = u1 < (int64_t)(blk + 1) * per ? u1 : (int64_t)(blk + 1) * per;
    // ---- the block's table, by one bulk copy
    __syncthreads();  // every warp is done with the previous table
    if (tid == 0) {
      const uint32_t bytes = (uint32_t)SM::tab_bytes(W);
      bk::fence_async();
      bk::mbar_expect(bar0, bytes);
      bk::load(stab_s, tab + (int64_t)blk * tab_stride(DS, W), bytes, bar0);
    }
    // this thread's two origins (slots tp and tp + 64): comparison masks
    // s[o][m][k] = all ones where bit k of o'_m is set, splits per sample
    uint32_t s[2][DS][kBits];
    bool real[2];
    uint32_t spP[2], spT[2];
#pragma unroll
    for (int o = 0; o < 2; ++o) {
      const int slot = tp + 64 * o;
      const int64_t q = (int64_t)blk * kOB + slot;
      real[o] = slot < kOB && q < no;
#pragma unroll
      for (int m = 0; m < DS; ++m) {
        const uint32_t v = oval[((int64_t)blk * DS + m) * kOC + slot];
#pragma unroll
        for (int k = 0; k < kBits; ++k) s[o][m][k] = 0u - ((v >> k) & 1u);
      }
      spP[o] = spT[o] = 0;
      if (real[o]) {
        const OriginMeta mt = meta[q];
        spP[o] = mt.sP;
        spT[o] = mt.sT;
      }
    }
    // groups wholly before / from the block's splits, per sample (the block's
    // origins are consecutive in dimension-0 order, so its splits increase)
    uint32_t wloP, whiP, wloT, whiT;
    {
      const int64_t q0 = (int64_t)blk * kOB;
      const int64_t qL = ((int64_t)(blk + 1) * kOB < no ? (int64_t)(blk + 1) * kOB : no) - 1;
      const OriginMeta m0 = meta[q0], mL = meta[qL];
      wloP = m0.sP >> 5;
      whiP = (mL.sP + 31) >> 5;
      wloT = m0.sT >> 5;
      whiT = (mL.sT + 31) >> 5;
    }
    const bool tok = bk::wait(bar0, visits & 1u, wait_ns);
    ++visits;
    if (__syncthreads_or(!tok)) {
      if (tid == 0) {
        atomicOr(flags, ddks::kFlagTimeout);
        bk::wait(bar0, (visits - 1) & 1u, bk::kDrainNs);
      }
      return;
    }
    const int64_t gi = u - (int64_t)blk * per, ge = bend - (int64_t)blk * per;
    for (int smp = 0; smp < 2; ++smp) {
      // sample-local groups [pa, pb) of this piece (the same for every thread)
      const int64_t pa = smp == 0 ? gi : (gi > GP ? gi - GP : 0);
      const int64_t pb = smp == 0 ? (ge < GP ? ge : GP) : ge - GP;
      if (pb <= pa) continue;
      const int64_t size = smp == 0 ? NP : NT;
      const int64_t lbase = smp == 0 ? 0 : NPpad;  // list position of the sample's first point
      const uint32_t wlo = smp == 0 ? wloP : wloT, whi = smp == 0 ? whiP : whiT;
      const uint32_t sp0 = smp == 0 ? spP[0] : spT[0], sp1 = smp == 0 ? spP[1] : spT[1];
      // acc_r[o][S]: this pair's points so far >= origin o in every dimension
      // of S.  A pair visits its groups in increasing order, so its groups
      // before an origin's split are wholly phase A and those after it wholly
      // phase B.  When the pair reaches the split it adds its phase-A count
      // so far to the shared phase-A counter and takes it off the phase-B
      // counter, which receives acc_r at the end.
      uint32_t acc_r[2][NS];
      bool crossed[2];
#pragma unroll
      for (int o = 0; o < 2; ++o) {
        crossed[o] = false;
#pragma unroll
        for (int S = 0; S < NS; ++S) acc_r[o][S] = 0u;
      }
      bool all_crossed = false;  // warp-uniform: past the block's window
      auto snapshot = [&](int o, int S, uint32_t v) {
        if (real[o] && v) {
          const int slot = tp + 64 * o;
          atomicAdd(&acc[(slot * 2 + 0) * NS + S], v);
          atomicSub(&acc[(slot * 2 + 1) * NS + S], v);
        }
      };
      const int nb = (int)((pb - pa + kBG - 1) / kBG);
      // thread 0 of the pair: the ranks of batch i into stage st
      auto issue = [&](int i, uint32_t st) {
        const int64_t g0 = pa + (int64_t)i * kBG;
        const uint32_t bytes = (uint32_t)((pb - g0 < kBG ? pb - g0 : kBG) * 128);
        const uint32_t bar = rbar + 8u * st;
        bk::fence_async();
        bk::mbar_expect(bar, bytes * DS);
#pragma unroll
        for (int m = 0; m < DS; ++m)
          bk::load(rbuf_s + (st * DS + m) * (kBG * 128u), rankL + (int64_t)m * Lrow + lbase + g0 * 32, bytes, bar);
      };
      if (tp == 0 && pair < nb) issue(pair, jj & 1u);
      bool aborted = false;
      for (int i = pair; i < nb; i += kPairs, ++jj) {
        const uint32_t st = jj & 1u;
        // stage st ^ 1 was released by the pair barrier of the previous batch
        if (tp == 0 && i + kPairs < nb) issue(i + kPairs, st ^ 1u);
        const bool ok = bk::wait(rbar + 8u * st, (jj >> 1) & 1u, wait_ns);
        const int64_t g0 = pa + (int64_t)i * kBG;
        const int n = (int)(pb - g0 < kBG ? pb - g0 : kBG);
        uint32_t* pl_st = pbuf + st * (kBG * DS * 8);
        if (ok) {
          // x' of the batch's points, 32 per group, turned into bit planes:
          // after the transpose lane 8m + k holds plane k of dimension m + 1.
          // Groups past the batch's end get zero planes (no point is >= a
          // real origin there).
          const uint32_t* rb = rbuf + st * (DS * kBG * 32);
          uint32_t keep[5];
          transpose_masks(lane, keep);
          for (int j = half; j < kBG; j += 2) {
            const int64_t pos = (g0 + j) * 32 + lane;  // sample-local position
            uint32_t w = 0;
            if (j < n && pos < size) {
#pragma unroll
              for (int m = 0; m < DS; ++m)
                w |= rerank(stab + (size_t)m * W, rb[m * (kBG * 32) + j * 32 + lane]) << (8 * m);
            }
            const uint32_t x = transpose32(w, lane, keep);
            if (lane < 8 * DS) pl_st[j * (DS * 8) + lane] = x;
          }
        }
        if (pair_or(pair_bar, !ok)) {
          // a rank copy did not arrive in time: wait (bounded) for this
          // pair's copies still in flight, then stop
          if (tp == 0) {
            atomicOr(flags, ddks::kFlagTimeout);
            bk::wait(rbar + 8u * st, (jj >> 1) & 1u, bk::kDrainNs);
            if (i + kPairs < nb) bk::wait(rbar + 8u * (st ^ 1u), ((jj + 1) >> 1) & 1u, bk::kDrainNs);
          }
          aborted = true;
          break;
        }
        const uint4* P4 = reinterpret_cast<const uint4*>(pl_st);
        // G[o][m] = the group's points >= origin o in dimension m + 1
        auto compare = [&](int j, uint32_t (&G)[2][DS]) {
#pragma unroll
          for (int m = 0; m < DS; ++m) {
            const uint4 x0 = P4[(j * DS + m) * 2], x1 = P4[(j * DS + m) * 2 + 1];
            const uint32_t pl[kBits] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z};
#pragma unroll
            for (int o = 0; o < 2; ++o) {
              uint32_t r = pl[0] | ~s[o][m][0];
#pragma unroll
              for (int k = 1; k < kBits; ++k) r = cmp_step(s[o][m][k], pl[k], r);
              G[o][m] = r;
            }
          }
        };
        auto accumulate = [&](const uint32_t (&G)[2][DS]) {
#pragma unroll
          for (int o = 0; o < 2; ++o) {
            uint32_t M[NS + 1];
            M[0] = 0xFFFFFFFFu;
#pragma unroll
            for (int S = 1; S <= NS; ++S) {
              const uint32_t gdim = (S & 1) ? G[o][0] : ((S & 2) ? G[o][DS > 1 ? 1 : 0] : G[o][DS > 2 ? 2 : 0]);
              M[S] = M[S & (S - 1)] & gdim;
            }
#pragma unroll
            for (int S = 1; S <= NS; ++S) acc_r[o][S - 1] += (uint32_t)__popc(M[S]);
          }
        };
        if (all_crossed || g0 + kBG <= (int64_t)wlo) {
          // no split in this batch for any origin of the block
#pragma unroll UNR
          for (int j = 0; j < kBG; ++j) {
            uint32_t G[2][DS];
            compare(j, G);
            accumulate(G);
          }
        } else {
          for (int j = 0; j < n; ++j) {
            const uint32_t gl = (uint32_t)(g0 + j);
            uint32_t G[2][DS];
            compare(j, G);
            if (!all_crossed && gl >= wlo) {
              if (gl >= whi) {
                // past every split of the block: the rest is phase B
#pragma unroll
                for (int o = 0; o < 2; ++o)
                  if (!crossed[o]) {
#pragma unroll
                    for (int S = 0; S < NS; ++S) snapshot(o, S, acc_r[o][S]);
                    crossed[o] = true;
                  }
                all_crossed = true;
              } else {
                // a group that may hold some origin's split
#pragma unroll
                for (int o = 0; o < 2; ++o) {
                  const uint32_t sp = o == 0 ? sp0 : sp1, pos0 = gl * 32u;
                  if (!crossed[o] && sp < pos0 + 32u) {
                    const uint32_t pam = sp > pos0 ? (1u << (sp - pos0)) - 1u : 0u;  // phase-A points
#pragma unroll
                    for (int S = 1; S <= NS; ++S) {
                      uint32_t Ms = pam;
#pragma unroll
                      for (int m = 0; m < DS; ++m)
                        if ((S >> m) & 1) Ms &= G[o][m];
                      snapshot(o, S - 1, acc_r[o][S - 1] + (uint32_t)__popc(Ms));
                    }
                    crossed[o] = true;
                  }
                }
              }
            }
            accumulate(G);
          }
        }
      }
      if (aborted) s_abort = 1u;
      // the pairs' counters, summed in shared memory: acc_r is phase A for
      // an origin whose split this pair never reached, else phase B
#pragma unroll
      for (int o = 0; o < 2; ++o) {
        if (!real[o]) continue;
        const int slot = tp + 64 * o;
#pragma unroll
        for (int S = 0; S < NS; ++S)
          if (acc_r[o][S]) atomicAdd(&acc[(slot * 2 + (crossed[o] ? 1 : 0)) * NS + S], acc_r[o][S]);
      }
      __syncthreads();
      const bool abort = s_abort != 0u;
      if (!abort) {
        // into the global counters [q][sample][phase][S]; acc is left zeroed
        for (int idx = tid; idx < kOC * 2 * NS; idx += kFThreads) {
          const uint32_t v = acc[idx];
          if (!v) continue;
          acc[idx] = 0u;
          const int slot = idx / (2 * NS), ph = (idx / NS) & 1, S = idx % NS;
          const int64_t q = (int64_t)blk * kOB + slot;
          atomicAdd(&gcnt[q * kCnt + (smp * 2 + ph) * NS + S], v);
        }
      }
      __threadfence();
      __syncthreads();
      if (abort) return;
      // ticket: the CTA that completes the block's GP + GT groups finishes it
      if (tid == 0) {
        const unsigned add = (unsigned)(pb - pa);
        s_last = (atomicAdd(&fin.done[blk], add) + add == (unsigned)per) ? 1u : 0u;
      }
      __syncthreads();
      if (s_last) {
        __threadfence();
        finish_block<DS, true>(gcnt, meta, no, NP, NT, blk, fin, &s_ticket);
      }
    }
    u = bend;
  }
}

// Kernel shapes of the fused count (plan.fused): warp pairs per CTA,
// resident CTAs per SM the registers are budgeted for, group-loop unroll.
//   1: 4 pairs, 2 CTAs/SM (128 registers), no unroll
//   2: 4 pairs, 1 CTA/SM (up to 255 registers), 16 groups unrolled
//   3: 2 pairs, 3 CTAs/SM (up to 170 registers), 4 groups unrolled
template <int DS>
size_t fused_smem(int variant, int W) {
  return variant == 3 ? FusedSmem<DS, 2>::total(W) : FusedSmem<DS, 4>::total(W);
}

size_t fused_smem_ds(int ds, int variant, int W) {
  return ds == 1 ? fused_smem<1>(variant, W) : ds == 2 ? fused_smem<2>(variant, W) : fused_smem<3>(variant, W);
}

}  // namespace

bool ddks_fused_supported(int ds, int64_t N, int variant) {
  if (ds < 1 || ds > 3 || N < 2 || N > (1 << 24) || variant < 1 || variant > 3) return false;
  const int W = (int)((N + 31) / 32);
  const size_t prep = (size_t)ds * W * 5;
  return fused_smem_ds(ds, variant, W) <= 220u * 1024u && prep <= 220u * 1024u;
}

size_t ddks_fused_scratch_bytes(int ds, int64_t N, int64_t blocks) {
  const int W = (int)((N + 31) / 32);
  return (size_t)blocks * tab_stride(ds, W) * 8 + (size_t)blocks * ds * kOC + 16;
}

cudaError_t ddks_fused_count(ddks_ctx* ctx, int ds, int variant, const uint32_t* rankL, const uint32_t* orank,
                             const void* meta, int64_t no, int64_t N, int64_t NP, int64_t NT, int64_t NPpad,
                             int64_t Lrow, uint32_t* gcnt, unsigned* done, unsigned long long* packed, uint64_t* best,
                             int32_t* bestj, int64_t ob, unsigned long long* out3, unsigned* flags,
                             void* scratch, cudaStream_t st, int* launches) {
  if (!ddks_fused_supported(ds, N, variant)) return cudaErrorInvalidValue;
  const int W = (int)((N + 31) / 32);
  const int64_t blocks = (no + kOB - 1) / kOB;
  uint2* tab = reinterpret_cast<uint2*>(scratch);
  uint8_t* oval = reinterpret_cast<uint8_t*>(tab + blocks * tab_stride(ds, W));
  const int GP = (int)((NP + 31) / 32), GT = (int)((NT + 31) / 32);
  const int64_t units = blocks * (GP + GT);
  const size_t prep_smem = (size_t)ds * W * 5;
  const size_t smem = fused_smem_ds(ds, variant, W);
  Final fin{out3, done, packed, best, bestj, ob, (int)blocks};
  const OriginMeta* mt = reinterpret_cast<const OriginMeta*>(meta);
  auto go = [&](auto prep, auto kern, int threads) -> cudaError_t {
    cudaError_t e = ddks_smem_attr(prep, (int)prep_smem);
    if (e != cudaSuccess) return e;
    prep<<<(unsigned)blocks, kPrepThreads, prep_smem, st>>>(orank, no, W, tab, oval);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    e = ddks_smem_attr(kern, (int)smem);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, smem);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    // persistent: one wave of resident CTAs, each with at least a few batches
    int64_t grid = (int64_t)ctx->num_sms * occ;
    const int64_t min_units = 4 * kBG;
    if (grid * min_units > units) grid = (units + min_units - 1) / min_units;
    if (grid < 1) grid = 1;
    kern<<<(unsigned)grid, threads, smem, st>>>(rankL, tab, oval, mt, no, NP, NT, NPpad, Lrow, W, GP, GT, units, gcnt,
                                               flags, fin, ctx->dev_wait_ns);
    *launches += 2;
    return cudaGetLastError();
  };
  auto pick = [&](auto prep, auto k1, auto k2, auto k3) -> cudaError_t {
    return variant == 1 ? go(prep, k1, 256) : variant == 2 ? go(prep, k2, 256) : go(prep, k3, 128);
  };
  if (ds == 1)
    return pick(k_fused_tables<1>, k_fused<1, 4, 2, 1>, k_fused<1, 4, 1, 16>, k_fused<1, 2, 3, 4>);
  if (ds == 2)
    return pick(k_fused_tables<2>, k_fused<2, 4, 2, 1>, k_fused<2, 4, 1, 16>, k_fused<2, 2, 3, 4>);
  return pick(k_fused_tables<3>, k_fused<3, 4, 2, 1>, k_fused<3, 4, 1, 16>, k_fused<3, 2, 3, 4>);
}
