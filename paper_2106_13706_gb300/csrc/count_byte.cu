// count_byte.cu -- orthant counts for larger d (5..16) on byte re-ranks, four
// dimensions per 32-bit compare.
//
// The statistic is that of every path (Sec. 2.1, Eq. ddks_tensor_definition;
// the ">=" of Sec. 2.2.1, Eq. g; the histogram of codes of Eq. membership and
// max |cP*NT - cT*NP| of Eq. d1 with the normalisation of Eq. abs_difference),
// with one shared-memory histogram of 2^d bins per origin as in the warp path.
// What changes is the compare:
//
// 1. Re-ranking.  Origins form blocks of 127 (consecutive pooled indices).
//    Per block and dimension every point is re-ranked as x' = #{distinct
//    values of the block's origins <= x} (<= 127), which keeps x >= o <=>
//    x' >= o' for every origin o of the block.  A pack kernel computes x' from
//    a bitmap of the block's origin ranks with per-word prefix counts and
//    stores it as a byte with bit 7 set; four dimensions share one word.
// 2. Compare.  For a point word x and an origin word o (bytes o' <= 127),
//    x - o leaves in bit 7 of each byte [x' >= o'] (each byte of x - o lies in
//    [1, 255]: no byte borrows from the next), so one subtract compares four
//    dimensions; (v & 0x80808080) * 0x00204081 gathers the four bits into
//    bits 28..31.  Dimensions past d are bytes 0x80 against 0 and fall outside
//    the code's mask.
// 3. Counting.  A CTA takes rounds of H origins of one block; each thread
//    keeps its points' words in registers and, origin by origin, adds 1 (P) or
//    1 << 16 (T) to bin code of that origin's histogram (N <= 65535 keeps both
//    counts in one 32-bit bin).  Then the CTA scans the H histograms for each
//    origin's largest numerator and lowest orthant.
#include "ddks_host.h"
#include "ddks_internal.cuh"

namespace {

constexpr int kBO = 127;         // origins per block (x' <= 127 fits 7 bits)
constexpr int kBThreads = 768;   // threads per CTA of the count kernel
constexpr int kBPrep = 256;      // threads per CTA of the pack kernel
constexpr int kMaxP = 12;        // points per thread held in registers per pass

// Grid (blocks, d): CTA (b, m) re-ranks every point in dimension m against
// block b's origins and writes byte m % 4 of X8[(b * NQ + m / 4) * N + i]
// (x' | 0x80) and of OW[(b * kBO + slot) * NQ + m / 4] (o').  X8 and OW were
// filled with 0x80 / 0 bytes first, so dimensions past d always compare >=.
__global__ void __launch_bounds__(kBPrep)
k_byte_pack(const uint32_t* __restrict__ rank, int64_t N, int d, int NQ, int64_t ob, int64_t no, int W,
            uint8_t* __restrict__ X8, uint8_t* __restrict__ OW) {
  extern __shared__ __align__(16) uint32_t bsm[];
  uint32_t* bits = bsm;                                   // [W]
  uint8_t* pf = reinterpret_cast<uint8_t*>(bsm + W);      // [W] prefix counts
  __shared__ uint32_t tmp[kBPrep / 32];
  const int blk = blockIdx.x, m = blockIdx.y, tid = threadIdx.x;
  const uint32_t* R = rank + (int64_t)m * N;
  for (int i = tid; i < W; i += kBPrep) bits[i] = 0u;
  __syncthreads();
  for (int s = tid; s < kBO; s += kBPrep) {
    const int64_t q = (int64_t)blk * kBO + s;
    if (q < no) {
      const uint32_t r = R[ob + q];
      atomicOr(&bits[r >> 5], 1u << (r & 31));
    }
  }
  __syncthreads();
  // exclusive prefix counts of the bitmap words (at most 127 set bits: bytes)
  const int seg = (W + kBPrep - 1) / kBPrep;
  const int wa = tid * seg < W ? tid * seg : W;
  const int wb = wa + seg < W ? wa + seg : W;
  uint32_t c = 0;
  for (int w = wa; w < wb; ++w) c += (uint32_t)__popc(bits[w]);
  {
    const int lane = tid & 31, warp = tid >> 5;
    uint32_t incl = c;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const uint32_t x = __shfl_up_sync(0xffffffffu, incl, off);
      if (lane >= off) incl += x;
    }
    if (lane == 31) tmp[warp] = incl;
    __syncthreads();
    uint32_t carry = 0;
    for (int q = 0; q < warp; ++q) carry += tmp[q];
    uint32_t run = carry + incl - c;
    for (int w = wa; w < wb; ++w) {
      pf[w] = (uint8_t)run;
      run += (uint32_t)__popc(bits[w]);
    }
  }
  __syncthreads();
  const int byte = m & 3, word = m >> 2;
  uint8_t* xo = X8 + ((int64_t)blk * NQ + word) * N * 4 + byte;
  for (int64_t i = tid; i < N; i += kBPrep) {
    const uint32_t r = R[i];
    const uint32_t v = pf[r >> 5] + (uint32_t)__popc(bits[r >> 5] << (31 - (r & 31)));
    xo[i * 4] = (uint8_t)(v | 0x80u);
  }
  for (int s = tid; s < kBO; s += kBPrep) {
    const int64_t q = (int64_t)blk * kBO + s;
    if (q < no) {
      const uint32_t r = R[ob + q];
      const uint32_t v = pf[r >> 5] + (uint32_t)__popc(bits[r >> 5] << (31 - (r & 31)));
      OW[(((int64_t)blk * kBO + s) * NQ + word) * 4 + byte] = (uint8_t)v;
    }
  }
}

// The code of one point against one origin: per word one subtract, the four
// byte sign bits gathered into bits 28..31 by one multiply.
template <int NQ>
DDKS_DEV uint32_t byte_code(const uint32_t (&x)[NQ], const uint32_t (&o)[NQ], uint32_t dmask) {
  uint32_t c = 0;
#pragma unroll
  for (int w = 0; w < NQ; ++w) c |= (((x[w] - o[w]) & 0x80808080u) * 0x00204081u) >> 28 << (4 * w);
  return c & dmask;
}

// Work items (block, round): round r of block b takes origin slots
// [r * H, r * H + H) of the block; CTAs pull items from a device counter.
// Shared memory: hist [H][nb] (P count | T count << 16, cleared after each
// scan), ow [H][NQ] origin words, part [warps][2] partial maxima.
template <int NQ>
__global__ void __launch_bounds__(kBThreads)
k_byte(const uint32_t* __restrict__ X8, const uint32_t* __restrict__ OW, int N, int NP, int NT, int d, int H,
       int64_t no, int nblocks, int rpb, unsigned long long* __restrict__ work, uint64_t* __restrict__ best,
       int32_t* __restrict__ bestj) {
  extern __shared__ __align__(16) uint32_t csm[];
  const int nb = 1 << d;
  const uint32_t dmask = (uint32_t)nb - 1u;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  constexpr int W = kBThreads / 32;
  uint32_t* hist = csm;                                  // [H][nb]
  uint32_t* ow = csm + (size_t)H * nb;                   // [H][NQ]
  unsigned long long* part = reinterpret_cast<unsigned long long*>(
      (reinterpret_cast<uintptr_t>(ow + (size_t)H * NQ) + 7) & ~(uintptr_t)7);  // [W]
  __shared__ long long item_s;
  for (int j = tid; j < H * nb; j += kBThreads) hist[j] = 0u;
  for (;;) {
    __syncthreads();  // histograms cleared, the previous round's partials consumed
    if (tid == 0) item_s = (long long)atomicAdd(work, 1ull);
    __syncthreads();
    const long long item = item_s;
    if (item >= (long long)nblocks * rpb) break;
    const int blk = (int)(item / rpb), first = (int)(item % rpb) * H;
    const int64_t q0 = (int64_t)blk * kBO + first;  // first origin (index into [0, no))
    int nh = kBO - first < H ? kBO - first : H;
    if (no - q0 < nh) nh = (int)(no - q0 > 0 ? no - q0 : 0);
    if (nh <= 0) continue;  // CTA-uniform
    for (int i = tid; i < nh * NQ; i += kBThreads) ow[i] = OW[(q0 + i / NQ) * NQ + i % NQ];
    __syncthreads();
    const uint32_t* X = X8 + (size_t)blk * NQ * N;
    for (int base = 0; base < N; base += kBThreads * kMaxP) {
      uint32_t x[kMaxP][NQ];
      uint32_t inc[kMaxP];
#pragma unroll
      for (int pt = 0; pt < kMaxP; ++pt) {
        const int p = base + pt * kBThreads + tid;
        inc[pt] = p < N ? (p < NP ? 1u : 65536u) : 0u;
#pragma unroll
        for (int w = 0; w < NQ; ++w) x[pt][w] = p < N ? __ldg(&X[(size_t)w * N + p]) : 0u;
      }
      for (int hh = 0; hh < nh; ++hh) {
        uint32_t o[NQ];
#pragma unroll
        for (int w = 0; w < NQ; ++w) o[w] = ow[hh * NQ + w];
        uint32_t* h = hist + (size_t)hh * nb;
#pragma unroll
        for (int pt = 0; pt < kMaxP; ++pt)
          if (inc[pt]) atomicAdd(&h[byte_code<NQ>(x[pt], o, dmask)], inc[pt]);
      }
    }
    __syncthreads();
    // scan: G warps per origin, each clears the bins it reads
    const int G = W / nh;  // >= 1: nh <= H <= W
    const int hsel = warp / G, g = warp - hsel * G;
    if (hsel < nh) {
      uint64_t bv = 0;
      int bj = 0;
      uint32_t* h = hist + (size_t)hsel * nb;
      for (int j = 32 * g + lane; j < nb; j += 32 * G) {
        const uint32_t v = h[j];
        h[j] = 0u;
        const uint64_t num = ddks::numer(v & 0xFFFFu, v >> 16, (uint64_t)NP, (uint64_t)NT);
        if (num > bv) { bv = num; bj = j; }
      }
      for (int off = 16; off > 0; off >>= 1) {
        const uint64_t v2 = __shfl_down_sync(0xffffffffu, bv, off);
        const int j2 = __shfl_down_sync(0xffffffffu, bj, off);
        if (v2 > bv || (v2 == bv && j2 < bj)) { bv = v2; bj = j2; }
      }
      if (lane == 0) part[warp] = (bv << 24) | (unsigned long long)(uint32_t)bj;  // numerators < 2^32, bins < 2^16
    }
    __syncthreads();
    if (hsel < nh && g == 0 && lane == 0) {
      unsigned long long bp = part[warp];
      for (int k = 1; k < G; ++k) {
        const unsigned long long v2 = part[warp + k];
        // larger numerator first, then the lower orthant
        if ((v2 >> 24) > (bp >> 24) || ((v2 >> 24) == (bp >> 24) && (v2 & 0xFFFFFFu) < (bp & 0xFFFFFFu))) bp = v2;
      }
      const uint64_t bv = bp >> 24;
      best[q0 + hsel] = bv;
      bestj[q0 + hsel] = bv ? (int32_t)(bp & 0xFFFFFFu) : 0;
    }
  }
}

size_t byte_smem(int d, int NQ, int H) {
  return (size_t)H * ((size_t)(1u << d) + NQ) * 4 + 16 + (size_t)(kBThreads / 32) * 8;
}

}  // namespace

bool ddks_byte_supported(int d, int64_t NP, int64_t NT) {
  const int64_t N = NP + NT;
  if (d < 2 || d > 15 || N < 2 || N > 32768) return false;
  return byte_smem(d, (d + 3) / 4, 1) <= 200u * 1024u;
}

cudaError_t ddks_launch_byte(ddks_ctx* ctx, const uint32_t* rank, int64_t N, int64_t NP, int64_t NT, int d,
                             int64_t ob, int64_t oe, uint64_t* best, int32_t* bestj, cudaStream_t st,
                             int* launches) {
  if (!ddks_byte_supported(d, NP, NT)) return cudaErrorInvalidValue;
  const int64_t no = oe - ob;
  if (no <= 0) return cudaSuccess;
  const int NQ = (d + 3) / 4;
  const int W = (int)((N + 31) / 32);
  const int64_t blocks = (no + kBO - 1) / kBO;
  const size_t x_words = (size_t)blocks * NQ * N, o_words = (size_t)blocks * kBO * NQ;
  if (ctx->warp_words.reserve(ctx, (x_words + o_words) * 4 + 64)) return cudaErrorMemoryAllocation;
  uint32_t* X8 = (uint32_t*)ctx->warp_words.ptr;
  uint32_t* OW = X8 + x_words;
  unsigned long long* work =
      reinterpret_cast<unsigned long long*>((reinterpret_cast<uintptr_t>(OW + o_words) + 7) & ~(uintptr_t)7);
  cudaError_t e = cudaMemsetAsync(X8, 0x80, x_words * 4, st);  // dimensions past d: always >=
  if (e == cudaSuccess) e = cudaMemsetAsync(OW, 0, o_words * 4, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(work, 0, 8, st);
  if (e != cudaSuccess) return e;
  const size_t psmem = (size_t)W * 5;
  e = ddks_smem_attr(k_byte_pack, (int)psmem);
  if (e != cudaSuccess) return e;
  k_byte_pack<<<dim3((unsigned)blocks, (unsigned)d), kBPrep, psmem, st>>>(rank, N, d, NQ, ob, no, W, (uint8_t*)X8,
                                                                         (uint8_t*)OW);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // H histograms of 2^d bins in up to ~200 KB, at most one per warp
  int H = (int)((200u * 1024u - 16 - (kBThreads / 32) * 8) / (((size_t)(1u << d) + NQ) * 4));
  if (H > kBThreads / 32) H = kBThreads / 32;
  if (H > kBO) H = kBO;
  if (H < 1) H = 1;
  const int rpb = (kBO + H - 1) / H;
  const size_t smem = byte_smem(d, NQ, H);
  auto go = [&](auto kern) -> cudaError_t {
    cudaError_t r = ddks_smem_attr(kern, (int)smem);
    if (r != cudaSuccess) return r;
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBThreads, smem);
    if (per_sm < 1) per_sm = 1;
    int64_t grid = (int64_t)ctx->num_sms * per_sm;
    if (grid > blocks * rpb) grid = blocks * rpb;
    kern<<<(unsigned)grid, kBThreads, smem, st>>>(X8, OW, (int)N, (int)NP, (int)NT, d, H, no, (int)blocks, rpb,
                                                  work, best, bestj);
    return cudaGetLastError();
  };
  switch (NQ) {
    case 1: e = go(k_byte<1>); break;
    case 2: e = go(k_byte<2>); break;
    case 3: e = go(k_byte<3>); break;
    default: e = go(k_byte<4>); break;
  }
  if (launches) *launches += 2;
  return e;
}
