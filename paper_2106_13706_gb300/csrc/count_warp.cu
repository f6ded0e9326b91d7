// count_warp.cu -- orthant counts with one shared-memory histogram per warp.
//
// For larger d (2^d bins) a lane-private histogram no longer fits, so each warp
// takes one origin o and its lanes split the pooled points: every lane forms
// the code c = sum_m [r_m(x) >= r_m(o)] 2^m (Sec. 2.2.1, Eq. g) of its points
// and adds 1 (P) or 1 << 16 (T) to bin c of the warp's histogram with a shared
// atomic; two 32-bit histograms are used when NP or NT exceed 65535.  The
// lanes then scan the 2^d bins for the largest |cP*NT - cT*NP| (Eq. d1) and
// the lowest orthant reaching it.  All warps of a CTA share the staged tiles
// of point ranks.
//
// For N <= 32767 (ranks below 2^15) the codes come from packed rank pairs
// instead (k_warp16): each point's ranks of dimensions 2w and 2w+1 sit in the
// two 16-bit halves of word w with bit 15 of each half set, so one 32-bit
// subtract of the origin's word leaves [x_2w >= o_2w] and [x_2w+1 >= o_2w+1]
// in bits 15 and 31 (a half never borrows from the other), and a shift and a
// mask move them into the code.  Warps take origins from a device counter, so
// the load stays even whatever the number of origins per CTA.
#include "ddks_host.h"
#include "ddks_internal.cuh"

namespace {

constexpr int kTile = 512;
constexpr int kW16Threads = 768;

template <bool WIDE>
__global__ void k_warp(const uint32_t* __restrict__ rank, int64_t N, int64_t NP, int64_t NT, int d,
                       int64_t o_begin, int64_t o_end, uint64_t* __restrict__ best,
                       int32_t* __restrict__ bestj) {
  extern __shared__ uint32_t sm[];
  const int nb = 1 << d;
  const int W = blockDim.x >> 5;
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  uint32_t* hist = sm + (size_t)warp * nb * (WIDE ? 2 : 1);
  uint32_t* tile = sm + (size_t)W * nb * (WIDE ? 2 : 1);   // [d][kTile]
  uint32_t* o = tile + (size_t)d * kTile + warp * ddks::kMaxD; // origin ranks per warp
  const int64_t k = o_begin + (int64_t)blockIdx.x * W + warp;
  const bool active = k < o_end;
  if (lane < d) o[lane] = active ? rank[(int64_t)lane * N + k] : 0u;
  for (int j = lane; j < nb * (WIDE ? 2 : 1); j += 32) hist[j] = 0;
  for (int64_t base = 0; base < N; base += kTile) {
    const int cnt = (int)((N - base) < kTile ? (N - base) : kTile);
    __syncthreads();
    for (int e = threadIdx.x; e < d * cnt; e += blockDim.x) {
      const int m = e / cnt;
      const int j = e - m * cnt;
      tile[m * kTile + j] = rank[(int64_t)m * N + base + j];
    }
    __syncthreads();
    if (active) {
      for (int j = lane; j < cnt; j += 32) {
        uint32_t c = 0;
        for (int m = 0; m < d; ++m) c |= (uint32_t)(tile[m * kTile + j] >= o[m]) << m;
        const bool isP = base + j < NP;
        if (WIDE) atomicAdd(&hist[isP ? c : nb + c], 1u);
        else atomicAdd(&hist[c], isP ? 1u : (1u << 16));
      }
    }
  }
  if (!active) return;
  __syncwarp();
  uint64_t bv = 0;
  int bj = 0;
  for (int j = lane; j < nb; j += 32) {
    uint64_t a, b;
    if (WIDE) {
      a = hist[j];
      b = hist[nb + j];
    } else {
      const uint32_t v = hist[j];
      a = v & 0xFFFFu;
      b = v >> 16;
    }
    const uint64_t num = ddks::numer(a, b, (uint64_t)NP, (uint64_t)NT);
    if (num > bv) { bv = num; bj = j; }
  }
  // warp arg-max: larger value first, then lower orthant
  for (int off = 16; off > 0; off >>= 1) {
    const uint64_t v2 = __shfl_down_sync(0xffffffffu, bv, off);
    const int j2 = __shfl_down_sync(0xffffffffu, bj, off);
    if (v2 > bv || (v2 == bv && j2 < bj)) { bv = v2; bj = j2; }
  }
  if (lane == 0) {
    best[k - o_begin] = bv;
    bestj[k - o_begin] = bv ? bj : 0;
  }
}

// X[w][i]: ranks of dimensions 2w (low half) and 2w+1 (high half) of pooled
// point i with bit 15 of each half set (rank of dimension d taken as 0)
__global__ void k_pair_pack(const uint32_t* __restrict__ rank, int64_t N, int d, int nw,
                            uint32_t* __restrict__ X) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)nw * N;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int w = (int)(e / N);
    const int64_t i = e - (int64_t)w * N;
    const uint32_t lo = rank[(int64_t)(2 * w) * N + i];
    const uint32_t hi = 2 * w + 1 < d ? rank[(int64_t)(2 * w + 1) * N + i] : 0u;
    X[e] = (lo | 0x8000u) | ((hi | 0x8000u) << 16);
  }
}

// the code of one point: bits 15 and 31 of each word's difference, moved to
// code bits 2w and 2w+1
template <int NW>
DDKS_DEV uint32_t pair_code(const uint32_t (&x)[NW], const uint32_t (&on)[NW], uint32_t dmask) {
  uint32_t c = 0;
#pragma unroll
  for (int w = 0; w < NW; ++w) c |= ((x[w] + on[w]) & 0x80008000u) >> (15 - 2 * w);
  return (c | (c >> 15)) & dmask;
}

// One CTA holds H histograms (one origin each).  Each round the CTA takes H
// origins from the device counter and puts their negated pair words in shared
// memory; every thread then takes points, loads a point's words once and adds
// it to all H histograms (the origin words are the same for the whole warp,
// so they are broadcast loads).  Then G = warps / H warps per origin scan
// (and clear) its bins, and the partial maxima are combined.  Indices fit 32
// bits here (N <= 32767); so do the numerators |cP*NT - cT*NP| < 2^30.
template <int NW>
__global__ void __launch_bounds__(kW16Threads)
k_warp16(const uint32_t* __restrict__ X, int N, int NP, int NT, int d, int H, int64_t o_begin,
         int64_t o_end, unsigned long long* __restrict__ work, uint64_t* __restrict__ best,
         int32_t* __restrict__ bestj) {
  extern __shared__ __align__(16) uint32_t sm[];
  const int nb = 1 << d;
  const uint32_t dmask = (uint32_t)nb - 1u;
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int W = blockDim.x >> 5;
  uint32_t* hist = sm;                                  // [H][nb]: cP low half, cT high half
  uint32_t* onw = sm + (((size_t)H * nb + 3) & ~(size_t)3);  // [H][8] negated origin words (16-byte aligned)
  uint32_t* part = onw + (size_t)H * 8;                 // [W][2] partial (value, bin)
  __shared__ unsigned long long round_base;
  for (int j = threadIdx.x; j < H * nb; j += blockDim.x) hist[j] = 0;
  for (;;) {
    __syncthreads();  // histograms cleared, previous round's partials consumed
    if (threadIdx.x == 0) round_base = atomicAdd(work, (unsigned long long)H);
    __syncthreads();
    const int64_t first = o_begin + (int64_t)round_base;
    if (first >= o_end) break;
    const int nh = (int)((o_end - first) < H ? (o_end - first) : H);
    for (int i = threadIdx.x; i < nh * 8; i += blockDim.x) {
      const int hh = i >> 3, w = i & 7;
      onw[i] = w < NW ? 0u - (X[w * N + (int)(first + hh)] & 0x7FFF7FFFu) : 0u;
    }
    __syncthreads();
    for (int p = threadIdx.x; p < N; p += blockDim.x) {
      uint32_t x[NW];
#pragma unroll
      for (int w = 0; w < NW; ++w) x[w] = __ldg(&X[w * N + p]);
      const uint32_t inc = p < NP ? 1u : 65536u;
      for (int hh = 0; hh < nh; ++hh) {
        // the origin's words: two vector broadcast loads
        const uint4 a = *reinterpret_cast<const uint4*>(onw + hh * 8);
        const uint4 b = *reinterpret_cast<const uint4*>(onw + hh * 8 + 4);
        const uint32_t all[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
        uint32_t on[NW];
#pragma unroll
        for (int w = 0; w < NW; ++w) on[w] = all[w];
        atomicAdd(&hist[hh * nb + pair_code<NW>(x, on, dmask)], inc);
      }
    }
    __syncthreads();
    const int G = W / nh;  // warps per origin in the scan (>= 1: nh <= H <= W)
    const int h = warp / G, g = warp - h * G;
    if (h < nh) {
      uint32_t bv = 0;
      int bj = 0;
      uint32_t* hh = hist + (size_t)h * nb;
      for (int j = 32 * g + lane; j < nb; j += 32 * G) {
        const uint32_t v = hh[j];
        hh[j] = 0;  // ready for the next round
        const int a = (int)(v & 0xFFFFu) * NT, b = (int)(v >> 16) * NP;
        const uint32_t num = (uint32_t)(a > b ? a - b : b - a);
        if (num > bv) { bv = num; bj = j; }
      }
      for (int off = 16; off > 0; off >>= 1) {
        const uint32_t v2 = __shfl_down_sync(0xffffffffu, bv, off);
        const int j2 = __shfl_down_sync(0xffffffffu, bj, off);
        if (v2 > bv || (v2 == bv && j2 < bj)) { bv = v2; bj = j2; }
      }
      if (lane == 0) {
        part[2 * warp] = bv;
        part[2 * warp + 1] = (uint32_t)bj;
      }
    }
    __syncthreads();
    if (h < nh && g == 0 && lane == 0) {
      uint32_t bv = part[2 * warp];
      int bj = (int)part[2 * warp + 1];
      for (int q = 1; q < G; ++q) {
        const uint32_t v2 = part[2 * (warp + q)];
        const int j2 = (int)part[2 * (warp + q) + 1];
        if (v2 > bv || (v2 == bv && j2 < bj)) { bv = v2; bj = j2; }
      }
      const int64_t k = first + h;
      best[k - o_begin] = bv;
      bestj[k - o_begin] = bv ? bj : 0;
    }
  }
}

size_t warp_smem(int d, bool wide, int warps) {
  return (size_t)warps * ((size_t)(1u << d) * (wide ? 2 : 1) + ddks::kMaxD) * 4u +
         (size_t)d * kTile * 4u;
}

}  // namespace

bool ddks_warp_supported(int d, int64_t NP, int64_t NT) {
  if (d < 1 || d > 13) return false;
  const bool wide = NP > 65535 || NT > 65535;
  return warp_smem(d, wide, 1) <= 200u * 1024u;
}

cudaError_t ddks_launch_warp(const uint32_t* rank, int64_t N, int64_t NP, int64_t NT, int d,
                             int64_t o_begin, int64_t o_end, uint64_t* best, int32_t* bestj,
                             cudaStream_t st, int warps) {
  if (!ddks_warp_supported(d, NP, NT)) return cudaErrorInvalidValue;
  const bool wide = NP > 65535 || NT > 65535;
  while (warps > 1 && warp_smem(d, wide, warps) > 200u * 1024u) --warps;
  if (warps < 1) warps = 1;
  const size_t sm = warp_smem(d, wide, warps);
  const int64_t no = o_end - o_begin;
  const unsigned grid = (unsigned)((no + warps - 1) / warps);
  if (grid == 0) return cudaSuccess;
  cudaError_t e;
  if (wide) {
    e = ddks_smem_attr(k_warp<true>, (int)sm);
    if (e != cudaSuccess) return e;
    k_warp<true><<<grid, warps * 32, sm, st>>>(rank, N, NP, NT, d, o_begin, o_end, best, bestj);
  } else {
    e = ddks_smem_attr(k_warp<false>, (int)sm);
    if (e != cudaSuccess) return e;
    k_warp<false><<<grid, warps * 32, sm, st>>>(rank, N, NP, NT, d, o_begin, o_end, best, bestj);
  }
  return cudaGetLastError();
}

bool ddks_warp16_supported(int d, int64_t NP, int64_t NT) {
  return d >= 1 && d <= 13 && NP + NT <= 32767;
}

// The packed-pair variant: needs the context for its scratch (pair words and
// the origin counter).
cudaError_t ddks_launch_warp16(ddks_ctx* ctx, const uint32_t* rank, int64_t N, int64_t NP, int64_t NT,
                               int d, int64_t o_begin, int64_t o_end, uint64_t* best, int32_t* bestj,
                               cudaStream_t st, int* launches) {
  if (!ddks_warp16_supported(d, NP, NT)) return cudaErrorInvalidValue;
  const int64_t no = o_end - o_begin;
  if (no <= 0) return cudaSuccess;
  const int nw = (d + 1) / 2;
  if (ctx->warp_words.reserve(ctx, (size_t)nw * N * 4 + 64)) return cudaErrorMemoryAllocation;
  uint32_t* X = (uint32_t*)ctx->warp_words.ptr;
  unsigned long long* work = reinterpret_cast<unsigned long long*>(
      (reinterpret_cast<uintptr_t>(X + (size_t)nw * N) + 7) & ~(uintptr_t)7);
  int64_t g = ((int64_t)nw * N + 255) / 256;
  if (g > 152 * 16) g = 152 * 16;
  k_pair_pack<<<(unsigned)g, 256, 0, st>>>(rank, N, d, nw, X);
  cudaError_t e = cudaMemsetAsync(work, 0, 8, st);
  if (e != cudaSuccess) return e;
  // H histograms of 2^d words in up to ~200 KB (at most one per warp)
  const size_t per_hist = (size_t)(1u << d) * 4u;
  int H = (int)((200u * 1024u) / per_hist);
  const int W = kW16Threads / 32;
  if (H > W) H = W;
  if (H < 1) H = 1;
  if ((int64_t)H > no) H = (int)no;
  const size_t sm = per_hist * H + 16 + (size_t)H * 8 * 4 + (size_t)W * 8;
  auto go = [&](auto kern) -> cudaError_t {
    cudaError_t r = ddks_smem_attr(kern, (int)sm);
    if (r != cudaSuccess) return r;
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kW16Threads, sm);
    if (per_sm < 1) per_sm = 1;
    int64_t grid = (int64_t)ctx->num_sms * per_sm;
    const int64_t need = (no + H - 1) / H;
    if (grid > need) grid = need;
    kern<<<(unsigned)grid, kW16Threads, sm, st>>>(X, (int)N, (int)NP, (int)NT, d, H, o_begin, o_end, work, best,
                                                  bestj);
    return cudaGetLastError();
  };
  switch (nw) {
    case 1: e = go(k_warp16<1>); break;
    case 2: e = go(k_warp16<2>); break;
    case 3: e = go(k_warp16<3>); break;
    case 4: e = go(k_warp16<4>); break;
    case 5: e = go(k_warp16<5>); break;
    case 6: e = go(k_warp16<6>); break;
    default: e = go(k_warp16<7>); break;
  }
  if (launches) *launches += 2;
  return e;
}
