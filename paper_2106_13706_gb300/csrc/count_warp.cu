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
#include "ddks_internal.cuh"

namespace {

constexpr int kTile = 512;

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
    e = cudaFuncSetAttribute(k_warp<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_warp<true><<<grid, warps * 32, sm, st>>>(rank, N, NP, NT, d, o_begin, o_end, best, bestj);
  } else {
    e = cudaFuncSetAttribute(k_warp<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_warp<false><<<grid, warps * 32, sm, st>>>(rank, N, NP, NT, d, o_begin, o_end, best, bestj);
  }
  return cudaGetLastError();
}
