// count_lane.cu -- orthant counts with lane-private shared-memory histograms.
//
// One thread per origin o (Sec. 2.1: every pooled point is a test point).  The
// CTA stages tiles of the pooled sample's ranks in shared memory; every thread
// walks each tile, forms the d-bit code  c = sum_m [r_m(x) >= r_m(o)] 2^m
// (Eq. g; bit m set on the ">=" side), and increments bin c of its own column
// of a [2^d][threads] histogram (bank = lane, so increments never conflict).
// A P point adds 1, a T point adds 1 << 16 to the packed (cP | cT << 16) bin;
// when NP or NT exceed 65535 two separate 32-bit histograms are used.  After
// the last tile each thread scans its 2^d bins for the largest
// |cP*NT - cT*NP| (Eq. d1 with Eq. abs_difference) and the lowest orthant
// reaching it.
#include "ddks_internal.cuh"

namespace {

constexpr int kTile = 1024;

template <int D, bool WIDE>
__global__ void k_lane(const uint32_t* __restrict__ rank, int64_t N, int64_t NP, int64_t NT,
                       int64_t o_begin, int64_t o_end, uint64_t* __restrict__ best,
                       int32_t* __restrict__ bestj) {
  extern __shared__ uint32_t sm[];
  constexpr int NB = 1 << D;
  const int T = blockDim.x;
  const int tid = threadIdx.x;
  uint32_t* histP = sm;                              // [NB][T]
  uint32_t* histT = WIDE ? sm + NB * T : sm;         // [NB][T] when WIDE
  uint32_t* tile = sm + (WIDE ? 2 : 1) * NB * T;     // [D][kTile]
  const int64_t k = o_begin + (int64_t)blockIdx.x * T + tid;
  const bool active = k < o_end;
  uint32_t o[D];
#pragma unroll
  for (int m = 0; m < D; ++m) o[m] = active ? rank[(int64_t)m * N + k] : 0u;
  for (int j = 0; j < NB; ++j) {
    histP[j * T + tid] = 0;
    if (WIDE) histT[j * T + tid] = 0;
  }
  for (int64_t base = 0; base < N; base += kTile) {
    const int cnt = (int)((N - base) < kTile ? (N - base) : kTile);
    __syncthreads();
    for (int e = tid; e < D * cnt; e += T) {
      const int m = e / cnt;
      const int j = e - m * cnt;
      tile[m * kTile + j] = rank[(int64_t)m * N + base + j];
    }
    __syncthreads();
    int pend = (int)(NP - base);
    pend = pend < 0 ? 0 : (pend > cnt ? cnt : pend);
#pragma unroll 4
    for (int j = 0; j < pend; ++j) {
      uint32_t c = 0;
#pragma unroll
      for (int m = 0; m < D; ++m) c |= (uint32_t)(tile[m * kTile + j] >= o[m]) << m;
      atomicAdd(&histP[c * T + tid], 1u);
    }
#pragma unroll 4
    for (int j = pend; j < cnt; ++j) {
      uint32_t c = 0;
#pragma unroll
      for (int m = 0; m < D; ++m) c |= (uint32_t)(tile[m * kTile + j] >= o[m]) << m;
      if (WIDE) atomicAdd(&histT[c * T + tid], 1u);
      else atomicAdd(&histP[c * T + tid], 1u << 16);
    }
  }
  if (!active) return;
  uint64_t bv = 0;
  int bj = 0;
  for (int j = 0; j < NB; ++j) {
    uint64_t a, b;
    if (WIDE) {
      a = histP[j * T + tid];
      b = histT[j * T + tid];
    } else {
      const uint32_t v = histP[j * T + tid];
      a = v & 0xFFFFu;
      b = v >> 16;
    }
    const uint64_t num = ddks::numer(a, b, (uint64_t)NP, (uint64_t)NT);
    if (num > bv) { bv = num; bj = j; }
  }
  best[k - o_begin] = bv;
  bestj[k - o_begin] = bj;
}

size_t lane_smem(int d, bool wide, int threads) {
  return (size_t)(wide ? 2 : 1) * (size_t)(1u << d) * threads * 4u + (size_t)d * kTile * 4u;
}

template <int D, bool WIDE>
cudaError_t launch_t(const uint32_t* rank, int64_t N, int64_t NP, int64_t NT, int64_t ob,
                     int64_t oe, uint64_t* best, int32_t* bestj, cudaStream_t st, int threads) {
  const size_t sm = lane_smem(D, WIDE, threads);
  cudaError_t e = cudaFuncSetAttribute(k_lane<D, WIDE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sm);
  if (e != cudaSuccess) return e;
  const int64_t no = oe - ob;
  const unsigned grid = (unsigned)((no + threads - 1) / threads);
  if (grid == 0) return cudaSuccess;
  k_lane<D, WIDE><<<grid, threads, sm, st>>>(rank, N, NP, NT, ob, oe, best, bestj);
  return cudaGetLastError();
}

template <bool WIDE>
cudaError_t launch_w(int d, const uint32_t* rank, int64_t N, int64_t NP, int64_t NT, int64_t ob,
                     int64_t oe, uint64_t* best, int32_t* bestj, cudaStream_t st, int threads) {
  switch (d) {
    case 1: return launch_t<1, WIDE>(rank, N, NP, NT, ob, oe, best, bestj, st, threads);
    case 2: return launch_t<2, WIDE>(rank, N, NP, NT, ob, oe, best, bestj, st, threads);
    case 3: return launch_t<3, WIDE>(rank, N, NP, NT, ob, oe, best, bestj, st, threads);
    case 4: return launch_t<4, WIDE>(rank, N, NP, NT, ob, oe, best, bestj, st, threads);
    case 5: return launch_t<5, WIDE>(rank, N, NP, NT, ob, oe, best, bestj, st, threads);
    case 6: return launch_t<6, WIDE>(rank, N, NP, NT, ob, oe, best, bestj, st, threads);
    case 7: return launch_t<7, WIDE>(rank, N, NP, NT, ob, oe, best, bestj, st, threads);
    case 8: return launch_t<8, WIDE>(rank, N, NP, NT, ob, oe, best, bestj, st, threads);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

bool ddks_lane_supported(int d, int64_t NP, int64_t NT, int threads) {
  if (d < 1 || d > 8 || threads < 32 || threads > 1024 || (threads & 31)) return false;
  const bool wide = NP > 65535 || NT > 65535;
  return lane_smem(d, wide, threads) <= 200u * 1024u;
}

cudaError_t ddks_launch_lane(const uint32_t* rank, int64_t N, int64_t NP, int64_t NT, int d,
                             int64_t o_begin, int64_t o_end, uint64_t* best, int32_t* bestj,
                             cudaStream_t st, int threads) {
  if (!ddks_lane_supported(d, NP, NT, threads)) return cudaErrorInvalidValue;
  const bool wide = NP > 65535 || NT > 65535;
  return wide ? launch_w<true>(d, rank, N, NP, NT, o_begin, o_end, best, bestj, st, threads)
              : launch_w<false>(d, rank, N, NP, NT, o_begin, o_end, best, bestj, st, threads);
}
