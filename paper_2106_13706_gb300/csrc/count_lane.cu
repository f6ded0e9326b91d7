// count_lane.cu -- orthant counts with lane-private shared-memory histograms.
//
// Each origin o (Sec. 2.1: every pooled point is a test point) is served by S
// adjacent threads that split the pooled points between them.  The CTA stages
// tiles of the pooled sample's ranks in shared memory (point-major, padded to
// 4 or 8 words so a point is one or two 16-byte loads); every thread forms the
// d-bit code  c = sum_m [r_m(x) >= r_m(o)] 2^m  (Eq. g: bit m set on the ">="
// side) of its points and increments bin c of its own column of a
// [2^d][threads] histogram (bank = lane, so increments never conflict).  A P
// point adds 1, a T point 1 << 16 to the packed (cP | cT << 16) bin; when NP
// or NT exceed 65535 two 32-bit histograms are used.  At the end the S
// threads of an origin sum their columns, scan the 2^d bins for the largest
// |cP*NT - cT*NP| (Eq. d1 with Eq. abs_difference) and the lowest orthant
// reaching it, and combine their partial maxima with shuffles.
#include "ddks_internal.cuh"

namespace {

constexpr int kTile = 1024;

template <int D>
struct Pad { static constexpr int W = D <= 4 ? 4 : 8; };

template <int D, bool WIDE>
__global__ void __launch_bounds__(256)
k_lane(const uint32_t* __restrict__ rank, int64_t N, int64_t NP, int64_t NT, int64_t o_begin,
       int64_t o_end, int S, uint64_t* __restrict__ best, int32_t* __restrict__ bestj) {
  extern __shared__ __align__(16) uint32_t sm[];
  constexpr int NB = 1 << D;
  constexpr int W = Pad<D>::W;
  const int T = blockDim.x;
  const int tid = threadIdx.x;
  const int TO = T / S;                      // origins per CTA
  const int ol = tid / S, s = tid - ol * S;  // origin slot, slice
  uint32_t* histP = sm;                              // [NB][T]
  uint32_t* histT = WIDE ? sm + NB * T : sm;         // [NB][T] when WIDE
  uint32_t* tile = sm + (WIDE ? 2 : 1) * NB * T;     // [kTile][W]
  const int64_t k = o_begin + (int64_t)blockIdx.x * TO + ol;
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
      tile[j * W + m] = rank[(int64_t)m * N + base + j];
    }
    __syncthreads();
    int pend = (int)(NP - base);
    pend = pend < 0 ? 0 : (pend > cnt ? cnt : pend);
    for (int j = s; j < cnt; j += S) {
      uint32_t x[W];
      const uint4* src = reinterpret_cast<const uint4*>(tile + j * W);
      const uint4 a = src[0];
      x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w;
      if constexpr (W == 8) {
        const uint4 b = src[1];
        x[4] = b.x; x[5] = b.y; x[6] = b.z; x[7] = b.w;
      }
      uint32_t c = 0;
#pragma unroll
      for (int m = 0; m < D; ++m) c |= (uint32_t)(x[m] >= o[m]) << m;
      if (j < pend) atomicAdd(&histP[c * T + tid], 1u);
      else if (WIDE) atomicAdd(&histT[c * T + tid], 1u);
      else atomicAdd(&histP[c * T + tid], 1u << 16);
    }
  }
  __syncthreads();
  uint64_t bv = 0;
  int bj = 0;
  if (active) {
    for (int j = s; j < NB; j += S) {
      uint64_t a = 0, b = 0;
      for (int q = 0; q < S; ++q) {
        const int col = ol * S + q;
        if (WIDE) {
          a += histP[j * T + col];
          b += histT[j * T + col];
        } else {
          const uint32_t v = histP[j * T + col];
          a += v & 0xFFFFu;
          b += v >> 16;
        }
      }
      const uint64_t num = ddks::numer(a, b, (uint64_t)NP, (uint64_t)NT);
      if (num > bv) { bv = num; bj = j; }
    }
  }
  // combine the S slices of this origin (adjacent lanes)
  for (int off = 1; off < S; off <<= 1) {
    const uint64_t v2 = __shfl_xor_sync(0xffffffffu, bv, off);
    const int j2 = __shfl_xor_sync(0xffffffffu, bj, off);
    if (v2 > bv || (v2 == bv && j2 < bj)) { bv = v2; bj = j2; }
  }
  if (active && s == 0) {
    best[k - o_begin] = bv;
    bestj[k - o_begin] = bv ? bj : 0;
  }
}

size_t lane_smem(int d, bool wide, int threads) {
  const int w = d <= 4 ? 4 : 8;
  return (size_t)(wide ? 2 : 1) * (size_t)(1u << d) * threads * 4u + (size_t)w * kTile * 4u;
}

template <int D, bool WIDE>
cudaError_t launch_t(const uint32_t* rank, int64_t N, int64_t NP, int64_t NT, int64_t ob,
                     int64_t oe, uint64_t* best, int32_t* bestj, cudaStream_t st, int threads,
                     int S) {
  const size_t sm = lane_smem(D, WIDE, threads);
  cudaError_t e = ddks_smem_attr(k_lane<D, WIDE>, (int)sm);
  if (e != cudaSuccess) return e;
  const int64_t no = oe - ob;
  const int TO = threads / S;
  const unsigned grid = (unsigned)((no + TO - 1) / TO);
  if (grid == 0) return cudaSuccess;
  k_lane<D, WIDE><<<grid, threads, sm, st>>>(rank, N, NP, NT, ob, oe, S, best, bestj);
  return cudaGetLastError();
}

template <bool WIDE>
cudaError_t launch_w(int d, const uint32_t* rank, int64_t N, int64_t NP, int64_t NT, int64_t ob,
                     int64_t oe, uint64_t* best, int32_t* bestj, cudaStream_t st, int threads, int S) {
  switch (d) {
    case 1: return launch_t<1, WIDE>(rank, N, NP, NT, ob, oe, best, bestj, st, threads, S);
    case 2: return launch_t<2, WIDE>(rank, N, NP, NT, ob, oe, best, bestj, st, threads, S);
    case 3: return launch_t<3, WIDE>(rank, N, NP, NT, ob, oe, best, bestj, st, threads, S);
    case 4: return launch_t<4, WIDE>(rank, N, NP, NT, ob, oe, best, bestj, st, threads, S);
    case 5: return launch_t<5, WIDE>(rank, N, NP, NT, ob, oe, best, bestj, st, threads, S);
    case 6: return launch_t<6, WIDE>(rank, N, NP, NT, ob, oe, best, bestj, st, threads, S);
    case 7: return launch_t<7, WIDE>(rank, N, NP, NT, ob, oe, best, bestj, st, threads, S);
    case 8: return launch_t<8, WIDE>(rank, N, NP, NT, ob, oe, best, bestj, st, threads, S);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

bool ddks_lane_supported(int d, int64_t NP, int64_t NT, int threads) {
  if (d < 1 || d > 8 || threads < 32 || threads > 256 || (threads & 31)) return false;
  const bool wide = NP > 65535 || NT > 65535;
  return lane_smem(d, wide, threads) <= 200u * 1024u;
}

// S (slices per origin, a power of two <= 16) is chosen so the grid has about
// 64 resident warps' worth of threads per SM.
cudaError_t ddks_launch_lane(const uint32_t* rank, int64_t N, int64_t NP, int64_t NT, int d,
                             int64_t o_begin, int64_t o_end, uint64_t* best, int32_t* bestj,
                             cudaStream_t st, int threads, int num_sms) {
  if (!ddks_lane_supported(d, NP, NT, threads)) return cudaErrorInvalidValue;
  const bool wide = NP > 65535 || NT > 65535;
  const int64_t no = o_end - o_begin;
  const int64_t target = (int64_t)num_sms * 2048;
  int S = 1;
  while (S < 16 && S * 2 <= threads && no * S * 2 <= target) S <<= 1;
  return wide ? launch_w<true>(d, rank, N, NP, NT, o_begin, o_end, best, bestj, st, threads, S)
              : launch_w<false>(d, rank, N, NP, NT, o_begin, o_end, best, bestj, st, threads, S);
}
