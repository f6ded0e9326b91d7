// ddks_internal.cuh -- device-side declarations shared by the library's .cu files.
//
// Data layout in device memory (one problem):
//   pooled sample X = [P; T], N = NP + NT points, P rows first.
//   keys   u64 [d][N]   order-preserving integer image of each coordinate
//   rank   u32 [d][N]   rank[m][i] = #{j : X[j][m] < X[i][m]}  (min-rank), so
//                       X[i][m] >= X[k][m]  <=>  rank[m][i] >= rank[m][k]   (Eq. g)
//   best   u64 [no]     each origin's max over orthants of |cP*NT - cT*NP|
//   bestj  i32 [no]     the lowest orthant code reaching it
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#define DDKS_DEV __device__ __forceinline__

namespace ddks {

constexpr int kMaxD = 30;

// error flags raised by kernels and read back by the host
// (kFlagRange: a coordinate range that cannot be rescaled to [0, 1], the
// normalisation of the vdKS / rdKS approximations; kFlagRedo: not an error,
// a fast path met data it does not take and the host reruns the call on the
// general path)
enum : unsigned { kFlagNaN = 1u, kFlagTimeout = 2u, kFlagBounds = 4u, kFlagRange = 8u, kFlagRedo = 16u };

// Order-preserving image of a float as an unsigned integer: x <= y (IEEE, no
// NaN) <=> key(x) <= key(y).  -0.0 is mapped like +0.0 so the two compare equal.
DDKS_DEV uint64_t order_key(float v) {
  uint32_t u = __float_as_uint(v == 0.0f ? 0.0f : v);
  u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
  return (uint64_t)u;
}
DDKS_DEV uint64_t order_key(double v) {
  uint64_t u = (uint64_t)__double_as_longlong(v);
  if ((u << 1) == 0) u = 0;  // -0.0 as +0.0 (an integer test: FP64 compares are costly here)
  u = (u & 0x8000000000000000ull) ? ~u : (u | 0x8000000000000000ull);
  return u;
}

// Lanes of the (fully active) warp whose 8-bit digit equals this lane's: one
// ballot per digit bit that differs somewhere in the warp (a fixed cost;
// match.any slows down with the number of distinct values in the warp).
DDKS_DEV uint32_t same_digit(uint32_t dg) {
  const uint32_t vary = __reduce_or_sync(0xffffffffu, dg) ^ __reduce_and_sync(0xffffffffu, dg);
  uint32_t m = 0xffffffffu;
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    if ((vary >> b) & 1u) {
      const bool bit = (dg >> b) & 1u;
      const uint32_t bal = __ballot_sync(0xffffffffu, bit);
      m &= bit ? bal : ~bal;
    }
  }
  return m;
}

// |a*NT - b*NP| for counts a <= NP, b <= NT with NP*NT < 2^62 (no overflow).
DDKS_DEV uint64_t numer(uint64_t a, uint64_t b, uint64_t NP, uint64_t NT) {
  uint64_t x = a * NT, y = b * NP;
  return x > y ? x - y : y - x;
}

}  // namespace ddks

// The dynamic shared-memory limit of a kernel, raised to at least `bytes`
// (never lowered: contexts on several threads launch the same kernels with
// different sizes, and a lowered limit would fail another thread's launch
// between its own set and launch).  Per device; thread-safe.
cudaError_t ddks_smem_attr_raw(const void* func, size_t bytes);
template <class F>
inline cudaError_t ddks_smem_attr(F* func, size_t bytes) {
  return ddks_smem_attr_raw(reinterpret_cast<const void*>(func), bytes);
}

// Launch wrappers implemented in the .cu files (all enqueue on `st`).
struct DdksProblemDev {
  const uint32_t* rank;  // [d][N]
  int64_t N, NP, NT;
  int32_t d;
};

cudaError_t ddks_launch_encode(const void* P, const void* T, int64_t NP, int64_t NT, int d,
                               int is_f64, uint64_t* keys, unsigned* flags, cudaStream_t st);
cudaError_t ddks_launch_rank(const uint64_t* keys, int64_t N, int64_t NP, int d, uint64_t* tmp_keys,
                             uint32_t* tmp_idx, uint64_t* tmp_keys2, uint32_t* tmp_idx2,
                             uint32_t* rank, uint32_t* sorted_idx0, uint32_t* pprefix0, uint32_t* cpfx,
                             int* pfx_done, cudaStream_t st, int* launches, int key_bits = 64,
                             uint32_t* radix_scratch = nullptr, const uint32_t** sorted_rows = nullptr);
size_t ddks_rank_pfx_elems(int64_t N);
size_t ddks_rank_scratch_elems(int64_t N);
cudaError_t ddks_launch_sort_segments(const uint64_t* keys, int64_t N, int64_t NP, int S, uint64_t* k1,
                                      uint32_t* i1, uint32_t* p1, uint64_t* k2, uint32_t* i2,
                                      uint32_t* p2, const uint64_t** out_k, const uint32_t** out_i,
                                      const uint32_t** out_p, cudaStream_t st, int* launches);

cudaError_t ddks_launch_lane(const uint32_t* rank, int64_t N, int64_t NP, int64_t NT, int d,
                             int64_t o_begin, int64_t o_end, uint64_t* best, int32_t* bestj,
                             cudaStream_t st, int threads, int num_sms);
cudaError_t ddks_launch_warp(const uint32_t* rank, int64_t N, int64_t NP, int64_t NT, int d,
                             int64_t o_begin, int64_t o_end, uint64_t* best, int32_t* bestj,
                             cudaStream_t st, int warps);
cudaError_t ddks_launch_sort(const uint32_t* rank, int64_t N, int64_t NP, int64_t NT, int d,
                             int64_t o_begin, int64_t o_end, uint64_t* best, int32_t* bestj,
                             cudaStream_t st);
size_t ddks_reduce_scratch_bytes();
cudaError_t ddks_launch_reduce(const uint64_t* best, const int32_t* bestj, int64_t no,
                               int64_t o_begin, unsigned long long* out3, void* scratch,
                               cudaStream_t st);

// radix.cu: stable LSD radix sort of key rows carrying their positions, and
// min-ranks / P prefixes / dimension-0 order from the sorted rows.
size_t ddks_radix_scratch_words(int64_t n, int64_t rows, int64_t pfx_rows);
cudaError_t ddks_radix_sort(const uint64_t* keys, uint64_t* ka, uint32_t* ia, uint64_t* kb, uint32_t* ib, int64_t n,
                            int64_t stride, int64_t rows, int nbits, uint32_t* scratch, const uint64_t** out_k,
                            const uint32_t** out_i, cudaStream_t st, int* launches);
cudaError_t ddks_radix_ranks(const uint64_t* sk, const uint32_t* si, int64_t n, int64_t stride, int64_t rows,
                             int64_t NP, uint32_t* rank, uint32_t* pfx, int64_t pfx_rows, uint32_t* sorted_idx0,
                             uint32_t* scratch, cudaStream_t st, int* launches);

size_t ddks_scan_tmp_elems(int64_t rows, int64_t n);
cudaError_t ddks_scan_rows(const uint32_t* in, uint32_t* out, int64_t rows, int64_t n, bool exclusive,
                           uint32_t* tmp, cudaStream_t st, int* launches);

bool ddks_lane_supported(int d, int64_t NP, int64_t NT, int threads);
bool ddks_warp_supported(int d, int64_t NP, int64_t NT);
bool ddks_sort_supported(int d, int64_t N);
