// noalloc.cu -- ddks_distance_noalloc: the exact distance without any device
// allocation, for callers that must not allocate device memory after start-up.
//
// All scratch lives in one file-scope device array of kNoallocScratch bytes
// that every GPU loading the library holds until the process exits.  Host code
// never passes the array's name to a kernel (in host code that name is only a
// host-side stand-in, not a device address): every call, with the device
// current, asks cudaGetSymbolAddress for the array's device address on that
// device and passes it to the kernels.  Every call
// reuses the same array, so calls whose work overlaps on the GPU (different
// streams, or host threads, on one device) race; the NaN flag, the only state
// that must start at zero, is cleared by each call.
//
// Sizes: N = NP + NT <= 16384 and d <= 8.  Ranks are computed by one CTA per
// dimension that sorts the N coordinates in shared memory (no global sort
// buffers); the orthant counts use the lane-private histogram kernel; the
// maximum uses the two-level reduction.
#include <cstring>
#include <mutex>

#include "../../include/ddks.h"
#include "ddks_internal.cuh"

namespace {

constexpr int64_t kMaxN = 16384;
constexpr int kMaxDim = 8;
constexpr size_t kRankBytes = (size_t)kMaxDim * kMaxN * 4;
constexpr size_t kBestBytes = (size_t)kMaxN * 8;
constexpr size_t kBestjBytes = (size_t)kMaxN * 4;
constexpr size_t kOutBytes = 64;
constexpr size_t kReduceBytes = 8192;
constexpr size_t kFlagBytes = 256;
constexpr size_t kNoallocScratch =
    kRankBytes + kBestBytes + kBestjBytes + kOutBytes + kReduceBytes + kFlagBytes;

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratch];

std::mutex g_mu;
int g_sms[128] = {};

DDKS_DEV bool pair_less(uint64_t ka, uint32_t ia, uint64_t kb, uint32_t ib) {
  return ka < kb || (ka == kb && ia < ib);
}

// one CTA per dimension m: order keys, bitonic sort of (key, index) in shared
// memory, then each point's min-rank by lower_bound in the sorted keys
template <typename V>
__global__ void __launch_bounds__(1024)
k_noalloc_rank(const V* __restrict__ P, const V* __restrict__ T, int64_t NP, int64_t NT, int d,
               uint32_t* __restrict__ rank, unsigned* __restrict__ flags) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int m = blockIdx.x;
  const int64_t N = NP + NT;
  int P2 = 1;
  while (P2 < N) P2 <<= 1;
  uint64_t* sk = reinterpret_cast<uint64_t*>(smraw);
  uint32_t* si = reinterpret_cast<uint32_t*>(sk + P2);
  for (int i = threadIdx.x; i < P2; i += blockDim.x) {
    uint64_t key = ~0ull;
    if (i < N) {
      const V v = i < NP ? P[(int64_t)i * d + m] : T[(int64_t)(i - NP) * d + m];
      if (v != v) atomicOr(flags, ddks::kFlagNaN);
      key = ddks::order_key(v);
    }
    sk[i] = key;
    si[i] = (uint32_t)i;
  }
  __syncthreads();
  for (int size = 2; size <= P2; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int t = threadIdx.x; t < P2 / 2; t += blockDim.x) {
        const int lo = 2 * t - (t & (stride - 1));
        const int hi = lo + stride;
        const bool asc = ((lo & size) == 0);
        const uint64_t ka = sk[lo], kb = sk[hi];
        const uint32_t ia = si[lo], ib = si[hi];
        const bool swap = asc ? pair_less(kb, ib, ka, ia) : pair_less(ka, ia, kb, ib);
        if (swap) { sk[lo] = kb; sk[hi] = ka; si[lo] = ib; si[hi] = ia; }
      }
      __syncthreads();
    }
  }
  for (int p = threadIdx.x; p < N; p += blockDim.x) {
    const uint64_t key = sk[p];
    int lo = 0, hi = p;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (sk[mid] < key) lo = mid + 1; else hi = mid;
    }
    rank[(int64_t)m * N + si[p]] = (uint32_t)lo;
  }
}

int fail(cudaError_t e) {
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? DDKS_ENOMEM : DDKS_ECUDA;
}

// Device address of the scratch array on the current device, looked up on
// every call (no allocation; a device reset reloads the module, so a cached
// address could go stale), and the device's SM count (cached per device).
int scratch_on_device(int dev, void** addr, int* sms) {
  if (dev < 0 || dev >= 128) return DDKS_EINVAL;
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return fail(e);
  std::lock_guard<std::mutex> g(g_mu);
  if (!g_sms[dev]) {
    int n = 0;
    e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return fail(e);
    g_sms[dev] = n;
  }
  *addr = p;
  *sms = g_sms[dev];
  return DDKS_OK;
}

}  // namespace

int ddks_distance_noalloc(const void* P, int64_t NP, const void* T, int64_t NT, int32_t d,
                          int32_t dtype, void* stream, ddks_result* out) {
  if (!out) return DDKS_EINVAL;
  if (!P || !T || NP < 1 || NT < 1 || d < 1 || d > DDKS_MAX_D ||
      (dtype != DDKS_F32 && dtype != DDKS_F64))
    return out->status = DDKS_EINVAL;
  if (NP + NT > kMaxN || d > kMaxDim) return out->status = DDKS_EUNSUPPORTED;
  cudaPointerAttributes pa, ta;
  if (cudaPointerGetAttributes(&pa, P) != cudaSuccess || cudaPointerGetAttributes(&ta, T) != cudaSuccess) {
    cudaGetLastError();
    return out->status = DDKS_EINVAL;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return out->status = fail(e);
  // inputs must already be device memory of this device (or managed memory)
  if (ddks_classify_pointer((int32_t)pa.type, (int32_t)pa.device, dev) != 1 ||
      ddks_classify_pointer((int32_t)ta.type, (int32_t)ta.device, dev) != 1)
    return out->status = DDKS_EINVAL;
  void* base = nullptr;
  int sms = 0;
  int rc = scratch_on_device(dev, &base, &sms);
  if (rc) return out->status = rc;
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t N = NP + NT;
  unsigned char* b = (unsigned char*)base;
  uint32_t* rank = (uint32_t*)b;
  uint64_t* best = (uint64_t*)(b + kRankBytes);
  int32_t* bestj = (int32_t*)(b + kRankBytes + kBestBytes);
  unsigned long long* out3 = (unsigned long long*)(b + kRankBytes + kBestBytes + kBestjBytes);
  void* red = b + kRankBytes + kBestBytes + kBestjBytes + kOutBytes;
  unsigned* flags = (unsigned*)(b + kRankBytes + kBestBytes + kBestjBytes + kOutBytes + kReduceBytes);
  if (ddks_reduce_scratch_bytes() > kReduceBytes) return out->status = DDKS_EUNSUPPORTED;
  e = cudaMemsetAsync(flags, 0, sizeof(unsigned), st);
  if (e != cudaSuccess) return out->status = fail(e);
  int P2 = 1;
  while (P2 < N) P2 <<= 1;
  const size_t smem = (size_t)P2 * 12;
  if (dtype == DDKS_F64) {
    e = ddks_smem_attr(k_noalloc_rank<double>, (int)smem);
    if (e == cudaSuccess)
      k_noalloc_rank<double><<<d, 1024, smem, st>>>((const double*)P, (const double*)T, NP, NT, d, rank, flags);
  } else {
    e = ddks_smem_attr(k_noalloc_rank<float>, (int)smem);
    if (e == cudaSuccess)
      k_noalloc_rank<float><<<d, 1024, smem, st>>>((const float*)P, (const float*)T, NP, NT, d, rank, flags);
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  const int threads = d <= 4 ? 256 : (d <= 6 ? 128 : 64);
  if (e == cudaSuccess) e = ddks_launch_lane(rank, N, NP, NT, d, 0, N, best, bestj, st, threads, sms);
  if (e == cudaSuccess) e = ddks_launch_reduce(best, bestj, N, 0, out3, red, st);
  unsigned long long h[3] = {0, 0, 0};
  unsigned hf = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, out3, sizeof h, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hf, flags, sizeof hf, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return out->status = fail(e);
  if (hf & ddks::kFlagNaN) return out->status = DDKS_ENAN;
  out->num_max = h[0];
  out->denom = (uint64_t)NP * (uint64_t)NT;
  out->D = (double)out->num_max / (double)out->denom;
  out->argmax_origin = (int64_t)h[1];
  out->argmax_orthant = (int32_t)h[2];
  out->status = DDKS_OK;
  return DDKS_OK;
}
