// scan.cu -- row-wise prefix sums of u32 arrays over many CTAs (used by the
// preparation kernels of the register path).  Three passes: per-chunk sums,
// a scan of the chunk sums of each row, then each chunk scanned locally with
// its offset added.
#include "ddks_internal.cuh"

namespace {

constexpr int kThreads = 1024;
constexpr int kPer = 4;
constexpr int kChunk = kThreads * kPer;

DDKS_DEV uint32_t block_incl_scan(uint32_t v, uint32_t* ws, uint32_t* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int off = 1; off < 32; off <<= 1) {
    const uint32_t a = __shfl_up_sync(0xffffffffu, v, off);
    if (lane >= off) v += a;
  }
  if (lane == 31) ws[warp] = v;
  __syncthreads();
  if (warp == 0) {
    uint32_t s = lane < (int)(blockDim.x >> 5) ? ws[lane] : 0u;
    for (int off = 1; off < 32; off <<= 1) {
      const uint32_t a = __shfl_up_sync(0xffffffffu, s, off);
      if (lane >= off) s += a;
    }
    ws[lane] = s;
  }
  __syncthreads();
  const uint32_t r = v + (warp ? ws[warp - 1] : 0u);
  if (total) *total = ws[(blockDim.x >> 5) - 1];
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(kThreads)
k_chunk_sums(const uint32_t* __restrict__ in, int64_t n, int64_t nch, uint32_t* __restrict__ sums) {
  __shared__ uint32_t ws[32];
  const int64_t row = blockIdx.y;
  const int64_t base = (int64_t)blockIdx.x * kChunk;
  const uint32_t* x = in + row * n;
  uint32_t v = 0;
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
    const int64_t i = base + (int64_t)threadIdx.x * kPer + q;
    if (i < n) v += x[i];
  }
  uint32_t tot;
  block_incl_scan(v, ws, &tot);
  if (threadIdx.x == 0) sums[row * nch + blockIdx.x] = tot;
}

// exclusive scan of each row of sums (nch entries), in place
__global__ void __launch_bounds__(kThreads)
k_chunk_offsets(uint32_t* __restrict__ sums, int64_t nch) {
  __shared__ uint32_t ws[32];
  uint32_t* s = sums + (int64_t)blockIdx.x * nch;
  uint32_t carry = 0;
  for (int64_t base = 0; base < nch; base += kThreads) {
    const int64_t i = base + threadIdx.x;
    const uint32_t v = i < nch ? s[i] : 0u;
    uint32_t tot;
    const uint32_t inc = block_incl_scan(v, ws, &tot);
    if (i < nch) s[i] = carry + inc - v;
    carry += tot;
  }
}

__global__ void __launch_bounds__(kThreads)
k_chunk_scan(const uint32_t* __restrict__ in, uint32_t* __restrict__ out, int64_t n, int64_t nch,
             const uint32_t* __restrict__ offs, int exclusive) {
  __shared__ uint32_t ws[32];
  const int64_t row = blockIdx.y;
  const int64_t base = (int64_t)blockIdx.x * kChunk;
  const uint32_t* x = in + row * n;
  uint32_t* y = out + row * n;
  uint32_t v[kPer];
  uint32_t t = 0;
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
    const int64_t i = base + (int64_t)threadIdx.x * kPer + q;
    v[q] = i < n ? x[i] : 0u;
    t += v[q];
  }
  const uint32_t inc = block_incl_scan(t, ws, nullptr);
  uint32_t run = offs[row * nch + blockIdx.x] + inc - t;
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
    const int64_t i = base + (int64_t)threadIdx.x * kPer + q;
    if (exclusive) {
      if (i < n) y[i] = run;
      run += v[q];
    } else {
      run += v[q];
      if (i < n) y[i] = run;
    }
  }
}

}  // namespace

size_t ddks_scan_tmp_elems(int64_t rows, int64_t n) {
  return (size_t)rows * (size_t)((n + kChunk - 1) / kChunk);
}

// out[r][i] = sum of in[r][0..i] (inclusive) or in[r][0..i) (exclusive); in == out allowed.
cudaError_t ddks_scan_rows(const uint32_t* in, uint32_t* out, int64_t rows, int64_t n, bool exclusive,
                           uint32_t* tmp, cudaStream_t st, int* launches) {
  if (rows <= 0 || n <= 0) return cudaSuccess;
  const int64_t nch = (n + kChunk - 1) / kChunk;
  dim3 g((unsigned)nch, (unsigned)rows);
  k_chunk_sums<<<g, kThreads, 0, st>>>(in, n, nch, tmp);
  k_chunk_offsets<<<(unsigned)rows, kThreads, 0, st>>>(tmp, nch);
  k_chunk_scan<<<g, kThreads, 0, st>>>(in, out, n, nch, tmp, exclusive ? 1 : 0);
  if (launches) *launches += 3;
  return cudaGetLastError();
}
