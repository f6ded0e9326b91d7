// reduce.cu -- A5/A6: the maximum over origins (Eq. d1 takes the max over the
// concatenation of the per-origin sets) and its arg-max.
//
// One CTA walks the per-origin maxima twice: first the largest value, then the
// lowest origin index holding it.  out[0] = num_max, out[1] = that origin's
// pooled index (o_begin + position), out[2] = its lowest orthant.
#include "ddks_internal.cuh"

namespace {

__global__ void __launch_bounds__(1024)
k_reduce(const uint64_t* __restrict__ best, const int32_t* __restrict__ bestj, int64_t no,
         int64_t o_begin, unsigned long long* __restrict__ out) {
  __shared__ unsigned long long sv[32];
  __shared__ long long si[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned long long v = 0;
  for (int64_t i = threadIdx.x; i < no; i += blockDim.x) v = best[i] > v ? best[i] : v;
  for (int off = 16; off > 0; off >>= 1) {
    const unsigned long long v2 = __shfl_down_sync(0xffffffffu, v, off);
    v = v2 > v ? v2 : v;
  }
  if (lane == 0) sv[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long b = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b = sv[w] > b ? sv[w] : b;
    sv[0] = b;
  }
  __syncthreads();
  const unsigned long long vmax = sv[0];
  long long idx = no;  // lowest position holding vmax
  for (int64_t i = threadIdx.x; i < no; i += blockDim.x)
    if (best[i] == vmax) { idx = i; break; }
  for (int off = 16; off > 0; off >>= 1) {
    const long long i2 = __shfl_down_sync(0xffffffffu, idx, off);
    idx = i2 < idx ? i2 : idx;
  }
  __syncthreads();
  if (lane == 0) si[warp] = idx;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long b = no;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b = si[w] < b ? si[w] : b;
    out[0] = vmax;
    if (b < no) {
      out[1] = (unsigned long long)(o_begin + b);
      out[2] = (unsigned long long)(long long)bestj[b];
    } else {
      out[1] = ~0ull;  // empty origin range
      out[2] = 0;
    }
  }
}

}  // namespace

cudaError_t ddks_launch_reduce(const uint64_t* best, const int32_t* bestj, int64_t no,
                               int64_t o_begin, unsigned long long* out3, cudaStream_t st) {
  k_reduce<<<1, 1024, 0, st>>>(best, bestj, no, o_begin, out3);
  return cudaGetLastError();
}
