// reduce.cu -- A5/A6: the maximum over origins (Eq. d1 takes the max over the
// concatenation of the per-origin sets) and its arg-max.
//
// Two launches: each CTA of the first reduces a contiguous range of origins to
// (largest value, lowest origin holding it, that origin's orthant); one CTA
// then combines the partials in range order.  out[0] = num_max,
// out[1] = arg-max origin (pooled index, o_begin + position; ~0 if empty),
// out[2] = its lowest orthant.
#include "ddks_internal.cuh"

namespace {

constexpr int kThreads = 512;
constexpr int kMaxParts = 256;

struct Part {
  unsigned long long v;
  long long i;
};

DDKS_DEV void better(Part& a, const Part& b) {
  if (b.v > a.v || (b.v == a.v && b.i < a.i)) a = b;
}

DDKS_DEV Part block_best(Part p, Part* sh) {
  for (int off = 16; off > 0; off >>= 1) {
    Part q;
    q.v = __shfl_down_sync(0xffffffffu, p.v, off);
    q.i = __shfl_down_sync(0xffffffffu, p.i, off);
    better(p, q);
  }
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = p;
  __syncthreads();
  if (threadIdx.x == 0) {
    Part b = sh[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) better(b, sh[w]);
    sh[0] = b;
  }
  __syncthreads();
  return sh[0];
}

__global__ void __launch_bounds__(kThreads)
k_reduce_part(const uint64_t* __restrict__ best, int64_t no, int64_t per, Part* __restrict__ parts) {
  __shared__ Part sh[kThreads / 32];
  const int64_t a = (int64_t)blockIdx.x * per;
  const int64_t b = (a + per) < no ? (a + per) : no;
  Part p{0ull, (long long)no};
  for (int64_t i = a + threadIdx.x; i < b; i += blockDim.x) {
    const Part q{best[i], (long long)i};
    better(p, q);
  }
  p = block_best(p, sh);
  if (threadIdx.x == 0) parts[blockIdx.x] = p;
}

__global__ void __launch_bounds__(kThreads)
k_reduce_final(const Part* __restrict__ parts, int nparts, const int32_t* __restrict__ bestj,
               int64_t no, int64_t o_begin, unsigned long long* __restrict__ out) {
  __shared__ Part sh[kThreads / 32];
  Part p{0ull, (long long)no};
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) better(p, parts[i]);
  p = block_best(p, sh);
  if (threadIdx.x == 0) {
    out[0] = p.v;
    if (p.i < no) {
      out[1] = (unsigned long long)(o_begin + p.i);
      out[2] = (unsigned long long)(long long)bestj[p.i];
    } else {
      out[1] = ~0ull;
      out[2] = 0;
    }
  }
}

}  // namespace

size_t ddks_reduce_scratch_bytes() { return sizeof(Part) * kMaxParts; }

// scratch: ddks_reduce_scratch_bytes() of device memory
cudaError_t ddks_launch_reduce(const uint64_t* best, const int32_t* bestj, int64_t no,
                               int64_t o_begin, unsigned long long* out3, void* scratch,
                               cudaStream_t st) {
  Part* parts = reinterpret_cast<Part*>(scratch);
  int64_t nparts = (no + 4095) / 4096;
  if (nparts > kMaxParts) nparts = kMaxParts;
  if (nparts < 1) nparts = 1;
  const int64_t per = (no + nparts - 1) / nparts;
  k_reduce_part<<<(unsigned)nparts, kThreads, 0, st>>>(best, no, per > 0 ? per : 1, parts);
  k_reduce_final<<<1, kThreads, 0, st>>>(parts, (int)nparts, bestj, no, o_begin, out3);
  return cudaGetLastError();
}
