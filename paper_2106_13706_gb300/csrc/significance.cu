// significance.cu -- A9: analytic significance of a ddKS statistic (Sec. 3).
//
// Eq. (ddks_significance): S = 1 - prod over every pooled origin k and orthant j
// of p(delta <= D; lam_kj).  Each cell's rate lam is estimated from its T count
// cT (Sec. 3: cT/NT, or the Bayes estimator (cT + 1)/(NT + 2)), so the cell
// probability depends on the cell only through cT and
//     log prod = sum_m  cells[m] * log p(delta <= D; lam(m)),
// cells[m] = number of (origin, orthant) cells with cT = m.
//
// K_cells: one warp per origin counts the T points of every orthant in a
//   shared histogram and adds each orthant's cT into cells[] (zeros are summed
//   per warp first).
// K_logp: for each m, p(delta <= D) = sum over (nP, nT) with
//   |nP*NT - nT*NP| <= num_max of pmf(nP; NP) * pmf(nT; NT)
//   (Eq. binomial_probability, or the Poisson pmf with mean m*lam).  For fixed
//   nP the admissible nT form one interval [lo, hi], so the inner sum is a
//   difference of cumulative sums of pmf(.; NT): the CTA writes the T pmf,
//   its prefix sums L and suffix sums R, and adds pmf(nP) * (L[lo-1] +
//   R[hi+1]) = the mass outside the interval.  For the binomial (masses sum
//   to one) log p = log1p(-outside mass) keeps full precision when p is near 1.
// K_final: log prod and S = -expm1(log prod), in double.
#include <cstring>

#include "ddks_host.h"
#include "ddks_internal.cuh"

namespace {

constexpr int kMaxSigD = 13;

__global__ void k_sig_cells(const uint32_t* __restrict__ rank, int64_t N, int64_t NP, int d,
                            unsigned long long* __restrict__ cells) {
  extern __shared__ uint32_t hsm[];
  const int nb = 1 << d;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int W = blockDim.x >> 5;
  uint32_t* hist = hsm + (size_t)warp * (nb + ddks::kMaxD);
  uint32_t* o = hist + nb;
  for (int64_t k = (int64_t)blockIdx.x * W + warp; k < N; k += (int64_t)gridDim.x * W) {
    for (int j = lane; j < nb; j += 32) hist[j] = 0;
    if (lane < d) o[lane] = rank[(int64_t)lane * N + k];
    __syncwarp();
    for (int64_t i = NP + lane; i < N; i += 32) {
      uint32_t c = 0;
      for (int m = 0; m < d; ++m) c |= (uint32_t)(rank[(int64_t)m * N + i] >= o[m]) << m;
      atomicAdd(&hist[c], 1u);
    }
    __syncwarp();
    unsigned long long zeros = 0;
    for (int j = lane; j < nb; j += 32) {
      const uint32_t ct = hist[j];
      if (ct == 0) ++zeros;
      else atomicAdd(&cells[ct], 1ull);
    }
    for (int off = 16; off > 0; off >>= 1) zeros += __shfl_down_sync(0xffffffffu, zeros, off);
    if (lane == 0 && zeros) atomicAdd(&cells[0], zeros);
    __syncwarp();
  }
}

__global__ void k_sig_lgamma(double* __restrict__ lg, int64_t nmax) {
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n <= nmax;
       n += (int64_t)gridDim.x * blockDim.x)
    lg[n] = lgamma((double)n + 1.0);
}

// pmf of n successes in m trials at rate lam (Eq. binomial_probability), or the
// Poisson pmf with mean m*lam (model 1); lg[n] = log(n!).
DDKS_DEV double pmf(int64_t n, int64_t m, double lam, double loglam, double log1m, int model,
                    const double* __restrict__ lg) {
  if (lam <= 0.0) return n == 0 ? 1.0 : 0.0;
  if (model == 1) {
    const double mu = (double)m * lam;
    return exp((double)n * log(mu) - mu - lg[n]);
  }
  if (lam >= 1.0) return n == m ? 1.0 : 0.0;
  return exp(lg[m] - lg[n] - lg[m - n] + (double)n * loglam + (double)(m - n) * log1m);
}

DDKS_DEV double block_sum(double v, double* red) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0;
  if (threadIdx.x == 0) {
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    red[0] = s;
  }
  __syncthreads();
  s = red[0];
  __syncthreads();
  return s;
}

// In-place scan of x[0..n) with blockDim threads: forward = inclusive prefix,
// otherwise inclusive suffix (x[i] = sum_{j >= i}).
DDKS_DEV void block_scan(double* __restrict__ x, int64_t n, bool forward, double* red) {
  double carry = 0.0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int W = blockDim.x >> 5;
  for (int64_t base = 0; base < n; base += blockDim.x) {
    const int64_t t = base + threadIdx.x;
    const int64_t idx = forward ? t : n - 1 - t;
    double v = t < n ? x[idx] : 0.0;
    for (int off = 1; off < 32; off <<= 1) {
      const double a = __shfl_up_sync(0xffffffffu, v, off);
      if (lane >= off) v += a;
    }
    if (lane == 31) red[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      double acc = 0;
      for (int w = 0; w < W; ++w) { const double s = red[w]; red[w] = acc; acc += s; }
      red[32] = acc;
    }
    __syncthreads();
    v += red[warp] + carry;
    if (t < n) x[idx] = v;
    carry += red[32];
    __syncthreads();
  }
}

__global__ void __launch_bounds__(1024)
k_sig_logp(int64_t NP, int64_t NT, unsigned long long num_max, int estimator, int model,
           const double* __restrict__ lg, const unsigned long long* __restrict__ cells,
           double* __restrict__ scratch, double* __restrict__ logp) {
  __shared__ double red[33];
  double* L = scratch + (int64_t)blockIdx.x * 2 * (NT + 1);
  double* R = L + (NT + 1);
  for (int64_t m = blockIdx.x; m <= NT; m += gridDim.x) {
    if (cells[m] == 0) {  // no cell has this count: its probability is not needed
      if (threadIdx.x == 0) logp[m] = 0.0;
      continue;
    }
    const double lam = estimator == 1 ? ((double)m + 1.0) / ((double)NT + 2.0)
                                      : (double)m / (double)NT;
    const double loglam = lam > 0.0 ? log(lam) : 0.0;
    const double log1m = lam < 1.0 ? log1p(-lam) : 0.0;
    for (int64_t n = threadIdx.x; n <= NT; n += blockDim.x) {
      const double v = pmf(n, NT, lam, loglam, log1m, model, lg);
      L[n] = v;
      R[n] = v;
    }
    __syncthreads();
    block_scan(L, NT + 1, true, red);
    block_scan(R, NT + 1, false, red);
    double outside = 0.0, massP = 0.0;
    for (int64_t np = threadIdx.x; np <= NP; np += blockDim.x) {
      const double pp = pmf(np, NP, lam, loglam, log1m, model, lg);
      const long long x = (long long)np * NT - (long long)num_max;
      int64_t lo = x <= 0 ? 0 : (int64_t)((x + NP - 1) / NP);
      int64_t hi = (int64_t)(((unsigned long long)np * NT + num_max) / (unsigned long long)NP);
      if (lo > NT + 1) lo = NT + 1;
      if (hi > NT) hi = NT;
      const double left = lo >= 1 ? L[lo - 1] : 0.0;
      const double right = hi + 1 <= NT ? R[hi + 1] : 0.0;
      outside += pp * (left + right);
      massP += pp;
    }
    outside = block_sum(outside, red);
    massP = block_sum(massP, red);
    if (threadIdx.x == 0) {
      if (model == 1) {
        const double p = massP * L[NT] - outside;  // mass inside the admissible set
        logp[m] = log(p);
      } else {
        logp[m] = log1p(-outside);
      }
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(1024)
k_sig_final(const unsigned long long* __restrict__ cells, const double* __restrict__ logp,
            int64_t NT, double* __restrict__ out) {
  __shared__ double red[33];
  double s = 0.0;
  for (int64_t m = threadIdx.x; m <= NT; m += blockDim.x)
    if (cells[m]) s += (double)cells[m] * logp[m];
  s = block_sum(s, red);
  if (threadIdx.x == 0) {
    out[0] = -expm1(s);  // S = 1 - prod
    out[1] = s;          // log prod
  }
}

}  // namespace

int ddks_significance(ddks_ctx* ctx, const void* P, int64_t NP, const void* T, int64_t NT,
                      int32_t d, int32_t dtype, uint64_t num_max, int32_t estimator,
                      int32_t model, void* stream, double* S, double* log_prod) {
  if (!ctx || !S) return DDKS_EINVAL;
  int rc = ddks_check_problem(P, NP, T, NT, d, dtype);
  if (rc) return rc;
  if (d > kMaxSigD || (estimator != 0 && estimator != 1) || (model != 0 && model != 1))
    return d > kMaxSigD ? DDKS_EUNSUPPORTED : DDKS_EINVAL;
  if (num_max > (uint64_t)NP * (uint64_t)NT) return DDKS_EINVAL;
  const int64_t N = NP + NT;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return ctx_cuda_fail(ctx, e, "cudaSetDevice");
  const void *dP, *dT;
  if ((rc = ddks_stage_inputs(ctx, P, NP, T, NT, d, dtype, st, &dP, &dT))) return rc;
  if ((rc = ddks_encode_problem(ctx, dP, NP, dT, NT, d, dtype, st, false))) return rc;
  const int64_t nmax = NP > NT ? NP : NT;
  const int sig_ctas = ctx->num_sms * 2;
  const int64_t lo_ctas = (NT + 1) < sig_ctas ? (NT + 1) : sig_ctas;
  if ((rc = ctx->sig_cells.reserve(ctx, 8 * (size_t)(NT + 1) + 8 * 4))) return rc;
  if ((rc = ctx->sig_logp.reserve(ctx, 8 * ((size_t)(NT + 1) + (size_t)(nmax + 1) +
                                            (size_t)lo_ctas * 2 * (NT + 1) + 4))))
    return rc;
  unsigned long long* cells = (unsigned long long*)ctx->sig_cells.ptr;
  double* logp = (double*)ctx->sig_logp.ptr;
  double* lg = logp + (NT + 1);
  double* scratch = lg + (nmax + 1);
  double* outd = (double*)(cells + (NT + 1));
  e = cudaMemsetAsync(cells, 0, 8 * (size_t)(NT + 1), st);
  if (e == cudaSuccess) {
    int warps = 8;
    while (warps > 1 && (size_t)warps * ((size_t)(1u << d) + ddks::kMaxD) * 4 > 160u * 1024u) --warps;
    const size_t smem = (size_t)warps * ((size_t)(1u << d) + ddks::kMaxD) * 4;
    e = ddks_smem_attr(k_sig_cells, (int)smem);
    if (e == cudaSuccess) {
      int64_t g = (N + warps - 1) / warps;
      if (g > (int64_t)ctx->num_sms * 8) g = (int64_t)ctx->num_sms * 8;
      k_sig_cells<<<(unsigned)g, warps * 32, smem, st>>>((const uint32_t*)ctx->rank.ptr, N, NP, d, cells);
      e = cudaGetLastError();
    }
  }
  if (e == cudaSuccess) {
    k_sig_lgamma<<<(unsigned)((nmax + 256) / 256 < 1024 ? (nmax + 256) / 256 : 1024), 256, 0, st>>>(lg, nmax);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    k_sig_logp<<<(unsigned)lo_ctas, 1024, 0, st>>>(NP, NT, (unsigned long long)num_max, estimator, model,
                                                   lg, cells, scratch, logp);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    k_sig_final<<<1, 1024, 0, st>>>(cells, logp, NT, outd);
    e = cudaGetLastError();
  }
  ctx->launches += 4;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ctx->h_out, outd, 2 * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ctx->h_out + 4, ctx->flags.ptr, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return ctx_cuda_fail(ctx, e, "significance");
  if ((unsigned)(ctx->h_out[4] & 0xFFFFFFFFull) & ddks::kFlagNaN) return DDKS_ENAN;
  if ((unsigned)(ctx->h_out[4] & 0xFFFFFFFFull) & ddks::kFlagTimeout) return DDKS_ETIMEOUT;
  double v[2];
  memcpy(v, ctx->h_out, sizeof v);
  *S = v[0];
  if (log_prod) *log_prod = v[1];
  return DDKS_OK;
}
