// dominance.cu -- exact ddKS for d = 2 in O(N log N) work (DDKS_PATH_DOMINANCE).
//
// Not in the paper: a sub-quadratic restatement of the same statistic
// (Eq. ddks_tensor_definition with the ">=" split of Eq. g) that skips the
// pairwise compares.  With min-ranks (K0), a point x is on the upper side of
// origin o in dimension m iff rank_m(x) >= rank_m(o).  In the order of
// dimension 0 (K0's sorted_idx0), the points with x_0 >= o_0 are exactly the
// positions >= rank_0(o), so the upper-upper count of a sample is a range
// query: #{positions k >= rank_0(o) : y(k) >= rank_1(o)}, y(k) the
// dimension-1 rank of the point at position k.  The other three quadrants
// follow from the marginals: #{x_0 >= o_0} = N - rank_0(o) (its P part from
// K0's P prefix at that position), #{x_1 >= o_1} = N - rank_1(o) (its P part
// by a second query over the whole range).
//
// The range queries run on two wavelet matrices (the wavelet tree variant of
// Information Systems 47, 2015): one over the y ranks of all points in
// dimension-0 order, one
// over the P points only.  Level l of a matrix holds one bit per position
// (bit L-1-l of the value), a per-word prefix count of ones, and the next
// level's order: a stable partition, zeros first.  A query walks the L levels
// with two rank lookups each.  Build: per level a bit kernel (warp ballots), a
// scan of the word counts and a scatter kernel; query: one thread per origin.
#include <cstring>

#include "../../include/ddks.h"
#include "ddks_host.h"
#include "ddks_internal.cuh"

namespace {

constexpr int kThreads = 256;

// One wavelet matrix in device memory: level lv's bit words at
// B + lv * bstride, its prefix counts (ones before each word, nw + 1 entries)
// at R + lv * rstride.
struct WMView {
  const uint32_t* B;
  const uint32_t* R;
  uint32_t n, nw;
  uint32_t bstride, rstride;
  int L;
};

DDKS_DEV uint32_t rank1(const uint32_t* B, const uint32_t* R, uint32_t k) {
  const uint32_t w = k >> 5, b = k & 31;
  return R[w] + (b ? (uint32_t)__popc(B[w] & ((1u << b) - 1u)) : 0u);
}

// #{k in [l, r) : value(k) >= v}
DDKS_DEV uint32_t count_ge(const WMView& wm, uint32_t l, uint32_t r, uint32_t v) {
  const uint32_t len = r - l;
  uint32_t less = 0;
  for (int lv = 0; lv < wm.L; ++lv) {
    if (l >= r) break;
    const uint32_t* B = wm.B + (size_t)lv * wm.bstride;
    const uint32_t* R = wm.R + (size_t)lv * wm.rstride;
    const uint32_t ol = rank1(B, R, l), orr = rank1(B, R, r);
    const uint32_t Z = wm.n - R[wm.nw];
    if ((v >> (wm.L - 1 - lv)) & 1u) {
      less += (r - l) - (orr - ol);  // the zeros of this level are smaller
      l = Z + ol;
      r = Z + orr;
    } else {
      l -= ol;
      r -= orr;
    }
  }
  return len - less;
}

// Level-0 values: y ranks in dimension-0 order, for all points (matrix 0) and
// for the P points (matrix 1, positions = P points before the position).
__global__ void __launch_bounds__(kThreads)
k_dom_init(const uint32_t* __restrict__ rank, const uint32_t* __restrict__ sorted_idx0,
           const uint32_t* __restrict__ pprefix0, int64_t N, int64_t NP, uint32_t* __restrict__ v_all,
           uint32_t* __restrict__ v_p) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t i = sorted_idx0[k];
    const uint32_t y = rank[N + i];
    v_all[k] = y;
    if (i < (uint64_t)NP) v_p[pprefix0[k]] = y;
  }
}

// Bit words of one level for both matrices (blockIdx.y = matrix): cnt[w] =
// ones of word w (0 past the matrix's last word, up to nwmax + 1 words).
__global__ void __launch_bounds__(kThreads)
k_dom_bits(const uint32_t* __restrict__ vals, uint32_t n0, uint32_t n1, uint32_t nmax, uint32_t nwmax, int bit,
           uint32_t* __restrict__ Bout, uint32_t* __restrict__ cnt) {
  const int mtx = blockIdx.y;
  const uint32_t n = mtx ? n1 : n0;
  const uint32_t* v = vals + (size_t)mtx * nmax;
  uint32_t* B = Bout + (size_t)mtx * nwmax;
  uint32_t* C = cnt + (size_t)mtx * (nwmax + 1);
  const uint32_t words = nwmax + 1;
  for (uint32_t w0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w0 < words;
       w0 += (gridDim.x * blockDim.x) >> 5) {
    const uint32_t k = w0 * 32 + (threadIdx.x & 31);
    const bool one = k < n && ((v[k] >> bit) & 1u);
    const uint32_t word = __ballot_sync(0xffffffffu, one);
    if ((threadIdx.x & 31) == 0) {
      if (w0 < nwmax) B[w0] = word;
      C[w0] = (uint32_t)__popc(word);
    }
  }
}

// Stable partition of one level (zeros first) into the next level's order.
__global__ void __launch_bounds__(kThreads)
k_dom_scatter(const uint32_t* __restrict__ vin, uint32_t* __restrict__ vout, uint32_t n0, uint32_t n1,
              uint32_t nmax, uint32_t nwmax, int bit, const uint32_t* __restrict__ Bl,
              const uint32_t* __restrict__ Rl) {
  const int mtx = blockIdx.y;
  const uint32_t n = mtx ? n1 : n0;
  const uint32_t nw = (n + 31) / 32;
  const uint32_t* v = vin + (size_t)mtx * nmax;
  uint32_t* o = vout + (size_t)mtx * nmax;
  const uint32_t* B = Bl + (size_t)mtx * nwmax;
  const uint32_t* R = Rl + (size_t)mtx * (nwmax + 1);
  const uint32_t Z = n - R[nw];
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const uint32_t x = v[k];
    const uint32_t ones = rank1(B, R, k);
    o[((x >> bit) & 1u) ? Z + ones : k - ones] = x;
  }
}

// Per origin: the four quadrant counts of each sample and the best orthant.
__global__ void __launch_bounds__(kThreads)
k_dom_query(const uint32_t* __restrict__ rank, const uint32_t* __restrict__ pprefix0, int64_t N, int64_t NP,
            int64_t NT, int64_t ob, int64_t oe, WMView wa, WMView wp, uint64_t* __restrict__ best,
            int32_t* __restrict__ bestj) {
  for (int64_t o = ob + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < oe;
       o += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t rx = rank[o], ry = rank[N + o];
    const uint32_t lxp = rx < (uint64_t)N ? pprefix0[rx] : (uint32_t)NP;  // P points with x_0 < o_0
    const uint64_t a3 = count_ge(wa, rx, (uint32_t)N, ry);                // both >=, all points
    const uint64_t p3 = count_ge(wp, lxp, (uint32_t)NP, ry);              // both >=, P
    const uint64_t pyu = count_ge(wp, 0, (uint32_t)NP, ry);               // P with x_1 >= o_1
    const uint64_t axu = (uint64_t)N - rx, pxu = (uint64_t)NP - lxp;      // x_0 >= o_0
    const uint64_t ayu = (uint64_t)N - ry;                                // x_1 >= o_1
    uint64_t cp[4], ca[4];
    cp[3] = p3;
    cp[1] = pxu - p3;  // code 1: x_0 >= o_0, x_1 < o_1
    cp[2] = pyu - p3;  // code 2: x_0 < o_0, x_1 >= o_1
    cp[0] = (uint64_t)NP - cp[1] - cp[2] - cp[3];
    ca[3] = a3;
    ca[1] = axu - a3;
    ca[2] = ayu - a3;
    ca[0] = (uint64_t)N - ca[1] - ca[2] - ca[3];
    uint64_t b = 0;
    int bj = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const uint64_t v = ddks::numer(cp[j], ca[j] - cp[j], (uint64_t)NP, (uint64_t)NT);
      if (v > b) { b = v; bj = j; }
    }
    best[o - ob] = b;
    bestj[o - ob] = bj;
  }
}

int grid_for(int64_t work, int threads, int cap) {
  int64_t g = (work + threads - 1) / threads;
  if (g > cap) g = cap;
  return (int)(g < 1 ? 1 : g);
}

}  // namespace

bool ddks_dominance_supported(int d, int64_t NP, int64_t NT) {
  return d == 2 && NP + NT < ((int64_t)1 << 31) && NP >= 1 && NT >= 1;
}

// Requires K0 with sorted_idx0 and its P prefix (ctx->pfx0_valid).
cudaError_t ddks_launch_dominance(ddks_ctx* ctx, const uint32_t* rank, int64_t N, int64_t NP, int64_t NT,
                                  int64_t ob, int64_t oe, uint64_t* best, int32_t* bestj, cudaStream_t st,
                                  int* launches) {
  int n = 0;
  int L = 1;
  while (((int64_t)1 << L) < N) ++L;  // values (ranks) < N <= 2^L
  const uint32_t n0 = (uint32_t)N, n1 = (uint32_t)NP, nmax = n0;
  const uint32_t nwmax = (nmax + 31) / 32;
  // scratch: values [2 bufs][2 matrices][nmax], bits [L][2][nwmax], prefixes
  // [L][2][nwmax + 1], counts [2][nwmax + 1], scan temp
  const size_t scan_tmp = ddks_scan_tmp_elems(2, nwmax + 1);
  const size_t words = (size_t)4 * nmax + (size_t)L * 2 * nwmax + (size_t)L * 2 * (nwmax + 1) +
                       2 * (size_t)(nwmax + 1) + scan_tmp;
  int rc = ctx->dom_work.reserve(ctx, 4 * words);
  if (rc) return cudaErrorMemoryAllocation;
  uint32_t* base = (uint32_t*)ctx->dom_work.ptr;
  uint32_t* vbuf[2] = {base, base + 2 * (size_t)nmax};
  uint32_t* Bw = base + 4 * (size_t)nmax;
  uint32_t* Rw = Bw + (size_t)L * 2 * nwmax;
  uint32_t* cnt = Rw + (size_t)L * 2 * (nwmax + 1);
  uint32_t* tmp = cnt + 2 * (size_t)(nwmax + 1);
  const uint32_t* sorted_idx0 = (const uint32_t*)ctx->sidx0.ptr;
  const uint32_t* pprefix0 = (const uint32_t*)ctx->pfx0.ptr;
  k_dom_init<<<grid_for(N, kThreads, ctx->num_sms * 8), kThreads, 0, st>>>(rank, sorted_idx0, pprefix0, N, NP,
                                                                         vbuf[0], vbuf[0] + nmax);
  ++n;
  const dim3 gw((unsigned)grid_for((int64_t)(nwmax + 1) * 32, kThreads, ctx->num_sms * 8), 2);
  const dim3 gs((unsigned)grid_for(nmax, kThreads, ctx->num_sms * 8), 2);
  for (int lv = 0; lv < L; ++lv) {
    const int bit = L - 1 - lv;
    uint32_t* Bl = Bw + (size_t)lv * 2 * nwmax;
    uint32_t* Rl = Rw + (size_t)lv * 2 * (nwmax + 1);
    k_dom_bits<<<gw, kThreads, 0, st>>>(vbuf[lv & 1], n0, n1, nmax, nwmax, bit, Bl, cnt);
    ++n;
    int sl = 0;
    cudaError_t e = ddks_scan_rows(cnt, Rl, 2, nwmax + 1, true, tmp, st, &sl);
    if (e != cudaSuccess) return e;
    n += sl;
    if (lv + 1 < L) {
      k_dom_scatter<<<gs, kThreads, 0, st>>>(vbuf[lv & 1], vbuf[(lv + 1) & 1], n0, n1, nmax, nwmax, bit, Bl, Rl);
      ++n;
    }
  }
  // query views: levels are [lv][matrix][words]
  const WMView wa{Bw, Rw, n0, (n0 + 31) / 32, 2 * nwmax, 2 * (nwmax + 1), L};
  const WMView wp{Bw + nwmax, Rw + (nwmax + 1), n1, (n1 + 31) / 32, 2 * nwmax, 2 * (nwmax + 1), L};
  const int64_t no = oe - ob;
  if (no > 0) {
    k_dom_query<<<grid_for(no, kThreads, ctx->num_sms * 16), kThreads, 0, st>>>(rank, pprefix0, N, NP, NT, ob, oe,
                                                                              wa, wp, best, bestj);
    ++n;
  }
  if (launches) *launches += n;
  return cudaGetLastError();
}
