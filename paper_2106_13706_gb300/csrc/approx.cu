// approx.cu -- the two approximations of Sec. 2.2 on the device: the voxel
// statistic vdKS (Alg. vdKS) and the radial statistic rdKS (Alg. rdKS), with
// the readings stated in include/ddks.h for their garbled or silent points.
//
// Shared first step (NormalizeData): k_minmax reduces each dimension's
// minimum and maximum over the pooled sample; every later kernel rescales a
// coordinate as x' = (x - lo) / (hi - lo) with correctly rounded IEEE double
// subtract and divide (0 for a constant dimension), so x' is the same double
// the host arithmetic of the definition gives.
//
// vdKS
//   k_vdks_voxel     voxel of every pooled point, c_m = floor(x'_m * V) (V - 1
//                    for x'_m = 1); counts (nP, nT) per voxel, warp-aggregated.
//                    With few voxels per dimension the coordinates come from
//                    exact thresholds (k_vdks_thresholds) by integer key
//                    compares instead of a double divide per coordinate: FP64
//                    runs at a small fraction of the integer rate on this GPU.
//   k_vdks_suffix*   d passes of suffix sums: U(c) = sum over the voxels c' with
//                    c'_m >= c_m in every dimension of nT*NP - nP*NT (the first
//                    pass forms the differences from the counts)
//   k_vdks_eval      at every filled voxel c: F(A) = U(c with the coordinates
//                    outside A set to 0) for each dimension subset A is the sum
//                    over the voxels on the upper side of the dimensions in A;
//                    the orthant sums follow by inclusion-exclusion,
//                    g(j) = sum over S within ~j of (-1)^|S| F(j u S), done as a
//                    Moebius transform one dimension at a time (lanes hold
//                    subsets and exchange by shuffles).  max |g| with the lowest
//                    voxel and then the lowest orthant; the last CTA reduces
//                    the CTAs' partial results.
// rdKS
//   k_rdks_dist_*    squared distance of each point to each corner, summed in
//                    dimension order; corner 0 is the origin, corner m + 1 the
//                    unit vector of dimension m.  The running sum over the
//                    first m terms is shared by corner m + 1.
//   sort             the K0 chunk sort and merge passes over the d + 1 corner
//                    segments, carrying the P count before each position
//   k_rdks_walk      at the last position of every run of equal distances:
//                    |cP*NT - cT*NP| of the counts up to and including it
//                    (both empirical CDFs evaluated after the tied values);
//                    max per corner
//   k_rdks_final     max over corners, lowest corner
#include <climits>
#include <cstring>

#include "../../include/ddks.h"
#include "ddks_internal.cuh"
#include "ddks_host.h"

namespace {

using ull = unsigned long long;
constexpr int kThreads = 256;
constexpr int kVdksMaxD = DDKS_VDKS_MAX_D;
constexpr int kRdksThreadMaxD = 16;  // up to here one thread computes all corners of a point
constexpr uint64_t kVdksMaxCells = 1ull << 28;
constexpr int64_t kVdksMaxThresholds = 4096;  // d * (V - 1) keys staged in shared memory

// Inverse of ddks::order_key for doubles (-0.0 comes back as +0.0).
DDKS_DEV double key_value(ull k) {
  const ull b = (k >> 63) ? (k & 0x7FFFFFFFFFFFFFFFull) : ~k;
  return __longlong_as_double((long long)b);
}

DDKS_DEV double rescale(double v, double lo, double span) {
  return span > 0.0 ? __ddiv_rn(__dsub_rn(v, lo), span) : 0.0;
}

template <typename V>
DDKS_DEV const V* point_row(const V* P, const V* T, int64_t NP, int d, int64_t i) {
  return i < NP ? P + i * d : T + (i - NP) * d;
}

// Order keys in the input type's own width: u32 for float, u64 for double
// (ddks::order_key's mapping, -0.0 like +0.0), and back.
template <typename V> struct NativeKey;
template <> struct NativeKey<float> {
  using K = uint32_t;
  static DDKS_DEV K key(float v) { return (K)ddks::order_key(v); }
  static DDKS_DEV float value(K k) { return __uint_as_float((k >> 31) ? (k & 0x7FFFFFFFu) : ~k); }
};
template <> struct NativeKey<double> {
  using K = ull;
  static DDKS_DEV K key(double v) { return (K)ddks::order_key(v); }
  static DDKS_DEV double value(K k) { return key_value(k); }
};

// Voxel coordinate of value v in a dimension of range [lo, lo + span]:
// floor(x' * V) with x' = (v - lo) / span, the last voxel for x' = 1.
DDKS_DEV int voxel_coord(double v, double lo, double span, int Vd) {
  const double x = rescale(v, lo, span);
  const int c = (int)floor(__dmul_rn(x, (double)Vd));
  return c > Vd - 1 ? Vd - 1 : (c < 0 ? 0 : c);
}

DDKS_DEV bool better(ull an, long long ac, int aj, ull bn, long long bc, int bj) {
  return an > bn || (an == bn && (ac < bc || (ac == bc && aj < bj)));
}

// Arg-max of (num, index, code) over the CTA: largest num, then lowest index,
// then lowest code.  Valid in thread 0; every thread of the CTA must call it.
DDKS_DEV void block_best(ull& n, long long& c, int& j) {
  __shared__ ull sn[kThreads / 32];
  __shared__ long long sc[kThreads / 32];
  __shared__ int sj[kThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  for (int off = 16; off > 0; off >>= 1) {
    const ull on = __shfl_down_sync(0xffffffffu, n, off);
    const long long oc = __shfl_down_sync(0xffffffffu, c, off);
    const int oj = __shfl_down_sync(0xffffffffu, j, off);
    if (lane + off < 32 && better(on, oc, oj, n, c, j)) { n = on; c = oc; j = oj; }
  }
  if (lane == 0) { sn[warp] = n; sc[warp] = c; sj[warp] = j; }
  __syncthreads();
  if (warp == 0) {
    n = lane < nw ? sn[lane] : 0ull;
    c = lane < nw ? sc[lane] : LLONG_MAX;
    j = lane < nw ? sj[lane] : INT_MAX;
    for (int off = 16; off > 0; off >>= 1) {
      const ull on = __shfl_down_sync(0xffffffffu, n, off);
      const long long oc = __shfl_down_sync(0xffffffffu, c, off);
      const int oj = __shfl_down_sync(0xffffffffu, j, off);
      if (lane + off < 32 && better(on, oc, oj, n, c, j)) { n = on; c = oc; j = oj; }
    }
  }
}

// Per-dimension minimum and maximum of the pooled sample (the range
// NormalizeData rescales by), reduced as order keys of the input type and
// stored as order keys of doubles.  Thread tid reads elements tid, tid + S,
// ... of the pooled row-major array, S a multiple of d, so all of them lie in
// dimension tid mod d.  gmin / gmax start at ~0 / 0.  NaN and infinite
// coordinates raise kFlagNaN / kFlagRange.
template <typename V>
__global__ void __launch_bounds__(kThreads)
k_minmax(const V* __restrict__ P, const V* __restrict__ T, int64_t NP, int64_t NT, int d,
         ull* __restrict__ gmin, ull* __restrict__ gmax, unsigned* __restrict__ flags) {
  using NK = NativeKey<V>;
  using K = typename NK::K;
  extern __shared__ __align__(16) unsigned char smm_raw[];
  K* smin = reinterpret_cast<K*>(smm_raw);  // [2][d]
  K* smax = smin + d;
  for (int m = threadIdx.x; m < d; m += blockDim.x) { smin[m] = ~(K)0; smax[m] = (K)0; }
  __syncthreads();
  const int64_t nP = NP * d, total = (NP + NT) * d;
  const int64_t S = ((int64_t)gridDim.x * blockDim.x / d) * d;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid < S && tid < total) {
    K lo = ~(K)0, hi = (K)0;
    unsigned bad = 0;
    for (int64_t e = tid; e < total; e += S) {
      const V v = e < nP ? P[e] : T[e - nP];
      if (v != v) bad |= ddks::kFlagNaN;
      else if (isinf(v)) bad |= ddks::kFlagRange;
      const K k = NK::key(v);
      lo = k < lo ? k : lo;
      hi = k > hi ? k : hi;
    }
    const int m = (int)(tid % d);
    atomicMin(&smin[m], lo);
    atomicMax(&smax[m], hi);
    if (bad) atomicOr(flags, bad);
  }
  __syncthreads();
  for (int m = threadIdx.x; m < d; m += blockDim.x)
    if (smin[m] != ~(K)0) {
      atomicMin(&gmin[m], (ull)ddks::order_key((double)NK::value(smin[m])));
      atomicMax(&gmax[m], (ull)ddks::order_key((double)NK::value(smax[m])));
    }
}

// CTA 0 flags a range hi - lo that overflows to infinity.
DDKS_DEV void check_spans(const ull* gmin, const ull* gmax, int d, unsigned* flags) {
  if (blockIdx.x != 0) return;
  for (int m = threadIdx.x; m < d; m += blockDim.x)
    if (isinf(__dsub_rn(key_value(gmax[m]), key_value(gmin[m])))) atomicOr(flags, ddks::kFlagRange);
}

// ------------------------------------------------------------------ vdKS

// Threshold path of the voxel step.  A point's voxel coordinate in dimension
// m is a non-decreasing step function of its value (every operation of the
// rescaling is monotone), so it equals the number of thresholds t_k <= v,
// t_k = the least value of the input type with coordinate >= k, k = 1..V-1.
// Thread (m, k) finds t_k by bisection over the input type's order keys in
// [key(lo), key(hi)] with the exact double arithmetic of voxel_coord;
// thr[m * (V - 1) + k - 1] = key(t_k), or ~0 (never reached) for a constant
// dimension.
template <typename V>
__global__ void __launch_bounds__(kThreads)
k_vdks_thresholds(const ull* __restrict__ gmin, const ull* __restrict__ gmax, int d, int Vd,
                  typename NativeKey<V>::K* __restrict__ thr) {
  using NK = NativeKey<V>;
  using K = typename NK::K;
  const int per = Vd - 1;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= d * per) return;
  const int m = t / per, k = t - m * per + 1;
  const double lo = key_value(gmin[m]), hi = key_value(gmax[m]);
  const double span = __dsub_rn(hi, lo);
  K res = ~(K)0;
  if (span > 0.0 && !isinf(span)) {
    K a = NK::key((V)lo), b = NK::key((V)hi);  // the coordinate of hi is V - 1 >= k
    while (a < b) {
      const K mid = a + (b - a) / 2;
      if (voxel_coord((double)NK::value(mid), lo, span, Vd) >= k) b = mid; else a = mid + 1;
    }
    res = a;
  }
  thr[t] = res;
}

// Voxel of every pooled point; cnt[2 * voxel + (point is in T)] += 1.
// use_thr: coordinates from the thresholds (staged in shared memory, a binary
// search of integer keys per dimension); else from the double rescaling.
template <typename V>
__global__ void __launch_bounds__(kThreads)
k_vdks_voxel(const V* __restrict__ P, const V* __restrict__ T, int64_t NP, int64_t NT, int d, int Vd,
             const ull* __restrict__ gmin, const ull* __restrict__ gmax,
             const typename NativeKey<V>::K* __restrict__ thr, int use_thr, uint32_t* __restrict__ cnt,
             unsigned* __restrict__ flags) {
  using NK = NativeKey<V>;
  using K = typename NK::K;
  extern __shared__ __align__(16) unsigned char vox_raw[];
  K* sthr = reinterpret_cast<K*>(vox_raw);  // [d][V - 1] on the threshold path
  __shared__ double slo[kVdksMaxD], sspan[kVdksMaxD];
  const int per = Vd - 1;
  if (threadIdx.x < d) {
    const double lo = key_value(gmin[threadIdx.x]);
    slo[threadIdx.x] = lo;
    sspan[threadIdx.x] = __dsub_rn(key_value(gmax[threadIdx.x]), lo);
  }
  if (use_thr)
    for (int t = threadIdx.x; t < d * per; t += blockDim.x) sthr[t] = thr[t];
  check_spans(gmin, gmax, d, flags);
  __syncthreads();
  const int64_t N = NP + NT;
  const int lane = threadIdx.x & 31;
  // warp-uniform loop: every lane reaches the match, invalid ones with a key
  // no voxel has
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x - lane; b < N;
       b += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = b + lane;
    uint32_t key = 0xFFFFFFFFu;
    if (i < N) {
      const V* row = point_row(P, T, NP, d, i);
      uint32_t idx = 0, stride = 1;
#pragma unroll
      for (int m = 0; m < kVdksMaxD; ++m) {
        if (m < d) {
          int c;
          if (use_thr) {
            const K kv = NK::key(row[m]);
            const K* tm = sthr + m * per;
            int a = 0, z = per;
            while (a < z) {
              const int mid = (a + z) >> 1;
              if (tm[mid] <= kv) a = mid + 1; else z = mid;
            }
            c = a;
          } else {
            c = voxel_coord((double)row[m], slo[m], sspan[m], Vd);
          }
          idx += (uint32_t)c * stride;
          stride *= (uint32_t)Vd;
        }
      }
      key = 2u * idx + (i >= NP ? 1u : 0u);
    }
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    if (i < N && lane == __ffs(peers) - 1) atomicAdd(&cnt[key], (uint32_t)__popc(peers));
  }
}

// Suffix sums along dimension 0 (lines of Vd consecutive voxels), one warp
// per line, forming the differences nT*NP - nP*NT from the counts.
__global__ void __launch_bounds__(kThreads)
k_vdks_suffix0(const uint32_t* __restrict__ cnt, long long* __restrict__ U, uint32_t lines, int Vd,
               long long NP, long long NT) {
  const int lane = threadIdx.x & 31;
  const uint32_t w0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t l = w0; l < lines; l += nw) {
    const uint64_t base = (uint64_t)l * Vd;
    long long carry = 0;
    for (int j0 = Vd - 32; j0 > -32; j0 -= 32) {
      const int j = j0 + lane;
      long long v = 0;
      if (j >= 0) {
        const uint64_t a = base + (uint64_t)j;
        v = (long long)cnt[2 * a + 1] * NP - (long long)cnt[2 * a] * NT;
      }
      for (int off = 1; off < 32; off <<= 1) {
        const long long o = __shfl_down_sync(0xffffffffu, v, off);
        if (lane + off < 32) v += o;
      }
      v += carry;
      if (j >= 0) U[base + (uint64_t)j] = v;
      carry = __shfl_sync(0xffffffffu, v, 0);
    }
  }
}

// Suffix sums along a dimension with stride `inner` (= Vd^m, m >= 1), one
// thread per line.
__global__ void __launch_bounds__(kThreads)
k_vdks_suffix(long long* __restrict__ U, uint32_t lines, int Vd, uint32_t inner) {
  for (uint32_t l = blockIdx.x * blockDim.x + threadIdx.x; l < lines; l += gridDim.x * blockDim.x) {
    const uint32_t lo = l % inner, hi = l / inner;
    const uint64_t base = (uint64_t)hi * inner * (uint64_t)Vd + lo;
    long long acc = 0;
    for (int j = Vd - 1; j >= 0; --j) {
      const uint64_t a = base + (uint64_t)j * inner;
      acc += U[a];
      U[a] = acc;
    }
  }
}

// Orthant sums at the filled voxels.  d <= 5: groups of 2^d lanes per voxel,
// lane = subset; d > 5: a warp per voxel, lane = the subset's low 5 bits and
// register k = its high bits (R = 2^(d-5) registers).
template <int R>
__global__ void __launch_bounds__(kThreads)
k_vdks_eval(const long long* __restrict__ U, const uint32_t* __restrict__ cnt, uint32_t cells, int d,
            int Vd, ull* __restrict__ part_n, long long* __restrict__ part_c, int* __restrict__ part_j,
            unsigned* __restrict__ ticket, ull* __restrict__ out3) {
  const int lane = threadIdx.x & 31;
  const int dl = d < 5 ? d : 5;
  const int sub = lane & ((1 << dl) - 1);
  const int slot = lane >> dl;
  const uint32_t cpw = 32u >> dl;
  ull bn = 0;
  long long bc = LLONG_MAX;
  int bj = INT_MAX;
  const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  for (uint64_t base = (uint64_t)gw * cpw; base < cells; base += (uint64_t)nw * cpw) {
    const uint64_t c = base + slot;
    const bool in = c < cells;
    const bool filled = in && (cnt[2 * c] | cnt[2 * c + 1]) != 0u;
    uint32_t off[kVdksMaxD];
    uint32_t r = in ? (uint32_t)c : 0u, pw = 1;
#pragma unroll
    for (int m = 0; m < kVdksMaxD; ++m) {
      off[m] = 0;
      if (m < d) {
        const uint32_t q = r / (uint32_t)Vd;
        off[m] = (r - q * (uint32_t)Vd) * pw;
        r = q;
        pw *= (uint32_t)Vd;
      }
    }
    long long val[R];
#pragma unroll
    for (int k = 0; k < R; ++k) {
      const int A = sub | (k << 5);
      uint32_t idx = 0;
#pragma unroll
      for (int m = 0; m < kVdksMaxD; ++m)
        if (m < d && ((A >> m) & 1)) idx += off[m];
      val[k] = filled ? U[idx] : 0;
    }
    // F(A) - F(A u {m}) for every A without m, over the register dimensions ...
#pragma unroll
    for (int b = 1; b < R; b <<= 1)
#pragma unroll
      for (int k = 0; k < R; ++k)
        if (!(k & b)) val[k] -= val[k | b];
    // ... and over the lane dimensions
    for (int m = 0; m < dl; ++m) {
#pragma unroll
      for (int k = 0; k < R; ++k) {
        const long long o = __shfl_xor_sync(0xffffffffu, val[k], 1 << m);
        if (!((sub >> m) & 1)) val[k] -= o;
      }
    }
    if (filled) {
#pragma unroll
      for (int k = 0; k < R; ++k) {
        const ull a = (ull)(val[k] < 0 ? -val[k] : val[k]);
        const int code = sub | (k << 5);
        if (better(a, (long long)c, code, bn, bc, bj)) { bn = a; bc = (long long)c; bj = code; }
      }
    }
  }
  block_best(bn, bc, bj);
  __shared__ bool last;
  if (threadIdx.x == 0) {
    part_n[blockIdx.x] = bn;
    part_c[blockIdx.x] = bc;
    part_j[blockIdx.x] = bj;
    __threadfence();
    last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  ull n = 0;
  long long cc = LLONG_MAX;
  int j = INT_MAX;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
    const ull pn = __ldcg(part_n + b);
    const long long pc = __ldcg(part_c + b);
    const int pj = __ldcg(part_j + b);
    if (better(pn, pc, pj, n, cc, j)) { n = pn; cc = pc; j = pj; }
  }
  block_best(n, cc, j);
  if (threadIdx.x == 0) {
    out3[0] = n;
    out3[1] = (ull)cc;
    out3[2] = (ull)(unsigned)j;
    *ticket = 0u;
  }
}

// ------------------------------------------------------------------ rdKS

DDKS_DEV ull dist_key(double s) { return (ull)__double_as_longlong(s); }  // s >= +0: bits are ordered

// One thread per point, all d + 1 corners (d <= kRdksThreadMaxD).
template <typename V>
__global__ void __launch_bounds__(kThreads)
k_rdks_dist_thread(const V* __restrict__ P, const V* __restrict__ T, int64_t NP, int64_t NT, int d,
                   const ull* __restrict__ gmin, const ull* __restrict__ gmax, ull* __restrict__ keys,
                   unsigned* __restrict__ flags) {
  __shared__ double slo[kRdksThreadMaxD], sspan[kRdksThreadMaxD];
  if (threadIdx.x < d) {
    const double lo = key_value(gmin[threadIdx.x]);
    slo[threadIdx.x] = lo;
    sspan[threadIdx.x] = __dsub_rn(key_value(gmax[threadIdx.x]), lo);
  }
  check_spans(gmin, gmax, d, flags);
  __syncthreads();
  const int64_t N = NP + NT;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const V* row = point_row(P, T, NP, d, i);
    double x[kRdksThreadMaxD], q[kRdksThreadMaxD];
#pragma unroll
    for (int m = 0; m < kRdksThreadMaxD; ++m) {
      x[m] = 0.0;
      q[m] = 0.0;
      if (m < d) {
        x[m] = rescale((double)row[m], slo[m], sspan[m]);
        q[m] = __dmul_rn(x[m], x[m]);
      }
    }
    double pre = 0.0;  // sum of q[0..m) in dimension order
#pragma unroll
    for (int m = 0; m < kRdksThreadMaxD; ++m) {
      if (m < d) {
        const double t = __dsub_rn(x[m], 1.0);
        double s = __dadd_rn(pre, __dmul_rn(t, t));
#pragma unroll
        for (int mm = m + 1; mm < kRdksThreadMaxD; ++mm)
          if (mm < d) s = __dadd_rn(s, q[mm]);
        keys[(int64_t)(m + 1) * N + i] = dist_key(s);
        pre = __dadd_rn(pre, q[m]);
      }
    }
    keys[i] = dist_key(pre);
  }
}

// One warp per point (any d): lanes rescale and square the coordinates into
// shared memory, lane 0 forms the running sums, lanes take one corner each.
template <typename V>
__global__ void __launch_bounds__(kThreads)
k_rdks_dist_warp(const V* __restrict__ P, const V* __restrict__ T, int64_t NP, int64_t NT, int d,
                 const ull* __restrict__ gmin, const ull* __restrict__ gmax, ull* __restrict__ keys,
                 unsigned* __restrict__ flags) {
  extern __shared__ double sd[];  // per warp: x'[d], x'^2[d], running sums[d]
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nwb = blockDim.x >> 5;
  double* xs = sd + (size_t)w * 3 * d;
  double* q = xs + d;
  double* pre = q + d;
  check_spans(gmin, gmax, d, flags);
  const int64_t N = NP + NT;
  for (int64_t i = (int64_t)blockIdx.x * nwb + w; i < N; i += (int64_t)gridDim.x * nwb) {
    const V* row = point_row(P, T, NP, d, i);
    for (int m = lane; m < d; m += 32) {
      const double lo = key_value(gmin[m]);
      const double x = rescale((double)row[m], lo, __dsub_rn(key_value(gmax[m]), lo));
      xs[m] = x;
      q[m] = __dmul_rn(x, x);
    }
    __syncwarp();
    if (lane == 0) {
      double s = 0.0;
      for (int m = 0; m < d; ++m) {
        pre[m] = s;
        s = __dadd_rn(s, q[m]);
      }
      keys[i] = dist_key(s);
    }
    __syncwarp();
    for (int m = lane; m < d; m += 32) {
      const double t = __dsub_rn(xs[m], 1.0);
      double s = __dadd_rn(pre[m], __dmul_rn(t, t));
      for (int mm = m + 1; mm < d; ++mm) s = __dadd_rn(s, q[mm]);
      keys[(int64_t)(m + 1) * N + i] = dist_key(s);
    }
    __syncwarp();
  }
}

// grid (x, S): corner blockIdx.y.  K, I, Pf are the sorted segments [S][Npad].
__global__ void __launch_bounds__(kThreads)
k_rdks_walk(const ull* __restrict__ K, const uint32_t* __restrict__ I, const uint32_t* __restrict__ Pf,
            int64_t N, int64_t Npad, int64_t NP, int64_t NT, ull* __restrict__ per_corner) {
  const int64_t s = blockIdx.y;
  const ull* Ks = K + s * Npad;
  const uint32_t* Is = I + s * Npad;
  const uint32_t* Ps = Pf + s * Npad;
  ull best = 0;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (int64_t)gridDim.x * blockDim.x) {
    if (p == N - 1 || Ks[p + 1] != Ks[p]) {
      const uint64_t cp = (uint64_t)Ps[p] + (Is[p] < (uint64_t)NP ? 1u : 0u);
      const uint64_t ct = (uint64_t)p + 1 - cp;
      const ull v = ddks::numer(cp, ct, (uint64_t)NP, (uint64_t)NT);
      best = v > best ? v : best;
    }
  }
  for (int off = 16; off > 0; off >>= 1) {
    const ull o = __shfl_down_sync(0xffffffffu, best, off);
    best = o > best ? o : best;
  }
  if ((threadIdx.x & 31) == 0 && best) atomicMax(per_corner + s, best);
}

__global__ void __launch_bounds__(kThreads)
k_rdks_final(const ull* __restrict__ per_corner, int S, ull* __restrict__ out3) {
  ull n = 0;
  long long c = LLONG_MAX;
  int j = 0;
  for (int s = threadIdx.x; s < S; s += blockDim.x)
    if (better(per_corner[s], s, 0, n, c, 0)) { n = per_corner[s]; c = s; }
  block_best(n, c, j);
  if (threadIdx.x == 0) {
    out3[0] = n;
    out3[1] = (ull)c;
    out3[2] = 0;
  }
}

// ------------------------------------------------------------------ host

int grid_cap(int64_t work, int per_block, int cap) {
  int64_t g = (work + per_block - 1) / per_block;
  if (g > cap) g = cap;
  return (int)(g < 1 ? 1 : g);
}

// Offsets into ctx->apx_small: out3 (4 u64), flags and ticket (u32), the
// per-dimension min / max keys, then per-corner maxima or eval partials.
struct SmallLayout {
  size_t flags = 32, ticket = 36, gmin = 64, gmax = 0, tail = 0, bytes = 0;
  SmallLayout(int d, size_t tail_bytes) {
    gmax = gmin + 8 * (size_t)d;
    tail = (gmax + 8 * (size_t)d + 15) & ~(size_t)15;
    bytes = tail + tail_bytes;
  }
};

int map_flags(ddks_ctx* ctx, unsigned flags) {
  (void)ctx;
  if (flags & ddks::kFlagNaN) return DDKS_ENAN;
  if (flags & ddks::kFlagRange) return DDKS_EINVAL;
  return DDKS_OK;
}

template <typename V>
cudaError_t launch_minmax(const void* P, const void* T, int64_t NP, int64_t NT, int d, ull* gmin, ull* gmax,
                          unsigned* flags, int num_sms, cudaStream_t st) {
  const int64_t total = (NP + NT) * d;
  int g = grid_cap(total, kThreads, num_sms * 8);
  const int need = (d + kThreads - 1) / kThreads;  // at least d threads
  if (g < need) g = need;
  const size_t smem = 2 * sizeof(typename NativeKey<V>::K) * (size_t)d;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_minmax<V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_minmax<V><<<g, kThreads, smem, st>>>((const V*)P, (const V*)T, NP, NT, d, gmin, gmax, flags);
  return cudaGetLastError();
}

template <int R>
cudaError_t launch_eval(const long long* U, const uint32_t* cnt, uint32_t cells, int d, int Vd, ull* part_n,
                        long long* part_c, int* part_j, unsigned* ticket, ull* out3, int blocks,
                        cudaStream_t st) {
  k_vdks_eval<R><<<blocks, kThreads, 0, st>>>(U, cnt, cells, d, Vd, part_n, part_c, part_j, ticket, out3);
  return cudaGetLastError();
}

int vdks_blocks(ddks_ctx* ctx, uint32_t cells, int d) {
  const int dl = d < 5 ? d : 5;
  const int64_t warps = ((int64_t)cells + (32 >> dl) - 1) / (32 >> dl);
  return grid_cap(warps, kThreads / 32, ctx->num_sms * 8);
}

int finish(ddks_ctx* ctx, cudaStream_t st, const SmallLayout& L, int64_t NP, int64_t NT, ddks_result* out,
           uint64_t* extra, const void* extra_src, size_t extra_bytes) {
  cudaError_t e = cudaMemcpyAsync(ctx->h_out, ctx->apx_small.ptr, 3 * sizeof(ull), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ctx->h_out + 4, (char*)ctx->apx_small.ptr + L.flags, sizeof(unsigned),
                        cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && extra) e = cudaMemcpyAsync(extra, extra_src, extra_bytes, cudaMemcpyDefault, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return out->status = ctx_cuda_fail(ctx, e, "result copy");
  ddks_stage_collect(ctx);
  const int rc = map_flags(ctx, (unsigned)(ctx->h_out[4] & 0xFFFFFFFFull));
  if (rc) return out->status = rc;
  out->num_max = ctx->h_out[0];
  out->denom = (uint64_t)NP * (uint64_t)NT;
  out->D = (double)out->num_max / (double)out->denom;
  out->argmax_origin = (int64_t)ctx->h_out[1];
  out->argmax_orthant = (int32_t)ctx->h_out[2];
  out->status = DDKS_OK;
  return DDKS_OK;
}

}  // namespace

int ddks_vdks(ddks_ctx* ctx, const void* P, int64_t NP, const void* T, int64_t NT, int32_t d,
              int32_t dtype, int32_t voxels_per_dim, void* stream, ddks_result* out) {
  if (!ctx || !out) return DDKS_EINVAL;
  int rc = ddks_check_problem(P, NP, T, NT, d, dtype);
  if (rc) return out->status = rc;
  const int Vd = voxels_per_dim;
  if (Vd < 1) return out->status = DDKS_EINVAL;
  if (d > kVdksMaxD) return out->status = DDKS_EUNSUPPORTED;
  uint64_t cells64 = 1;
  for (int m = 0; m < d; ++m) {
    cells64 *= (uint64_t)Vd;
    if (cells64 > kVdksMaxCells) return out->status = DDKS_EUNSUPPORTED;
  }
  const uint32_t cells = (uint32_t)cells64;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return out->status = ctx_cuda_fail(ctx, e, "cudaSetDevice");
  const void *dP, *dT;
  if ((rc = ddks_stage_inputs(ctx, P, NP, T, NT, d, dtype, st, &dP, &dT))) return out->status = rc;
  const int blocks = vdks_blocks(ctx, cells, d);
  // the threshold path of the voxel step when its thresholds fit shared
  // memory and cost much less than rescaling every point in double
  const int64_t nthr_all = (int64_t)d * (Vd - 1);
  const bool use_thr = nthr_all <= kVdksMaxThresholds && (int64_t)(Vd - 1) * 64 <= NP + NT;
  const SmallLayout L(d, (((size_t)blocks * 20 + 15) & ~(size_t)15) + 8 * (size_t)nthr_all);
  if ((rc = ctx->apx_small.reserve(ctx, L.bytes))) return out->status = rc;
  if ((rc = ctx->apx_cnt.reserve(ctx, 8 * (size_t)cells))) return out->status = rc;
  if ((rc = ctx->apx_U.reserve(ctx, 8 * (size_t)cells))) return out->status = rc;
  GraphKey key;
  key.add(7).add((uint64_t)NP).add((uint64_t)NT).add((uint64_t)d).add((uint64_t)dtype).add((uint64_t)Vd);
  key.add((uint64_t)use_thr).add((uint64_t)ctx->stage_timing);
  key.add_ptr(dP).add_ptr(dT);
  rc = ddks_graph_run(ctx, key.h, st, [&](cudaStream_t s) -> int {
    char* sm = (char*)ctx->apx_small.ptr;
    ull* gmin = (ull*)(sm + L.gmin);
    ull* gmax = (ull*)(sm + L.gmax);
    unsigned* flags = (unsigned*)(sm + L.flags);
    unsigned* ticket = (unsigned*)(sm + L.ticket);
    ull* part_n = (ull*)(sm + L.tail);
    long long* part_c = (long long*)(part_n + blocks);
    int* part_j = (int*)(part_c + blocks);
    void* thr = (void*)(sm + L.tail + (((size_t)blocks * 20 + 15) & ~(size_t)15));
    uint32_t* cnt = (uint32_t*)ctx->apx_cnt.ptr;
    long long* U = (long long*)ctx->apx_U.ptr;
    cudaError_t ee = cudaMemsetAsync(sm + L.flags, 0, 8, s);
    if (ee == cudaSuccess) ee = cudaMemsetAsync(gmin, 0xFF, 8 * (size_t)d, s);
    if (ee == cudaSuccess) ee = cudaMemsetAsync(gmax, 0, 8 * (size_t)d, s);
    if (ee == cudaSuccess) ee = cudaMemsetAsync(cnt, 0, 8 * (size_t)cells, s);
    if (ee != cudaSuccess) return ctx_cuda_fail(ctx, ee, "vdks memset");
    ddks_stage_mark(ctx, 0, s);
    const bool f64 = dtype == DDKS_F64;
    ee = f64 ? launch_minmax<double>(dP, dT, NP, NT, d, gmin, gmax, flags, ctx->num_sms, s)
             : launch_minmax<float>(dP, dT, NP, NT, d, gmin, gmax, flags, ctx->num_sms, s);
    if (ee != cudaSuccess) return ctx_cuda_fail(ctx, ee, "vdks range");
    ddks_stage_mark(ctx, 1, s);
    const int gv = grid_cap(NP + NT, kThreads, ctx->num_sms * 8);
    const int nthr = d * (Vd - 1);
    const size_t ks = f64 ? 8 : 4;
    if (use_thr && nthr > 0) {
      const int gt = (nthr + kThreads - 1) / kThreads;
      if (f64)
        k_vdks_thresholds<double><<<gt, kThreads, 0, s>>>(gmin, gmax, d, Vd, (ull*)thr);
      else
        k_vdks_thresholds<float><<<gt, kThreads, 0, s>>>(gmin, gmax, d, Vd, (uint32_t*)thr);
      ctx->launches += 1;
    }
    const size_t vsm = use_thr ? ks * (size_t)nthr : 0;
    if (f64)
      k_vdks_voxel<double><<<gv, kThreads, vsm, s>>>((const double*)dP, (const double*)dT, NP, NT, d, Vd, gmin,
                                                     gmax, (const ull*)thr, use_thr ? 1 : 0, cnt, flags);
    else
      k_vdks_voxel<float><<<gv, kThreads, vsm, s>>>((const float*)dP, (const float*)dT, NP, NT, d, Vd, gmin,
                                                    gmax, (const uint32_t*)thr, use_thr ? 1 : 0, cnt, flags);
    ddks_stage_mark(ctx, 2, s);
    const uint32_t lines = cells / (uint32_t)Vd;
    k_vdks_suffix0<<<grid_cap(lines, kThreads / 32, ctx->num_sms * 8), kThreads, 0, s>>>(cnt, U, lines, Vd,
                                                                                        NP, NT);
    uint32_t inner = (uint32_t)Vd;
    for (int m = 1; m < d; ++m, inner *= (uint32_t)Vd)
      k_vdks_suffix<<<grid_cap(lines, kThreads, ctx->num_sms * 8), kThreads, 0, s>>>(U, lines, Vd, inner);
    ctx->launches += 3 + (d - 1) + 1;
    ull* out3 = (ull*)sm;
    switch (d <= 5 ? 0 : d - 5) {
      case 0: ee = launch_eval<1>(U, cnt, cells, d, Vd, part_n, part_c, part_j, ticket, out3, blocks, s); break;
      case 1: ee = launch_eval<2>(U, cnt, cells, d, Vd, part_n, part_c, part_j, ticket, out3, blocks, s); break;
      case 2: ee = launch_eval<4>(U, cnt, cells, d, Vd, part_n, part_c, part_j, ticket, out3, blocks, s); break;
      case 3: ee = launch_eval<8>(U, cnt, cells, d, Vd, part_n, part_c, part_j, ticket, out3, blocks, s); break;
      case 4: ee = launch_eval<16>(U, cnt, cells, d, Vd, part_n, part_c, part_j, ticket, out3, blocks, s); break;
      default: ee = launch_eval<32>(U, cnt, cells, d, Vd, part_n, part_c, part_j, ticket, out3, blocks, s); break;
    }
    if (ee != cudaSuccess) return ctx_cuda_fail(ctx, ee, "vdks kernels");
    ddks_stage_mark(ctx, 3, s);
    return DDKS_OK;
  });
  if (rc) return out->status = rc;
  return finish(ctx, st, L, NP, NT, out, nullptr, nullptr, 0);
}

int ddks_rdks(ddks_ctx* ctx, const void* P, int64_t NP, const void* T, int64_t NT, int32_t d,
              int32_t dtype, void* stream, ddks_result* out, uint64_t* per_corner) {
  if (!ctx || !out) return DDKS_EINVAL;
  if (d < 1 || d > DDKS_RDKS_MAX_D) return out->status = DDKS_EINVAL;
  int rc = ddks_check_problem(P, NP, T, NT, 1, dtype);
  if (rc) return out->status = rc;
  const int64_t N = NP + NT;
  const int S = d + 1;
  const int64_t Npad = (int64_t)ddks_rank_scratch_elems(N);
  if ((double)S * (double)Npad >= 4.0e9) return out->status = DDKS_EOVERFLOW;  // u32 positions per buffer
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return out->status = ctx_cuda_fail(ctx, e, "cudaSetDevice");
  const void *dP, *dT;
  if ((rc = ddks_stage_inputs(ctx, P, NP, T, NT, d, dtype, st, &dP, &dT))) return out->status = rc;
  const SmallLayout L(d, 8 * (size_t)S);
  const size_t segs = (size_t)S * (size_t)Npad;
  if ((rc = ctx->apx_small.reserve(ctx, L.bytes))) return out->status = rc;
  if ((rc = ctx->keys.reserve(ctx, 8 * (size_t)S * (size_t)N))) return out->status = rc;
  if ((rc = ctx->tk1.reserve(ctx, 8 * segs))) return out->status = rc;
  if ((rc = ctx->tk2.reserve(ctx, 8 * segs))) return out->status = rc;
  if ((rc = ctx->ti1.reserve(ctx, 4 * segs))) return out->status = rc;
  if ((rc = ctx->ti2.reserve(ctx, 4 * segs))) return out->status = rc;
  if ((rc = ctx->apx_cnt.reserve(ctx, 4 * segs))) return out->status = rc;  // P prefixes
  if ((rc = ctx->apx_U.reserve(ctx, 4 * segs))) return out->status = rc;
  // warp kernel: shared memory of 3 * d doubles per warp
  int nwb = 1;
  if (d > kRdksThreadMaxD) {
    nwb = (int)((200 * 1024) / (24 * (size_t)d));
    nwb = nwb < 1 ? 1 : (nwb > kThreads / 32 ? kThreads / 32 : nwb);
  }
  GraphKey key;
  key.add(8).add((uint64_t)NP).add((uint64_t)NT).add((uint64_t)d).add((uint64_t)dtype);
  key.add_ptr(dP).add_ptr(dT).add((uint64_t)ctx->stage_timing);
  rc = ddks_graph_run(ctx, key.h, st, [&](cudaStream_t s) -> int {
    char* sm = (char*)ctx->apx_small.ptr;
    ull* gmin = (ull*)(sm + L.gmin);
    ull* gmax = (ull*)(sm + L.gmax);
    unsigned* flags = (unsigned*)(sm + L.flags);
    ull* pc = (ull*)(sm + L.tail);
    ull* keys = (ull*)ctx->keys.ptr;
    cudaError_t ee = cudaMemsetAsync(sm + L.flags, 0, 8, s);
    if (ee == cudaSuccess) ee = cudaMemsetAsync(gmin, 0xFF, 8 * (size_t)d, s);
    if (ee == cudaSuccess) ee = cudaMemsetAsync(gmax, 0, 8 * (size_t)d, s);
    if (ee == cudaSuccess) ee = cudaMemsetAsync(pc, 0, 8 * (size_t)S, s);
    if (ee != cudaSuccess) return ctx_cuda_fail(ctx, ee, "rdks memset");
    ddks_stage_mark(ctx, 0, s);
    const bool f64 = dtype == DDKS_F64;
    ee = f64 ? launch_minmax<double>(dP, dT, NP, NT, d, gmin, gmax, flags, ctx->num_sms, s)
             : launch_minmax<float>(dP, dT, NP, NT, d, gmin, gmax, flags, ctx->num_sms, s);
    if (ee != cudaSuccess) return ctx_cuda_fail(ctx, ee, "rdks range");
    if (d <= kRdksThreadMaxD) {
      const int g = grid_cap(N, kThreads, ctx->num_sms * 8);
      if (f64)
        k_rdks_dist_thread<double><<<g, kThreads, 0, s>>>((const double*)dP, (const double*)dT, NP, NT, d,
                                                          gmin, gmax, keys, flags);
      else
        k_rdks_dist_thread<float><<<g, kThreads, 0, s>>>((const float*)dP, (const float*)dT, NP, NT, d, gmin,
                                                         gmax, keys, flags);
    } else {
      const size_t smem = (size_t)nwb * 24 * (size_t)d;
      const int g = grid_cap(N, nwb, ctx->num_sms * 8);
      if (f64) {
        ee = cudaFuncSetAttribute(k_rdks_dist_warp<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (ee == cudaSuccess)
          k_rdks_dist_warp<double><<<g, 32 * nwb, smem, s>>>((const double*)dP, (const double*)dT, NP, NT, d,
                                                             gmin, gmax, keys, flags);
      } else {
        ee = cudaFuncSetAttribute(k_rdks_dist_warp<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (ee == cudaSuccess)
          k_rdks_dist_warp<float><<<g, 32 * nwb, smem, s>>>((const float*)dP, (const float*)dT, NP, NT, d,
                                                            gmin, gmax, keys, flags);
      }
      if (ee != cudaSuccess) return ctx_cuda_fail(ctx, ee, "rdks distance attribute");
    }
    ctx->launches += 2;
    ddks_stage_mark(ctx, 1, s);
    const uint64_t* sk;
    const uint32_t *si, *sp;
    int n = 0;
    ee = ddks_launch_sort_segments((const uint64_t*)keys, N, NP, S, (uint64_t*)ctx->tk1.ptr, (uint32_t*)ctx->ti1.ptr,
                                   (uint32_t*)ctx->apx_cnt.ptr, (uint64_t*)ctx->tk2.ptr, (uint32_t*)ctx->ti2.ptr,
                                   (uint32_t*)ctx->apx_U.ptr, &sk, &si, &sp, s, &n);
    ctx->launches += n;
    if (ee != cudaSuccess) return ctx_cuda_fail(ctx, ee, "rdks sort");
    ddks_stage_mark(ctx, 2, s);
    int gx = grid_cap(N, kThreads, ctx->num_sms * 8);
    const int per = (ctx->num_sms * 8 + S - 1) / S;
    if (gx > per) gx = per < 1 ? 1 : per;
    k_rdks_walk<<<dim3((unsigned)gx, (unsigned)S), kThreads, 0, s>>>((const ull*)sk, si, sp, N, Npad, NP, NT,
                                                                      pc);
    k_rdks_final<<<1, kThreads, 0, s>>>(pc, S, (ull*)sm);
    ctx->launches += 2;
    ee = cudaGetLastError();
    if (ee != cudaSuccess) return ctx_cuda_fail(ctx, ee, "rdks kernels");
    ddks_stage_mark(ctx, 3, s);
    return DDKS_OK;
  });
  if (rc) return out->status = rc;
  rc = finish(ctx, st, L, NP, NT, out, per_corner, (char*)ctx->apx_small.ptr + L.tail, 8 * (size_t)S);
  if (rc == DDKS_OK) out->argmax_orthant = 0;
  return rc;
}
