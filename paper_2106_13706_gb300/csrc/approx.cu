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
//   k_vdks_suffix    d passes of suffix sums: U(c) = sum over the voxels c' with
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
//   k_rdks_dist_*    squared distance of each point to each corner: corner 0
//                    (the origin) is the squared norm s (squares added in
//                    dimension order), corner m + 1 (the unit vector of
//                    dimension m) is (s - 2 x'_m) + 1, so a point costs O(d)
//   sort             the d + 1 corner lists: from 131,072 points the LSD
//                    radix sort of radix.cu (then k_rdks_ptile counts each
//                    tile's P points and k_rdks_walk_tiles walks with in-tile
//                    prefixes), else the K0 chunk sort and merge passes,
//                    carrying the P count before each position
//   k_rdks_walk      at the last position of every run of equal distances:
//                    |cP*NT - cT*NP| of the counts up to and including it
//                    (both empirical CDFs evaluated after the tied values);
//                    max per corner
//   k_rdks_final     max over corners, lowest corner
#include <climits>
#include <cmath>
#include <cstring>

#include "../../include/ddks.h"
#include "bulk_copy.cuh"
#include "ddks_internal.cuh"
#include "ddks_host.h"

namespace {

using ull = unsigned long long;
constexpr int kThreads = 256;
constexpr int kVdksMaxD = DDKS_VDKS_MAX_D;
constexpr int kRdksThreadMaxD = 16;  // up to here one thread computes all corners of a point
constexpr uint64_t kVdksMaxCells = 1ull << 28;
constexpr int64_t kVdksMaxThresholds = 4096;  // d * (V - 1) keys staged in shared memory
constexpr size_t kVdksMaxHistSmem = 200 * 1024;   // private histogram + thresholds per CTA

// Inverse of ddks::order_key for doubles (-0.0 comes back as +0.0).
DDKS_DEV double key_value(ull k) {
  const ull b = (k >> 63) ? (k & 0x7FFFFFFFFFFFFFFFull) : ~k;
  return __longlong_as_double((long long)b);
}

DDKS_DEV double rescale(double v, double lo, double span) {
  return span > 0.0 ? __ddiv_rn(__dsub_rn(v, lo), span) : 0.0;
}

// The same correctly rounded x' = (v - lo) / span with fewer FP64
// instructions (GB300's FP64 rate is low, and the division sequence and
// floating-point compares all issue on that pipe).  rcp = RN(1 / span), or
// 0 for a span outside [2^-900, 2^1000) (division used throughout).
// q0 = RN(a * rcp), one correction q = RN(q0 + r0 * rcp) with the exact
// remainder r0 = a - q0 * span (Markstein's step).  q is returned only when
// certified: with the exact remainder r = a - q * span, q is the nearest
// double to a / span when |r| <= span * g / 2, g the smaller of the gaps
// next to q (a quotient of doubles is never a midpoint, so the nearest double
// is unique).  The range checks and the certificate compare bit patterns of
// non-negative doubles as integers, and span * g / 2 is span with its
// exponent field raised (everything stays normal for a, q0 >= 2^-900).
// Otherwise, or when the certificate fails, the IEEE division.
DDKS_DEV double rescale_rcp(double v, double lo, double span, double rcp) {
  constexpr long long kMinBits = 0x07B0000000000000ll;  // bit pattern of 2^-900
  const double a = __dsub_rn(v, lo);                    // >= +0: lo is the minimum
  const long long ab = __double_as_longlong(a);
  if (ab >= kMinBits && __double_as_longlong(rcp) != 0) {
    const double q0 = __dmul_rn(a, rcp);
    if (__double_as_longlong(q0) >= kMinBits) {
      const double q = __fma_rn(__fma_rn(-q0, span, a), rcp, q0);
      const double r = __fma_rn(-q, span, a);
      const long long qb = __double_as_longlong(q);
      // g / 2 = 2^(E - 53), or 2^(E - 54) when q is a power of two (E its exponent)
      const long long sh = ((qb >> 52) & 0x7FF) - 1023 - ((qb & 0xFFFFFFFFFFFFFll) == 0 ? 54 : 53);
      const long long lim = __double_as_longlong(span) + sh * (1ll << 52);
      if ((__double_as_longlong(r) & 0x7FFFFFFFFFFFFFFFll) <= lim) return q;
    }
  }
  if (ab == 0 || !(span > 0.0)) return 0.0;
  return __ddiv_rn(a, span);
}

// RN(1 / span) for rescale_rcp, or 0 where it takes the division path.
DDKS_DEV double rescale_rcp_of(double span) {
  return (span >= 0x1p-900 && span < 0x1p1000) ? __drcp_rn(span) : 0.0;
}

template <typename V>
DDKS_DEV const V* point_row(const V* P, const V* T, int64_t NP, int d, int64_t i) {
  return i < NP ? P + i * d : T + (i - NP) * d;
}

// Order keys in the input type's own width: u32 for float, u64 for double
// (ddks::order_key's mapping, -0.0 like +0.0), and back.
template <typename V> struct NativeKey;
// raw(v) is the same map without the -0.0 fix (-0.0 just below +0.0): NaNs
// land outside [raw(-inf), raw(+inf)].
template <> struct NativeKey<float> {
  using K = uint32_t;
  static DDKS_DEV K key(float v) { return (K)ddks::order_key(v); }
  static DDKS_DEV K raw(float v) {  // = u ^ (sign ? 0xFFFFFFFF : 0x80000000), two ALU ops
    const int32_t i = __float_as_int(v);
    return (K)(i ^ ((i >> 31) | (int32_t)0x80000000));
  }
  static DDKS_DEV float value(K k) { return __uint_as_float((k >> 31) ? (k & 0x7FFFFFFFu) : ~k); }
};
template <> struct NativeKey<double> {
  using K = ull;
  static DDKS_DEV K key(double v) { return (K)ddks::order_key(v); }
  static DDKS_DEV K raw(double v) {
    const long long i = __double_as_longlong(v);
    return (K)(i ^ ((i >> 63) | (long long)0x8000000000000000ll));
  }
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
// stored as order keys of doubles (an all-zero dimension may come back as
// -0.0, which rescales every coordinate the same way as +0.0).  Each thread
// reads 16-byte vectors of VEC
// consecutive elements at t0, t0 + S, ... of P's and then T's row-major
// array, S a multiple of both d and VEC, so element j of its vectors always
// lies in dimension (t0 + j) mod d.  gmin / gmax start at ~0 / 0.  NaN and
// infinite coordinates raise kFlagNaN / kFlagRange, found from each CTA's
// extreme keys.
template <typename V>
__global__ void __launch_bounds__(kThreads)
k_minmax(const V* __restrict__ P, const V* __restrict__ T, int64_t NP, int64_t NT, int d, int64_t S,
         ull* __restrict__ gmin, ull* __restrict__ gmax, unsigned* __restrict__ flags) {
  using NK = NativeKey<V>;
  using K = typename NK::K;
  constexpr int VEC = 16 / (int)sizeof(V);
  extern __shared__ __align__(16) unsigned char smm_raw[];
  K* smin = reinterpret_cast<K*>(smm_raw);  // [2][d]
  K* smax = smin + d;
  for (int m = threadIdx.x; m < d; m += blockDim.x) { smin[m] = ~(K)0; smax[m] = (K)0; }
  __syncthreads();
  const int64_t t0 = (int64_t)VEC * ((int64_t)blockIdx.x * blockDim.x + threadIdx.x);
  if (t0 < S) {
    K lo[VEC], hi[VEC];
#pragma unroll
    for (int j = 0; j < VEC; ++j) { lo[j] = ~(K)0; hi[j] = (K)0; }
    for (int a = 0; a < 2; ++a) {
      const V* X = a ? T : P;
      const int64_t n = (a ? NT : NP) * d;
      const bool vec_ok = ((uintptr_t)X & 15) == 0;
      constexpr int B = 4;  // vectors whose loads are issued together
      for (int64_t e0 = t0; e0 < n; e0 += (int64_t)B * S) {
        V v[B][VEC];
        int cnt[B];  // elements of each vector inside the array
#pragma unroll
        for (int u = 0; u < B; ++u) {
          const int64_t e = e0 + (int64_t)u * S;
          cnt[u] = e >= n ? 0 : (n - e < VEC ? (int)(n - e) : VEC);
          if (vec_ok && cnt[u] == VEC) {
            if constexpr (VEC == 4) {
              const float4 q = *reinterpret_cast<const float4*>(X + e);
              v[u][0] = q.x; v[u][1] = q.y; v[u][2] = q.z; v[u][3] = q.w;
            } else {
              const double2 q = *reinterpret_cast<const double2*>(X + e);
              v[u][0] = q.x; v[u][1] = q.y;
            }
          } else {
#pragma unroll
            for (int j = 0; j < VEC; ++j) v[u][j] = j < cnt[u] ? X[e + j] : (V)0;
          }
        }
#pragma unroll
        for (int u = 0; u < B; ++u) {
#pragma unroll
          for (int j = 0; j < VEC; ++j) {
            if (j >= cnt[u]) continue;
            const K k = NK::raw(v[u][j]);
            lo[j] = k < lo[j] ? k : lo[j];
            hi[j] = k > hi[j] ? k : hi[j];
          }
        }
      }
    }
#pragma unroll
    for (int j = 0; j < VEC; ++j) {
      if (lo[j] != ~(K)0) {  // element j of some vector was seen
        const int m = (int)((t0 + j) % d);
        atomicMin(&smin[m], lo[j]);
        atomicMax(&smax[m], hi[j]);
      }
    }
  }
  __syncthreads();
  // NaN keys lie outside [raw(-inf), raw(+inf)]; infinities at its ends
  const K kninf = NK::raw(-__int_as_float(0x7f800000)), kpinf = NK::raw(__int_as_float(0x7f800000));
  for (int m = threadIdx.x; m < d; m += blockDim.x)
    if (smin[m] != ~(K)0) {
      if (smin[m] < kninf || smax[m] > kpinf) atomicOr(flags, ddks::kFlagNaN);
      else if (smin[m] == kninf || smax[m] == kpinf) atomicOr(flags, ddks::kFlagRange);
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
// Warp (m, k) finds t_k by a 32-way search over the input type's order keys
// in [key(lo), key(hi)], each lane evaluating voxel_coord (the exact double
// arithmetic) at one probe per round; thr[m * (V - 1) + k - 1] = key(t_k),
// or ~0 (never reached) for a constant dimension.
template <typename V>
__global__ void __launch_bounds__(kThreads)
k_vdks_thresholds(const ull* __restrict__ gmin, const ull* __restrict__ gmax, int d, int Vd,
                  typename NativeKey<V>::K* __restrict__ thr) {
  using NK = NativeKey<V>;
  using K = typename NK::K;
  const int per = Vd - 1;
  const int lane = threadIdx.x & 31;
  const int t = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);  // warp-uniform
  if (t >= d * per) return;
  const int m = t / per, k = t - m * per + 1;
  const double lo = key_value(gmin[m]), hi = key_value(gmax[m]);
  const double span = __dsub_rn(hi, lo);
  K res = ~(K)0;
  if (span > 0.0 && !isinf(span)) {
    // invariant: the answer is in [a, b] and the coordinate of b is >= k
    K a = NK::key((V)lo), b = NK::key((V)hi);
    while (a < b) {
      const K step = (b - a) / 32 + 1;
      const K c = a + (K)lane * step;
      const bool pr = c >= b || voxel_coord((double)NK::value(c), lo, span, Vd) >= k;
      const unsigned bal = __ballot_sync(0xffffffffu, pr);
      const int f = __ffs(bal) - 1;
      if (f < 0) {
        a = a + (K)31 * step + 1;
      } else if (f == 0) {
        b = a;
      } else {
        const K cf = a + (K)f * step;
        a = a + (K)(f - 1) * step + 1;
        b = cf < b ? cf : b;
      }
    }
    res = a;
  }
  if (lane == 0) thr[t] = res;
}

// Thresholds staged in shared memory: per dimension V + 1 slots, slot k
// (1 <= k <= V - 1) holding t_k and sentinels below (slot 0) and above
// (slot V).  Float inputs keep the threshold values (compared as floats,
// -0.0 == +0.0), double inputs their order keys.
template <typename V> struct StagedThr { using T = typename NativeKey<V>::K; };
template <> struct StagedThr<float> { using T = float; };

template <typename V>
DDKS_DEV void stage_thresholds(typename StagedThr<V>::T* sthr, const typename NativeKey<V>::K* thr, int d, int Vd) {
  using S = typename StagedThr<V>::T;
  const int per = Vd - 1, w = Vd + 1;
  for (int t = threadIdx.x; t < d * w; t += blockDim.x) {
    const int m = t / w, k = t - m * w;
    S v;
    if constexpr (sizeof(V) == 4) {
      v = k == 0 ? -__int_as_float(0x7f800000) : (k == Vd ? __int_as_float(0x7f800000)
                                                         : NativeKey<float>::value(thr[m * per + k - 1]));
    } else {
      v = k == 0 ? (S)0 : (k == Vd ? ~(S)0 : thr[m * per + k - 1]);
    }
    sthr[t] = v;
  }
}

// Voxel index sum_m c_m V^m of a point row: from the staged thresholds, or
// from the double rescaling.  DM = d when d <= 4, else an upper bound.
// Float inputs: a single-precision estimate of the coordinate is within one
// of the exact one (its relative error is below 2^-22 and V <= 4096 here), so
// one compare with each neighbouring threshold gives the exact count
// #{k : t_k <= v}.  Double inputs (whose float estimate can be far off) walk
// from the estimate to the count by order-key compares.
template <typename V, int DM>
DDKS_DEV uint32_t voxel_index(const V* row, int d, int Vd, const typename StagedThr<V>::T* sthr, bool use_thr,
                              const double* slo, const double* sspan, const float* flo, const float* fsc) {
  using NK = NativeKey<V>;
  using K = typename NK::K;
  constexpr bool exact = DM <= 4;
  const int per = Vd - 1, w = Vd + 1;
  uint32_t idx = 0, stride = 1;
#pragma unroll
  for (int m = 0; m < DM; ++m) {
    if (exact || m < d) {
      int c;
      if (use_thr) {
        const V v = row[m];
        const float e = fminf(fmaxf(((float)v - flo[m]) * fsc[m], 0.0f), (float)per);
        const int c0 = (int)e;
        const typename StagedThr<V>::T* tm = sthr + m * w;
        if constexpr (sizeof(V) == 4) {
          c = c0 + (v >= tm[c0 + 1] ? 1 : 0) - (v < tm[c0] ? 1 : 0);
          c = c < 0 ? 0 : (c > per ? per : c);
        } else {
          const K kv = NK::key(v);
          c = c0;
          while (c < per && tm[c + 1] <= kv) ++c;
          while (c > 0 && tm[c] > kv) --c;
        }
      } else {
        c = voxel_coord((double)row[m], slo[m], sspan[m], Vd);
      }
      idx += (uint32_t)c * stride;
      stride *= (uint32_t)Vd;
    }
  }
  return idx;
}

// Voxel of every pooled point; cnt[2 * voxel + (point is in T)] += 1.
// use_thr: coordinates from the thresholds (staged in shared memory); else
// from the double rescaling.
template <typename V>
__global__ void __launch_bounds__(kThreads)
k_vdks_voxel(const V* __restrict__ P, const V* __restrict__ T, int64_t NP, int64_t NT, int d, int Vd,
             const ull* __restrict__ gmin, const ull* __restrict__ gmax,
             const typename NativeKey<V>::K* __restrict__ thr, int use_thr, uint32_t* __restrict__ cnt,
             unsigned* __restrict__ flags) {
  using NK = NativeKey<V>;
  using K = typename NK::K;
  extern __shared__ __align__(16) unsigned char vox_raw[];
  using SK = typename StagedThr<V>::T;
  SK* sthr = reinterpret_cast<SK*>(vox_raw);  // [d][V + 1] on the threshold path
  __shared__ double slo[kVdksMaxD], sspan[kVdksMaxD];
  __shared__ float flo[kVdksMaxD], fsc[kVdksMaxD];
  const int per = Vd - 1;
  if (threadIdx.x < d) {
    const double lo = key_value(gmin[threadIdx.x]);
    const double sp = __dsub_rn(key_value(gmax[threadIdx.x]), lo);
    slo[threadIdx.x] = lo;
    sspan[threadIdx.x] = sp;
    flo[threadIdx.x] = (float)lo;
    fsc[threadIdx.x] = sp > 0.0 ? (float)((double)Vd / sp) : 0.0f;
  }
  if (use_thr) stage_thresholds<V>(sthr, thr, d, Vd);
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
      key = 2u * voxel_index<V, kVdksMaxD>(row, d, Vd, sthr, use_thr != 0, slo, sspan, flo, fsc) +
            (i >= NP ? 1u : 0u);
    }
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    if (i < N && lane == __ffs(peers) - 1) atomicAdd(&cnt[key], (uint32_t)__popc(peers));
  }
}

constexpr int kVoxThreads = 512;

// Voxel counts in a CTA-private shared-memory histogram: CTAs [0, bP) take
// equal slices of P, the others of T.  Each CTA writes its whole histogram
// (zeros included) to hist_all[blockIdx.x][cells]; k_vdks_gather sums them.
// U points per thread per round, their loads issued together; DM >= d.
template <typename V, int U, int DM>
__global__ void __launch_bounds__(kVoxThreads)
k_vdks_voxel_smem(const V* __restrict__ P, const V* __restrict__ T, int64_t NP, int64_t NT, int d, int Vd,
                  const ull* __restrict__ gmin, const ull* __restrict__ gmax,
                  const typename NativeKey<V>::K* __restrict__ thr, int use_thr, uint32_t cells, int bP,
                  uint32_t* __restrict__ hist_all, unsigned* __restrict__ flags) {
  using K = typename NativeKey<V>::K;
  extern __shared__ __align__(16) unsigned char vs_raw[];
  uint32_t* hist = reinterpret_cast<uint32_t*>(vs_raw);
  using SK = typename StagedThr<V>::T;
  SK* sthr = reinterpret_cast<SK*>(vs_raw + (((size_t)cells * 4 + 15) & ~(size_t)15));
  __shared__ double slo[kVdksMaxD], sspan[kVdksMaxD];
  __shared__ float flo[kVdksMaxD], fsc[kVdksMaxD];
  const int per = Vd - 1;
  for (uint32_t c = threadIdx.x; c < cells; c += blockDim.x) hist[c] = 0u;
  if (threadIdx.x < d) {
    const double lo = key_value(gmin[threadIdx.x]);
    const double sp = __dsub_rn(key_value(gmax[threadIdx.x]), lo);
    slo[threadIdx.x] = lo;
    sspan[threadIdx.x] = sp;
    flo[threadIdx.x] = (float)lo;
    fsc[threadIdx.x] = sp > 0.0 ? (float)((double)Vd / sp) : 0.0f;
  }
  if (use_thr) stage_thresholds<V>(sthr, thr, d, Vd);
  check_spans(gmin, gmax, d, flags);
  __syncthreads();
  const bool isT = (int)blockIdx.x >= bP;
  const V* X = isT ? T : P;
  const int64_t n = isT ? NT : NP;
  const int nb = isT ? (int)gridDim.x - bP : bP;
  const int b = isT ? (int)blockIdx.x - bP : (int)blockIdx.x;
  const int64_t beg = n * b / nb, end = n * (b + 1) / nb;
  for (int64_t i0 = beg + threadIdx.x; i0 < end; i0 += (int64_t)U * blockDim.x) {
    V v[U][DM];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t i = i0 + (int64_t)u * blockDim.x;
#pragma unroll
      for (int m = 0; m < DM; ++m)
        v[u][m] = (m < d && i < end) ? X[i * d + m] : (V)0;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (i0 + (int64_t)u * blockDim.x < end)
        atomicAdd(&hist[voxel_index<V, DM>(v[u], d, Vd, sthr, use_thr != 0, slo, sspan, flo, fsc)], 1u);
    }
  }
  __syncthreads();
  uint32_t* out = hist_all + (size_t)blockIdx.x * cells;
  for (uint32_t c = threadIdx.x; c < cells; c += blockDim.x) out[c] = hist[c];
}

constexpr int kVoxStages = 3;                    // bulk-copy ring depth
constexpr int kVoxBulkThreads = 1024;
constexpr size_t kVoxMaxDynSmem = 227 * 1024 - 1024;  // dynamic shared memory of one CTA

// The same counts with the CTA's rows streamed into shared memory by bulk
// asynchronous copies: a ring of kVoxStages chunks of rc rows, so that two
// chunks are in flight while one is counted.  CTA boundaries and rc are
// multiples of r0 rows (r0 rows = a multiple of 16 bytes; the sample bases
// are 16-byte aligned), so every copy starts and ends on 16 bytes; rows past
// the last such boundary (fewer than r0, at the sample's end) are read
// directly.  A wait that runs out (the context's device wait bound, 1 s by
// default) sets kFlagTimeout, waits (bounded)
// for the CTA's copies still in flight and returns without its counts.
// Shared memory: hist [cells] u32 at 0, thresholds at thr_off, stages at
// stage_off (stage_bytes each).
template <typename V, int DM>
__global__ void __launch_bounds__(kVoxBulkThreads)
k_vdks_voxel_bulk(const V* __restrict__ P, const V* __restrict__ T, int64_t NP, int64_t NT, int d, int Vd,
                  const ull* __restrict__ gmin, const ull* __restrict__ gmax,
                  const typename NativeKey<V>::K* __restrict__ thr, int use_thr, uint32_t cells, int bP, int r0,
                  int rc, uint32_t thr_off, uint32_t stage_off, uint32_t stage_bytes,
                  uint32_t* __restrict__ hist_all, unsigned* __restrict__ flags, unsigned long long wait_ns) {
  namespace bk = ddks::bulk;
  using K = typename NativeKey<V>::K;
  extern __shared__ __align__(16) unsigned char vb_raw[];
  __shared__ __align__(8) unsigned long long bars[kVoxStages];
  uint32_t* hist = reinterpret_cast<uint32_t*>(vb_raw);
  using SK = typename StagedThr<V>::T;
  SK* sthr = reinterpret_cast<SK*>(vb_raw + thr_off);
  __shared__ double slo[kVdksMaxD], sspan[kVdksMaxD];
  __shared__ float flo[kVdksMaxD], fsc[kVdksMaxD];
  const int tid = threadIdx.x;
  const int per = Vd - 1;
  for (uint32_t c = tid; c < cells; c += blockDim.x) hist[c] = 0u;
  if (tid < d) {
    const double lo = key_value(gmin[tid]);
    const double sp = __dsub_rn(key_value(gmax[tid]), lo);
    slo[tid] = lo;
    sspan[tid] = sp;
    flo[tid] = (float)lo;
    fsc[tid] = sp > 0.0 ? (float)((double)Vd / sp) : 0.0f;
  }
  if (use_thr) stage_thresholds<V>(sthr, thr, d, Vd);
  check_spans(gmin, gmax, d, flags);
  const uint32_t bar_s = (uint32_t)__cvta_generic_to_shared(bars);
  const uint32_t stage_s = (uint32_t)__cvta_generic_to_shared(vb_raw + stage_off);
  if (tid == 0) {
    for (int k = 0; k < kVoxStages; ++k) bk::mbar_init(bar_s + 8u * k, 1);
    bk::mbar_init_fence();
  }
  __syncthreads();
  const bool isT = (int)blockIdx.x >= bP;
  const V* X = isT ? T : P;
  const int64_t n = isT ? NT : NP;
  const int nb = isT ? (int)gridDim.x - bP : bP;
  const int b = isT ? (int)blockIdx.x - bP : (int)blockIdx.x;
  const int64_t beg = (n * b / nb) / r0 * r0;
  const int64_t end = b + 1 >= nb ? n : (n * (b + 1) / nb) / r0 * r0;
  const int64_t end_al = beg + (end - beg) / r0 * r0;
  const int64_t nrows = end_al - beg;
  const int nch = (int)((nrows + rc - 1) / rc);
  // chunks run from the end of the slice backwards: the range pass just read
  // the arrays forwards, so their ends are the likeliest to be still in L2
  auto chunk_row = [&](int c) -> int64_t { return beg + (int64_t)(nch - 1 - c) * rc; };
  auto issue = [&](int c) {  // thread 0: chunk c into stage c % kVoxStages
    const int64_t r = chunk_row(c);
    const int64_t cnt = end_al - r < rc ? end_al - r : rc;
    const uint32_t bar = bar_s + 8u * (uint32_t)(c % kVoxStages);
    bk::fence_async();
    bk::mbar_expect(bar, (uint32_t)(cnt * d * (int64_t)sizeof(V)));
    bk::load(stage_s + (uint32_t)(c % kVoxStages) * stage_bytes, X + r * d, (uint32_t)(cnt * d * (int64_t)sizeof(V)),
             bar);
  };
  if (tid == 0)
    for (int c = 0; c < kVoxStages - 1 && c < nch; ++c) issue(c);
  for (int c = 0; c < nch; ++c) {
    // stage (c - 1) % kVoxStages was released by the barrier that ended chunk c - 1
    if (tid == 0 && c + kVoxStages - 1 < nch) issue(c + kVoxStages - 1);
    const bool ok = bk::wait(bar_s + 8u * (uint32_t)(c % kVoxStages), (uint32_t)((c / kVoxStages) & 1), wait_ns);
    if (ok) {
      const int64_t r = chunk_row(c);
      const int cnt = (int)(end_al - r < rc ? end_al - r : rc);
      const V* st = reinterpret_cast<const V*>(vb_raw + stage_off + (size_t)(c % kVoxStages) * stage_bytes);
      for (int q = tid; q < cnt; q += blockDim.x)
        atomicAdd(&hist[voxel_index<V, DM>(st + (size_t)q * d, d, Vd, sthr, use_thr != 0, slo, sspan, flo, fsc)],
                  1u);
    }
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        atomicOr(flags, ddks::kFlagTimeout);
        // copies of chunks c .. c + kVoxStages - 2 may still be in flight
        for (int k = c; k < c + kVoxStages - 1 && k < nch; ++k)
          bk::wait(bar_s + 8u * (uint32_t)(k % kVoxStages), (uint32_t)((k / kVoxStages) & 1), bk::kDrainNs);
      }
      return;
    }
  }
  for (int64_t i = end_al + tid; i < end; i += blockDim.x)
    atomicAdd(&hist[voxel_index<V, DM>(X + i * d, d, Vd, sthr, use_thr != 0, slo, sspan, flo, fsc)], 1u);
  __syncthreads();
  uint32_t* out = hist_all + (size_t)blockIdx.x * cells;
  for (uint32_t c = tid; c < cells; c += blockDim.x) out[c] = hist[c];
}

// cnt[2c] = sum of the P CTAs' counts of voxel c, cnt[2c + 1] the T CTAs'.
// CTA of 32 voxels x 8 groups of slices (threadIdx.y), reduced in shared memory.
__global__ void __launch_bounds__(kThreads)
k_vdks_gather(const uint32_t* __restrict__ hist_all, uint32_t cells, int bP, int nb, uint32_t* __restrict__ cnt) {
  __shared__ uint32_t sa[8][32], st[8][32];
  const uint32_t c = blockIdx.x * 32 + threadIdx.x;
  const int g = threadIdx.y;
  uint32_t a = 0, t = 0;
  if (c < cells) {
    for (int b = g; b < nb; b += 8) {
      const uint32_t v = hist_all[(size_t)b * cells + c];
      if (b < bP) a += v; else t += v;
    }
  }
  sa[g][threadIdx.x] = a;
  st[g][threadIdx.x] = t;
  __syncthreads();
  if (g == 0 && c < cells) {
    for (int k = 1; k < 8; ++k) { a += sa[k][threadIdx.x]; t += st[k][threadIdx.x]; }
    cnt[2 * c] = a;
    cnt[2 * c + 1] = t;
  }
}

// Suffix sums along one dimension: voxel lines of Vd elements at stride
// `inner` (= Vd^m for dimension m), one warp per line scanning 32 elements
// at a time from the top end.  With cnt (the pass of dimension 0) the line
// values are first formed from the counts, nT*NP - nP*NT.
__global__ void __launch_bounds__(kThreads)
k_vdks_suffix(const uint32_t* __restrict__ cnt, long long* __restrict__ U, uint32_t lines, int Vd,
              uint32_t inner, long long NP, long long NT) {
  const int lane = threadIdx.x & 31;
  const uint32_t w0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t l = w0; l < lines; l += nw) {
    const uint32_t lo = l % inner, hi = l / inner;
    const uint64_t base = (uint64_t)hi * inner * (uint64_t)Vd + lo;
    long long carry = 0;
    for (int j0 = Vd - 32; j0 > -32; j0 -= 32) {
      const int j = j0 + lane;
      const uint64_t a = base + (uint64_t)(j >= 0 ? j : 0) * inner;
      long long v = 0;
      if (j >= 0) v = cnt ? (long long)cnt[2 * a + 1] * NP - (long long)cnt[2 * a] * NT : U[a];
      for (int off = 1; off < 32; off <<= 1) {
        const long long o = __shfl_down_sync(0xffffffffu, v, off);
        if (lane + off < 32) v += o;
      }
      v += carry;
      if (j >= 0) U[a] = v;
      carry = __shfl_sync(0xffffffffu, v, 0);
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

// Squared distances are ordered through ddks::order_key (a rounded
// (s - 2x) + 1 can be a little below zero; -0.0 keys like +0.0).
DDKS_DEV ull dist_key(double r) { return (ull)ddks::order_key(r); }

// |x' - e_m|^2 from the squared norm s: (s - 2 x'_m) + 1, each step rounded;
// 2 x'_m is exact, so one FMA rounds s - 2 x'_m.
DDKS_DEV double corner_dist(double s, double x) { return __dadd_rn(__fma_rn(-2.0, x, s), 1.0); }

__global__ void __launch_bounds__(kThreads)
k_rescale(const double* __restrict__ v, int64_t n, double lo, double span, double* __restrict__ out) {
  const double rcp = rescale_rcp_of(span);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = rescale_rcp(v[i], lo, span, rcp);
}

// One thread per point, all d + 1 corners (d <= kRdksThreadMaxD).
template <typename V>
__global__ void __launch_bounds__(kThreads)
k_rdks_dist_thread(const V* __restrict__ P, const V* __restrict__ T, int64_t NP, int64_t NT, int d,
                   const ull* __restrict__ gmin, const ull* __restrict__ gmax, ull* __restrict__ keys,
                   unsigned* __restrict__ flags) {
  __shared__ double slo[kRdksThreadMaxD], sspan[kRdksThreadMaxD], srcp[kRdksThreadMaxD];
  if (threadIdx.x < d) {
    const double lo = key_value(gmin[threadIdx.x]);
    const double span = __dsub_rn(key_value(gmax[threadIdx.x]), lo);
    slo[threadIdx.x] = lo;
    sspan[threadIdx.x] = span;
    srcp[threadIdx.x] = rescale_rcp_of(span);
  }
  check_spans(gmin, gmax, d, flags);
  __syncthreads();
  const int64_t N = NP + NT;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const V* row = point_row(P, T, NP, d, i);
    double x[kRdksThreadMaxD];
    x[0] = rescale_rcp((double)row[0], slo[0], sspan[0], srcp[0]);
    double s = __dmul_rn(x[0], x[0]);  // squared norm, added in dimension order (0 + x0^2 = x0^2)
#pragma unroll
    for (int m = 1; m < kRdksThreadMaxD; ++m) {
      x[m] = 0.0;
      if (m < d) {
        x[m] = rescale_rcp((double)row[m], slo[m], sspan[m], srcp[m]);
        s = __dadd_rn(s, __dmul_rn(x[m], x[m]));
      }
    }
    keys[i] = dist_key(s);
#pragma unroll
    for (int m = 0; m < kRdksThreadMaxD; ++m)
      if (m < d) keys[(int64_t)(m + 1) * N + i] = dist_key(corner_dist(s, x[m]));
  }
}

// Any d: one warp per point.  Lanes rescale coordinates into shared memory,
// lane 0 adds the squares in dimension order, lanes then write the corners.
template <typename V>
__global__ void __launch_bounds__(kThreads)
k_rdks_dist_warp(const V* __restrict__ P, const V* __restrict__ T, int64_t NP, int64_t NT, int d,
                 const ull* __restrict__ gmin, const ull* __restrict__ gmax, ull* __restrict__ keys,
                 unsigned* __restrict__ flags) {
  extern __shared__ double sd[];  // per warp: x'[d], x'^2[d]
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nwb = blockDim.x >> 5;
  double* xs = sd + (size_t)w * 2 * d;
  double* q = xs + d;
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
    double s = 0.0;
    if (lane == 0) {  // in dimension order; loads run ahead of the dependent adds
      int m = 0;
      for (; m + 8 <= d; m += 8) {
        double t[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) t[u] = q[m + u];
#pragma unroll
        for (int u = 0; u < 8; ++u) s = __dadd_rn(s, t[u]);
      }
      for (; m < d; ++m) s = __dadd_rn(s, q[m]);
      keys[i] = dist_key(s);
    }
    s = __shfl_sync(0xffffffffu, s, 0);
    for (int m = lane; m < d; m += 32) keys[(int64_t)(m + 1) * N + i] = dist_key(corner_dist(s, xs[m]));
    __syncwarp();
  }
}

// grid (x, S): corner blockIdx.y.  K, I, Pf are the sorted segments, rows Npad apart.
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

// The walk over radix-sorted lists (rows N apart) without a stored P prefix.
// Tiles of kWalkTile positions, grid (tiles, S).  k_rdks_ptile counts each
// tile's P points; k_rdks_walk_tiles adds the earlier tiles' counts (a CTA
// sum) to in-tile prefixes of ballot counts over warp segments of 32
// positions, then evaluates the run ends as k_rdks_walk does.
constexpr int kWalkEach = 8;
constexpr int kWalkTile = kThreads * kWalkEach;  // 2048 positions
constexpr int kWalkSeg = kWalkTile / 32;          // 64 segments

__global__ void __launch_bounds__(kThreads)
k_rdks_ptile(const uint32_t* __restrict__ I, int64_t N, int64_t NP, uint32_t* __restrict__ tp) {
  __shared__ uint32_t ws[kThreads / 32];
  const int64_t s = blockIdx.y, base = (int64_t)blockIdx.x * kWalkTile;
  const uint32_t* Is = I + s * N + base;
  const int nvalid = (int)(N - base < kWalkTile ? N - base : kWalkTile);
  uint32_t c = 0;
#pragma unroll
  for (int j = 0; j < kWalkEach; ++j) {
    const int q = j * kThreads + threadIdx.x;
    c += (q < nvalid && (uint64_t)Is[q] < (uint64_t)NP) ? 1u : 0u;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) c += __shfl_xor_sync(0xffffffffu, c, off);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = 0;
    for (int w = 0; w < kThreads / 32; ++w) t += ws[w];
    tp[s * gridDim.x + blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(kThreads)
k_rdks_walk_tiles(const ull* __restrict__ K, const uint32_t* __restrict__ I, const uint32_t* __restrict__ tp,
                  int64_t N, int64_t NP, int64_t NT, ull* __restrict__ per_corner) {
  __shared__ uint32_t seg[kWalkSeg];
  __shared__ uint32_t ws[kThreads / 32];
  __shared__ ull wbest[kThreads / 32];
  const int64_t s = blockIdx.y, tile = blockIdx.x, base = tile * kWalkTile;
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const ull* Ks = K + s * N;
  const uint32_t* Is = I + s * N;
  const int nvalid = (int)(N - base < kWalkTile ? N - base : kWalkTile);
  // P points in the earlier tiles of this list
  uint32_t c = 0;
  for (int64_t q = t; q < tile; q += kThreads) c += tp[s * gridDim.x + q];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) c += __shfl_xor_sync(0xffffffffu, c, off);
  if (lane == 0) ws[w] = c;
  uint32_t ix[kWalkEach], pm[kWalkEach];
#pragma unroll
  for (int j = 0; j < kWalkEach; ++j) {
    const int q = j * kThreads + t;
    ix[j] = q < nvalid ? Is[base + q] : 0u;
    pm[j] = __ballot_sync(0xffffffffu, q < nvalid && (uint64_t)ix[j] < (uint64_t)NP);
    if (lane == 0) seg[j * (kThreads / 32) + w] = (uint32_t)__popc(pm[j]);
  }
  __syncthreads();
  if (w == 0) {  // exclusive sums over the 64 segments (positions s * 32 + lane)
    const uint32_t a = seg[2 * lane], b = seg[2 * lane + 1];
    uint32_t incl = a + b;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const uint32_t x = __shfl_up_sync(0xffffffffu, incl, off);
      if (lane >= off) incl += x;
    }
    const uint32_t ex = incl - a - b;
    seg[2 * lane] = ex;
    seg[2 * lane + 1] = ex + a;
  }
  __syncthreads();
  uint32_t carry = 0;
#pragma unroll
  for (int q = 0; q < kThreads / 32; ++q) carry += ws[q];
  const uint32_t below = (1u << lane) - 1u;  // lane 0: none
  ull best = 0;
#pragma unroll
  for (int j = 0; j < kWalkEach; ++j) {
    const int q = j * kThreads + t;
    if (q < nvalid) {
      const int64_t p = base + q;
      if (p == N - 1 || Ks[p + 1] != Ks[p]) {
        const uint64_t cp = (uint64_t)carry + seg[j * (kThreads / 32) + w] + (uint32_t)__popc(pm[j] & below) +
                            ((uint64_t)ix[j] < (uint64_t)NP ? 1u : 0u);
        const uint64_t ct = (uint64_t)p + 1 - cp;
        const ull v = ddks::numer(cp, ct, (uint64_t)NP, (uint64_t)NT);
        best = v > best ? v : best;
      }
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const ull o = __shfl_down_sync(0xffffffffu, best, off);
    best = o > best ? o : best;
  }
  if (lane == 0) wbest[w] = best;
  __syncthreads();
  if (t == 0) {
    ull b = 0;
    for (int q = 0; q < kThreads / 32; ++q) b = wbest[q] > b ? wbest[q] : b;
    if (b) atomicMax(per_corner + s, b);
  }
}

// Small samples (N <= 1024): one warp per corner sorts the corner's (key,
// index) pairs in registers -- lane l holds positions l*E .. l*E+E-1 of the
// 32*E >= N padded list; bitonic stages of stride < E stay in the lane,
// larger strides pair lane l with l ^ (stride / E) by shuffles -- then walks
// the sorted list (P counts by a warp scan) and writes the corner's maximum.
template <int E>
__global__ void __launch_bounds__(kThreads)
k_rdks_small(const ull* __restrict__ keys, int N, int64_t NP, int64_t NT, int S, ull* __restrict__ per_corner) {
  constexpr int n = 32 * E;
  const int lane = threadIdx.x & 31;
  const int s = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);  // warp-uniform
  if (s >= S) return;
  ull k[E];
  uint32_t ix[E];
#pragma unroll
  for (int j = 0; j < E; ++j) {
    const int p = lane * E + j;
    k[j] = p < N ? keys[(int64_t)s * N + p] : ~0ull;  // pads sort last
    ix[j] = (uint32_t)p;
  }
  for (int size = 2; size <= n; size <<= 1) {
    int stride = size >> 1;
    for (; stride >= E; stride >>= 1) {
      const int xm = stride / E;
      const bool lower = (lane & xm) == 0;
#pragma unroll
      for (int j = 0; j < E; ++j) {
        const ull ok = __shfl_xor_sync(0xffffffffu, k[j], xm);
        const uint32_t oi = __shfl_xor_sync(0xffffffffu, ix[j], xm);
        const bool asc = ((lane * E + j) & size) == 0;
        const bool less = k[j] < ok || (k[j] == ok && ix[j] < oi);
        if ((lower == asc) != less) { k[j] = ok; ix[j] = oi; }
      }
    }
#pragma unroll
    for (int sd = E / 2; sd >= 1; sd >>= 1) {
      if (sd > stride) continue;
#pragma unroll
      for (int a = 0; a < E; ++a) {
        if (a & sd) continue;
        const int b = a | sd;
        const bool asc = ((lane * E + a) & size) == 0;
        const bool bl = k[b] < k[a] || (k[b] == k[a] && ix[b] < ix[a]);
        if (asc == bl) {
          const ull tk = k[a]; k[a] = k[b]; k[b] = tk;
          const uint32_t ti = ix[a]; ix[a] = ix[b]; ix[b] = ti;
        }
      }
    }
  }
  // P points before each position: lane totals, then an exclusive warp scan
  uint32_t cnt = 0;
#pragma unroll
  for (int j = 0; j < E; ++j) cnt += ix[j] < (uint64_t)NP ? 1u : 0u;
  uint32_t incl = cnt;
  for (int off = 1; off < 32; off <<= 1) {
    const uint32_t x = __shfl_up_sync(0xffffffffu, incl, off);
    if (lane >= off) incl += x;
  }
  uint32_t cp = incl - cnt;
  const ull next0 = __shfl_down_sync(0xffffffffu, k[0], 1);  // first key of the next lane
  ull best = 0;
#pragma unroll
  for (int j = 0; j < E; ++j) {
    const int p = lane * E + j;
    cp += ix[j] < (uint64_t)NP ? 1u : 0u;
    const ull nk = j + 1 < E ? k[j + 1 < E ? j + 1 : j] : next0;
    if (p < N && (p == N - 1 || nk != k[j])) {
      const ull v = ddks::numer(cp, (uint64_t)(p + 1) - cp, (uint64_t)NP, (uint64_t)NT);
      best = v > best ? v : best;
    }
  }
  for (int off = 16; off > 0; off >>= 1) {
    const ull o = __shfl_down_sync(0xffffffffu, best, off);
    best = o > best ? o : best;
  }
  if (lane == 0) per_corner[s] = best;
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

// ------------------------------------------------------------------ rdKS by histogram
//
// GetDFromCornerLists without a full sort.  The statistic of a corner is
// sup over run ends r of |D(r)|, D(r) = #P(dist <= r) * NT - #T(dist <= r) * NP
// (exact integers).  The corner's keys are counted into 2^15 buckets of equal
// width in key space between the row's smallest and largest key (one pass:
// shared-memory counts per chunk of keys, then a sum over the chunks, P and
// T counts in one 64-bit word).  Equal keys share a
// bucket, so every bucket end is a run end and D there is exact; inside a
// bucket D moves by +NT per P point and -NP per T point, so a bucket holding
// one sample only has its extremes at its ends, and a mixed bucket can exceed
// the best bucket end LB only if max(|D_start + nP*NT|, |D_start - nT*NP|) >
// LB.  Only those candidate buckets are gathered (a bitmap of them lets the
// other keys skip the slot table) and refined from D_start, one CTA each: up
// to kWarpRefineMax points without a sort (each point counts the points of
// each sample with a key <= its own, the warps splitting the points), larger
// ones by a bitonic sort in shared memory and a walk of the run ends.  A row
// with more than kMaxCand candidates, or a candidate with more than
// kRefineCap points, sets kFlagRedo and the host reruns the call on the
// sorting path.
constexpr int kHistBits = 15;
constexpr int kHistB = 1 << kHistBits;
constexpr int kMaxCand = 1024;
constexpr int kRefineCap = 8192;
constexpr int kCandThreads = 1024;

constexpr size_t kRefineSmem = (size_t)kRefineCap * 9;
constexpr int kWarpRefineMax = 512;  // candidates of up to this many points: one warp each, no sort

struct RdksCand {
  long long dstart;   // D before the bucket's first point
  uint32_t off;       // first slot of the bucket's points in the gather buffer (row-local)
  uint32_t n;         // points in the bucket
};

DDKS_DEV int hist_shift(ull kmin, ull kmax) {
  const ull range = kmax - kmin;
  if (range == 0) return 0;
  const int bits = 64 - __clzll((long long)range);
  return bits > kHistBits ? bits - kHistBits : 0;
}

// per corner: the smallest and largest key
__global__ void __launch_bounds__(kThreads)
k_rdks_krange(const ull* __restrict__ keys, int64_t N, ull* __restrict__ kmin, ull* __restrict__ kmax) {
  const int s = blockIdx.y;
  const ull* row = keys + (int64_t)s * N;
  ull lo = ~0ull, hi = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  for (; i + 3 * stride < N; i += 4 * stride) {  // four loads in flight
    ull k[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) k[u] = row[i + u * stride];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      lo = k[u] < lo ? k[u] : lo;
      hi = k[u] > hi ? k[u] : hi;
    }
  }
  for (; i < N; i += stride) {
    const ull k = row[i];
    lo = k < lo ? k : lo;
    hi = k > hi ? k : hi;
  }
  for (int off = 16; off > 0; off >>= 1) {
    const ull a = __shfl_xor_sync(0xffffffffu, lo, off), b = __shfl_xor_sync(0xffffffffu, hi, off);
    lo = a < lo ? a : lo;
    hi = b > hi ? b : hi;
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMin(&kmin[s], lo);
    atomicMax(&kmax[s], hi);
  }
}

// Per chunk of kHistChunk keys of a corner (grid (chunks, S)), the bucket
// counts in shared memory, P | T << 16 (a chunk has fewer than 2^16 keys),
// written out whole: part[s][chunk][b].
constexpr int kHistChunk = 65535;
constexpr int kHistThreads = 1024;

__global__ void __launch_bounds__(kHistThreads)
k_rdks_hist(const ull* __restrict__ keys, int64_t N, int64_t NP, const ull* __restrict__ kmin,
            const ull* __restrict__ kmax, uint32_t* __restrict__ part) {
  extern __shared__ __align__(16) uint32_t hsm[];  // [kHistB]
  const int s = blockIdx.y;
  const ull* row = keys + (int64_t)s * N;
  const ull k0 = kmin[s];
  const int sh = hist_shift(k0, kmax[s]);
  for (int b = threadIdx.x; b < kHistB; b += kHistThreads) hsm[b] = 0u;
  __syncthreads();
  const int64_t i0 = (int64_t)blockIdx.x * kHistChunk;
  const int64_t i1 = i0 + kHistChunk < N ? i0 + kHistChunk : N;
  for (int64_t i = i0 + threadIdx.x; i < i1; i += kHistThreads) {
    const uint32_t b = (uint32_t)((row[i] - k0) >> sh);
    atomicAdd(&hsm[b], i < NP ? 1u : (1u << 16));
  }
  __syncthreads();
  uint32_t* out = part + ((int64_t)s * gridDim.x + blockIdx.x) * kHistB;
  for (int b = threadIdx.x; b < kHistB; b += kHistThreads) out[b] = hsm[b];
}

// H[s][b] = sum over the chunks, as P | T << 32
__global__ void __launch_bounds__(kThreads)
k_rdks_hist_sum(const uint32_t* __restrict__ part, int chunks, ull* __restrict__ H) {
  const int s = blockIdx.y;
  for (int b = blockIdx.x * kThreads + threadIdx.x; b < kHistB; b += gridDim.x * kThreads) {
    ull p = 0, t = 0;
    for (int c = 0; c < chunks; ++c) {
      const uint32_t v = part[((int64_t)s * chunks + c) * kHistB + b];
      p += v & 0xFFFFu;
      t += v >> 16;
    }
    H[(int64_t)s * kHistB + b] = p | (t << 32);
  }
}

// One CTA per corner: D at every bucket end (LB = their maximum, the row's
// statistic so far), then the candidate buckets with their D_start and
// places in the gather buffer (taken in any order); slot[s][b] = candidate
// index or -1.  Warp w walks buckets [w * kPerW, (w + 1) * kPerW), 32 at a time.
__global__ void __launch_bounds__(kCandThreads)
k_rdks_cands(const ull* __restrict__ H, int64_t NP, int64_t NT, ull* __restrict__ pc, int* __restrict__ slot,
             RdksCand* __restrict__ cand, int* __restrict__ ccount, unsigned* __restrict__ fill,
             uint32_t* __restrict__ cbits, unsigned* __restrict__ flags) {
  constexpr int kW = kCandThreads / 32;
  constexpr int kPerW = kHistB / kW;
  __shared__ unsigned long long ws[kW];
  __shared__ unsigned long long s_lb;
  __shared__ unsigned s_nc, s_np;
  const int s = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const ull* h = H + (int64_t)s * kHistB + warp * kPerW;
  const long long nt = (long long)NT, np = (long long)NP;
  auto D = [&](ull c) { return (long long)(c & 0xFFFFFFFFull) * nt - (long long)(c >> 32) * np; };
  auto ab = [](long long v) { return (ull)(v < 0 ? -v : v); };
  // inclusive scan of the packed (P, T) counts over the warp's lanes (the
  // halves cannot carry: NP, NT < 2^32)
  auto wscan = [&](ull v) {
    for (int off = 1; off < 32; off <<= 1) {
      const ull y = __shfl_up_sync(0xffffffffu, v, off);
      if (lane >= off) v += y;
    }
    return v;
  };
  ull sum = 0;
#pragma unroll 8
  for (int j = lane; j < kPerW; j += 32) sum += h[j];
  for (int off = 16; off > 0; off >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, off);
  if (lane == 0) ws[warp] = sum;
  if (tid == 0) { s_nc = 0; s_np = 0; }
  __syncthreads();
  ull base = 0;
  for (int w = 0; w < warp; ++w) base += ws[w];
  // LB: the largest |D| at a bucket end
  ull lb = 0, carry = base;
  for (int j0 = 0; j0 < kPerW; j0 += 32 * 8) {
    ull hv[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) hv[u] = h[j0 + 32 * u + lane];  // eight loads in flight
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const ull inc = wscan(hv[u]);
      const ull v = ab(D(carry + inc));
      lb = v > lb ? v : lb;
      carry += __shfl_sync(0xffffffffu, inc, 31);
    }
  }
  for (int off = 16; off > 0; off >>= 1) {
    const ull y = __shfl_xor_sync(0xffffffffu, lb, off);
    lb = y > lb ? y : lb;
  }
  __syncthreads();  // ws is reused
  if (lane == 0) ws[warp] = lb;
  __syncthreads();
  if (tid == 0) {
    ull m = 0;
    for (int w = 0; w < kW; ++w) m = ws[w] > m ? ws[w] : m;
    s_lb = m;
    pc[s] = m;
  }
  __syncthreads();
  lb = s_lb;
  // candidates: mixed buckets whose reachable extreme beats LB
  static_assert(kPerW % 256 == 0, "eight chunks of 32 buckets per step");
  carry = base;
  for (int j0 = 0; j0 < kPerW; j0 += 32) {
    const ull hb = h[j0 + lane];
    const ull inc = wscan(hb);
    const long long ds = D(carry + inc - hb);
    const ull nP = hb & 0xFFFFFFFFull, nT = hb >> 32;
    int sl = -1;
    if (nP && nT && (ab(ds + (long long)nP * nt) > lb || ab(ds - (long long)nT * np) > lb)) {
      const unsigned k = atomicAdd(&s_nc, 1u);
      const unsigned off = atomicAdd(&s_np, (unsigned)(nP + nT));
      if (k < (unsigned)kMaxCand) {
        sl = (int)k;
        RdksCand cd;
        cd.dstart = ds;
        cd.off = off;
        cd.n = (unsigned)(nP + nT);
        cand[(int64_t)s * kMaxCand + k] = cd;
        fill[(int64_t)s * kMaxCand + k] = 0u;
        if (cd.n > (unsigned)kRefineCap) atomicOr(flags, ddks::kFlagRedo);
      }
    }
    slot[(int64_t)s * kHistB + warp * kPerW + j0 + lane] = sl;
    const uint32_t bm = __ballot_sync(0xffffffffu, sl >= 0);  // 32 buckets, one word of the bitmap
    if (lane == 0) cbits[(int64_t)s * (kHistB / 32) + (warp * kPerW + j0) / 32] = bm;
    carry += __shfl_sync(0xffffffffu, inc, 31);
  }
  __syncthreads();
  if (tid == 0) {
    ccount[s] = s_nc < (unsigned)kMaxCand ? (int)s_nc : kMaxCand;
    if (s_nc > (unsigned)kMaxCand) atomicOr(flags, ddks::kFlagRedo);
  }
}

// the points of the candidate buckets, with their sample (1 = P)
__global__ void __launch_bounds__(kThreads)
k_rdks_gather(const ull* __restrict__ keys, int64_t N, int64_t NP, const ull* __restrict__ kmin,
              const ull* __restrict__ kmax, const int* __restrict__ slot, const RdksCand* __restrict__ cand,
              const uint32_t* __restrict__ cbits, unsigned* __restrict__ fill, ull* __restrict__ gk,
              uint8_t* __restrict__ gl) {
  // the row's candidate buckets as a bitmap in shared memory: only keys in a
  // candidate bucket read the slot table
  __shared__ uint32_t sbits[kHistB / 32];
  const int s = blockIdx.y;
  for (int w = threadIdx.x; w < kHistB / 32; w += blockDim.x) sbits[w] = cbits[(int64_t)s * (kHistB / 32) + w];
  __syncthreads();
  const ull* row = keys + (int64_t)s * N;
  const ull k0 = kmin[s];
  const int sh = hist_shift(k0, kmax[s]);
  const int* sl = slot + (int64_t)s * kHistB;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i0 < N; i0 += 4 * stride) {
    // four keys at a time: their loads, then their buckets' slots, in flight together
    ull k[4];
    int c[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) k[u] = i0 + u * stride < N ? row[i0 + u * stride] : k0;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const uint32_t b = (uint32_t)((k[u] - k0) >> sh);
      c[u] = (i0 + u * stride < N && ((sbits[b >> 5] >> (b & 31)) & 1u)) ? sl[b] : -1;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (c[u] < 0) continue;
      const int64_t i = i0 + u * stride;
      const RdksCand cd = cand[(int64_t)s * kMaxCand + c[u]];
      const unsigned pos = atomicAdd(&fill[(int64_t)s * kMaxCand + c[u]], 1u);
      if (pos >= cd.n || cd.n > (unsigned)kRefineCap) continue;  // never past the bucket's places
      gk[(int64_t)s * N + cd.off + pos] = k[u];
      gl[(int64_t)s * N + cd.off + pos] = i < NP ? 1 : 0;
    }
  }
}

// One CTA per candidate of at most kWarpRefineMax points: its 8 warps split
// the candidate's points (warp w: points w * 32 * E .. ), each warp counting
// against all of them.
// This warp's points are [first, end) of the candidate's n points.
template <int E>
DDKS_DEV ull warp_refine_part(const ull* __restrict__ sk, const uint8_t* __restrict__ sp, int n, int first, int end,
                              long long dstart, long long nt, long long np, int lane) {
  ull mine[E];
  unsigned cpn[E], cnn[E];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int i = first + e * 32 + lane;
    mine[e] = i < end ? sk[i] : 0ull;
    cpn[e] = cnn[e] = 0;
  }
  for (int j = 0; j < n; ++j) {
    const ull kj = sk[j];
    const unsigned pj = sp[j];
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const unsigned le = kj <= mine[e] ? 1u : 0u;
      cpn[e] += le & pj;
      cnn[e] += le;
    }
  }
  ull best = 0;
#pragma unroll
  for (int e = 0; e < E; ++e) {
    if (first + e * 32 + lane >= end) break;
    const long long dv = dstart + (long long)cpn[e] * nt - (long long)(cnn[e] - cpn[e]) * np;
    const ull v = (ull)(dv < 0 ? -dv : dv);
    best = v > best ? v : best;
  }
  return best;
}

__global__ void __launch_bounds__(kThreads)
k_rdks_refine_warp(const ull* __restrict__ gk, const uint8_t* __restrict__ gl, int64_t N, int64_t NP, int64_t NT,
                   const RdksCand* __restrict__ cand, const int* __restrict__ ccount, ull* __restrict__ pc) {
  constexpr int kW = kThreads / 32;
  constexpr int kE = kWarpRefineMax / kThreads;  // points per lane at most
  __shared__ ull sk[kWarpRefineMax];
  __shared__ uint8_t sp[kWarpRefineMax];
  __shared__ ull wbest[kW];
  const int s = blockIdx.y;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const long long nt = (long long)NT, np = (long long)NP;
  for (int ci = blockIdx.x; ci < ccount[s]; ci += gridDim.x) {
    const RdksCand cd = cand[(int64_t)s * kMaxCand + ci];
    const int n = (int)cd.n;
    if (n > kWarpRefineMax) continue;  // the sorting kernel's
    __syncthreads();  // the buffers are free
    for (int i = tid; i < n; i += kThreads) {
      sk[i] = gk[(int64_t)s * N + cd.off + i];
      sp[i] = gl[(int64_t)s * N + cd.off + i];
    }
    __syncthreads();
    const int per = (n + kW - 1) / kW;  // points of each warp
    const int first = warp * per, cnt = n - first < per ? (n - first > 0 ? n - first : 0) : per;
    ull best = 0;
    if (cnt > 0) {  // warp-uniform
      best = cnt <= 32 ? warp_refine_part<1>(sk, sp, n, first, first + cnt, cd.dstart, nt, np, lane)
                       : warp_refine_part<kE>(sk, sp, n, first, first + cnt, cd.dstart, nt, np, lane);
    }
    for (int off = 16; off > 0; off >>= 1) {
      const ull y = __shfl_xor_sync(0xffffffffu, best, off);
      best = y > best ? y : best;
    }
    if (lane == 0) wbest[warp] = best;
    __syncthreads();
    if (tid == 0) {
      ull m = 0;
      for (int w = 0; w < kW; ++w) m = wbest[w] > m ? wbest[w] : m;
      atomicMax(&pc[s], m);
    }
  }
}

// One CTA per candidate bucket (a grid-stride over them): sort its points
// in shared memory and walk its run ends from D_start; the row's statistic
// is the maximum with LB.
__global__ void __launch_bounds__(kThreads)
k_rdks_refine(const ull* __restrict__ gk, const uint8_t* __restrict__ gl, int64_t N, int64_t NP, int64_t NT,
              const RdksCand* __restrict__ cand, const int* __restrict__ ccount, ull* __restrict__ pc) {
  extern __shared__ __align__(16) unsigned char rsm[];
  ull* sk = reinterpret_cast<ull*>(rsm);                     // [kRefineCap]
  uint8_t* sp = reinterpret_cast<uint8_t*>(sk + kRefineCap);  // [kRefineCap]
  __shared__ unsigned long long wsum[kThreads / 32], wmax[kThreads / 32];
  const int s = blockIdx.y;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int kW = kThreads / 32;
  const long long nt = (long long)NT, np = (long long)NP;
  for (int ci = blockIdx.x; ci < ccount[s]; ci += gridDim.x) {
    const RdksCand cd = cand[(int64_t)s * kMaxCand + ci];
    const int n = (int)cd.n;
    if (n > kRefineCap) continue;  // flagged: the host reruns on the sorting path
    if (n <= kWarpRefineMax) continue;  // refined by k_rdks_refine_warp
    int P2 = 1;
    while (P2 < n) P2 <<= 1;
    __syncthreads();
    for (int i = tid; i < P2; i += kThreads) {
      sk[i] = i < n ? gk[(int64_t)s * N + cd.off + i] : ~0ull;
      sp[i] = i < n ? gl[(int64_t)s * N + cd.off + i] : 0;
    }
    __syncthreads();
    for (int size = 2; size <= P2; size <<= 1) {
      for (int stride = size >> 1; stride > 0; stride >>= 1) {
        for (int t = tid; t < P2 / 2; t += kThreads) {
          const int lo = 2 * t - (t & (stride - 1)), hi = lo + stride;
          const bool asc = (lo & size) == 0;
          const ull a = sk[lo], b = sk[hi];
          if (asc ? b < a : a < b) {
            sk[lo] = b;
            sk[hi] = a;
            const uint8_t x = sp[lo];
            sp[lo] = sp[hi];
            sp[hi] = x;
          }
        }
        __syncthreads();
      }
    }
    // inclusive prefix of P points over the sorted positions, chunk per thread
    const int seg = (n + kThreads - 1) / kThreads;
    const int a0 = tid * seg < n ? tid * seg : n, a1 = a0 + seg < n ? a0 + seg : n;
    unsigned long long cp = 0;
    for (int i = a0; i < a1; ++i) cp += sp[i];
    unsigned long long inc = cp;
    for (int off = 1; off < 32; off <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xffffffffu, inc, off);
      if (lane >= off) inc += y;
    }
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    unsigned long long run = inc - cp;
    for (int w = 0; w < warp; ++w) run += wsum[w];
    ull best = 0;
    for (int i = a0; i < a1; ++i) {
      run += sp[i];
      if (i + 1 == n || sk[i + 1] != sk[i]) {  // a run end
        const long long dv = cd.dstart + (long long)run * nt - (long long)(i + 1 - (long long)run) * np;
        const ull v = (ull)(dv < 0 ? -dv : dv);
        best = v > best ? v : best;
      }
    }
    for (int off = 16; off > 0; off >>= 1) {
      const ull y = __shfl_xor_sync(0xffffffffu, best, off);
      best = y > best ? y : best;
    }
    if (lane == 0) wmax[warp] = best;
    __syncthreads();
    if (tid == 0) {
      ull m = 0;
      for (int w = 0; w < kW; ++w) m = wmax[w] > m ? wmax[w] : m;
      atomicMax(&pc[s], m);
    }
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
  if (flags & ddks::kFlagTimeout) return DDKS_ETIMEOUT;
  return DDKS_OK;
}

template <typename V>
cudaError_t launch_minmax(const void* P, const void* T, int64_t NP, int64_t NT, int d, ull* gmin, ull* gmax,
                          unsigned* flags, int num_sms, cudaStream_t st) {
  constexpr int VEC = 16 / (int)sizeof(V);
  const int64_t total = (NP + NT) * d;
  const int64_t L = (d % VEC == 0) ? d : (d % 2 == 0 && VEC == 4 ? 2 * (int64_t)d : (int64_t)VEC * d);  // lcm(VEC, d)
  int g = grid_cap((total + VEC - 1) / VEC, kThreads, num_sms * 8);
  const int need = (int)((L + (int64_t)VEC * kThreads - 1) / ((int64_t)VEC * kThreads));  // S >= L
  if (g < need) g = need;
  const int64_t S = ((int64_t)g * kThreads * VEC / L) * L;
  const size_t smem = 2 * sizeof(typename NativeKey<V>::K) * (size_t)d;
  if (smem > 48 * 1024) {
    cudaError_t e = ddks_smem_attr(k_minmax<V>, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_minmax<V><<<g, kThreads, smem, st>>>((const V*)P, (const V*)T, NP, NT, d, S, gmin, gmax, flags);
  return cudaGetLastError();
}

template <typename V>
cudaError_t launch_voxel_smem(const void* P, const void* T, int64_t NP, int64_t NT, int d, int Vd, const ull* gmin,
                              const ull* gmax, const void* thr, bool use_thr, uint32_t cells, int bP, int nb,
                              uint32_t* hall, unsigned* flags, size_t smem, cudaStream_t st) {
  using K = typename NativeKey<V>::K;
  constexpr int U4 = sizeof(V) == 4 ? 4 : 2;
  auto go = [&](auto kern) -> cudaError_t {
    cudaError_t e = ddks_smem_attr(kern, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<nb, kVoxThreads, smem, st>>>((const V*)P, (const V*)T, NP, NT, d, Vd, gmin, gmax, (const K*)thr,
                                       use_thr ? 1 : 0, cells, bP, hall, flags);
    return cudaGetLastError();
  };
  if (d == 1) return go(k_vdks_voxel_smem<V, U4, 1>);
  if (d == 2) return go(k_vdks_voxel_smem<V, U4, 2>);
  if (d == 3) return go(k_vdks_voxel_smem<V, U4, 3>);
  if (d == 4) return go(k_vdks_voxel_smem<V, U4, 4>);
  return go(k_vdks_voxel_smem<V, 1, kVdksMaxD>);
}

// Shared-memory plan of k_vdks_voxel_bulk; false when it does not fit.
struct BulkPlan {
  int r0 = 0, rc = 0;
  uint32_t thr_off = 0, stage_off = 0, stage_bytes = 0;
  size_t smem = 0;
};
bool plan_voxel_bulk(uint32_t cells, int d, size_t ks, int64_t nthr, size_t es, BulkPlan* bp) {
  const size_t rowb = (size_t)d * es;
  size_t g = 16, a = rowb;  // r0 = 16 / gcd(16, row bytes)
  while (a) { const size_t t = g % a; g = a; a = t; }
  bp->r0 = (int)(16 / g);
  bp->thr_off = (uint32_t)(((size_t)cells * 4 + 15) & ~(size_t)15);
  bp->stage_off = (uint32_t)((bp->thr_off + ks * (size_t)nthr + 15) & ~(size_t)15);
  if (bp->stage_off >= kVoxMaxDynSmem) return false;
  size_t ch = (kVoxMaxDynSmem - bp->stage_off) / kVoxStages;
  if (ch > 32 * 1024) ch = 32 * 1024;
  const size_t unit = (size_t)bp->r0 * rowb;  // a multiple of 16
  bp->rc = (int)(ch / unit) * bp->r0;
  if (bp->rc < bp->r0 || bp->rc * rowb < 4096) return false;
  bp->stage_bytes = (uint32_t)((size_t)bp->rc * rowb);
  bp->smem = bp->stage_off + (size_t)kVoxStages * bp->stage_bytes;
  return bp->smem <= kVoxMaxDynSmem;
}

template <typename V>
cudaError_t launch_voxel_bulk(const void* P, const void* T, int64_t NP, int64_t NT, int d, int Vd, const ull* gmin,
                              const ull* gmax, const void* thr, bool use_thr, uint32_t cells, int bP, int nb,
                              uint32_t* hall, unsigned* flags, const BulkPlan& bp, cudaStream_t st,
                              unsigned long long wait_ns) {
  using K = typename NativeKey<V>::K;
  auto go = [&](auto kern) -> cudaError_t {
    cudaError_t e = ddks_smem_attr(kern, (int)bp.smem);
    if (e != cudaSuccess) return e;
    kern<<<nb, kVoxBulkThreads, bp.smem, st>>>((const V*)P, (const V*)T, NP, NT, d, Vd, gmin, gmax, (const K*)thr,
                                              use_thr ? 1 : 0, cells, bP, bp.r0, bp.rc, bp.thr_off, bp.stage_off,
                                          bp.stage_bytes, hall, flags, wait_ns);
    return cudaGetLastError();
  };
  if (d == 1) return go(k_vdks_voxel_bulk<V, 1>);
  if (d == 2) return go(k_vdks_voxel_bulk<V, 2>);
  if (d == 3) return go(k_vdks_voxel_bulk<V, 3>);
  if (d == 4) return go(k_vdks_voxel_bulk<V, 4>);
  return go(k_vdks_voxel_bulk<V, kVdksMaxD>);
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
  // CTA-private shared-memory histograms (one CTA per SM, P and T CTAs apart)
  // when the voxels fit and every CTA has many points per voxel to count
  const size_t ks = dtype == DDKS_F64 ? 8 : 4;
  const int64_t nstaged = (int64_t)d * (Vd + 1);  // staged thresholds with their sentinels
  const size_t hsm = (((size_t)cells * 4 + 15) & ~(size_t)15) + (use_thr ? ks * (size_t)nstaged : 0);
  const int nbh = ctx->num_sms;
  const bool smem_hist = hsm <= kVdksMaxHistSmem && NP + NT >= 16 * (int64_t)cells && nbh >= 2;
  int bP = (int)((double)nbh * (double)NP / (double)(NP + NT) + 0.5);
  bP = bP < 1 ? 1 : (bP > nbh - 1 ? nbh - 1 : bP);
  if ((rc = ctx->apx_small.reserve(ctx, L.bytes))) return out->status = rc;
  if ((rc = ctx->apx_cnt.reserve(ctx, 8 * (size_t)cells))) return out->status = rc;
  if ((rc = ctx->apx_U.reserve(ctx, 8 * (size_t)cells))) return out->status = rc;
  if (smem_hist && (rc = ctx->apx_hist.reserve(ctx, 4 * (size_t)cells * nbh))) return out->status = rc;
  // stream the rows with bulk copies when the ring fits beside the histogram
  // and both sample bases are 16-byte aligned
  BulkPlan bp;
  const bool bulk = smem_hist && ((uintptr_t)dP & 15) == 0 && ((uintptr_t)dT & 15) == 0 &&
                    plan_voxel_bulk(cells, d, ks, use_thr ? nstaged : 0, ks, &bp);
  GraphKey key;
  key.add(7).add((uint64_t)NP).add((uint64_t)NT).add((uint64_t)d).add((uint64_t)dtype).add((uint64_t)Vd);
  key.add((uint64_t)use_thr).add((uint64_t)smem_hist).add((uint64_t)bulk).add((uint64_t)ctx->stage_timing);
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
    if (ee == cudaSuccess && !smem_hist) ee = cudaMemsetAsync(cnt, 0, 8 * (size_t)cells, s);
    if (ee != cudaSuccess) return ctx_cuda_fail(ctx, ee, "vdks memset");
    ddks_stage_mark(ctx, 0, s);
    const bool f64 = dtype == DDKS_F64;
    ee = f64 ? launch_minmax<double>(dP, dT, NP, NT, d, gmin, gmax, flags, ctx->num_sms, s)
             : launch_minmax<float>(dP, dT, NP, NT, d, gmin, gmax, flags, ctx->num_sms, s);
    if (ee != cudaSuccess) return ctx_cuda_fail(ctx, ee, "vdks range");
    ddks_stage_mark(ctx, 1, s);
    const int gv = grid_cap(NP + NT, kThreads, ctx->num_sms * 8);
    const int nthr = d * (Vd - 1);
    if (use_thr && nthr > 0) {
      const int gt = (int)(((int64_t)nthr * 32 + kThreads - 1) / kThreads);  // a warp per threshold
      if (f64)
        k_vdks_thresholds<double><<<gt, kThreads, 0, s>>>(gmin, gmax, d, Vd, (ull*)thr);
      else
        k_vdks_thresholds<float><<<gt, kThreads, 0, s>>>(gmin, gmax, d, Vd, (uint32_t*)thr);
      ctx->launches += 1;
    }
    if (smem_hist) {
      uint32_t* hall = (uint32_t*)ctx->apx_hist.ptr;
      if (bulk)
        ee = f64 ? launch_voxel_bulk<double>(dP, dT, NP, NT, d, Vd, gmin, gmax, thr, use_thr, cells, bP, nbh, hall,
                                             flags, bp, s, ctx->dev_wait_ns)
                 : launch_voxel_bulk<float>(dP, dT, NP, NT, d, Vd, gmin, gmax, thr, use_thr, cells, bP, nbh, hall,
                                            flags, bp, s, ctx->dev_wait_ns);
      else
        ee = f64 ? launch_voxel_smem<double>(dP, dT, NP, NT, d, Vd, gmin, gmax, thr, use_thr, cells, bP, nbh, hall,
                                             flags, hsm, s)
                 : launch_voxel_smem<float>(dP, dT, NP, NT, d, Vd, gmin, gmax, thr, use_thr, cells, bP, nbh, hall,
                                            flags, hsm, s);
      if (ee != cudaSuccess) return ctx_cuda_fail(ctx, ee, "vdks voxel attribute");
      k_vdks_gather<<<(cells + 31) / 32, dim3(32, 8), 0, s>>>(hall, cells, bP, nbh, cnt);
      ctx->launches += 1;
    } else {
      const size_t vsm = use_thr ? ks * (size_t)nstaged : 0;
      if (f64)
        k_vdks_voxel<double><<<gv, kThreads, vsm, s>>>((const double*)dP, (const double*)dT, NP, NT, d, Vd, gmin,
                                                       gmax, (const ull*)thr, use_thr ? 1 : 0, cnt, flags);
      else
        k_vdks_voxel<float><<<gv, kThreads, vsm, s>>>((const float*)dP, (const float*)dT, NP, NT, d, Vd, gmin,
                                                      gmax, (const uint32_t*)thr, use_thr ? 1 : 0, cnt, flags);
    }
    ddks_stage_mark(ctx, 2, s);
    const uint32_t lines = cells / (uint32_t)Vd;
    const int gs = grid_cap(lines, kThreads / 32, ctx->num_sms * 8);
    uint32_t inner = 1;
    for (int m = 0; m < d; ++m, inner *= (uint32_t)Vd)
      k_vdks_suffix<<<gs, kThreads, 0, s>>>(m == 0 ? cnt : nullptr, U, lines, Vd, inner, NP, NT);
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

int ddks_rescale(ddks_ctx* ctx, const double* v, int64_t n, double lo, double span, double* out, void* stream) {
  if (!ctx || n < 0 || (n > 0 && (!v || !out))) return DDKS_EINVAL;
  if (!std::isfinite(lo) || !std::isfinite(span) || span < 0.0) return DDKS_EINVAL;
  if (n == 0) return DDKS_OK;
  const int kv = ddks_pointer_kind(v, ctx->device), kout = ddks_pointer_kind(out, ctx->device);
  if (kv < 0 || kout < 0 || kv != kout) return DDKS_EINVAL;
  const bool dv = kv == 1;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return ctx_cuda_fail(ctx, e, "cudaSetDevice");
  const double* dvp = v;
  double* dop = out;
  if (!dv) {
    int rc = ctx->inP.reserve(ctx, 8 * (size_t)n);
    if (rc == DDKS_OK) rc = ctx->inT.reserve(ctx, 8 * (size_t)n);
    if (rc) return rc;
    e = cudaMemcpyAsync(ctx->inP.ptr, v, 8 * (size_t)n, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return ctx_cuda_fail(ctx, e, "copy rescale input");
    dvp = (const double*)ctx->inP.ptr;
    dop = (double*)ctx->inT.ptr;
  }
  k_rescale<<<grid_cap(n, kThreads, ctx->num_sms * 8), kThreads, 0, st>>>(dvp, n, lo, span, dop);
  e = cudaGetLastError();
  if (e != cudaSuccess) return ctx_cuda_fail(ctx, e, "rescale");
  ctx->launches += 1;
  if (!dv) {
    e = cudaMemcpyAsync(out, dop, 8 * (size_t)n, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return ctx_cuda_fail(ctx, e, "copy rescale output");
  }
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return ctx_cuda_fail(ctx, e, "rescale sync");
  return DDKS_OK;
}

// pooled sizes from which rdKS takes the histogram path (below: sort and walk),
// for up to kRdksHistMaxS corners (its buckets take 12 bytes x 2^16 per corner)
constexpr int64_t kRdksHistMinN = 8192;
constexpr int kRdksHistMaxS = 64;

static int rdks_run(ddks_ctx* ctx, const void* P, int64_t NP, const void* T, int64_t NT, int32_t d, int32_t dtype,
                    void* stream, ddks_result* out, uint64_t* per_corner, bool allow_hist, bool* redo);

int ddks_rdks(ddks_ctx* ctx, const void* P, int64_t NP, const void* T, int64_t NT, int32_t d,
              int32_t dtype, void* stream, ddks_result* out, uint64_t* per_corner) {
  bool redo = false;
  int rc = rdks_run(ctx, P, NP, T, NT, d, dtype, stream, out, per_corner, true, &redo);
  if (rc == DDKS_OK && redo)  // the histogram path met a bucket it does not refine: sort instead
    rc = rdks_run(ctx, P, NP, T, NT, d, dtype, stream, out, per_corner, false, &redo);
  return rc;
}

static int rdks_run(ddks_ctx* ctx, const void* P, int64_t NP, const void* T, int64_t NT, int32_t d, int32_t dtype,
                    void* stream, ddks_result* out, uint64_t* per_corner, bool allow_hist, bool* redo) {
  *redo = false;
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
  const bool hist = allow_hist && N >= kRdksHistMinN && S <= kRdksHistMaxS;
  const bool radix = !hist && N > 1024 && ddks_use_radix(ctx, N, 64);
  if (radix && (rc = ctx->radix.reserve(ctx, 4 * ddks_radix_scratch_words(N, S, 0)))) return out->status = rc;
  // histogram path scratch: partial histograms [S][chunks][B] u32, H [S][B]
  // u64, slot [S][B] i32, cand [S][kMaxCand], fill [S][kMaxCand] u32, kmin
  // [S], kmax [S], ccount [S]
  const int hchunks = (int)((N + kHistChunk - 1) / kHistChunk);
  const size_t a_part = 0, a_H = a_part + 4 * (size_t)S * hchunks * kHistB;
  const size_t a_slot = a_H + 8 * (size_t)S * kHistB, a_cand = a_slot + 4 * (size_t)S * kHistB;
  const size_t a_fill = a_cand + sizeof(RdksCand) * (size_t)S * kMaxCand;
  const size_t a_kmin = (a_fill + 4 * (size_t)S * kMaxCand + 15) & ~(size_t)15;
  const size_t a_kmax = a_kmin + 8 * (size_t)S, a_cc = a_kmax + 8 * (size_t)S;
  const size_t a_bits = (a_cc + 4 * (size_t)S + 15) & ~(size_t)15, a_end = a_bits + 4 * (size_t)S * (kHistB / 32);
  if (hist && (rc = ctx->rdks_aux.reserve(ctx, a_end))) return out->status = rc;
  // warp kernel: shared memory of 2 * d doubles per warp
  int nwb = (int)((96 * 1024) / (16 * (size_t)d));
  nwb = nwb < 1 ? 1 : (nwb > 2 ? 2 : nwb);
  GraphKey key;
  key.add(8).add((uint64_t)NP).add((uint64_t)NT).add((uint64_t)d).add((uint64_t)dtype);
  key.add_ptr(dP).add_ptr(dT).add((uint64_t)ctx->stage_timing).add((uint64_t)hist);
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
      const size_t smem = (size_t)nwb * 16 * (size_t)d;
      const int g = grid_cap(N, nwb, ctx->num_sms * 16);
      if (f64) {
        ee = ddks_smem_attr(k_rdks_dist_warp<double>, (int)smem);
        if (ee == cudaSuccess)
          k_rdks_dist_warp<double><<<g, 32 * nwb, smem, s>>>((const double*)dP, (const double*)dT, NP, NT, d,
                                                             gmin, gmax, keys, flags);
      } else {
        ee = ddks_smem_attr(k_rdks_dist_warp<float>, (int)smem);
        if (ee == cudaSuccess)
          k_rdks_dist_warp<float><<<g, 32 * nwb, smem, s>>>((const float*)dP, (const float*)dT, NP, NT, d,
                                                            gmin, gmax, keys, flags);
      }
      if (ee != cudaSuccess) return ctx_cuda_fail(ctx, ee, "rdks distance attribute");
    }
    ctx->launches += 2;
    ddks_stage_mark(ctx, 1, s);
    if (N <= 1024) {  // sort and walk each corner in one warp
      const int gsm = (int)(((int64_t)S * 32 + kThreads - 1) / kThreads);
      const int E = N <= 32 ? 1 : N <= 64 ? 2 : N <= 128 ? 4 : N <= 256 ? 8 : N <= 512 ? 16 : 32;
      const ull* kk = (const ull*)keys;
      switch (E) {
        case 1: k_rdks_small<1><<<gsm, kThreads, 0, s>>>(kk, (int)N, NP, NT, S, pc); break;
        case 2: k_rdks_small<2><<<gsm, kThreads, 0, s>>>(kk, (int)N, NP, NT, S, pc); break;
        case 4: k_rdks_small<4><<<gsm, kThreads, 0, s>>>(kk, (int)N, NP, NT, S, pc); break;
        case 8: k_rdks_small<8><<<gsm, kThreads, 0, s>>>(kk, (int)N, NP, NT, S, pc); break;
        case 16: k_rdks_small<16><<<gsm, kThreads, 0, s>>>(kk, (int)N, NP, NT, S, pc); break;
        default: k_rdks_small<32><<<gsm, kThreads, 0, s>>>(kk, (int)N, NP, NT, S, pc); break;
      }
      ddks_stage_mark(ctx, 2, s);
      k_rdks_final<<<1, kThreads, 0, s>>>(pc, S, (ull*)sm);
      ctx->launches += 2;
      ee = cudaGetLastError();
      if (ee != cudaSuccess) return ctx_cuda_fail(ctx, ee, "rdks kernels");
      ddks_stage_mark(ctx, 3, s);
      return DDKS_OK;
    }
    if (hist) {
      char* ax = (char*)ctx->rdks_aux.ptr;
      ull* H = (ull*)(ax + a_H);
      uint32_t* part = (uint32_t*)(ax + a_part);
      int* slot = (int*)(ax + a_slot);
      RdksCand* cand = (RdksCand*)(ax + a_cand);
      unsigned* fill = (unsigned*)(ax + a_fill);
      ull* kmin = (ull*)(ax + a_kmin);
      ull* kmax = (ull*)(ax + a_kmax);
      int* ccount = (int*)(ax + a_cc);
      uint32_t* cbits = (uint32_t*)(ax + a_bits);
      ull* gk = (ull*)ctx->tk1.ptr;
      uint8_t* gl = (uint8_t*)ctx->ti1.ptr;
      ee = cudaMemsetAsync(kmin, 0xFF, 8 * (size_t)S, s);
      if (ee == cudaSuccess) ee = ddks_smem_attr(k_rdks_hist, (int)(4 * kHistB));
      if (ee == cudaSuccess) ee = cudaMemsetAsync(kmax, 0, 8 * (size_t)S, s);
      if (ee == cudaSuccess) ee = ddks_smem_attr(k_rdks_refine, (int)kRefineSmem);
      if (ee != cudaSuccess) return ctx_cuda_fail(ctx, ee, "rdks histogram setup");
      int gx = grid_cap(N, kThreads, ctx->num_sms * 8);
      const int per = (ctx->num_sms * 8 + S - 1) / S;
      if (gx > per) gx = per < 1 ? 1 : per;
      const dim3 g2((unsigned)gx, (unsigned)S);
      k_rdks_krange<<<g2, kThreads, 0, s>>>(keys, N, kmin, kmax);
      k_rdks_hist<<<dim3((unsigned)hchunks, (unsigned)S), kHistThreads, 4 * kHistB, s>>>(keys, N, NP, kmin, kmax,
                                                                                        part);
      k_rdks_hist_sum<<<dim3((kHistB + kThreads - 1) / kThreads, (unsigned)S), kThreads, 0, s>>>(part, hchunks, H);
      ddks_stage_mark(ctx, 2, s);
      k_rdks_cands<<<S, kCandThreads, 0, s>>>(H, NP, NT, pc, slot, cand, ccount, fill, cbits, flags);
      k_rdks_gather<<<g2, kThreads, 0, s>>>(keys, N, NP, kmin, kmax, slot, cand, cbits, fill, gk, gl);
      k_rdks_refine_warp<<<dim3(kMaxCand / 2, (unsigned)S), kThreads, 0, s>>>(gk, gl, N, NP, NT, cand, ccount, pc);
      k_rdks_refine<<<dim3(16, (unsigned)S), kThreads, kRefineSmem, s>>>(gk, gl, N, NP, NT, cand, ccount, pc);
      k_rdks_final<<<1, kThreads, 0, s>>>(pc, S, (ull*)sm);
      ctx->launches += 8;
      ee = cudaGetLastError();
      if (ee != cudaSuccess) return ctx_cuda_fail(ctx, ee, "rdks histogram kernels");
      ddks_stage_mark(ctx, 3, s);
      return DDKS_OK;
    }
    const uint64_t* sk;
    const uint32_t *si, *sp;
    int n = 0;
    if (radix) {
      uint32_t* rsx = (uint32_t*)ctx->radix.ptr;
      ee = ddks_radix_sort((const uint64_t*)keys, (uint64_t*)ctx->tk1.ptr, (uint32_t*)ctx->ti1.ptr,
                           (uint64_t*)ctx->tk2.ptr, (uint32_t*)ctx->ti2.ptr, N, N, S, 64, rsx, &sk, &si, s, &n);
      ctx->launches += n;
      if (ee != cudaSuccess) return ctx_cuda_fail(ctx, ee, "rdks sort");
      ddks_stage_mark(ctx, 2, s);
      // per-tile P counts, then the walk with in-tile prefixes
      const unsigned wt = (unsigned)((N + kWalkTile - 1) / kWalkTile);
      uint32_t* tp = (uint32_t*)ctx->apx_cnt.ptr;  // [S][wt]
      k_rdks_ptile<<<dim3(wt, (unsigned)S), kThreads, 0, s>>>(si, N, NP, tp);
      k_rdks_walk_tiles<<<dim3(wt, (unsigned)S), kThreads, 0, s>>>((const ull*)sk, si, tp, N, NP, NT, pc);
      k_rdks_final<<<1, kThreads, 0, s>>>(pc, S, (ull*)sm);
      ctx->launches += 3;
      ee = cudaGetLastError();
      if (ee != cudaSuccess) return ctx_cuda_fail(ctx, ee, "rdks kernels");
      ddks_stage_mark(ctx, 3, s);
      return DDKS_OK;
    } else {
      ee = ddks_launch_sort_segments((const uint64_t*)keys, N, NP, S, (uint64_t*)ctx->tk1.ptr, (uint32_t*)ctx->ti1.ptr,
                                     (uint32_t*)ctx->apx_cnt.ptr, (uint64_t*)ctx->tk2.ptr, (uint32_t*)ctx->ti2.ptr,
                                     (uint32_t*)ctx->apx_U.ptr, &sk, &si, &sp, s, &n);
    }
    ctx->launches += n;
    if (ee != cudaSuccess) return ctx_cuda_fail(ctx, ee, "rdks sort");
    ddks_stage_mark(ctx, 2, s);
    int gx = grid_cap(N, kThreads, ctx->num_sms * 8);
    const int per = (ctx->num_sms * 8 + S - 1) / S;
    if (gx > per) gx = per < 1 ? 1 : per;
    k_rdks_walk<<<dim3((unsigned)gx, (unsigned)S), kThreads, 0, s>>>((const ull*)sk, si, sp, N, Npad, NP, NT, pc);
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
  if (rc == DDKS_OK && (ctx->h_out[4] & ddks::kFlagRedo)) *redo = true;
  return rc;
}
