/*
 * ddks_oracle.c -- plain, slow, obviously correct CPU oracle for the exact
 * d-dimensional Kolmogorov-Smirnov distance (ddKS) of arXiv 2106.13706.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file: only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header, table or helper with the CUDA
 * path.
 *
 * What it follows, written out loop by loop:
 *   - Sec. 2.1, Eq. (ddks_definition) and Eq. (ddks_tensor_definition): the
 *     statistic is the largest absolute difference of the two samples' orthant
 *     counts, evaluated at every point of P and of T (the pooled sample).
 *   - Sec. 2.1, the loop-based method: for each test point, split space into
 *     the 2^d orthants ("greater than or less than" in every dimension) and
 *     count how many points of each sample fall in each orthant.
 *   - Sec. 2.2.1, Eq. (g): the split uses ">=": coordinate m of point x is on
 *     the "greater" side of the test point o iff x_m >= o_m (ties included).
 *     All pairs are compared, the test point with itself included.
 *   - Sec. 3, Eq. (abs_difference): the counts enter as fractions M/N, so the
 *     cell value is |cP/NP - cT/NT|.  The oracle keeps it as the exact integer
 *     numerator |cP*NT - cT*NP| over the denominator NP*NT.
 *   - Sec. 3, Eq. (binomial_probability) and Eq. (ddks_significance): the
 *     analytic significance, as a plain double sum per cell.
 *   - Sec. 4.2: permutation test over relabellings of the pooled sample.
 *
 * Orthant code convention: bit m of the code is 1 iff x_m >= o_m.
 * Coordinates are compared as stored (float or double) with the C ">="
 * operator, so -0.0 == +0.0 and +-inf are ordinary values.  NaN is rejected.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_EINVAL -1
#define ORC_ENAN -2
#define ORC_EOVERFLOW -3
#define ORC_ENOMEM -4
#define ORC_RDKS_MAX_D 4096

/* coordinate m of pooled point i: P rows first, then T rows */
static double pooled_coord(const void* P, const void* T, int64_t NP, int d,
                           int is_f64, int64_t i, int m) {
  if (i < NP) {
    return is_f64 ? ((const double*)P)[i * d + m] : (double)((const float*)P)[i * d + m];
  }
  int64_t t = i - NP;
  return is_f64 ? ((const double*)T)[t * d + m] : (double)((const float*)T)[t * d + m];
}

static int check_args_dmax(const void* P, int64_t NP, const void* T, int64_t NT, int d, int is_f64,
                           int dmax) {
  if (!P || !T || NP < 1 || NT < 1 || d < 1 || d > dmax) return ORC_EINVAL;
  /* NP*NT must stay below 2^62 so every numerator fits an int64 */
  if ((double)NP * (double)NT >= 4.611686018427387904e18) return ORC_EOVERFLOW;
  int64_t N = NP + NT;
  for (int64_t i = 0; i < N; ++i)
    for (int m = 0; m < d; ++m) {
      double v = pooled_coord(P, T, NP, d, is_f64, i, m);
      if (v != v) return ORC_ENAN;
    }
  return ORC_OK;
}

static int check_args(const void* P, int64_t NP, const void* T, int64_t NT, int d, int is_f64) {
  return check_args_dmax(P, NP, T, NT, d, is_f64, 30);
}

static int cmp_u64(const void* a, const void* b) {
  uint64_t x = *(const uint64_t*)a, y = *(const uint64_t*)b;
  return (x > y) - (x < y);
}

/*
 * The orthant counts of one test point o (pooled index k): for every orthant
 * code j, cP[j] = #{x in P : code(x, o) = j}, cT[j] likewise for T.  Returns
 * the largest |cP[j]*NT - cT[j]*NP| over j and the lowest j reaching it.
 * For d <= 16 the counts live in a dense 2^d array; above that the codes of
 * all points are sorted and equal codes counted, which gives the same counts
 * without a 2^d array (orthants with no point have cP = cT = 0 and add 0).
 */
static uint64_t origin_max(const void* P, const void* T, int64_t NP, int64_t NT, int d,
                           int is_f64, int64_t k, int64_t* cP, int64_t* cT,
                           uint64_t* keys, int32_t* best_j) {
  int64_t N = NP + NT;
  uint64_t best = 0;
  int32_t bj = 0;
  if (d <= 16) {
    int64_t nb = (int64_t)1 << d;
    memset(cP, 0, sizeof(int64_t) * nb);
    memset(cT, 0, sizeof(int64_t) * nb);
    for (int64_t i = 0; i < N; ++i) {
      uint64_t code = 0;
      for (int m = 0; m < d; ++m) {
        double x = pooled_coord(P, T, NP, d, is_f64, i, m);
        double o = pooled_coord(P, T, NP, d, is_f64, k, m);
        if (x >= o) code |= (uint64_t)1 << m;
      }
      if (i < NP) cP[code] += 1; else cT[code] += 1;
    }
    for (int64_t j = 0; j < nb; ++j) {
      int64_t diff = cP[j] * NT - cT[j] * NP;
      uint64_t num = (uint64_t)(diff < 0 ? -diff : diff);
      if (num > best) { best = num; bj = (int32_t)j; }
    }
  } else {
    /* key = code * 2 + (point is from T) */
    for (int64_t i = 0; i < N; ++i) {
      uint64_t code = 0;
      for (int m = 0; m < d; ++m) {
        double x = pooled_coord(P, T, NP, d, is_f64, i, m);
        double o = pooled_coord(P, T, NP, d, is_f64, k, m);
        if (x >= o) code |= (uint64_t)1 << m;
      }
      keys[i] = code * 2 + (i < NP ? 0 : 1);
    }
    qsort(keys, (size_t)N, sizeof(uint64_t), cmp_u64);
    int64_t i = 0;
    int found = 0;
    while (i < N) {
      uint64_t code = keys[i] >> 1;
      int64_t np = 0, nt = 0;
      while (i < N && (keys[i] >> 1) == code) {
        if (keys[i] & 1) nt += 1; else np += 1;
        ++i;
      }
      int64_t diff = np * NT - nt * NP;
      uint64_t num = (uint64_t)(diff < 0 ? -diff : diff);
      /* codes arrive in increasing order, so the first strict improvement is
         the lowest orthant reaching the running maximum */
      if (!found || num > best) { best = num; bj = (int32_t)code; found = 1; }
    }
    /* an empty orthant (count 0, numerator 0) wins only if best is 0 and a
       lower code was empty: report orthant 0 when it is empty then */
    if (best == 0) bj = 0;
  }
  *best_j = bj;
  return best;
}

/*
 * oracle_ddks: exact ddKS over origins [o_begin, o_end) of the pooled sample.
 *   P: NP x d row-major, T: NT x d row-major; is_f64 selects double, else float.
 *   num_max: max numerator |cP*NT - cT*NP|; the distance is num_max/(NP*NT).
 *   argmax_origin: lowest pooled index reaching num_max (P rows first);
 *   argmax_orthant: lowest orthant code reaching it at that origin.
 *   per_origin (optional, length o_end - o_begin): each origin's maximum.
 *   nthreads: OpenMP threads over origins (<= 0: library default).
 */
int oracle_ddks(const void* P, int64_t NP, const void* T, int64_t NT, int d, int is_f64,
                int64_t o_begin, int64_t o_end, int nthreads, uint64_t* num_max,
                int64_t* argmax_origin, int32_t* argmax_orthant, uint64_t* per_origin) {
  int rc = check_args(P, NP, T, NT, d, is_f64);
  if (rc) return rc;
  int64_t N = NP + NT;
  if (o_begin < 0 || o_end > N || o_begin > o_end) return ORC_EINVAL;
  int64_t no = o_end - o_begin;
  uint64_t* po = per_origin ? per_origin : (uint64_t*)malloc(sizeof(uint64_t) * (no > 0 ? no : 1));
  int32_t* pj = (int32_t*)malloc(sizeof(int32_t) * (no > 0 ? no : 1));
  if (!po || !pj) { if (!per_origin) free(po); free(pj); return ORC_ENOMEM; }
  int failed = 0;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel reduction(| : failed)
#endif
  {
    int64_t nb = d <= 16 ? ((int64_t)1 << d) : 1;
    int64_t* cP = (int64_t*)malloc(sizeof(int64_t) * nb);
    int64_t* cT = (int64_t*)malloc(sizeof(int64_t) * nb);
    uint64_t* keys = d > 16 ? (uint64_t*)malloc(sizeof(uint64_t) * N) : NULL;
    if (!cP || !cT || (d > 16 && !keys)) {
      failed = 1;
    } else {
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
      for (int64_t k = o_begin; k < o_end; ++k) {
        po[k - o_begin] = origin_max(P, T, NP, NT, d, is_f64, k, cP, cT, keys, &pj[k - o_begin]);
      }
    }
    free(cP); free(cT); free(keys);
  }
  if (failed) { if (!per_origin) free(po); free(pj); return ORC_ENOMEM; }
  uint64_t best = 0;
  int64_t bk = no > 0 ? o_begin : -1;
  int32_t bj = 0;
  for (int64_t k = 0; k < no; ++k) {
    if (po[k] > best) { best = po[k]; bk = o_begin + k; bj = pj[k]; }
  }
  if (no > 0 && best == 0) bj = pj[0];
  *num_max = best;
  if (argmax_origin) *argmax_origin = bk;
  if (argmax_orthant) *argmax_orthant = bj;
  if (!per_origin) free(po);
  free(pj);
  return ORC_OK;
}

/* ---------------------------------------------------------------------------
 * Philox4x64-10 counter-based generator (Salmon, Moraes, Dror, Shaw, "Parallel
 * random numbers: as easy as 1, 2, 3", SC 2011): ten rounds of two 64x64->128
 * multiplies with the round key bumped by two Weyl constants between rounds.
 * Used to draw the permutation labels of the permutation test (Sec. 4.2).
 * ------------------------------------------------------------------------- */
static void mulhilo64(uint64_t a, uint64_t b, uint64_t* hi, uint64_t* lo) {
  unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
  *hi = (uint64_t)(p >> 64);
  *lo = (uint64_t)p;
}

void oracle_philox4x64_10(const uint64_t ctr_in[4], const uint64_t key_in[2], uint64_t out[4]) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
  const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
  uint64_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint64_t k0 = key_in[0], k1 = key_in[1];
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += W0; k1 += W1; }
    uint64_t hi0, lo0, hi1, lo1;
    mulhilo64(M0, c0, &hi0, &lo0);
    mulhilo64(M1, c2, &hi1, &lo1);
    uint64_t n0 = hi1 ^ c1 ^ k0;
    uint64_t n1 = lo1;
    uint64_t n2 = hi0 ^ c3 ^ k1;
    uint64_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/*
 * Random sort key of pooled point i in permutation b: word (i mod 4) of
 * Philox4x64-10 with counter (i / 4, b, 0, 0) and key (seed, 0).
 */
uint64_t oracle_perm_key(uint64_t seed, int64_t b, int64_t i) {
  uint64_t ctr[4] = {(uint64_t)i / 4, (uint64_t)b, 0, 0};
  uint64_t key[2] = {seed, 0};
  uint64_t out[4];
  oracle_philox4x64_10(ctr, key, out);
  return out[i % 4];
}

typedef struct { uint64_t key; int64_t idx; } keyidx;
static int cmp_keyidx(const void* a, const void* b) {
  const keyidx* x = (const keyidx*)a; const keyidx* y = (const keyidx*)b;
  if (x->key != y->key) return x->key < y->key ? -1 : 1;
  return (x->idx > y->idx) - (x->idx < y->idx);
}

/*
 * Labels of permutation b: the NP pooled points with the smallest
 * (key, index) pairs form the permuted P, the rest the permuted T.
 * is_p[i] = 1 if pooled point i goes to P.
 */
int oracle_perm_labels(uint64_t seed, int64_t b, int64_t NP, int64_t NT, uint8_t* is_p) {
  int64_t N = NP + NT;
  keyidx* ki = (keyidx*)malloc(sizeof(keyidx) * N);
  if (!ki) return ORC_ENOMEM;
  for (int64_t i = 0; i < N; ++i) { ki[i].key = oracle_perm_key(seed, b, i); ki[i].idx = i; }
  qsort(ki, (size_t)N, sizeof(keyidx), cmp_keyidx);
  memset(is_p, 0, (size_t)N);
  for (int64_t r = 0; r < NP; ++r) is_p[ki[r].idx] = 1;
  free(ki);
  return ORC_OK;
}

/*
 * Permutation test (Sec. 4.2): the observed numerator, then for b in [0, B)
 * the numerator of the relabelled pooled sample.  p-value reading:
 * (1 + #{b : num_b >= num_obs}) / (1 + B).
 */
int oracle_permutation_test(const void* P, int64_t NP, const void* T, int64_t NT, int d,
                            int is_f64, int64_t B, uint64_t seed, int nthreads,
                            uint64_t* num_obs, uint64_t* perm_num_max, double* p_value) {
  int rc = check_args(P, NP, T, NT, d, is_f64);
  if (rc) return rc;
  if (B < 0) return ORC_EINVAL;
  int64_t N = NP + NT;
  size_t es = is_f64 ? sizeof(double) : sizeof(float);
  rc = oracle_ddks(P, NP, T, NT, d, is_f64, 0, N, nthreads, num_obs, NULL, NULL, NULL);
  if (rc) return rc;
  uint8_t* is_p = (uint8_t*)malloc((size_t)N);
  char* Pb = (char*)malloc(es * (size_t)NP * d);
  char* Tb = (char*)malloc(es * (size_t)NT * d);
  if (!is_p || !Pb || !Tb) { free(is_p); free(Pb); free(Tb); return ORC_ENOMEM; }
  int64_t ge = 0;
  for (int64_t b = 0; b < B && rc == ORC_OK; ++b) {
    rc = oracle_perm_labels(seed, b, NP, NT, is_p);
    if (rc) break;
    int64_t ip = 0, it = 0;
    for (int64_t i = 0; i < N; ++i) {
      const char* src = i < NP ? (const char*)P + es * (size_t)i * d
                               : (const char*)T + es * (size_t)(i - NP) * d;
      if (is_p[i]) memcpy(Pb + es * (size_t)(ip++) * d, src, es * d);
      else memcpy(Tb + es * (size_t)(it++) * d, src, es * d);
    }
    uint64_t nb = 0;
    rc = oracle_ddks(Pb, NP, Tb, NT, d, is_f64, 0, N, nthreads, &nb, NULL, NULL, NULL);
    if (perm_num_max) perm_num_max[b] = nb;
    if (nb >= *num_obs) ++ge;
  }
  free(is_p); free(Pb); free(Tb);
  if (rc) return rc;
  if (p_value) *p_value = (double)(1 + ge) / (double)(1 + B);
  return ORC_OK;
}

/* ---------------------------------------------------------------------------
 * Analytic significance (Sec. 3).
 * ------------------------------------------------------------------------- */

/* Eq. (binomial_probability): C(m, n) lam^n (1 - lam)^(m - n); model 1 uses
   the Poisson pmf with mean m*lam instead (the large-m variant of Sec. 3). */
static double cell_pmf(int64_t n, int64_t m, double lam, int model) {
  /* degenerate rates: all mass on n = 0 (lam = 0) or, binomially, n = m */
  if (lam <= 0.0) return n == 0 ? 1.0 : 0.0;
  if (lam >= 1.0 && model != 1) return n == m ? 1.0 : 0.0;
  if (model == 1) {
    double mu = (double)m * lam;
    return exp((double)n * log(mu) - mu - lgamma((double)n + 1.0));
  }
  return exp(lgamma((double)m + 1.0) - lgamma((double)n + 1.0) - lgamma((double)(m - n) + 1.0) +
             (double)n * log(lam) + (double)(m - n) * log1p(-lam));
}

/*
 * p(delta <= D) for one cell with rate lam: the sum over every pair
 * (nP, nT), 0 <= nP <= NP, 0 <= nT <= NT, whose normalised difference
 * |nP/NP - nT/NT| does not exceed D = num_max/(NP*NT), of
 * pmf(nP; NP, lam) * pmf(nT; NT, lam).  The test is done on the exact
 * integers: |nP*NT - nT*NP| <= num_max.
 */
double oracle_cell_p_le(int64_t NP, int64_t NT, uint64_t num_max, double lam, int model) {
  double s = 0.0;
  for (int64_t np = 0; np <= NP; ++np) {
    for (int64_t nt = 0; nt <= NT; ++nt) {
      int64_t diff = np * NT - nt * NP;
      uint64_t a = (uint64_t)(diff < 0 ? -diff : diff);
      if (a <= num_max) s += cell_pmf(np, NP, lam, model) * cell_pmf(nt, NT, lam, model);
    }
  }
  return s;
}

/*
 * Eq. (ddks_significance): S = 1 - prod over every origin k of the pooled
 * sample and every orthant j of p(delta <= D; lam_kj), lam_kj estimated from
 * the T count of that cell: (cT + 1)/(NT + 2) (Bayes estimator with a uniform
 * prior, estimator 1) or cT/NT (estimator 0).  The product is accumulated as
 * a sum of logs.  The cell probability depends on the cell only through cT,
 * so it is evaluated once per distinct cT value.  log_prod receives the
 * log of the product (S = 1 - exp(log_prod)).
 */
int oracle_significance(const void* P, int64_t NP, const void* T, int64_t NT, int d, int is_f64,
                        uint64_t num_max, int estimator, int model, double* S, double* log_prod) {
  int rc = check_args(P, NP, T, NT, d, is_f64);
  if (rc) return rc;
  if (d > 16) return ORC_EINVAL;
  int64_t N = NP + NT;
  int64_t nb = (int64_t)1 << d;
  double* memo = (double*)malloc(sizeof(double) * (NT + 1));
  char* have = (char*)calloc((size_t)(NT + 1), 1);
  int64_t* cP = (int64_t*)malloc(sizeof(int64_t) * nb);
  int64_t* cT = (int64_t*)malloc(sizeof(int64_t) * nb);
  if (!memo || !have || !cP || !cT) { free(memo); free(have); free(cP); free(cT); return ORC_ENOMEM; }
  double acc = 0.0;
  for (int64_t k = 0; k < N; ++k) {
    memset(cP, 0, sizeof(int64_t) * nb);
    memset(cT, 0, sizeof(int64_t) * nb);
    for (int64_t i = 0; i < N; ++i) {
      uint64_t code = 0;
      for (int m = 0; m < d; ++m) {
        double x = pooled_coord(P, T, NP, d, is_f64, i, m);
        double o = pooled_coord(P, T, NP, d, is_f64, k, m);
        if (x >= o) code |= (uint64_t)1 << m;
      }
      if (i < NP) cP[code] += 1; else cT[code] += 1;
    }
    for (int64_t j = 0; j < nb; ++j) {
      int64_t mt = cT[j];
      if (!have[mt]) {
        double lam = estimator == 1 ? ((double)mt + 1.0) / ((double)NT + 2.0)
                                    : (double)mt / (double)NT;
        memo[mt] = oracle_cell_p_le(NP, NT, num_max, lam, model);
        have[mt] = 1;
      }
      acc += log(memo[mt]);
    }
  }
  free(memo); free(have); free(cP); free(cT);
  if (log_prod) *log_prod = acc;
  if (S) *S = 1.0 - exp(acc);
  return ORC_OK;
}

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------ vdKS, rdKS
 *
 * The two approximations of Sec. 2.2 (Alg. vdKS, Alg. rdKS), step by step in
 * the algorithms' order, with the readings of the garbled or silent points:
 *   - NormalizeData / the normalised sample space: per dimension, the pooled
 *     sample is shifted and rescaled to [0, 1] with its minimum and maximum,
 *     x' = (x - lo) / (hi - lo); a constant dimension maps to 0.  The
 *     rescaling needs a finite range: an infinite coordinate, or a range
 *     hi - lo that overflows to infinity, is rejected (ORC_EINVAL).
 *   - vdKS IndexFromPoint: voxel coordinate c_m = floor(x'_m * V), with
 *     x'_m = 1 put in the last voxel V - 1.
 *   - vdKS SumOrthants: the orthants around a filled voxel c split the voxel
 *     grid with the same ">=" convention as ddKS (voxel c' is on the upper
 *     side of dimension m iff c'_m >= c_m); the statistic is the largest
 *     ABSOLUTE orthant sum of Diff = (T fraction - P fraction) over the voxels
 *     filled by either sample.  Exact integer numerator: Diff * NP * NT =
 *     nT * NP - nP * NT per voxel.
 *   - rdKS IdentifyCorners: the d + 1 corners are the origin and the d unit
 *     vectors of the normalised space; distances are Euclidean, compared as
 *     squared distances.  rdKS is linear in d (Sec. 2.2, Sec. 4), so a
 *     point's squared distances come from its squared norm
 *     s = x'_0^2 + ... + x'_{d-1}^2 (added in dimension order): s itself for
 *     the origin and (s - 2 x'_m) + 1 for the unit vector e_m, each operation
 *     rounded in IEEE double (no fused multiply-add).
 *   - rdKS GetDFromCornerLists: the two-sample Kolmogorov-Smirnov statistic
 *     of the two sorted distance lists, sup_r |F_P(r) - F_T(r)| with
 *     F(r) = #{distance <= r} / n, i.e. evaluated after all distances equal
 *     to r; the statistic is the largest over the corners.
 */

static int normalise(const void* P, int64_t NP, const void* T, int64_t NT, int d, int is_f64,
                     double* out) {
  const int64_t N = NP + NT;
  for (int m = 0; m < d; ++m) {
    double lo = pooled_coord(P, T, NP, d, is_f64, 0, m), hi = lo;
    for (int64_t i = 1; i < N; ++i) {
      const double v = pooled_coord(P, T, NP, d, is_f64, i, m);
      if (v < lo) lo = v;
      if (v > hi) hi = v;
    }
    const double span = hi - lo;
    if (!isfinite(lo) || !isfinite(hi) || !isfinite(span)) return ORC_EINVAL;
    for (int64_t i = 0; i < N; ++i) {
      const double v = pooled_coord(P, T, NP, d, is_f64, i, m);
      out[i * d + m] = span > 0.0 ? (v - lo) / span : 0.0;
    }
  }
  return ORC_OK;
}

int oracle_vdks(const void* P, int64_t NP, const void* T, int64_t NT, int d, int is_f64, int V,
                uint64_t* num_max, int64_t* argmax_voxel /* or NULL */, int32_t* argmax_orthant /* or NULL */) {
  int rc = check_args(P, NP, T, NT, d, is_f64);
  if (rc) return rc;
  if (V < 1 || !num_max) return ORC_EINVAL;
  double cells_d = 1.0;
  for (int m = 0; m < d; ++m) cells_d *= V;
  if (cells_d > (double)(1 << 24)) return ORC_EINVAL;
  const int64_t cells = (int64_t)cells_d, N = NP + NT;
  double* xn = (double*)malloc(sizeof(double) * (size_t)(N * d));
  int64_t* diff = (int64_t*)calloc((size_t)cells, sizeof(int64_t));
  unsigned char* filled = (unsigned char*)calloc((size_t)cells, 1);
  int* coord = (int*)malloc(sizeof(int) * (size_t)d);
  int* ccur = (int*)malloc(sizeof(int) * (size_t)d);
  int64_t* osum = (int64_t*)malloc(sizeof(int64_t) * ((size_t)1 << d));
  if (!xn || !diff || !filled || !coord || !ccur || !osum) {
    free(xn); free(diff); free(filled); free(coord); free(ccur); free(osum);
    return ORC_ENOMEM;
  }
  if (normalise(P, NP, T, NT, d, is_f64, xn) != ORC_OK) {
    free(xn); free(diff); free(filled); free(coord); free(ccur); free(osum);
    return ORC_EINVAL;
  }
  /* voxel occupation: Diff numerator nT * NP - nP * NT */
  for (int64_t i = 0; i < N; ++i) {
    int64_t idx = 0, stride = 1;
    for (int m = 0; m < d; ++m) {
      int c = (int)floor(xn[i * d + m] * (double)V);
      if (c > V - 1) c = V - 1;
      idx += (int64_t)c * stride;
      stride *= V;
    }
    diff[idx] += i < NP ? -(int64_t)NT : (int64_t)NP;
    filled[idx] = 1;
  }
  uint64_t best = 0;
  int64_t bf = -1; /* the lowest filled voxel, then the lowest orthant, reaching the max */
  int bjj = 0;
  for (int64_t f = 0; f < cells; ++f) {
    if (!filled[f]) continue;
    int64_t r = f;
    for (int m = 0; m < d; ++m) { coord[m] = (int)(r % V); r /= V; }
    for (int j = 0; j < (1 << d); ++j) osum[j] = 0;
    /* every voxel goes to the orthant of its sides relative to voxel f */
    for (int64_t c = 0; c < cells; ++c) {
      int64_t t = c;
      int code = 0;
      for (int m = 0; m < d; ++m) {
        ccur[m] = (int)(t % V);
        t /= V;
        if (ccur[m] >= coord[m]) code |= 1 << m;
      }
      osum[code] += diff[c];
    }
    for (int j = 0; j < (1 << d); ++j) {
      const uint64_t a = (uint64_t)(osum[j] < 0 ? -osum[j] : osum[j]);
      if (a > best || bf < 0) { best = a; bf = f; bjj = j; }
    }
  }
  *num_max = best;
  if (argmax_voxel) *argmax_voxel = bf;
  if (argmax_orthant) *argmax_orthant = bjj;
  free(xn); free(diff); free(filled); free(coord); free(ccur); free(osum);
  return ORC_OK;
}

typedef struct {
  double r;
  int is_t;
} orc_dist;

static int cmp_dist(const void* a, const void* b) {
  const double x = ((const orc_dist*)a)->r, y = ((const orc_dist*)b)->r;
  return x < y ? -1 : (x > y ? 1 : 0);
}

int oracle_rdks(const void* P, int64_t NP, const void* T, int64_t NT, int d, int is_f64,
                uint64_t* num_max, uint64_t* per_corner /* d + 1 entries or NULL */) {
  /* rdKS is linear in d (Sec. 2.2, and the 1000-dimensional study of Sec. 4),
     so it takes up to ORC_RDKS_MAX_D dimensions rather than ddKS's 30 */
  int rc = check_args_dmax(P, NP, T, NT, d, is_f64, ORC_RDKS_MAX_D);
  if (rc) return rc;
  if (!num_max) return ORC_EINVAL;
  const int64_t N = NP + NT;
  double* xn = (double*)malloc(sizeof(double) * (size_t)(N * d));
  double* norm2 = (double*)malloc(sizeof(double) * (size_t)N);
  orc_dist* list = (orc_dist*)malloc(sizeof(orc_dist) * (size_t)N);
  if (!xn || !norm2 || !list) { free(xn); free(norm2); free(list); return ORC_ENOMEM; }
  if (normalise(P, NP, T, NT, d, is_f64, xn) != ORC_OK) {
    free(xn); free(norm2); free(list);
    return ORC_EINVAL;
  }
  uint64_t best = 0;
  /* squared norms in the normalised space, added in dimension order */
  for (int64_t i = 0; i < N; ++i) {
    double s = 0.0;
    for (int m = 0; m < d; ++m) {
      const double x = xn[i * d + m];
      const double sq = x * x;
      s = s + sq;
    }
    norm2[i] = s;
  }
  for (int corner = 0; corner <= d; ++corner) {
    /* corner 0: the origin, |x'|^2; corner m + 1: unit vector m,
       |x' - e_m|^2 = (|x'|^2 - 2 x'_m) + 1 */
    for (int64_t i = 0; i < N; ++i) {
      double r = norm2[i];
      if (corner > 0) {
        const double x = xn[i * d + corner - 1];
        const double t = r - 2.0 * x;
        r = t + 1.0;
      }
      list[i].r = r;
      list[i].is_t = i >= NP;
    }
    qsort(list, (size_t)N, sizeof(orc_dist), cmp_dist);
    int64_t cp = 0, ct = 0;
    uint64_t cb = 0;
    for (int64_t i = 0; i < N; ++i) {
      if (list[i].is_t) ++ct; else ++cp;
      if (i + 1 < N && list[i + 1].r == list[i].r) continue;  /* after all equal distances */
      const int64_t x = cp * NT, y = ct * NP;
      const uint64_t v = (uint64_t)(x > y ? x - y : y - x);
      if (v > cb) cb = v;
    }
    if (per_corner) per_corner[corner] = cb;
    if (cb > best) best = cb;
  }
  *num_max = best;
  free(xn); free(norm2); free(list);
  return ORC_OK;
}
