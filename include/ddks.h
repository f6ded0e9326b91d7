/*
 * ddks.h -- C ABI of the GB300-native exact ddKS library (libddks.so).
 *
 * The d-dimensional Kolmogorov-Smirnov distance of arXiv 2106.13706:
 *
 *   Sec. 2.1, Eq. (ddks_tensor_definition): every point of the pooled sample
 *   P u T is taken in turn as a test point (origin) o.  Every point x of P and
 *   of T gets the orthant code  c(x, o) = sum_m [x_m >= o_m] * 2^m  (the ">="
 *   split of Sec. 2.2.1, Eq. (g): equal coordinates and the origin itself go
 *   to the ">=" side).  cP(o, j) and cT(o, j) count the points of each sample
 *   with code j (Eq. membership), and the statistic is the largest normalised
 *   difference |cP/NP - cT/NT| over origins and orthants (Eq. d1 with the
 *   normalisation of Eq. abs_difference).
 *
 * The library reports the exact integer numerator  num_max =
 * max |cP*NT - cT*NP|  and the denominator NP*NT, so results are bit-exact;
 * D = num_max / (NP*NT) is given as a double for convenience.
 *
 * Conventions shared by every entry point
 *   - P is NP x d, T is NT x d, row-major and contiguous, of element type
 *     dtype (DDKS_F32 = float, DDKS_F64 = double).  Coordinates are compared
 *     as stored: -0.0 equals +0.0, +-inf are ordinary values, NaN is rejected
 *     with DDKS_ENAN.
 *   - P and T may be device pointers (read in place) or host pointers
 *     (pageable or pinned; copied into context-owned device memory first).
 *     The library tells them apart with cudaPointerGetAttributes.  Inputs are
 *     read-only and are not retained after the call returns.
 *   - stream is a cudaStream_t (NULL = the legacy default stream).  Calls are
 *     synchronous: they enqueue their kernels on stream and wait for it.
 *   - 1 <= d <= DDKS_MAX_D; NP, NT >= 1; NP*NT < 2^62.
 *   - Orthant code bit m is [x_m >= o_m].  argmax_origin is the lowest pooled
 *     index (P rows first, then T rows) whose best orthant reaches num_max,
 *     argmax_orthant the lowest code reaching it there (0 when num_max = 0).
 *   - Every function returns DDKS_OK (0) or a negative error code; no
 *     exception crosses the ABI and no device code traps.  A context is not
 *     thread-safe: one host thread at a time (submit/poll excepted, which
 *     lock internally).
 */
#ifndef DDKS_H_
#define DDKS_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DDKS_MAX_D 30
#define DDKS_VDKS_MAX_D 10    /* ddks_vdks: most dimensions */
#define DDKS_RDKS_MAX_D 4096  /* ddks_rdks: most dimensions */

/* return codes */
#define DDKS_OK 0
#define DDKS_PENDING 1          /* ddks_poll: request not finished yet */
#define DDKS_EINVAL (-1)        /* bad shape, dtype, pointer or option */
#define DDKS_ENAN (-2)          /* a coordinate is NaN */
#define DDKS_EOVERFLOW (-3)     /* NP*NT >= 2^62 or a size beyond the kernels' index range */
#define DDKS_ENOMEM (-4)        /* device allocation failed, or a request exceeds the HBM budget */
#define DDKS_ECUDA (-5)         /* a CUDA runtime call failed (see ddks_last_cuda_error) */
#define DDKS_ETIMEOUT (-6)      /* a bounded wait ran out */
#define DDKS_ENOTFOUND (-7)     /* unknown ticket */
#define DDKS_EUNSUPPORTED (-8)  /* valid input that the selected kernel path cannot take */

typedef enum { DDKS_F32 = 0, DDKS_F64 = 1 } ddks_dtype;

/* kernel paths for the orthant counts (DDKS_PATH_AUTO lets the autotuner pick) */
typedef enum {
  DDKS_PATH_AUTO = 0,
  DDKS_PATH_REGISTER = 1,  /* bit-sliced compares, register counters (d = 2..4) */
  DDKS_PATH_LANE = 2,      /* lane-private shared-memory histograms (d <= 8) */
  DDKS_PATH_WARP = 3,      /* one shared-memory histogram per warp and origin (d <= 13) */
  DDKS_PATH_SORT = 4,      /* per-origin sort of codes and segmented counts (any d) */
  DDKS_PATH_DOMINANCE = 5, /* d = 2 only: quadrant counts by range queries, O(N log N) work */
  DDKS_PATH_BYTE = 6       /* byte re-ranks, four dimensions per 32-bit compare, per-origin histograms
                              (2 <= d <= 15, N <= 32768) */
} ddks_path;

typedef struct {
  int32_t device;             /* CUDA device ordinal; -1 = the current device */
  int32_t path;               /* a ddks_path; DDKS_PATH_AUTO by default */
  uint64_t hbm_budget_bytes;  /* serving: device bytes the resident requests may hold (0 = 8 GiB) */
  int32_t max_batch;          /* serving: most requests per device batch (0 = 64) */
  int32_t wait_limit_ms;      /* bound on each host wait (0 = 10000) and, when set, on each
                                 device-side wait for an asynchronous copy (0 = 1000 there) */
  const char* tune_cache;     /* autotuner cache file (NULL = $DDKS_TUNE_CACHE, else none) */
  int32_t graphs;             /* 1 (default): replay CUDA graphs for repeated calls, see below; 0 = off */
  int64_t radix_min_n;        /* pooled sizes N from which the key sorts (the per-dimension ranks of the
                                 exact paths, the rdKS distance orders) run as LSD radix sorts instead of
                                 chunk sorts + merges; 0 = the built-in defaults (16384 for float32
                                 inputs, 131072 for float64 and the rdKS distances), -1 = never */
  int32_t register_variant;   /* the bit-sliced kernel of DDKS_PATH_REGISTER (d = 2..4) when that path is
                                 forced: 0 = automatic (the bit planes staged in global memory by a
                                 pack kernel), 1 = staged by the pack kernel, 2..4 = built in shared
                                 memory by the count kernel itself (where the re-rank tables fit) with count
                                 kernel shape 1..3 (4 warp pairs at 2 CTAs/SM; 4 pairs at 1 CTA/SM,
                                 unrolled; 2 pairs at 3 CTAs/SM) */
  int32_t rank_kernel;        /* the per-dimension ranks of the exact paths: 0 = automatic (float32
                                 inputs: one launch of a thread-block cluster per dimension, sorting in
                                 distributed shared memory, up to about 125k points; otherwise the
                                 multi-launch sorts), 1 = always the multi-launch sorts, 2 = the cluster
                                 launch wherever it fits (float64 too) */
} ddks_config;

typedef struct {
  uint64_t num_max;        /* max over origins and orthants of |cP*NT - cT*NP| */
  uint64_t denom;          /* NP*NT */
  double D;                /* num_max / denom */
  int64_t argmax_origin;   /* see conventions above; -1 if the origin range is empty */
  int32_t argmax_orthant;
  int32_t status;          /* DDKS_OK, or the error of the call that produced it */
} ddks_result;

typedef struct ddks_ctx ddks_ctx;

/* Fill cfg with the defaults listed in ddks_config. */
void ddks_config_default(ddks_config* cfg);

/* Create a context on cfg->device (NULL cfg = defaults).  The context owns all
   device scratch; it grows on demand and is freed by ddks_ctx_destroy.

   Graph replay (cfg.graphs = 1): ddks_distance, ddks_distance_range,
   ddks_permutation_test and ddks_batch_distance enqueue their kernels as one
   CUDA graph when a call repeats an earlier one's shapes (NP, NT, d, dtype,
   origin range, B, the kernel path) and device input addresses.  The second
   such call captures the graph, later ones replay it with one launch.  The
   graph reads the inputs at replay time, so new values at the same addresses
   are seen; the permutation seed is uploaded per call, so it may change.  A
   capture is dropped when the context's scratch has been reallocated since.
   Host inputs are copied into context scratch first and so always repeat.
   While stage timing (ddks_set_stage_timing) is on, calls run kernel by
   kernel, so that the stage events bracket the stages. */
int ddks_ctx_create(const ddks_config* cfg, ddks_ctx** out);
int ddks_ctx_destroy(ddks_ctx* ctx);

/*
 * Exact ddKS of P (NP x d) and T (NT x d): Sec. 2.1, Eq. (ddks_tensor_definition),
 * with the ">=" split of Eq. (g) and the normalisation of Eq. (abs_difference).
 * Writes out->num_max, denom, D, argmax_origin, argmax_orthant.
 */
int ddks_distance(ddks_ctx* ctx, const void* P, int64_t NP, const void* T, int64_t NT,
                  int32_t d, int32_t dtype, void* stream, ddks_result* out);

/*
 * The same statistic restricted to the pooled origins [o_begin, o_end): the
 * building block of an origin-sharded (multi-GPU) computation, where the
 * shards' num_max are combined with max and the argmax is the lowest origin.
 * per_origin (optional, device or host, o_end - o_begin entries) receives
 * each origin's maximum over orthants.
 */
int ddks_distance_range(ddks_ctx* ctx, const void* P, int64_t NP, const void* T, int64_t NT,
                        int32_t d, int32_t dtype, int64_t o_begin, int64_t o_end,
                        uint64_t* per_origin, void* stream, ddks_result* out);

/*
 * Permutation test (Sec. 4.2): the observed statistic, then B relabellings of
 * the pooled sample.  Relabelling b puts into P the NP pooled points with the
 * smallest (key, index), key(b, i) = word (i mod 4) of Philox4x64-10 with
 * counter (i / 4, b, 0, 0) and key (seed, 0) (Salmon et al., SC 2011).
 * perm_num_max (optional host array of B) receives each relabelling's num_max;
 * p_value = (1 + #{b : num_b >= num_obs}) / (1 + B).
 * All B relabellings run as one batched launch; 0 <= B <= 2^20.
 */
int ddks_permutation_test(ddks_ctx* ctx, const void* P, int64_t NP, const void* T, int64_t NT,
                          int32_t d, int32_t dtype, int32_t B, uint64_t seed, void* stream,
                          ddks_result* observed, uint64_t* perm_num_max, double* p_value);

/*
 * One shard of a permutation test split across GPUs by relabelling: the
 * observed statistic and relabellings b in [b_begin, b_end) only, each drawn
 * exactly as in ddks_permutation_test (relabelling b depends on seed and b
 * alone), so the shards of one test reproduce its relabellings whatever the
 * split.  perm_num_max (optional host array of b_end - b_begin) receives their
 * num_max; count_ge (optional) the number with num_b >= num_obs.  Merge: sum
 * count_ge over the shards; p = (1 + sum) / (1 + B) for B relabellings in all.
 * 0 <= b_begin <= b_end, b_end - b_begin <= 2^20.
 */
int ddks_permutation_test_range(ddks_ctx* ctx, const void* P, int64_t NP, const void* T, int64_t NT,
                                int32_t d, int32_t dtype, int64_t b_begin, int64_t b_end, uint64_t seed,
                                void* stream, ddks_result* observed, uint64_t* perm_num_max,
                                uint64_t* count_ge);

/*
 * Analytic significance (Sec. 3, Eq. ddks_significance) of a statistic
 * num_max for these samples: S = 1 - prod over every pooled origin k and
 * orthant j of p(delta <= D; lam_kj), where p(delta <= D; lam) sums
 * Bi(nP; NP, lam) * Bi(nT; NT, lam) (Eq. binomial_probability) over all
 * (nP, nT) with |nP*NT - nT*NP| <= num_max, and lam_kj comes from that cell's
 * T count cT: (cT + 1)/(NT + 2) when estimator = 1 (Bayes, uniform prior),
 * cT/NT when estimator = 0.  model = 1 uses the Poisson pmf with mean m*lam
 * in place of the binomial (the large-sample variant of Sec. 3).
 * d <= 13.  S and log_prod (= log of the product) are written on the host.
 */
int ddks_significance(ddks_ctx* ctx, const void* P, int64_t NP, const void* T, int64_t NT,
                      int32_t d, int32_t dtype, uint64_t num_max, int32_t estimator,
                      int32_t model, void* stream, double* S, double* log_prod);

/*
 * Many independent problems of different sizes and dimensions (Sec. 2.1's
 * statistic for each) batched: problems of up to 16384 pooled points and
 * d <= 11 are ranked in one launch and counted by one persistent launch per
 * dimension present, whose CTAs pull (problem, origin tile) work units from a
 * device counter; larger problems go through ddks_distance.  Arrays have
 * count entries; P[i], T[i] follow the conventions above (all of one dtype,
 * all host or all device); out[i] receives problem i's result.
 */
int ddks_batch_distance(ddks_ctx* ctx, int32_t count, const void* const* P, const int64_t* NP,
                        const void* const* T, const int64_t* NT, const int32_t* d,
                        int32_t dtype, void* stream, ddks_result* out);

/*
 * Tile shape of the batched units for problems of dimension d (1..11).
 * Histogram units: origins per work unit (32, 64 or 128) and points per
 * shared-memory tile (256, 512 or 1024).  Bit-sliced unit (2 <= d <= 6 only):
 * origins_per_unit = 127 (the unit's origins re-rank every point to 7 bits;
 * Sec. 2.2.1, Eq. g) and points per tile 256, 512, 1024 or 2048, rounded to
 * groups of 32.  Byte unit (d = 7 or 8 only): origins_per_unit = 31, 63 or
 * 127 (one origin per thread, each point re-ranked to a byte per dimension)
 * and points per tile 256, 512, 1024 or 2048.  DDKS_EINVAL otherwise.  The
 * defaults: 127 x 512 for 2 <= d <= 8 (bit-sliced up to d = 6, bytes for
 * d = 7, 8), 64 x 512 otherwise.  The results do not depend on the shape.  The paper has no counterpart.
 */
int ddks_set_batch_shape(ddks_ctx* ctx, int32_t d, int32_t origins_per_unit, int32_t points_per_tile);

/*
 * Autotuner of the batched launch: runs this batch with each tile shape (the
 * nine histogram shapes, three bit-sliced shapes for 2 <= d <= 6 and four
 * byte shapes for d = 7, 8), times each dimension group's launch, keeps the fastest shape per
 * dimension in the context, and checks that every shape gives identical
 * results (DDKS_ECUDA if not).  shapes (optional host array of 12 x 2) gets
 * (origins per unit, points per tile) per dimension.  The paper has no
 * counterpart.
 */
int ddks_autotune_batch(ddks_ctx* ctx, int32_t count, const void* const* P, const int64_t* NP,
                        const void* const* T, const int64_t* NT, const int32_t* d, int32_t dtype,
                        void* stream, int32_t* shapes);

/*
 * Serving: submit copies the inputs into library memory (the caller may free
 * them on return) and queues the request; a scheduler thread admits queued
 * requests while their device footprint fits cfg.hbm_budget_bytes and runs
 * the admitted ones together, so requests that arrive while others run join
 * the next device batch.  A request larger than the whole budget is refused
 * with DDKS_ENOMEM.  poll returns DDKS_OK with out filled, DDKS_PENDING, or
 * an error; timeout_us bounds how long poll waits (0 = do not wait).
 * A ticket is released once poll has returned its result.
 */
int ddks_submit(ddks_ctx* ctx, const void* P, int64_t NP, const void* T, int64_t NT, int32_t d,
                int32_t dtype, uint64_t* ticket);
int ddks_poll(ddks_ctx* ctx, uint64_t ticket, int32_t timeout_us, ddks_result* out);

typedef struct {
  uint64_t submitted, admitted, completed, rejected;
  uint64_t batches;            /* device batches launched by the scheduler */
  uint64_t bytes_resident;     /* device bytes held by admitted requests now */
  uint64_t bytes_resident_peak;
  uint64_t kernel_launches;    /* kernels launched by this context so far (graph replays included) */
  uint64_t graph_captures;     /* CUDA graphs captured by this context */
  uint64_t graph_replays;      /* calls served by replaying a captured graph */
} ddks_stats;

int ddks_ctx_stats(ddks_ctx* ctx, ddks_stats* out);

/*
 * Autotune the orthant-count kernel for this problem shape: every kernel path
 * and launch shape that can take it (the bit-sliced register path built for 8,
 * 12 or 16 resident CTAs per SM; lane-private histograms with 64, 128 or 256
 * threads per CTA; per-warp histograms; the sort path; for d = 2 the
 * range-query path) runs on these inputs, timed
 * with CUDA events on stream; all must produce the same statistic.  The
 * fastest is kept for the shape's class (d, log2 NP, log2 NT) in the context
 * and written to the tune cache file when one is configured; later calls with
 * DDKS_PATH_AUTO use it.  chosen_path and best_ms (optional) report it.
 */
int ddks_autotune(ddks_ctx* ctx, const void* P, int64_t NP, const void* T, int64_t NT, int32_t d,
                  int32_t dtype, void* stream, int32_t* chosen_path, float* best_ms);

/*
 * Stage timing.  When enabled, every distance call records CUDA events on its
 * stream around its stages; ddks_stage_times then returns the last call's
 * durations in milliseconds: encode (K0: keys, sort, ranks, and the register
 * path's packing of the points), count (the orthant count kernel), reduce
 * (max over origins).  For ddks_vdks the three stages are the range
 * reduction, the voxel pass (thresholds and counts) and the suffix sums with
 * the orthant evaluation; for ddks_rdks the range reduction with the corner
 * distances, the sort, and the Kolmogorov-Smirnov walk.  Enabling it adds
 * event records, never extra synchronisation beyond the call's own.
 */
int ddks_set_stage_timing(ddks_ctx* ctx, int32_t enable);
int ddks_stage_times(ddks_ctx* ctx, float* encode_ms, float* count_ms, float* reduce_ms);

/*
 * ddks_distance_noalloc: the exact distance of ddks_distance for callers that
 * cannot allocate device memory once they are running -- a latency-critical
 * loop that must not pay cudaMalloc's synchronisation and unbounded latency,
 * a process whose device memory is already reserved by another allocator, or
 * code that must keep a fixed device footprint fixed at start-up.  The paper
 * has no counterpart; this is a calling convention of the library.
 *
 * No context is needed and nothing is allocated: the scratch is one static
 * device array of about 0.7 MiB that every GPU loading the library holds until
 * the process exits.  P and T must already be device memory of the current
 * device, or managed memory (DDKS_EINVAL otherwise, including device memory
 * of another GPU); out is written on the host after the call synchronises
 * stream.  Limits: NP + NT <= 16384 and d <= 8, else DDKS_EUNSUPPORTED.
 * Every call looks up the array's device address on the current device
 * (cudaGetSymbolAddress, which allocates nothing), so a device reset between
 * calls leaves no stale address; make the first call on a device before any
 * stream capture, since that lookup may load the module.  All calls
 * share the one array: calls whose work overlaps on the GPU (other streams or
 * host threads on the same device) race and must be serialised by the caller.
 */
int ddks_distance_noalloc(const void* P, int64_t NP, const void* T, int64_t NT, int32_t d,
                          int32_t dtype, void* stream, ddks_result* out);

/*
 * vdKS, the voxel approximation of Sec. 2.2 (Alg. vdKS).  NormalizeData
 * rescales every dimension of the pooled sample to [0, 1] by its minimum and
 * maximum, x' = (x - lo) / (hi - lo) in IEEE double (0 for a constant
 * dimension).  Each point falls in voxel c with c_m = floor(x'_m * V)
 * (x'_m = 1 in voxel V - 1) of the V^d voxels, V = voxels_per_dim; voxel c
 * holds Diff(c) = nT(c)/NT - nP(c)/NP.  For every voxel filled by either
 * sample, the 2^d orthants around it split the voxels with the ">=" side
 * convention of ddKS (voxel c' on the upper side of dimension m iff
 * c'_m >= c_m), and the statistic is the largest absolute orthant sum of Diff
 * (Alg. vdKS takes a "max" of the orthant sums: read as the largest |sum|,
 * as in Eq. d1).  num_max is that sum times NP*NT, an exact integer;
 * argmax_origin is the lowest filled voxel reaching it (linear index
 * sum_m c_m V^m) and argmax_orthant its lowest orthant code there.
 * 1 <= d <= DDKS_VDKS_MAX_D and V^d <= 2^28 (else DDKS_EUNSUPPORTED);
 * V >= 1.  Coordinates must be finite and every range hi - lo must not
 * overflow (DDKS_EINVAL); NaN gives DDKS_ENAN.  Conventions as above.
 */
int ddks_vdks(ddks_ctx* ctx, const void* P, int64_t NP, const void* T, int64_t NT, int32_t d,
              int32_t dtype, int32_t voxels_per_dim, void* stream, ddks_result* out);

/*
 * rdKS, the radial approximation of Sec. 2.2 (Alg. rdKS).  After the same
 * NormalizeData rescaling as ddks_vdks, the d + 1 corners are the origin
 * (corner 0) and the unit vectors e_m (corner m + 1).  For each corner, the
 * points' squared Euclidean distances to it are compared as two samples by
 * the two-sample Kolmogorov-Smirnov statistic
 * sup_r |F_P(r) - F_T(r)| with F(r) = #{distance <= r} / n (the merge of the
 * two sorted lists in Alg. rdKS, read with absolute differences and after
 * all distances equal to r).  The squared distance of a point is its
 * squared norm s (the squares of x'_m added in dimension order) for the
 * origin and (s - 2 x'_m) + 1 for e_m, each operation rounded in IEEE double,
 * which keeps a point's work linear in d.  num_max is the largest over corners times
 * NP*NT; argmax_origin is the lowest corner reaching it, argmax_orthant 0.
 * per_corner (optional, host or device, d + 1 entries) receives each
 * corner's numerator.  1 <= d <= DDKS_RDKS_MAX_D (rdKS is linear in d; the
 * paper runs it at d = 1000, Sec. 4); (NP + NT) * (d + 1) must stay below
 * about 4e9 (DDKS_EOVERFLOW).  Finite coordinates as for ddks_vdks.
 */
int ddks_rdks(ddks_ctx* ctx, const void* P, int64_t NP, const void* T, int64_t NT, int32_t d,
              int32_t dtype, void* stream, ddks_result* out, uint64_t* per_corner);

/*
 * The NormalizeData rescale of one dimension (Alg. vdKS, Alg. rdKS) as the
 * rdKS distance kernel computes it: out[i] = (v[i] - lo) / span, the
 * subtraction and the division each rounded to nearest in IEEE double (0 for
 * span == 0).  The kernel forms the quotient from RN(1 / span) with FMAs and
 * certifies it by its exact remainder (the division itself where the
 * certificate fails), so out must equal the plain IEEE expression bit for
 * bit.  v, out: n doubles, both device or both host memory.  span >= 0 and
 * finite, lo finite (DDKS_EINVAL otherwise); n >= 0.
 */
int ddks_rescale(ddks_ctx* ctx, const double* v, int64_t n, double lo, double span, double* out, void* stream);

/*
 * Bound on each device-side wait of a kernel for one of its own asynchronous
 * bulk copies (the streamed count and voxel kernels), in nanoseconds of the
 * GPU's global timer; 0 restores the value fixed at creation (the config's
 * wait_limit_ms, else 1 s).  A wait that runs out makes its CTA wait (at most
 * 1 s more) for its copies still in flight and return; the call then returns
 * DDKS_ETIMEOUT and the context stays usable.  A copy normally lands within
 * microseconds, so only a broken device reaches the default bound.  The
 * paper has no counterpart (failure handling of the library).
 */
int ddks_set_device_wait_limit(ddks_ctx* ctx, uint64_t limit_ns);

/*
 * Self-test of the bounded device wait: one kernel arms an mbarrier for a
 * 16-byte transaction that no copy ever delivers and waits with the
 * context's bound.  Returns DDKS_ETIMEOUT (the expected outcome) and the time
 * the wait took in *waited_ns (may be NULL); nothing faults or hangs, and the
 * context remains usable.  Synchronous on stream.  The paper has no
 * counterpart.
 */
int ddks_wait_selftest(ddks_ctx* ctx, void* stream, uint64_t* waited_ns);

/*
 * How every entry point treats an input pointer, from the memory type that
 * cudaPointerGetAttributes reports (cudaMemoryType: 0 unregistered, 1 host,
 * 2 device, 3 managed) and, for device memory, the device that holds it.
 * Returns 1 when the pointer is read in place (device memory of `device`, the
 * device the call runs on, or managed memory), 0 when the call copies it from
 * the host (pinned or pageable host memory), and DDKS_EINVAL for device
 * memory of another GPU or an unknown type: such inputs are refused rather
 * than read across devices.  Pure function; needs no GPU.  The paper has no
 * counterpart.
 */
int ddks_classify_pointer(int32_t memory_type, int32_t pointer_device, int32_t device);

/* Human-readable text for a return code. */
const char* ddks_strerror(int code);

/* The last CUDA error string seen by this context (empty if none). */
const char* ddks_last_cuda_error(ddks_ctx* ctx);

/* Library version, e.g. "0.1.0". */
const char* ddks_version(void);

#ifdef __cplusplus
}
#endif

#endif /* DDKS_H_ */
