/*
 * qwlsh.h -- C ABI of the GB300 LSH query-workload library (libqwlsh.so).
 *
 * The library builds an LSH index over n float32 vectors and answers a whole
 * workload of k-nearest-neighbour queries against it, following the method of
 * arXiv 1907.11803 and the LSH variants it builds on:
 *   - hash family (Section 3): h_i(v) = floor((a_i . v + b_i) / w),
 *     a_i ~ N(0, I_d), b_i ~ U[0, w);
 *   - collision counting over m hash functions with a threshold l and at most
 *     k + v candidates read per query (Section 3.1);
 *   - virtual rehashing: the lookup range of every projection grows by the
 *     factor c per level, served by range searches over one sorted structure
 *     per hash function (Section 2);
 *   - exact Euclidean top-k over the candidates (Section 3, c-k-ANN; Section 4
 *     workload of |Q| queries).
 *
 * Conventions shared by every entry point:
 *   - Arrays are row-major and contiguous.  float32 inputs, int32/int64 ids.
 *   - Ownership: every buffer passed in or out belongs to the caller and is
 *     only read / written during the call (or, for device-memory calls, by the
 *     work the call enqueues on `stream`).  The library owns the index handle
 *     and the device workspace inside it.
 *   - `mem` says where the caller's buffers live: QW_MEM_DEVICE (device
 *     pointers; the call enqueues work on `stream` and returns; outputs are
 *     valid once the stream reaches that point) or QW_MEM_HOST (host pointers;
 *     the call copies in, computes, copies out, and returns with the outputs
 *     written).
 *   - `stream` is a cudaStream_t passed as void*; NULL means the legacy default
 *     stream.
 *   - Errors: every function returns a qw_status; nothing throws across the
 *     ABI.  On failure qw_last_error() gives a message for the calling thread.
 *     Invalid arguments are rejected before any work is enqueued.
 *   - One index handle must not be used by two calls at the same time.
 */
#ifndef QWLSH_H
#define QWLSH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t qw_status;
#define QW_OK 0
#define QW_ERR_ARG 1      /* invalid argument (null pointer, bad size, unsupported field) */
#define QW_ERR_OOM 2      /* device or host allocation failed */
#define QW_ERR_CUDA 3     /* a CUDA runtime call or kernel launch failed */
#define QW_ERR_TIMEOUT 4  /* a bounded device loop ran out of iterations */
#define QW_ERR_RANGE 5    /* a bucket id or bucket span does not fit in int32 */

#define QW_MEM_DEVICE 0
#define QW_MEM_HOST 1

/* Number of int64 statistics written per query by qw_run_workload. */
#define QW_NSTAT 8
/* Statistic slots (per query):
 *  0 levels run (1 = stopped at radius R = 1)
 *  1 radius R of the last level
 *  2 |C_R|, candidates (collision count >= l) at the last level
 *  3 candidates kept after the k + v bound
 *  4 termination: 2 = |C_R| >= k + v; 3 = R exceeds every bucket id of the
 *    data and of the query, so no further level can change C_R (QALSH: every
 *    projection's interval holds the whole data)
 *  5 sorted index entries inside the last level's bucket ranges, summed over
 *    projections (the entries an incremental scan reads in total)
 *  6 sum over levels of the entries inside that level's ranges
 *  7 |C_{R/c}|, candidates at the level before the last */

/* Largest supported values. */
#define QW_MAX_M 127          /* projections per index (collision counts are 7-bit) */
#define QW_MAX_CLUSTER_TILES 96  /* index tiles the cluster path can hold */
#define QW_MAX_CAND 4096      /* k + v */

typedef struct qw_index qw_index;

/* Index parameters (Sections 3, 3.1, 6). */
typedef struct {
    int32_t m;     /* number of hash functions / projections, 1..QW_MAX_M */
    float w;       /* bucket width w > 0 */
    int32_t c;     /* approximation ratio, also the per-level radius factor; integer >= 2 */
    int32_t v;     /* allowed false positives (Section 3.1 uses 100); >= 0 */
    int32_t l;     /* collision threshold 1..m; 0 = derive from Eq. 1 (see
                      qw_collision_threshold) with beta = v / n */
    float delta;   /* error probability used when deriving l; <= 0 means 1/e (Section 6) */
    int32_t shadow_bf16;  /* non-zero: also keep a BF16 copy of the data for the
                             QW_RERANK_BF16 pre-filter: rows in the rerank's row order (the
                             locality order when bitmaps are built) grouped by 128, each stored
                             as the BF16 residual r~ to its group's mean C_g (kept in BF16),
                             with a residual-norm bound and the constants C_g . r~ and |r~|^2
                             per row (2 * n * d + 12 * n + 2 * d * ceil(n / 128) bytes) */
    int32_t bitmaps;      /* non-zero: also build the level bitmaps of QW_PATH_BITMAP: per
                             projection i, id tile and level L, one bitmap of the tile's ids
                             per level-L bucket; about m * n_tiles * (c/(c-1)) * (span_i + 1)
                             * 4 KiB (qw_index_info.bitmap_bytes) */
    int32_t host_bitmaps; /* non-zero (with bitmaps): keep the level bitmaps in pinned host
                             memory that the kernels read directly (on GB300 the Grace
                             memory, over NVLink-C2C) -- an index larger than the GPU's
                             memory, the paper's external-storage setting.  The bitmap path
                             then reads them with plain loads (QW_LOADS_TMA acts as
                             QW_LOADS_DIRECT).  Same results */
    uint64_t seed;        /* used only when qw_build_index gets A == NULL and b == NULL: the
                             projections are then drawn on the host by qw_draw_projections(seed,
                             m, d, w, ...); read them back with qw_index_get_projections */
    int32_t projection;   /* QW_PROJ_FP32 (default) or QW_PROJ_TENSOR: how the data are
                             projected at build time (same bucket ids) */
    int32_t family;       /* hash family (QW_FAMILY_*, below); default QW_FAMILY_E2LSH */
} qw_index_params;

/* Hash families (qw_index_params.family).
 *
 * QW_FAMILY_E2LSH (0): Section 3's h(v) = floor((a . v + b) / w) with anchored
 * bucket ids and virtual rehashing (C2LSH): at radius R an object collides on
 * projection i when floor(bid / R) equals the query's.
 *
 * QW_FAMILY_QALSH (1): QALSH's query-aware buckets (Section 2; the method the
 * paper's experiments build on, Section 6, w = 2.719).  The hash is the
 * projection p_i(v) = a_i . v itself (b is not used), computed in FP64 with the
 * products summed in coordinate order; at radius R an object collides on
 * projection i when |p_i(o) - p_i(q)| <= w R / 2 (the difference rounded once
 * in FP64, ends included).  The radius rule: a query stops at the first R at
 * which every projection's interval holds the whole data.  The threshold l,
 * the k + v bound, truncation and top-k are unchanged; l = 0 derives l from
 * QALSH's collision probability (qw_qalsh_collision_threshold).  Layout: per
 * projection and id tile, the tile's FP64 projections in ascending order with
 * their 16-bit in-tile ids (10 bytes per entry).  Runs on the level path only:
 * no bitmaps, learned start levels, multi-probe, tensor-core projection or
 * bucket-signature order (the workload runs in the given order). */
#define QW_FAMILY_E2LSH 0
#define QW_FAMILY_QALSH 1

/* Per-workload options.  Zero-initialise; unknown non-zero fields are rejected. */
typedef struct {
    int32_t batch;        /* queries per pass over the index; 0 = library choice */
    int32_t profile;      /* non-zero: time every kernel launch with CUDA events on the call's
                             stream and add the times to the index's profile (see
                             qw_index_profile); the call then waits for the stream */
    int32_t path;         /* QW_PATH_AUTO, QW_PATH_CLUSTER or QW_PATH_LEVELS (below) */
    int32_t clusters;     /* cluster path: most clusters resident at once; 0 = all that fit */
    int32_t order;        /* QW_ORDER_AUTO / QW_ORDER_SIGNATURE: answer queries grouped by a
                             coarse bucket signature (queries of one region share index
                             entries in L2); QW_ORDER_GIVEN: in the caller's order.  Results are
                             returned in the caller's order either way and do not depend on it */
    int32_t rerank;       /* QW_RERANK_FP32 (default), QW_RERANK_BF16 or QW_RERANK_BF16_TC
                             (both need shadow_bf16): the BF16 pre-filter on CUDA cores, or with
                             its dot products q . r~ on the tensor cores (tcgen05, FP32
                             accumulation in tensor memory, a certified bound per candidate);
                             both keep every candidate that could be among the k nearest for
                             the exact FP32 / FP64 stages.  Same results */
    int32_t start;        /* QW_START_PLAIN (default) or QW_START_LEARNED (level path; needs a
                             start model, see qw_index_set_start_model) */
    int32_t graph;        /* non-zero (level path): each batch's level loop runs as one CUDA
                             graph whose conditional WHILE node advances the level on the
                             device, so the host does not wait inside a batch; the call waits
                             for the stream once at its end.  Same kernels, same results */
    int32_t bitmap_loads; /* QW_PATH_BITMAP: QW_LOADS_TMA (default) stages the bucket bitmaps
                             in shared memory with TMA bulk copies in a persistent kernel;
                             QW_LOADS_DIRECT runs a summary filter, then counts the live
                             128-id groups with plain loads in a second launch;
                             QW_LOADS_FUSED does both in one launch, one warp per (query,
                             run of tiles).  Same results */
    int32_t l2_mode;      /* persisting-L2 division between the index and the data (the
                             workload cache split of Section 4, on the GPU's L2): QW_L2_OFF
                             (default) attaches no access-policy window; QW_L2_SPLIT gives
                             l2_index_permille of the set-aside to the index window and the
                             rest to the data window; QW_L2_MODEL takes the split from
                             qw_l2_split_model.  Speed only: the results do not change */
    int32_t l2_index_permille;  /* QW_L2_SPLIT: 0..1000, the paper's size(C_I) / size(C) */
    int32_t projection;   /* QW_PROJ_FP32 (default): the queries' projection on CUDA cores in
                             FP32; QW_PROJ_TENSOR: on the tensor cores (split BF16 products,
                             FP32 accumulation, m <= 128; see qw_hash_tc).  Same bucket ids */
    int32_t rerank_rows;  /* tile shape of the distance kernels: candidate rows a warp takes
                             at a time (2, 4 or 8; 0 = 4).  Same results */
    int32_t tiles_per_warp; /* tile shape of the bitmap path's filter and fused kernels: id
                             tiles a warp walks for one query (4, 8 or 16; 0 = 8).  Same
                             results */
    int32_t probes;       /* multi-probe (Section 2 on probing the neighbouring buckets of the
                             query's bucket): at radius R an object collides on projection i
                             when its level-R bucket floor(bid / R) lies within `probes` of the
                             query's, i.e. bid in [(beta_i - probes) R, (beta_i + probes + 1) R
                             - 1]; the radius rule then also waits for R > -g_i.  0 (default):
                             the plain rule.  0..64; > 0 runs on the level path (QW_PATH_AUTO
                             and QW_PATH_LEVELS; the bitmap and cluster paths refuse it).
                             Changes the candidate sets, as it changes the method */
} qw_query_params;

/* Persisting-L2 modes (qw_query_params.l2_mode).  With a window mode the call
 * attaches an access-policy window over the index structure that every
 * (query, tile, level) pass reads first (bucket summaries on the bitmap path,
 * sorted id arrays on the level path) to the collision-counting launches, and
 * one over the data rows the candidates are read from to the rerank launch,
 * each with the hit ratio that makes its persisting footprint its share of
 * the set-aside, and puts the stream's window attribute back before
 * returning.  The index's first such call raises the context's persisting-L2
 * set-aside (cudaLimitPersistingL2CacheSize) to the device maximum; it stays
 * raised, shared by the whole context, until qw_index_free, or a later call
 * on the index with QW_L2_OFF, puts back the value found and demotes the
 * persisting lines (cudaCtxResetPersistingL2Cache).
 * Nothing outlives the process.  On the legacy default stream (NULL), or where
 * the device has no set-aside (MIG, MPS), the call runs without windows. */
#define QW_L2_OFF 0
#define QW_L2_SPLIT 1
#define QW_L2_MODEL 2

#define QW_PROJ_FP32 0
#define QW_PROJ_TENSOR 1

#define QW_LOADS_TMA 0
#define QW_LOADS_DIRECT 1
#define QW_LOADS_FUSED 2

/* First level of the collision-counting loop.  QW_START_PLAIN: every query
 * starts at radius R = 1.  QW_START_LEARNED: the index's start model predicts,
 * per query, the level at which it stops; the query begins at the largest
 * level s whose predicted probability of stopping at or before s is at most
 * eps, counting its whole bucket range there.  A query that nevertheless stops
 * at its first level is answered again from R = 1, so the results (ids,
 * distances, statistics) equal the plain ones. */
#define QW_START_PLAIN 0
#define QW_START_LEARNED 1

/* Candidate distance stage.  QW_RERANK_FP32: FP32 distances of every kept
 * candidate, FP64 for neighbours FP32 cannot order.  QW_RERANK_BF16: distance
 * bounds from the residual BF16 copy first (see shadow_bf16): |q - C_g - r~|^2
 * expanded as |q - C_g|^2 - 2 q.r~ + 2 C_g.r~ + |r~|^2, so a candidate costs
 * one FP32 dot product with its BF16 row and |q - C_g|^2 is formed once per
 * distinct group, with a proven error bound; only candidates that could still
 * be among the k nearest go through the FP32/FP64 stage.  QW_RERANK_BF16_TC:
 * the same pre-filter with the
 * candidates' residual rows multiplied by the query on the tensor cores
 * (tcgen05.mma, BF16 operands, the query split into BF16 hi + lo parts, FP32
 * accumulation in tensor memory; the per-row constants C_g . r~ and |r~|^2
 * kept with the residual copy) and its own proven bound.  All three return the
 * same ids and distances. */
#define QW_RERANK_FP32 0
#define QW_RERANK_BF16 1
#define QW_RERANK_BF16_TC 2

#define QW_ORDER_AUTO 0
#define QW_ORDER_SIGNATURE 1
#define QW_ORDER_GIVEN 2

/* Execution paths of the query loop (identical results):
 * QW_PATH_LEVELS: one launch per level over (index tile, query) pairs, collision
 *   counters in device memory between levels; any index size.
 * QW_PATH_CLUSTER: one persistent launch of thread-block clusters; a cluster
 *   answers one query at a time with its counters in shared memory for all
 *   levels and pulls the next query from a work queue; indexes of up to
 *   96 tiles (3,145,728 points).
 * QW_PATH_BITMAP: the level loop of QW_PATH_LEVELS, but the collision counts
 *   of a (tile, query) are recomputed at every level as the bit-sliced sum of
 *   the m precomputed bitmaps of the query's level-L buckets (no per-entry
 *   work, no counters kept between levels); needs an index built with bitmaps.
 * QW_PATH_AUTO: the path qw_autotune chose for the index, else the level path. */
#define QW_PATH_AUTO 0
#define QW_PATH_CLUSTER 1
#define QW_PATH_LEVELS 2
#define QW_PATH_BITMAP 3

/* Kernel classes of the query path, for qw_profile. */
#define QW_K_PROJECT 0   /* query projection + FP64 boundary pass */
#define QW_K_SETUP 1     /* per-query state */
#define QW_K_LEVEL 2     /* bucket-range search + collision counting, one launch per level
                            (bitmap path with direct loads and a host-driven loop: the
                            summary filter and the count pass only, see QW_K_BUCKET) */
#define QW_K_DECIDE 3    /* per-level termination test */
#define QW_K_SELECT 4    /* candidate selection under the k + v bound */
#define QW_K_RERANK 5    /* candidate distances + top-k */
#define QW_K_CLUSTER 6   /* cluster path: every level, the stop test and the selection of a
                            query in one persistent launch */
#define QW_K_ORDER 7     /* workload ordering: signature sort, gather, scatter of results */
#define QW_K_START 8     /* learned start levels: features + network forward */
#define QW_K_BUCKET 9    /* bitmap path, direct loads, host-driven loop: the bitmap numbers of
                            the query's buckets before each level's filter (in graph mode they
                            are part of QW_K_LEVEL) */
#define QW_K_COUNT 10

/* Launch counts and (profile mode) summed kernel times of qw_run_workload /
 * qw_workload_candidates calls on one index since the last reset. */
typedef struct {
    int64_t launches[QW_K_COUNT];  /* kernels launched, per class (always counted) */
    double ms[QW_K_COUNT];         /* summed CUDA-event durations, per class (profile mode) */
    int64_t timed_launches[QW_K_COUNT];  /* launches included in ms[] */
    int64_t queries;               /* queries answered */
    int64_t rerank_candidates;     /* kept candidates reranked (profile mode) */
    int64_t rerank_fp32_rows;      /* of those, read in FP32 (profile mode; BF16 pre-filter) */
    int64_t start_levels_skipped;  /* levels skipped by learned starts (always counted) */
    int64_t start_fallbacks;       /* queries recomputed from R = 1 (always counted) */
    int64_t level_passes;          /* (query, level) pairs counted by the level paths
                                      (profile mode) */
    int64_t bitmap_fallbacks;      /* QW_PATH_BITMAP queries answered by the level path: a
                                      last level whose kept entries and tie class do not fit
                                      the candidate list even when rebuilt (always counted;
                                      same results) */
    int64_t bitmap_live_items;     /* QW_PATH_BITMAP, direct loads: (query, tile, level) items
                                      with a live 128-id group (profile mode) */
    int64_t bitmap_live_groups;    /* ... and live groups counted from the bitmaps */
    int64_t bitmap_live_words;     /* ... and the 16-byte bitmap words those groups read (the
                                      projections whose bucket summary touches the group) */
    int64_t l2_setaside_bytes;     /* last call with a window mode: persisting-L2 set-aside used
                                      (0: windows could not be attached) */
    int64_t l2_index_permille;     /* ... and the share of it given to the index window */
    int64_t bitmap_overflows;      /* QW_PATH_BITMAP queries whose last level held more
                                      candidates than the list: the list is rebuilt with the
                                      kept entries and the tie class only (profile mode) */
} qw_profile;

typedef struct {
    int64_t n;             /* data vectors */
    int32_t d;             /* dimension */
    int32_t m;             /* projections */
    float w;
    int32_t c;
    int32_t v;
    int32_t l;             /* collision threshold in use */
    int32_t tile;          /* ids per index tile (entries are grouped by id / tile) */
    int32_t n_tiles;
    int32_t span_max;      /* largest anchored bucket id over all projections */
    int64_t n_fixups;      /* data projections recomputed in FP64 at build time */
    int64_t device_bytes;  /* device memory held by the index (excluding workspace) */
    int64_t bitmap_bytes;  /* the level bitmaps (0 without them), in device memory unless
                              host_bitmaps */
    int64_t host_bytes;    /* pinned host memory held by the index (host_bitmaps) */
    int32_t family;        /* QW_FAMILY_E2LSH or QW_FAMILY_QALSH */
} qw_index_info;

/* Library version string. */
const char *qw_version(void);

/* Message describing the last failure on the calling thread ("" if none). */
const char *qw_last_error(void);

/* Eq. 1: collision probability P(r) of the hash family for two points at
 * distance r and bucket width w, in closed form
 *   1 - 2 Phi(-w/r) - (2 r / (sqrt(2 pi) w)) (1 - exp(-w^2 / (2 r^2))).
 * Returns NaN for r <= 0 or w <= 0. */
double qw_collision_probability(double r, double w);

/* Collision threshold l for m projections (Section 3.1; the paper gives no
 * value, so the collision-counting rule is used): with p1 = P(1), p2 = P(c),
 * beta = v / n and z = sqrt(ln(2 / beta) / ln(1 / delta)),
 *   alpha = (z p1 + p2) / (1 + z),  l = ceil(alpha m)  clamped to [1, m].
 * delta <= 0 means 1/e.  Returns -1 on invalid arguments. */
int32_t qw_collision_threshold(int32_t m, float w, int32_t c, int64_t n, int32_t v, float delta);

/* QALSH's collision probability (Section 2): for a projection a with i.i.d.
 * N(0, 1) entries, a . (o - q) is N(0, r^2) for ||o - q|| = r, and the bucket
 * of width w centred on the query catches it with probability
 *   P(|N(0, r^2)| <= w / 2) = erf(w / (2 sqrt(2) r)).
 * Returns NaN for r <= 0 or w <= 0. */
double qw_qalsh_collision_probability(double r, double w);

/* qw_collision_threshold with p1, p2 from qw_qalsh_collision_probability. */
int32_t qw_qalsh_collision_threshold(int32_t m, float w, int32_t c, int64_t n, int32_t v,
                                     float delta);

/* Hash vectors (Section 3): H[r * m + i] = floor((a_i . V_r + b_i) / w).
 * V: nv x d float32, A: m x d float32, b: m float32, H: nv x m int32; all
 * DEVICE pointers.  The projection runs in FP32; every result whose FP32 value
 * lies within a proven error bound (and at least 1e-5 w) of a bucket boundary
 * is recomputed in FP64 with the dot product summed in index order, so H
 * equals the FP64 result.  *n_fixups (optional, host) receives how many were
 * recomputed; passing it makes the call wait for the stream.
 * Errors: QW_ERR_ARG (null pointer, nv < 0, d < 1, m < 1, w <= 0),
 * QW_ERR_RANGE (a bucket id outside int32; H is then unspecified),
 * QW_ERR_CUDA. */
qw_status qw_hash(const float *V, int64_t nv, int32_t d, const float *A, const float *b,
                  int32_t m, float w, int32_t *H, int64_t *n_fixups, void *stream);

/* qw_hash on the fifth-generation tensor cores (tcgen05.mma, BF16 operands in
 * shared memory, FP32 accumulators in tensor memory), m <= 128.  Each FP32
 * input is split into BF16 hi and lo parts; the products hi*hi, hi*lo and
 * lo*hi are accumulated in FP32, which leaves an error of at most
 * (3.01 * 2^-16 + (d - 1) * 2^-22 + 2^-23) * ||a_i|| ||V_r|| for any order of
 * the tensor cores' additions, taking each to lose at most two units in the
 * last place.  Entries within that bound (and at least 1e-5 w) of a bucket
 * boundary are recomputed in FP64 as in qw_hash, so H equals the FP64 result;
 * the wider bound means more recomputations (*n_fixups).  Arguments, pointer
 * spaces and errors as qw_hash; QW_ERR_ARG also for m > 128. */
qw_status qw_hash_tc(const float *V, int64_t nv, int32_t d, const float *A, const float *b,
                     int32_t m, float w, int32_t *H, int64_t *n_fixups, void *stream);

/* The hash family's random draws (Section 3: a_i ~ N(0, I_d), b_i ~ U[0, w))
 * from a seed, on the host, the same on every machine.  The generator is
 * SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) used by counter: draw k is
 *   z = seed + (k + 1) * 0x9E3779B97F4A7C15 (mod 2^64),
 *   z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9,  z = (z ^ (z >> 27)) * 0x94D049BB133111EB,
 *   z = z ^ (z >> 31),   u_k = (z >> 11) * 2^-53  in [0, 1).
 * A (m x d, row-major, HOST) is filled in pairs by the Box-Muller transform:
 * entries 2j and 2j + 1 are r cos(2 pi u_{2j+1}) and r sin(2 pi u_{2j+1}) with
 * r = sqrt(-2 ln(1 - u_{2j})), computed in double and rounded to float.
 * b (m, HOST): b_i = float(u_{k0 + i} w) with k0 = m d rounded up to even,
 * replaced by the largest float below w if it rounds up to w.
 * Nothing is written for m < 1, d < 1 or a null pointer. */
void qw_draw_projections(uint64_t seed, int32_t m, int32_t d, float w, float *A, float *b);

/* Build an index over data (n x d float32) with projections A (m x d float32)
 * and offsets b (m float32), all in `mem` space; A and b both NULL: they are
 * drawn with qw_draw_projections(params->seed, m, d, w, ...).  The index keeps its own
 * device copies of data, A and b; the caller's buffers may be freed after the
 * call returns (device mode: after the stream has passed the call).
 * Layout built (Section 2: one sorted structure per hash function):
 *   anchor o_i = min over data of h_i, bucket id bid = h_i - o_i >= 0,
 *   and, for every projection, the (bid, id) pairs sorted by bid (ids within
 *   a bucket in the bank-spread order described at qw_index_export),
 *   grouped by id tile, with a directory of the distinct bids of each tile;
 * with QW_FAMILY_QALSH the sorted FP64 projections instead (anchors and spans
 * are then zero).
 * The call waits for the stream.  *out receives the handle (free with
 * qw_index_free).
 * Errors: QW_ERR_ARG (null pointer, n < 1, n >= 2^31, d < 1, bad params),
 * QW_ERR_RANGE (bucket id or span outside int32; QALSH: a projection not
 * finite), QW_ERR_OOM, QW_ERR_CUDA. */
qw_status qw_build_index(const float *data, int64_t n, int32_t d, const float *A,
                         const float *b, const qw_index_params *params, int32_t mem,
                         void *stream, qw_index **out);

/* The index's projections and anchors (Section 3's a_i and b_i, and the
 * anchors o_i = min over the data of h_i that make every data bucket id
 * non-negative): A (m x d float32), b (m float32), offsets (m int32), all
 * HOST pointers, each optional (NULL: not copied).  These are the values the
 * index hashes with -- the caller's A and b, or the ones drawn from the seed
 * -- so an independent implementation given them computes the same bucket
 * ids.  Waits for the device.  Errors: QW_ERR_ARG (null index), QW_ERR_CUDA. */
qw_status qw_index_get_projections(const qw_index *index, float *A, float *b, int32_t *offsets);

/* Answer a workload of nq queries (nq x d float32) for the k nearest
 * neighbours each (Sections 3.1, 4).  Per query: levels R = 1, c, c^2, ...;
 * C_R = { o : o collides with q on >= l projections at radius R }; stop at the
 * first level with |C_R| >= k + v, or when R exceeds every bucket id of the
 * data and the query; keep at most k + v candidates (those of the previous
 * level first, then more collisions, then smaller id); return the k nearest
 * by exact distance (ties by smaller id).  The optional stopping rule of
 * collision-counting LSH -- stop once k candidates lie within c R of the
 * query -- is not supported: a query stops by the k + v bound or the radius
 * rule only.
 * Outputs: ids (nq x k int64, -1 where fewer than k candidates), dists
 * (nq x k float32, Euclidean distance, +inf where id is -1), stats (optional,
 * nq x QW_NSTAT int64, slots above).  All in `mem` space.
 * Ids equal those of the FP64 definition: distances are computed in FP32 and
 * every candidate whose order against a neighbour is not certain under the
 * FP32 error bound is recomputed in FP64.
 * Errors: QW_ERR_ARG (null pointer, nq < 0, k < 1, k > n, k + v > QW_MAX_CAND,
 * unknown option values), QW_ERR_RANGE (query bucket id outside int32),
 * QW_ERR_OOM, QW_ERR_CUDA. */
qw_status qw_run_workload(qw_index *index, const float *queries, int64_t nq, int32_t k,
                          const qw_query_params *qparams, int64_t *ids, float *dists,
                          int64_t *stats, int32_t mem, void *stream);

/* The candidate sets of a workload, for inspection: runs the steps of
 * qw_run_workload up to and including the k + v bound and writes, per query,
 * the kept candidates in ascending id order with their collision counts at the
 * last level.  cand_ids: nq x (k + v) int64 padded with -1; cand_col:
 * nq x (k + v) int32 padded with 0 (optional); stats as in qw_run_workload
 * (optional).  All in `mem` space.  Errors as qw_run_workload. */
qw_status qw_workload_candidates(qw_index *index, const float *queries, int64_t nq, int32_t k,
                                 const qw_query_params *qparams, int64_t *cand_ids,
                                 int32_t *cand_col, int64_t *stats, int32_t mem, void *stream);

/* Bytes of the library-owned static device scratch used by
 * qw_run_workload_noalloc (held by every GPU that loads the library, until the
 * process exits). */
#define QW_STATIC_SCRATCH_BYTES (64u << 20)

/* qw_run_workload for callers that must not allocate device memory.
 *
 * The paper has no counterpart: this is a deployment variant of the
 * level-synchronous path.  Some callers cannot call cudaMalloc or cudaFree at
 * query time -- for example a process whose device memory is already fully
 * reserved by another framework's caching allocator, or a latency-critical
 * serving thread that must not trigger the device-wide synchronisation these
 * calls can imply.  This entry point allocates nothing: its working memory is
 * one file-scope device array of QW_STATIC_SCRATCH_BYTES, and queries are
 * processed in batches sized to fit it.  The index must already exist
 * (qw_build_index allocates; build it beforehand).
 *
 * Arguments as qw_run_workload, except that queries, ids, dists and stats
 * (optional) are DEVICE pointers and there are no per-call options.
 * Every call looks up the scratch array's device address on the current
 * device (cudaGetSymbolAddress); the first call on a device also loads the
 * library's module there, so make that first call before any stream capture.
 * The index must live on the current device.  Every call on a device shares the
 * same array, so calls whose work overlaps on the GPU (different streams or
 * threads without ordering between them) race and corrupt each other's
 * results: order them on one stream.  The call waits for `stream` once per
 * batch.
 * Errors: as qw_run_workload; QW_ERR_ARG also when the index is on another
 * device, or when one query's working memory exceeds the static array.  One
 * query needs n_tiles * (32768 + 528) + 12 m + 8 (k + v) bytes (collision
 * counters, per-tile candidate profiles and plans, bucket ids, candidate
 * lists) plus about 5.5 KB of block alignment, n_tiles = ceil(n / 32768):
 * indexes of up to about 65 million points fit. */
qw_status qw_run_workload_noalloc(qw_index *index, const float *queries, int64_t nq, int32_t k,
                                  int64_t *ids, float *dists, int64_t *stats, void *stream);

/* Cost model of the L2 split (Section 4, Eq. 4: choose size(C_I) +
 * size(C_D) = size(C) to minimise the workload's index IO plus data IO),
 * restated for a hardware cache.  A region X (index or data) of U_X bytes is
 * read A_X >= U_X bytes in total by the workload.  Its DRAM traffic with S_X
 * persisting bytes is modelled as
 *   D_X(S_X) = U_X + (A_X - U_X) * (1 - min(1, S_X / U_X)),
 * i.e. the first read of every byte misses and a re-read hits when the byte
 * is among the persisting share.  The function returns the permille p of the
 * set-aside S given to the index (S_I = p S / 1000, S_D = S - S_I) that
 * minimises D_I(S_I) + D_D(S_D); on a tie the smaller p.  The index reads
 * scale with the cardinality (the paper's alpha_card: every pass reads the
 * index of every tile) and the data reads with the dimensionality (alpha_dim:
 * at most k + v rows of 4 d bytes per query).
 * All sizes are bytes, >= 0.  Returns -1 on invalid arguments (negative or
 * non-finite values, setaside == 0). */
int32_t qw_l2_split_model(double setaside, double index_bytes, double index_reads,
                          double data_bytes, double data_reads);

/* Read bandwidth of a device buffer of `bytes` bytes (a measuring tool; the
 * paper has no counterpart): the library allocates the buffer and reads it
 * with 16-byte loads cached in L2 only, each thread the same elements on every
 * pass; each launch makes as many passes as come to about 2 GB; after three
 * untimed launches it times `reps` launches (CUDA events on `stream`) and
 * writes the best rate to *gbs in GB/s.  A buffer well below the L2 size (126 MB usable
 * on GB300) gives the rate L2 delivers to the SMs -- the ceiling of kernels
 * whose reads hit L2 -- and one well above it the HBM rate.  Waits for the
 * stream.  Errors: QW_ERR_ARG (bytes < 16, reps < 1, null gbs), QW_ERR_OOM,
 * QW_ERR_CUDA. */
qw_status qw_measure_read_bandwidth(int64_t bytes, int32_t reps, double *gbs, void *stream);

/* Copy the index's profile counters (launch counts of every call; kernel
 * times and work counters of calls made with qw_query_params.profile) into
 * the host struct *out; reset them afterwards when `reset` is non-zero.
 * QW_ERR_ARG for a NULL index or out. */
qw_status qw_index_profile(qw_index *index, qw_profile *out, int32_t reset);

/* Settings qw_autotune tried, with their median times. */
#define QW_TUNE_MAX 32
typedef struct {
    int32_t tried;                         /* entries filled below */
    qw_query_params params[QW_TUNE_MAX];   /* each setting tried */
    float ms[QW_TUNE_MAX];                 /* its median time over `reps` calls */
    int32_t best;                          /* index of the chosen setting */
} qw_tune_report;

/* Autotuner of the workload path (the paper has no counterpart; its settings
 * change speed only).  Times qw_run_workload on the given queries (a sample
 * of the workload, `mem` space) under candidate settings, one coordinate at a
 * time, keeping the fastest before moving on: start level (plain / learned,
 * when a start model is attached), queries per batch on the level path (the
 * default and 1/16, 1/4, 4x of it) and graph mode; the bitmap path (when the
 * index has bitmaps) with its default batch, 1/16 and 1/4 of it, and graph
 * mode and direct loads; then the cluster path against the best so far (when the index fits it
 * and the start is plain); order (signature / given), rerank (FP32 / BF16,
 * when the index has the BF16 copy) and the persisting-L2 windows (off /
 * QW_L2_MODEL).  Every setting returns the same results, so the choice cannot change
 * them.  Each setting runs once untimed, then `reps` (>= 1) times timed with
 * CUDA events on `stream`; the median counts.  The chosen setting is written
 * to *best (host) and stored in the index: later calls with QW_PATH_AUTO take
 * its path and, with batch 0, its batch size.  report (host, optional)
 * receives every setting tried.  base (optional) gives the fields not tuned
 * (profile); NULL means zero.  Waits for the stream.
 * Errors: as qw_run_workload; QW_ERR_ARG also for reps < 1 or best NULL. */
qw_status qw_autotune(qw_index *index, const float *queries, int64_t nq, int32_t k, int32_t mem,
                      int32_t reps, const qw_query_params *base, qw_query_params *best,
                      qw_tune_report *report, void *stream);

/* ---- The learned start model (the paper trains an offline model for its
 * cache split in Section 5.2 but prints no network).
 * A multilayer perceptron n_in -> hidden -> hidden -> classes with ReLU,
 * softmax cross-entropy, FP16 weight copies of FP32 master weights and FP32
 * accumulation; trained with Adam by the library's kernels.  Parameters are a
 * flat float array: W1 (hidden x n_in, row-major), b1, W2 (hidden x hidden),
 * b2, W3 (classes x hidden), b3.  The caller provides the initial values (the
 * random draws of the method are inputs).  Every call below that takes a
 * model returns QW_ERR_ARG for a NULL model or pointer argument (and names the
 * problem in qw_last_error), QW_ERR_OOM when device memory runs out and
 * QW_ERR_CUDA on a CUDA error.  qw_mlp_loss_grad and qw_mlp_train wait for
 * their stream; qw_mlp_predict only enqueues its kernels on it. */
typedef struct qw_mlp qw_mlp;

/* A model with zeroed parameters, owned by the caller until qw_mlp_free.
 * QW_ERR_ARG unless 1 <= n_in <= 65536, 1 <= hidden <= 65536 and
 * 2 <= classes <= 1024. */
qw_status qw_mlp_create(int32_t n_in, int32_t hidden, int32_t classes, qw_mlp **out);
/* Number of parameters (the flat array's length), -1 for a NULL model. */
int64_t qw_mlp_param_count(const qw_mlp *mlp);
/* Host arrays of qw_mlp_param_count floats (QW_ERR_ARG for another count),
 * copied in or out; set_params also resets Adam's moments. */
qw_status qw_mlp_set_params(qw_mlp *mlp, const float *params, int64_t count);
qw_status qw_mlp_get_params(const qw_mlp *mlp, float *params, int64_t count);
/* Mean loss (host *loss, optional) and its gradient (host grad of
 * qw_mlp_param_count floats, optional) over n rows, 1 <= n <= 2^20: X DEVICE
 * n x n_in float32 row-major, y DEVICE n int32 class labels in [0, classes). */
qw_status qw_mlp_loss_grad(qw_mlp *mlp, const float *X, const int32_t *y, int64_t n, float *loss,
                           float *grad, void *stream);
/* Adam (beta 0.9 / 0.999, step size lr > 0) over the rows in order, `batch`
 * rows per step, `epochs` passes (n, epochs, batch >= 1); X and y as in
 * qw_mlp_loss_grad.  *final_loss (host, optional) = mean loss of the last
 * epoch. */
qw_status qw_mlp_train(qw_mlp *mlp, const float *X, const int32_t *y, int64_t n, int32_t epochs,
                       int32_t batch, float lr, float *final_loss, void *stream);
/* Class probabilities (DEVICE n x classes float32, softmax) of DEVICE rows X
 * (n x n_in float32), n >= 0. */
qw_status qw_mlp_predict(qw_mlp *mlp, const float *X, int64_t n, float *prob, void *stream);
/* The same forward pass on the tensor cores (tcgen05.mma, FP16 activations
 * and weights, FP32 accumulators in tensor memory), 128 rows per CTA: the form
 * qw_run_workload uses for learned starts whenever the network has this shape
 * -- hidden = 256, classes a multiple of 16 up to 32, n_in a multiple of 64 up
 * to 576 -- and QW_ERR_ARG for any other shape.  Probabilities differ from
 * qw_mlp_predict by the FP16 rounding of the activations (about 1e-3).  Waits
 * for the stream; QW_ERR_TIMEOUT if a tensor-core wait gave up. */
qw_status qw_mlp_predict_tc(qw_mlp *mlp, const float *X, int64_t n, float *prob, void *stream);
void qw_mlp_free(qw_mlp *mlp);

/* Features of queries for the start model (DEVICE pointers): per query its
 * d coordinates divided by the data's RMS coordinate, then for each of the m
 * projections its position in the data's bucket-id range, (g + 0.5) /
 * (span + 1) - 0.5 clamped to [-1.5, 1.5]; F is nq x (d + m) float32
 * row-major, written by the library.  QW_ERR_ARG for a NULL index, NULL
 * pointers with nq > 0 or nq < 0; QW_ERR_RANGE if a query's bucket id leaves
 * the 32-bit range.  Waits for the stream. */
qw_status qw_query_features(qw_index *index, const float *queries, int64_t nq, float *F,
                            void *stream);
/* Attach a start model (not owned; it must outlive its use) with classes =
 * level index 0, 1, ...; eps in (0, 1) bounds the predicted probability of
 * starting too late.  NULL detaches.  QW_ERR_ARG for a NULL index, eps
 * outside (0, 1), or a model whose input size is not d + m. */
qw_status qw_index_set_start_model(qw_index *index, qw_mlp *mlp, float eps);

/* Copy index metadata into the host struct *info.  QW_ERR_ARG for a NULL
 * index or info. */
qw_status qw_index_get_info(const qw_index *index, qw_index_info *info);

/* Export the index for inspection, into HOST buffers: o and span (m int32),
 * and, per projection, every entry's bucket id and data id (m x n int32 each)
 * in the index's own order: by id tile (id / tile), then bucket id; within a
 * bucket, ids are arranged so that consecutive entries fall into different
 * shared-memory banks of the counting kernels (groups of 8 ids of one bank,
 * the groups cycling through the banks).
 * Any output pointer may be NULL.  Waits for the stream.  A QALSH index has no
 * bucket ids: entry_bid / entry_id are refused with QW_ERR_ARG. */
qw_status qw_index_export(const qw_index *index, int32_t *o, int32_t *span,
                          int32_t *entry_bid, int32_t *entry_id, void *stream);

/* Free an index and its device memory (synchronises the device first). */
void qw_index_free(qw_index *index);

#ifdef __cplusplus
}
#endif

#endif /* QWLSH_H */
