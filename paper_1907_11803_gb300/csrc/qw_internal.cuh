// qw_internal.cuh -- declarations shared by the library's translation units.
//
// Nothing here is shared with the CPU oracle; the oracle is a separate C file
// with its own arithmetic.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/qwlsh.h"

namespace qw {

// Ids per index tile.  Entries of one projection are grouped by tile
// (id / kTile), so a tile's collision counters fit in shared memory and its
// ids fit in 16 bits.
constexpr int kTile = 32768;
constexpr int kTileShift = 15;

// Bucket id written by the FP32 projection when the value is too close to a
// bucket boundary to trust; the FP64 pass replaces every such entry.
constexpr int32_t kNeedsFp64 = INT32_MIN;

// Per-(query, tile) candidate profile: [0] previous-level candidates,
// [1 + c] other candidates with collision count c (c <= QW_MAX_M).
constexpr int kHistBins = QW_MAX_M + 2;

// Thread-local error text behind qw_last_error().
void set_error(const std::string &msg);
void clear_error();

qw_status cuda_status(cudaError_t e, const char *what);

#define QW_CUDA_TRY(call)                                           \
    do {                                                            \
        cudaError_t qw_e_ = (call);                                 \
        if (qw_e_ != cudaSuccess) return qw::cuda_status(qw_e_, #call); \
    } while (0)

#define QW_TRY(call)                        \
    do {                                    \
        qw_status qw_s_ = (call);           \
        if (qw_s_ != QW_OK) return qw_s_;   \
    } while (0)

// Grow-only device buffer.
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    ~DevBuf() { release(); }
    qw_status ensure(size_t want);
    void release();
    template <class T> T *as() const { return reinterpret_cast<T *>(p); }
};

// ---------------------------------------------------------------- projection
// H[r * ld_row + i * ld_col] = floor((a_i . V_r + b_i) / w), FP32 with an
// FP64 recomputation of every entry near a bucket boundary.  err (device int)
// gets bit 1 set when a bucket id falls outside int32.  fixups (device
// unsigned long long, may be null) counts FP64 recomputations.
// tensor_cores (m <= 128): the projection on the tensor cores (split BF16
// products, FP32 accumulation) with its own proven bound; same bucket ids.
qw_status launch_hash(const float *V, int64_t nv, int d, const float *A, const float *b, int m,
                      float w, int32_t *H, int64_t ld_row, int64_t ld_col, int *err,
                      unsigned long long *fixups, cudaStream_t s, bool tensor_cores = false);

// ---------------------------------------------------------------- QALSH (qw_qalsh.cu)
// out[r * ld_r + i * ld_i] = a_i . V_r in FP64, summed in coordinate order.
qw_status launch_fp64_project(const float *V, int64_t nv, int d, const float *A, int m,
                              double *out, int64_t ld_r, int64_t ld_i, cudaStream_t s);
// qmin / qmax (device, m) of the projections P (m rows of ldp doubles, n used);
// kscratch: 2 m words; err bit 1 when one is not finite.
qw_status launch_qalsh_extent(const double *P, int64_t n, int64_t ldp, int m,
                              unsigned long long *kscratch, double *qmin, double *qmax, int *err,
                              cudaStream_t s);
// Sort every (tile, projection) segment of P (m rows of nT * kTile doubles,
// overwritten) into qkey / lid; tlid: scratch of the same shape in uint16.
qw_status launch_qalsh_sort(double *P, int64_t n, int m, int nT, uint16_t *tlid, double *qkey,
                            uint16_t *lid, cudaStream_t s);

// ---------------------------------------------------------------- index build
qw_status launch_minmax(const int32_t *Ht, int64_t n, int m, int32_t *hmin, int32_t *hmax,
                        cudaStream_t s);
qw_status launch_tile_sort(const int32_t *Ht, int64_t n, int m, int nT, const int32_t *o,
                           uint16_t *lid, int32_t *dir_bid, int32_t *dir_off,
                           const int64_t *dir_start, int32_t *dir_cnt, cudaStream_t s);
qw_status launch_export(const uint16_t *lid, const int32_t *dir_bid, const int32_t *dir_off,
                        const int64_t *dir_start, const int32_t *dir_cnt, int64_t n, int m,
                        int nT, int32_t *entry_bid, int32_t *entry_id, cudaStream_t s);

// ---------------------------------------------------------------- queries
struct IndexView {
    const float *X;
    int64_t n;
    int d;
    int m;
    int nT;
    const int32_t *o;
    const int32_t *span;
    const uint16_t *lid;
    const int32_t *dir_bid;
    const int32_t *dir_off;
    const int64_t *dir_start;
    const int32_t *dir_cnt;
    // level bitmaps (null when the index was built without them): for every
    // projection i, tile t, level L <= bm_J[i] and level-L bucket beta, the
    // tile's ids whose bid / c^L == beta, as kTile bits (kTile / 128 uint4):
    // bitmap number bm_base[i] + t * bm_nb[i] + bm_lvl[i * kBmLevels + L] + beta.
    // Bitmaps number ids in locality order: internal id j is data object
    // perm[j] (groups of 128 consecutive internal ids are spatially compact);
    // bm_sum holds per bitmap 256 bits, bit g set when 128-id group g has an id.
    const uint4 *bm;
    const int32_t *perm;
    const uint32_t *bm_sum;
    const float *Xloc;        // the data in locality order (row j = data id perm[j])
    const int32_t *inv;       // data id -> internal id
    const int64_t *bm_base;
    const int32_t *bm_nb;
    const int32_t *bm_lvl;
    const int32_t *bm_J;
    // per projection i, bid_prefix[prefix_off[i] + b] = data objects with bid < b,
    // b = 0 .. span_i + 1 (built with the bitmaps; entries scanned per range)
    const int64_t *bid_prefix;
    const int64_t *prefix_off;
    // anchored bucket ids in locality order, row j = internal id j (m entries
    // of hloc_bytes = 1, 2 or 4 bytes each, rows hloc_stride bytes apart, a
    // multiple of 16; built with the bitmaps)
    const void *hloc;
    int hloc_bytes;
    int hloc_stride;
    // QALSH index (null for the bucketed family): per projection i and tile t
    // the FP64 projections a_i . x of the tile's objects, ascending and aligned
    // with lid (qkey[i * nT * kTile + t * kTile + p] belongs to lid[same]);
    // per projection the smallest and largest projection over the data; and
    // w / 2 in FP64 (the level-R interval is p_i(q) +- qhalf * R)
    const double *qkey = nullptr;
    const double *qmin = nullptr;
    const double *qmax = nullptr;
    double qhalf = 0.0;
};

// Entries-scanned statistics from the bid prefix counts (bitmap path), for
// the decision kernel; prefix == null: the level kernel accumulated them.
struct ScanStats {
    const int64_t *prefix = nullptr;
    const int64_t *off = nullptr;
    const int32_t *span = nullptr;
    int m = 0;
    int cgrow = 2;
    // bitmap path, learned starts: a query that stops at its first level > 0
    // stops there and is marked for the previous-level recount (no rerun)
    bool recount_first = false;
};

// Most levels a bitmap table describes per projection (c >= 2, bids < 2^31).
constexpr int kBmLevels = 32;
constexpr int kBmUint4 = kTile / 128;  // uint4 per bitmap

// Bitmap path: the rebuild of a last level's overflowing candidate list.
struct RdPlan {
    int32_t q;      // query of the batch
    int32_t np;     // candidates of the previous level
    int32_t cstar;  // boundary count
    int32_t take;   // ids kept at the boundary count
    int32_t mode;   // 0: not rebuilt, 1: whole tie class listed, 2: its take smallest ids
    int32_t pad0;
    int32_t pos;    // entries of the rebuilt list
    int32_t prev_recount;  // learned first level: previous level from its bitmaps
    int32_t pad[8];
};

// Per-batch query state, all device arrays of length nb (or nb x m).
struct QueryState {
    // multi-probe: buckets looked into on each side of the query's (0: none;
    // level path only)
    int32_t probes = 0;
    int64_t *g = nullptr;             // nb x m: h_i(q) - o_i
    int64_t *top = nullptr;           // nb: max_i max(span_i, g_i)
    int32_t *active = nullptr;        // nb
    int32_t *ncand = nullptr;         // nb: |C_R| after the last finished level
    int32_t *nprev = nullptr;         // nb
    int32_t *cross = nullptr;         // nb: candidates of the running level, summed over tiles
    int32_t *term = nullptr;          // nb
    int32_t *levels = nullptr;        // nb
    int64_t *finalR = nullptr;        // nb
    int64_t *scan_level = nullptr;    // nb
    int64_t *scan_last = nullptr;     // nb
    int64_t *scan_full = nullptr;     // nb
    int32_t *nkeep = nullptr;         // nb
    unsigned long long *max_top = nullptr;  // 1
    uint32_t *counters = nullptr;     // nb x (nT * kTile / 4)
    int32_t *cand = nullptr;          // nb x cap
    int32_t *cand_col = nullptr;      // nb x cap
    int32_t *tile_hist = nullptr;     // nb x nT x kHistBins
    int32_t *tile_plan = nullptr;     // nb x nT x 3: first output slot, count-c* ids before the tile,
                            //   ids kept in the tile
    int32_t *qplan = nullptr;         // nb x 2: c*, how many count-c* ids are kept
    int32_t *start = nullptr;         // nb: first level of the query (0 unless learned)
    int32_t *fb = nullptr;            // nb: query stopped at a learned first level > 0
    unsigned long long *fb_count = nullptr;  // 2: queries to recompute, levels skipped
    unsigned long long *level_passes = nullptr;  // profile mode: (query, level) passes run, else null
    uint4 *cbits = nullptr;           // bitmap path: 2 (level parity) x nb x nT candidate bitmaps
    int64_t cb_par = 0;         // uint4 per parity (batch capacity x nT x kBmUint4)
    // bitmap path: per (level parity, query, tile) the number of candidates
    // (0: the tile's candidate bitmap was not written at that level)
    int32_t *clist_n = nullptr;
    int64_t cln_par = 0;        // entries of clist_n per parity (batch capacity x nT)
    // bitmap path: per (level parity, query) every candidate of the level as
    // (internal id << 32) | (was a candidate at the previous level << 8) | count,
    // up to kQCap of them (qbuf_n counts beyond: more means overflow)
    uint64_t *qbuf = nullptr;
    int32_t *qbuf_n = nullptr;
    int64_t qb_par = 0;         // entries of qbuf per parity (batch capacity x kQCap)
    int64_t qbn_par = 0;        // entries of qbuf_n per parity (batch capacity)
    // bitmap path selection: per query "answer on the level path" flags, and
    // tie lists of kEqCap original ids
    int32_t *bm_ovf = nullptr;
    int32_t *eqbuf = nullptr;
    int32_t *recount = nullptr;     // per query: stopped at its learned first level (bitmap path)
    // bitmap path, last levels whose candidates overflowed the list: the
    // number of such queries, per slot its plan and its count histogram
    int32_t *rd_ctl = nullptr;      // [0]: slots
    struct RdPlan *rd_plan = nullptr;
    int32_t *rd_hist = nullptr;     // slots x kHistBins: counts of candidates not of C_{R/c}
    int64_t *rd_bq = nullptr;       // slots x 2 x QW_MAX_M: bitmap numbers in tile 0 (L, L - 1)
    uint4 *rd_store = nullptr;      // per slot of a wave, per group: 7 count planes + prev word
    // bitmap path, two-pass level: item slots (query, tile) with their m bitmap
    // numbers, and the work list of live (slot << 8 | group) entries
    int32_t *bm_nitems = nullptr;   // 2 counters: items, work entries (per level)
    int32_t *bm_nwork = nullptr;
    int2 *bm_item_qt = nullptr;
    int64_t *bm_bq = nullptr;       // per (query, projection): bitmap number in tile 0, or -1
    int32_t *bm_item_bi = nullptr;  // per item, (m + 3) / 4 * 4 bitmap numbers (-1: none)
    uint32_t *bm_amask = nullptr;   // per (level parity, query, tile): live groups, 8 words
    int32_t *bm_work = nullptr;
    // per work entry, (m + 63) / 64 words: the projections whose bucket touches
    // the group (its summary bit); the others' words are zero and not read
    unsigned long long *bm_wmask = nullptr;
    int32_t bm_item_cap = 0;
    int32_t bm_work_cap = 0;
    unsigned long long *bm_prof = nullptr;  // profile mode: live items, groups, words (summed)
};

// Candidates per query and level the bitmap path holds (more: the query is
// answered by the level path).  4 MiB of lists per query (two levels).
constexpr int kQCap = 262144;
// Tie-list capacity per query on the bitmap path (larger tie classes are
// answered by the level path).
constexpr int kEqCap = 16384;


// Level of a loop that runs on the device (graph mode): the level kernels
// read level, R and R/c from here, and the loop-control kernel advances it.
struct LoopCtl {
    int64_t R;
    int64_t Rp;
    int32_t level;
    int32_t pass;                 // 0, then 1 for the recomputed queries (learned start)
    unsigned long long iters;     // level passes run, summed over the call's batches
    unsigned long long fb_total;  // learned start: queries recomputed, summed over batches
    unsigned long long skipped_total;  // learned start: levels skipped, summed over batches
    int32_t min_start;            // smallest first level of the batch's queries
    uint32_t active;              // queries still running or not yet started after a level
};

// QALSH: the queries' FP64 projections are in st.g (as double bits); sets
// every query's radius-rule bound and resets its state (err bit 1: no radius
// of int64 reaches the whole data).
qw_status launch_qalsh_setup(const IndexView &ix, int nb, QueryState &st, int cgrow, int *err,
                             cudaStream_t s);
qw_status launch_query_setup(const IndexView &ix, const int32_t *HQ, int nb, QueryState &st,
                             cudaStream_t s);
// Learned first levels: at most each query's last useful level.
qw_status launch_clamp_start(int nb, QueryState &st, int cgrow, cudaStream_t s);
qw_status launch_level(const IndexView &ix, int nb, int level, int64_t R, int64_t Rp, int l,
                       int cgrow, QueryState &st, cudaStream_t s, const LoopCtl *ctl = nullptr);
qw_status launch_fallback(int nb, QueryState &st, cudaStream_t s);
qw_status launch_decide(int nb, int level, int64_t R, int cap, QueryState &st, cudaStream_t s,
                        LoopCtl *ctl = nullptr, const ScanStats &ss = ScanStats());
// Bitmap path (qw_bitmap.cu).
struct BitmapLayout {
    std::vector<int64_t> base;   // per projection, first bitmap
    std::vector<int32_t> nb;     // per projection, bitmaps per tile
    std::vector<int32_t> lvl;    // m x kBmLevels, first bitmap of each level in a tile's block
    std::vector<int32_t> J;      // per projection, last level stored (c^J > span)
    int64_t total = 0;           // bitmaps
};
qw_status bitmap_layout(const std::vector<int32_t> &span, int nT, int c, BitmapLayout *out);
// Internal order of the bitmaps: a two-means tree over the data (host
// copies X n x d, A m x d), leaves of at most kGroupIds ids aligned to groups.
constexpr int kGroupIds = 128;
qw_status locality_order(const float *X, int64_t n, int d, const float *A, int m,
                         std::vector<int32_t> &perm);
qw_status launch_bitmap_build(const IndexView &ix, int c, int maxJ, const int32_t *Ht, uint4 *bm,
                              uint32_t *bm_sum, int64_t total_bitmaps, cudaStream_t s);
qw_status launch_bid_prefix(const IndexView &ix, int64_t *prefix, const int64_t *off,
                            cudaStream_t s);
ScanStats scan_stats_of(const IndexView &ix, int c);
// loads: QW_LOADS_TMA stages the bitmaps with TMA bulk copies in a persistent
// kernel; QW_LOADS_DIRECT filters on the summaries, then counts the live groups
// in a second launch; QW_LOADS_FUSED does both in one launch.  err bit 4: a
// staged-copy wait gave up.
// part (direct and fused loads): 0 every launch of the level, 1 the bucket
// numbers, 2 the summary filter and the count pass (and the profile counters).
// tpw: tiles a warp of the filter / fused kernel takes (4, 8 or 16; else 8).
qw_status launch_bm_level(const IndexView &ix, int nb, int level, int64_t R, int64_t Rp, int l,
                          int cgrow, QueryState &st, int *err, int loads, cudaStream_t s,
                          const LoopCtl *ctl = nullptr, int part = 0, int tpw = 8);
// Rebuild the candidate lists of the queries whose last level overflowed them
// (kept entries and tie class only); tma: the level ran bm_level_tma_kernel.
qw_status launch_bm_reduce(const IndexView &ix, int nb, int l, int cap, int cgrow,
                           QueryState &st, bool tma, int wave_slots, cudaStream_t s);
// Bytes of the rebuild's plane store, and how many slots it holds for an index
// of nT tiles (more overflowing queries in one batch keep the level-path
// answer).
constexpr int64_t kRdStoreBytes = (int64_t)1 << 32;
int bm_reduce_wave(int nT);
// sorted: the kept lists in ascending original id (else in no particular order)
qw_status launch_bm_collect(const IndexView &ix, int nb, int l, int cap, QueryState &st,
                            int64_t *stats_out, bool sorted, cudaStream_t s);
qw_status launch_select_plan(const IndexView &ix, int nb, int l, int cap, QueryState &st,
                             int64_t *stats_out, cudaStream_t s);
// Queries of the batch to answer again (workload indices): list0 / count[0]
// those whose candidates overflowed the bitmap path's lists, list1 / count[1]
// those whose learned first level was too late.
qw_status launch_bm_overflow_list(const QueryState &st, int nb, const int32_t *order_perm,
                                  int64_t b0, int32_t *list0, int32_t *list1, int32_t *count,
                                  cudaStream_t s);

// Device-driven loop control (qw_graph.cu builds the graphs that use them).
qw_status launch_loop_init(LoopCtl *ctl, const QueryState &st, int nb, int cgrow, cudaStream_t s);
qw_status launch_loop_ctl(LoopCtl *ctl, const unsigned long long *max_top, int cgrow,
                          cudaGraphConditionalHandle h, int *err, cudaStream_t s);
qw_status launch_fallback_graph(int nb, QueryState &st, LoopCtl *ctl,
                                cudaGraphConditionalHandle h, cudaStream_t s);

// Graph mode of the level loop: one CUDA graph per batch shape, cached.
struct LevelGraphCache;
LevelGraphCache *level_graph_cache_new();
void level_graph_cache_free(LevelGraphCache *c);
qw_status run_level_graph(LevelGraphCache *c, const IndexView &ix, int nb, int l, int cgrow,
                          int cap, bool learned, bool bitmap, int loads, int tpw, QueryState &st,
                          LoopCtl *ctl, int *err, cudaStream_t s);
qw_status launch_collect(const IndexView &ix, int nb, int l, int cap, QueryState &st,
                         int64_t *stats_out, cudaStream_t s);
bool cluster_path_fits(const IndexView &ix, int *cluster_size, int *tiles_per_cta);
qw_status launch_cluster_query(const IndexView &ix, const int32_t *HQ, int nq, int l, int c,
                               int cap, int cluster_size, int tpc, int max_clusters,
                               QueryState &st, int *queue, int64_t *stats_out, int *err,
                               cudaStream_t s, int *clusters_used);
size_t order_hist_ints();
qw_status launch_order(const int32_t *HQ, int64_t nq, const IndexView &ix, uint32_t *keys,
                       int32_t *hist, int32_t *perm, cudaStream_t s);
qw_status launch_gather(const float *Q, const int32_t *HQ, const int32_t *perm, int64_t b0, int nb,
                        int d, int m, float *Qb, int32_t *HQb, cudaStream_t s);
qw_status launch_scatter(const int32_t *perm, int64_t b0, int nb, int k, int cap,
                         const int64_t *ids_b, const float *dists_b, const int64_t *stats_b,
                         const int64_t *cids_b, const int32_t *ccol_b, int64_t *ids, float *dists,
                         int64_t *stats, int64_t *cids, int32_t *ccol, cudaStream_t s);
qw_status launch_sum_i32(const int32_t *v, int n, unsigned long long *out, cudaStream_t s);
qw_status launch_candidates_out(const QueryState &st, int nb, int cap, int64_t *cand_ids,
                                int32_t *cand_col, cudaStream_t s);
// BF16 pre-filter then the FP32 / FP64 stages.  Rb, rnorm, C: the residual
// BF16 copy built by launch_shadow_bf16 over the index's row order (the
// locality order when the index has bitmaps, read through ix.inv).
qw_status launch_rerank_bf16(const IndexView &ix, const void *Rb, const float *rnorm,
                             const float2 *rcr, const void *C, const float *Qb, int nb, int k,
                             int cap,
                             const QueryState &st, int64_t *ids_out, float *dists_out,
                             unsigned long long *rows_fp32, cudaStream_t s, int rows = 4);
// Rows Xs (n x d) grouped by 128: C (ceil(n / 128) x d BF16) the group means,
// Rb (n x d BF16) the residuals to them, rnorm (n) bounds of the residual norms,
// rcr (n, optional) per row (C_g . r~, |r~|^2).
qw_status launch_shadow_bf16(const float *Xs, int64_t n, int d, void *Rb, float *rnorm,
                             void *C, cudaStream_t s, float2 *rcr = nullptr);
// The BF16 pre-filter with q . r~ on the tensor cores (tcgen05), then the
// FP32 / FP64 stages; rcr from launch_shadow_bf16.  err bit 32: a tensor-core
// wait gave up (the query's candidates then all go to the exact stages).
qw_status launch_rerank_tc(const IndexView &ix, const void *Rb, const float *rnorm,
                           const float2 *rcr, const void *C, const float *Qb, int nb, int k,
                           int cap, const QueryState &st, int64_t *ids_out, float *dists_out,
                           unsigned long long *rows_fp32, int *err, cudaStream_t s);
// Xrows/row_of (optional): read data id `id` from row row_of[id] of Xrows
// (the bitmap path's copy of the data in locality order).
// rows: candidate rows a warp takes at a time (2, 4 or 8; other values: 4).
qw_status launch_rerank(const IndexView &ix, const float *Qb, int nb, int k, int cap,
                        const QueryState &st, int64_t *ids_out, float *dists_out,
                        cudaStream_t s, const float *Xrows = nullptr,
                        const int32_t *row_of = nullptr, int rows = 4);
// The data in locality order (Xloc[j] = X[perm[j]]) and the inverse order.
qw_status launch_locality_copy(const float *X, const int32_t *perm, int64_t n, int d, float *Xloc,
                               int32_t *inv, cudaStream_t s);
// Anchored bucket ids in locality order: row j (ix.hloc_stride bytes, zero
// padded) holds Ht[i][perm[j]] - o[i] for i < m, as ix.hloc_bytes-byte
// unsigned integers (every anchored id fits).
qw_status launch_hloc_build(const IndexView &ix, const int32_t *Ht, void *hloc, cudaStream_t s);

// The learned start model (qw_mlp.cu).
int mlp_inputs(const qw_mlp *mp);
int mlp_classes(const qw_mlp *mp);
qw_status mlp_predict_dev(qw_mlp *mp, const float *X, int64_t n, float *prob, cudaStream_t s);
qw_status launch_features(const float *Q, const int32_t *HQ, int64_t nq, const IndexView &ix,
                          float xs, float *F, cudaStream_t s);
qw_status launch_start_levels(const float *prob, int n, int C, float eps, int32_t *start,
                              cudaStream_t s);
// Features, network, softmax and first-level rule in one launch (inference).
qw_status launch_start_model(qw_mlp *mp, const float *Q, const int32_t *HQ, int nq,
                             const IndexView &ix, float xs, float eps, int shift, int32_t *start,
                             cudaStream_t s);
// Bitmap path: previous-level flags of the queries marked for recount.
qw_status launch_bm_recount(const IndexView &ix, int nb, int l, int cap, int cgrow, QueryState &st,
                            cudaStream_t s);
qw_status data_rms(const float *X, int64_t count, double *dev_acc, double *out, cudaStream_t s);

// Read-only view of a built index for entry points outside qw_api.cu.
struct IndexParams {
    IndexView view;
    const float *A;
    const float *b;
    float w;
    int c, v, l;
};
qw_status index_params(const qw_index *ix, IndexParams *out);

}  // namespace qw
