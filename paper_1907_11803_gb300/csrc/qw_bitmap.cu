// qw_bitmap.cu -- the bitmap path of collision counting.
//
// The level path counts collisions by scanning the index entries of every
// projection's bucket range and incrementing one counter per entry: one
// shared-memory atomic per (entry, query), plus one counter byte per (id,
// query) kept in device memory between levels.  On workloads whose ranges are
// dense (a query's range holds a quarter of the ids of a projection) that is
// both atomic-bound and counter-traffic-bound.
//
// The bitmap path trades HBM capacity for that work.  At build time it stores,
// for every projection i, id tile t, level L (radius R = c^L, Section 2's
// virtual rehashing) and level-L bucket beta, the set of the tile's ids whose
// anchored bucket id satisfies floor(bid / R) == beta, as a bitmap of kTile
// bits (4 KiB).  A query collides with an object on projection i at radius R
// exactly when the object lies in the bucket beta_i = floor(g_i / R) of the
// query, so at every level the collision count of each id is the number of
// the m bitmaps B_i(beta_i) that contain it (Section 3.1).  Counts are summed
// bit-sliced (a carry-save adder tree keeps, per 32 ids, the seven bit planes
// of their counts in registers) and recomputed from scratch at every level:
// no atomics per entry and no counters kept between levels.
//
// Ids are numbered in a locality order (a two-means tree over the data, leaves
// of 128 ids): a 128-id group holds nearby points.  Every bitmap carries a
// 256-bit summary (which groups it touches).  A group touched by fewer than l
// of the query's m buckets cannot hold a candidate, so a level runs in two
// passes: a filter on the summaries finds the live groups of every (query,
// tile), and only those are counted from the bitmaps.  Candidates go to a
// per-query list with their counts; the k + v bound and the tie rule (smallest
// original id) are applied per query at the end.  Results -- candidate sets,
// counts, statistics -- are those of the level path; a query whose candidates
// overflow the fixed lists is answered by the level path.
//
// Storage: per (projection, tile), sum over levels L of (span / c^L + 1)
// bitmaps, i.e. about (c / (c - 1)) * (span + 1) * 4 KiB, plus 32 bytes of
// summary each.  A level-L bitmap is the OR of its c children at level L - 1;
// the finest level comes from the data's bucket ids.
#include "qw_internal.cuh"
#include "qw_dir.cuh"
#include "qw_scan.cuh"
#include "qw_tma.cuh"

#include <algorithm>
#include <thread>
#include <cmath>
#include <atomic>
#include <new>
#include <vector>

namespace qw {

qw_status bitmap_layout(const std::vector<int32_t> &span, int nT, int c, BitmapLayout *out)
{
    const int m = (int)span.size();
    out->base.assign(m, 0);
    out->nb.assign(m, 0);
    out->lvl.assign((size_t)m * kBmLevels, 0);
    out->J.assign(m, 0);
    int64_t total = 0;
    for (int i = 0; i < m; ++i) {
        int J = 0;
        int64_t R = 1;
        while (R <= (int64_t)span[i]) {
            R *= c;
            ++J;
        }
        if (J >= kBmLevels) {
            set_error("qw_build_index: too many levels for the bitmap table");
            return QW_ERR_RANGE;
        }
        int32_t acc = 0;
        R = 1;
        for (int L = 0; L <= J; ++L) {
            out->lvl[(size_t)i * kBmLevels + L] = acc;
            const int64_t nbk = (int64_t)span[i] / R + 1;
            if ((int64_t)acc + nbk > INT32_MAX) {
                set_error("qw_build_index: bitmap table too large");
                return QW_ERR_RANGE;
            }
            acc += (int32_t)nbk;
            R *= c;
        }
        out->J[i] = J;
        out->nb[i] = acc;
        out->base[i] = total;
        total += (int64_t)nT * acc;
    }
    out->total = total;
    return QW_OK;
}

namespace {

constexpr int BM_THREADS = kBmUint4;  // one thread per 16 bytes (128 ids) of a tile bitmap

// Level 0: bit j of bitmap (i, t, 0, bid) for every internal id j of tile t
// whose object has anchored bucket id bid on projection i.  A warp covers one
// 32-bit word (32 consecutive internal ids); lanes with equal bids share one
// atomic OR.  The buffer is cleared first.
__global__ void __launch_bounds__(BM_THREADS) bm_fill_level0_kernel(IndexView ix,
                                                                    const int32_t *__restrict__ Ht,
                                                                    uint4 *bm)
{
    const int t = blockIdx.x, i = blockIdx.y;
    const int len = (int)min((int64_t)kTile, ix.n - (int64_t)t * kTile);
    const int64_t blk = ix.bm_base[i] + (int64_t)t * ix.bm_nb[i] + ix.bm_lvl[i * kBmLevels + 0];
    const int32_t oi = ix.o[i];
    uint32_t *bw = reinterpret_cast<uint32_t *>(bm);
    const int lane = threadIdx.x & 31;
    for (int j = threadIdx.x; j < kTile; j += BM_THREADS) {
        const bool valid = j < len;
        const int32_t bid =
            valid ? Ht[(int64_t)i * ix.n + ix.perm[(int64_t)t * kTile + j]] - oi : -1;
        const uint32_t same = __match_any_sync(0xffffffffu, bid);
        if (valid && lane == __ffs(same) - 1)
            atomicOr(&bw[(blk + bid) * (kTile / 32) + (j >> 5)], same);
    }
}

// Row j of Xloc is data row perm[j]; inv is the inverse of perm.
__global__ void locality_copy_kernel(const float *__restrict__ X, const int32_t *__restrict__ perm,
                                     int64_t n, int d, float *__restrict__ Xloc,
                                     int32_t *__restrict__ inv)
{
    for (int64_t j = blockIdx.x; j < n; j += gridDim.x) {
        const int64_t src = perm[j];
        for (int c = threadIdx.x; c < d; c += blockDim.x) Xloc[j * d + c] = X[src * d + c];
        if (threadIdx.x == 0) inv[src] = (int32_t)j;
    }
}

// Per bitmap, one bit per 128-id group: the group has at least one id.
__global__ void __launch_bounds__(BM_THREADS) bm_summary_kernel(const uint4 *__restrict__ bm,
                                                                int64_t total,
                                                                uint32_t *__restrict__ sum)
{
    for (int64_t b = blockIdx.x; b < total; b += gridDim.x) {
        const uint4 v = bm[b * kBmUint4 + threadIdx.x];
        const uint32_t word = __ballot_sync(0xffffffffu, (v.x | v.y | v.z | v.w) != 0);
        if ((threadIdx.x & 31) == 0) sum[b * (kBmUint4 / 32) + (threadIdx.x >> 5)] = word;
    }
}

// Level L >= 1: bucket beta is the union of buckets c*beta .. c*beta + c - 1
// of level L - 1 (floor(floor(bid / R) / c) == floor(bid / (R c))).
__global__ void __launch_bounds__(BM_THREADS) bm_or_level_kernel(IndexView ix, uint4 *bm, int L,
                                                                 int64_t R, int c)
{
    const int t = blockIdx.x, i = blockIdx.y;
    if (L > ix.bm_J[i]) return;
    const int64_t sp = ix.span[i];
    const int64_t nbk = sp / R + 1;
    const int64_t nbk_child = sp / (R / c) + 1;
    const int64_t blk = ix.bm_base[i] + (int64_t)t * ix.bm_nb[i];
    const uint4 *child = bm + (blk + ix.bm_lvl[i * kBmLevels + L - 1]) * kBmUint4;
    uint4 *out = bm + (blk + ix.bm_lvl[i * kBmLevels + L]) * kBmUint4;
    for (int64_t beta = 0; beta < nbk; ++beta) {
        uint4 acc = make_uint4(0, 0, 0, 0);
        for (int u = 0; u < c; ++u) {
            const int64_t ch = beta * c + u;
            if (ch >= nbk_child) break;
            const uint4 x = child[ch * kBmUint4 + threadIdx.x];
            acc.x |= x.x;
            acc.y |= x.y;
            acc.z |= x.z;
            acc.w |= x.w;
        }
        out[beta * kBmUint4 + threadIdx.x] = acc;
    }
}


// Full adder on 32 lanes of bits: lo = a ^ b ^ c, hi = majority(a, b, c).
__device__ __forceinline__ void csa(uint32_t &hi, uint32_t &lo, uint32_t a, uint32_t b, uint32_t c)
{
    const uint32_t u = a ^ b;
    hi = (a & b) | (u & c);
    lo = u ^ c;
}

// Seven bit planes of the counts of 4 x 32 ids: bit k of the count of id
// (word w, bit b) is bit b of s[k][w].
struct Planes {
    uint32_t s[7][4];
};

// Add eight one-bit inputs per id (x[0..8)) to the planes.  Ones, twos and
// fours are carry-save; eights are a binary counter incremented by ripple.
__device__ __forceinline__ void add8(Planes &P, const uint4 (&x)[8])
{
#pragma unroll
    for (int w = 0; w < 4; ++w) {
        uint32_t xs[8];
#pragma unroll
        for (int u = 0; u < 8; ++u)
            xs[u] = w == 0 ? x[u].x : (w == 1 ? x[u].y : (w == 2 ? x[u].z : x[u].w));
        uint32_t t2a, t2b, t4a, t4b, t8;
        csa(t2a, P.s[0][w], P.s[0][w], xs[0], xs[1]);
        csa(t2b, P.s[0][w], P.s[0][w], xs[2], xs[3]);
        csa(t4a, P.s[1][w], P.s[1][w], t2a, t2b);
        csa(t2a, P.s[0][w], P.s[0][w], xs[4], xs[5]);
        csa(t2b, P.s[0][w], P.s[0][w], xs[6], xs[7]);
        csa(t4b, P.s[1][w], P.s[1][w], t2a, t2b);
        csa(t8, P.s[2][w], P.s[2][w], t4a, t4b);
        uint32_t cy = t8, nx;
        nx = P.s[3][w] & cy; P.s[3][w] ^= cy; cy = nx;
        nx = P.s[4][w] & cy; P.s[4][w] ^= cy; cy = nx;
        nx = P.s[5][w] & cy; P.s[5][w] ^= cy; cy = nx;
        P.s[6][w] ^= cy;  // counts stay below 128 (m <= 127)
    }
}


// Bits of word w whose count is >= l (l in 1..127).
__device__ __forceinline__ uint32_t count_ge_planes(const Planes &P, int w, int l)
{
    uint32_t gt = 0, eq = 0xffffffffu;
#pragma unroll
    for (int k = 6; k >= 0; --k) {
        const uint32_t sk = P.s[k][w];
        if ((l >> k) & 1) {
            eq &= sk;
        } else {
            gt |= eq & sk;
            eq &= ~sk;
        }
    }
    return gt | eq;
}

__device__ __forceinline__ int count_of(const Planes &P, int w, int b)
{
    int c = 0;
#pragma unroll
    for (int k = 0; k < 7; ++k) c |= (int)((P.s[k][w] >> b) & 1u) << k;
    return c;
}

__device__ __forceinline__ uint32_t word_of(const uint4 &v, int w)
{
    return w == 0 ? v.x : (w == 1 ? v.y : (w == 2 ? v.z : v.w));
}


// The candidate bits (count >= l) of the thread's 4 x 32 ids.
__device__ __forceinline__ uint4 candidates_of(const Planes &P, int l)
{
    uint4 cand;
    cand.x = count_ge_planes(P, 0, l);
    cand.y = count_ge_planes(P, 1, l);
    cand.z = count_ge_planes(P, 2, l);
    cand.w = count_ge_planes(P, 3, l);
    return cand;
}

// Append this thread's candidates (128 ids, ascending) to the query's list
// for the level from position pos: (internal id << 32) | (prev << 8) | count.
__device__ __forceinline__ void append_candidates(const Planes &P, const uint4 &cand,
                                                  const uint4 &prev, uint64_t *list, int pos,
                                                  int64_t id_base)
{
#pragma unroll
    for (int w = 0; w < 4; ++w) {
        uint32_t x = word_of(cand, w);
        const uint32_t pw = word_of(prev, w);
        while (x) {
            const int b = __ffs(x) - 1;
            x &= x - 1;
            if (pos < kQCap)
                list[pos] = ((uint64_t)(id_base + w * 32 + b) << 32) |
                            ((uint64_t)((pw >> b) & 1u) << 8) | (uint64_t)count_of(P, w, b);
            ++pos;
        }
    }
}

// Bitmap number of the level-`level` bucket beta of projection i in tile t,
// or -1 when the bucket holds no data (beta below zero or past the span).
// Past the last stored level a single bucket (beta == 0) holds every id.
__device__ __forceinline__ int64_t bm_index(const IndexView &ix, int i, int t, int level,
                                            int64_t R, int64_t beta)
{
    const int J = ix.bm_J[i];
    int L = level;
    if (level > J) {
        if (beta != 0) return -1;
        L = J;
    } else if (beta < 0 || beta > (int64_t)ix.span[i] / R) {
        return -1;
    }
    return ix.bm_base[i] + (int64_t)t * ix.bm_nb[i] + ix.bm_lvl[i * kBmLevels + L] + beta;
}

// ---- the same level in two passes (the bitmap path's default)
//
// Pass 1, one warp per (query, tile), the tasks taken tile-major (a wave of
// warps covers one run of tiles for many queries, whose bucket bitmaps then
// serve all of them from L2): only the bucket summaries are read (8
// words of 32 bits per projection, one bit per 128-id group), and a carry-save
// sum over the m projections gives every group the number of the query's
// buckets that touch it.  Groups below l cannot hold a candidate.  A tile
// without live groups is done (its candidate count is 0); otherwise its live
// groups are recorded (a 256-bit mask: only their candidate words are written
// at this level), the item's m bitmap numbers are stored in a slot, and its
// live groups go to a work list.
// Pass 2, one thread per live group: the 128-id group's word of each of the
// m bitmaps, summed into bit planes; the group's candidates (count >= l) are
// written to the tile's candidate bitmap and the query's list.
constexpr int FL_WARPS = 8;                   // warps per block in pass 1
constexpr int kSumWords = kBmUint4 / 32;      // summary words per bitmap (8)

// Before pass 1, per (query, projection): the bitmap number of the query's
// bucket at this level in tile 0 (tile t adds t * bm_nb[i]), or -1 when the
// bucket holds no data.  Also clears the pass's item and work counters.
__global__ void bm_bucket_kernel(IndexView ix, int level, int64_t R, int nb, QueryState st,
                                 const LoopCtl *ctl)
{
    if (ctl) {
        level = ctl->level;
        R = ctl->R;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st.bm_nitems[0] = 0;
        st.bm_nwork[0] = 0;
    }
    const int m = ix.m;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)nb * m;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int q = (int)(e / m), i = (int)(e % m);
        if (!st.active[q] || level < st.start[q]) continue;
        st.bm_bq[e] = bm_index(ix, i, 0, level, R, floordiv64(st.g[e], R));
    }
}

// Bit transpose of a 32 x 32 block held one row per lane (bit b of lane i's
// word is element (i, b)): returns column `lane`, whose bit i is element
// (i, lane).  Five butterfly steps, each exchanging the off-diagonal halves
// of the blocks of that size.
__device__ __forceinline__ uint32_t transpose32(uint32_t a, int lane)
{
    const uint32_t keep[5] = {0x0000ffffu, 0x00ff00ffu, 0x0f0f0f0fu, 0x33333333u, 0x55555555u};
#pragma unroll
    for (int s = 0; s < 5; ++s) {
        const int j = 16 >> s;
        const uint32_t y = __shfl_xor_sync(0xffffffffu, a, j);
        a = (lane & j) ? (a & ~keep[s]) | ((y >> j) & keep[s])
                       : (a & keep[s]) | ((y << j) & ~keep[s]);
    }
    return a;
}

// One warp per (query, run of FL_TILES tiles).  Lane j holds the summaries of
// projections j, j + 32, ... (32 bytes each, two vector loads; the next tile's
// are loaded while the current one is counted).  For each summary word, the
// bit transpose of the lanes' rows gives lane g the projections touching group
// w * 32 + g: their number decides whether the group is live, and the same
// bits are the group's projection mask for pass 2.
constexpr int FL_TILES = 8;  // tiles per warp unless the caller picks 4 or 16

template <int NROW>
__device__ __forceinline__ void load_summaries(const IndexView &ix, const int64_t (&b0)[NROW],
                                               const int32_t (&nbp)[NROW], int t,
                                               uint4 (&sv)[NROW][2])
{
#pragma unroll
    for (int r = 0; r < NROW; ++r) {
        if (b0[r] >= 0) {
            const uint4 *p = reinterpret_cast<const uint4 *>(
                ix.bm_sum + (b0[r] + (int64_t)t * nbp[r]) * kSumWords);
            sv[r][0] = __ldg(p);
            sv[r][1] = __ldg(p + 1);
        } else {
            sv[r][0] = make_uint4(0, 0, 0, 0);
            sv[r][1] = make_uint4(0, 0, 0, 0);
        }
    }
}

template <int NROW, int TPW>
__global__ void __launch_bounds__(FL_WARPS * 32, NROW <= 2 ? 3 : 2) bm_filter_kernel(IndexView ix, int level, int l,
                                                                  int nb, QueryState st,
                                                                  const LoopCtl *ctl)
{
    constexpr int MW = (NROW + 1) / 2;
    // per warp: the projection masks of the current tile's groups
    __shared__ unsigned long long wmk[FL_WARPS][kSumWords][MW][32];
    if (ctl) level = ctl->level;
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
    const int m = ix.m, nT = ix.nT;
    const int mw = (m + 63) >> 6;
    const int nch = (nT + TPW - 1) / TPW;
    const int64_t tasks = (int64_t)nb * nch;
    const int par = level & 1;
    for (int64_t k = (int64_t)blockIdx.x * FL_WARPS + (threadIdx.x >> 5); k < tasks;
         k += (int64_t)gridDim.x * FL_WARPS) {
        // tile-major: the warps of a wave take one run of tiles for many
        // queries, so the bitmaps they touch (and the count pass after them)
        // stay in L2 across queries
        const int q = (int)(k % nb);
        const int t0 = (int)(k / nb) * TPW, t1 = min(nT, t0 + TPW);
        if (!st.active[q] || level < st.start[q]) continue;
        int64_t b0[NROW];
        int32_t nbp[NROW];
#pragma unroll
        for (int r = 0; r < NROW; ++r) {
            const int i = lane + 32 * r;
            b0[r] = i < m ? st.bm_bq[(int64_t)q * m + i] : -1;
            nbp[r] = i < m ? ix.bm_nb[i] : 0;
        }
        uint4 sv[NROW][2];
        load_summaries<NROW>(ix, b0, nbp, t0, sv);
        for (int t = t0; t < t1; ++t) {
            uint4 cur[NROW][2];
#pragma unroll
            for (int r = 0; r < NROW; ++r) {
                cur[r][0] = sv[r][0];
                cur[r][1] = sv[r][1];
            }
            if (t + 1 < t1) load_summaries<NROW>(ix, b0, nbp, t + 1, sv);
            const int64_t qt = (int64_t)q * nT + t;
            uint32_t x[kSumWords];
            int n_alive = 0;
#pragma unroll
            for (int w = 0; w < kSumWords; ++w) {
                int cnt = 0;
                unsigned long long mk[MW];
#pragma unroll
                for (int h = 0; h < MW; ++h) mk[h] = 0ull;
#pragma unroll
                for (int r = 0; r < NROW; ++r) {
                    const uint32_t c = transpose32(word_of(cur[r][w >> 2], w & 3), lane);
                    cnt += __popc(c);
                    mk[r >> 1] |= (unsigned long long)c << (32 * (r & 1));
                }
#pragma unroll
                for (int h = 0; h < MW; ++h) wmk[wi][w][h][lane] = mk[h];
                x[w] = __ballot_sync(0xffffffffu, cnt >= l);
                n_alive += __popc(x[w]);
            }
            if (lane == 0) st.clist_n[(int64_t)par * st.cln_par + qt] = 0;
            if (n_alive == 0) continue;
            // which groups have a candidate word at this level
            uint32_t xl = 0;
#pragma unroll
            for (int w = 0; w < kSumWords; ++w) xl = lane == w ? x[w] : xl;
            if (lane < kSumWords) st.bm_amask[((int64_t)par * st.cln_par + qt) * kSumWords + lane] = xl;
            int slot = 0, base = 0;
            if (lane == 0) {
                slot = atomicAdd(st.bm_nitems, 1);
                base = atomicAdd(st.bm_nwork, n_alive);
            }
            slot = __shfl_sync(0xffffffffu, slot, 0);
            base = __shfl_sync(0xffffffffu, base, 0);
            if (slot >= st.bm_item_cap) continue;
            const int mpad = (m + 3) & ~3;
#pragma unroll
            for (int r = 0; r < NROW; ++r)
                if (lane + 32 * r < mpad)
                    st.bm_item_bi[(int64_t)slot * mpad + lane + 32 * r] =
                        b0[r] >= 0 ? (int32_t)(b0[r] + (int64_t)t * nbp[r]) : -1;
            if (lane == 0) st.bm_item_qt[slot] = make_int2(q, t);
            // live groups of the tile, in ascending order, after `base`
            int pos = base, words = 0;
#pragma unroll
            for (int w = 0; w < kSumWords; ++w) {
                if ((x[w] >> lane) & 1u) {
                    const int at = pos + __popc(x[w] & ((1u << lane) - 1u));
                    if (at < st.bm_work_cap) {
                        st.bm_work[at] = (slot << 8) | (w * 32 + lane);
#pragma unroll
                        for (int h = 0; h < MW; ++h)
                            if (h < mw) {
                                const unsigned long long mk = wmk[wi][w][h][lane];
                                st.bm_wmask[(int64_t)at * mw + h] = mk;
                                words += __popcll(mk);
                            }
                    }
                }
                pos += __popc(x[w]);
            }
            if (st.bm_prof) {
                words = __reduce_add_sync(0xffffffffu, words);
                if (lane == 0) atomicAdd(st.bm_prof + 2, (unsigned long long)words);
            }
        }
    }
}

// Profile mode: add this level's live items and live groups to the totals.
__global__ void bm_prof_kernel(QueryState st)
{
    st.bm_prof[0] += (unsigned long long)min(*st.bm_nitems, st.bm_item_cap);
    st.bm_prof[1] += (unsigned long long)min(*st.bm_nwork, st.bm_work_cap);
}

__global__ void __launch_bounds__(256, 3) bm_count_kernel(IndexView ix, int level, int l,
                                                       QueryState st, const LoopCtl *ctl)
{
    if (ctl) level = ctl->level;
    const int m = ix.m, nT = ix.nT;
    const int nwork = min(*st.bm_nwork, st.bm_work_cap);
    for (int wk = blockIdx.x * blockDim.x + threadIdx.x; wk < nwork;
         wk += gridDim.x * blockDim.x) {
        const int e = st.bm_work[wk];
        const int slot = e >> 8, g = e & 0xff;
        const int2 qt2 = st.bm_item_qt[slot];
        const int q = qt2.x, t = qt2.y;
        const int64_t qt = (int64_t)q * nT + t;
        const int4 *bi4 = reinterpret_cast<const int4 *>(st.bm_item_bi + (int64_t)slot * ((m + 3) & ~3));
        Planes P;
#pragma unroll
        for (int kk = 0; kk < 7; ++kk)
#pragma unroll
            for (int w = 0; w < 4; ++w) P.s[kk][w] = 0;
        // words of projections whose summary misses the group are zero
        const int mw = (m + 63) >> 6;
        const unsigned long long mk0 = st.bm_wmask[(int64_t)wk * mw];
        const unsigned long long mk1 = mw > 1 ? st.bm_wmask[(int64_t)wk * mw + 1] : 0ull;
        for (int i0 = 0; i0 < m; i0 += 8) {
            const uint32_t bits = (uint32_t)(((i0 < 64 ? mk0 : mk1) >> (i0 & 63)) & 0xffu);
            if (bits == 0) continue;
            // eight bitmap numbers in two vector loads (the row is padded to a
            // multiple of four; entries past m are never selected by the mask)
            const int4 ba = bits & 0x0fu ? bi4[i0 >> 2] : make_int4(-1, -1, -1, -1);
            const int4 bb = bits & 0xf0u ? bi4[(i0 >> 2) + 1] : make_int4(-1, -1, -1, -1);
            const int32_t bn[8] = {ba.x, ba.y, ba.z, ba.w, bb.x, bb.y, bb.z, bb.w};
            uint4 x[8];
#pragma unroll
            for (int u = 0; u < 8; ++u)
                x[u] = (bits >> u) & 1u ? __ldg(ix.bm + (int64_t)bn[u] * kBmUint4 + g)
                                        : make_uint4(0, 0, 0, 0);
            add8(P, x);
        }
        const uint4 cand = candidates_of(P, l);
        const int nc = __popc(cand.x) + __popc(cand.y) + __popc(cand.z) + __popc(cand.w);
        // A group without candidates (most live groups) writes no word: its
        // live bit is cleared instead, and every reader of candidate words
        // (the next level, the list rebuild) treats a cleared bit as an empty
        // word.  Lanes clearing bits of the same mask word combine them.
        {
            const int64_t mw = ((int64_t)(level & 1) * st.cln_par + qt) * kSumWords + (g >> 5);
            const uint32_t clear = nc == 0 ? (1u << (g & 31)) : 0u;
            const unsigned act = __activemask();
            const unsigned peers = __match_any_sync(act, (unsigned long long)mw);
            const uint32_t all = __reduce_or_sync(peers, clear);
            if (all != 0u && (threadIdx.x & 31) == __ffs(peers) - 1)
                atomicAnd(st.bm_amask + mw, ~all);
        }
        if (nc == 0) continue;
        st.cbits[(int64_t)(level & 1) * st.cb_par + qt * kBmUint4 + g] = cand;
        // the previous level's candidate word, needed only to flag the new
        // candidates: written there only if the tile had candidates and the
        // group was live
        const bool first = level == st.start[q];
        const int64_t pq = (int64_t)((level - 1) & 1) * st.cln_par + qt;
        const bool has_prev = !first && st.clist_n[pq] > 0 &&
                              ((st.bm_amask[pq * kSumWords + (g >> 5)] >> (g & 31)) & 1u);
        const uint4 prev = has_prev ? st.cbits[(int64_t)((level - 1) & 1) * st.cb_par + qt * kBmUint4 + g]
                                    : make_uint4(0, 0, 0, 0);
        atomicAdd(st.clist_n + (int64_t)(level & 1) * st.cln_par + qt, nc);
        atomicAdd(st.cross + q, nc);
        const int pos = atomicAdd(st.qbuf_n + (int64_t)(level & 1) * st.qbn_par + q, nc);
        append_candidates(P, cand, prev, st.qbuf + (int64_t)(level & 1) * st.qb_par + (int64_t)q * kQCap,
                          pos, (int64_t)t * kTile + (int64_t)g * 128);
    }
}

// ---- the same level in one pass (filter and count fused)
//
// One warp per (query, run of FL_TILES tiles), as in pass 1 above: the bucket
// summaries give every 128-id group the set of the query's buckets touching
// it, and the groups touched by at least l buckets are live.  The same warp
// then counts its live groups, 32 at a time (lane k takes the k-th live group
// of the tile): the m bitmap numbers of the tile stay in the lanes' registers
// (lane j holds projections j and j + 32) and are broadcast by shuffles, so a
// group's m word loads depend on nothing but its own projection mask, which
// the filter step left in shared memory.  No work list, item slots or masks go
// through global memory.  Results (candidate words, live-group masks, tile
// counts, candidate lists, profile counters) are those of the two passes.
// Position of the n-th (0-based) set bit of v; n < popc(v).
__device__ __forceinline__ int nth_set_bit(uint32_t v, int n)
{
    int pos = 0;
#pragma unroll
    for (int w = 16; w > 0; w >>= 1) {
        const int c = __popc(v & ((1u << w) - 1u));
        if (n >= c) {
            n -= c;
            v >>= w;
            pos += w;
        }
    }
    return pos;
}

template <int NROW, int TPW>
__global__ void __launch_bounds__(FL_WARPS * 32, 2) bm_fused_kernel(IndexView ix, int level,
                                                                   int l, int nb, QueryState st,
                                                                   const LoopCtl *ctl)
{
    constexpr int MW = (NROW + 1) / 2;
    __shared__ unsigned long long wmk[FL_WARPS][kSumWords][MW][32];
    __shared__ uint32_t wlive[FL_WARPS][kSumWords];
    if (ctl) level = ctl->level;
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
    const int m = ix.m, nT = ix.nT;
    const int nch = (nT + TPW - 1) / TPW;
    const int64_t tasks = (int64_t)nb * nch;
    const int par = level & 1;
    unsigned long long p_items = 0, p_groups = 0, p_words = 0;
    for (int64_t k = (int64_t)blockIdx.x * FL_WARPS + wi; k < tasks;
         k += (int64_t)gridDim.x * FL_WARPS) {
        // tile-major: the warps of a wave take one run of tiles for many
        // queries, so the bitmaps they touch (and the count pass after them)
        // stay in L2 across queries
        const int q = (int)(k % nb);
        const int t0 = (int)(k / nb) * TPW, t1 = min(nT, t0 + TPW);
        if (!st.active[q] || level < st.start[q]) continue;
        const bool first = level == st.start[q];
        int64_t b0[NROW];
        int32_t nbp[NROW];
#pragma unroll
        for (int r = 0; r < NROW; ++r) {
            const int i = lane + 32 * r;
            b0[r] = i < m ? st.bm_bq[(int64_t)q * m + i] : -1;
            nbp[r] = i < m ? ix.bm_nb[i] : 0;
        }
        uint4 sv[NROW][2];
        load_summaries<NROW>(ix, b0, nbp, t0, sv);
        for (int t = t0; t < t1; ++t) {
            const int64_t qt = (int64_t)q * nT + t;
            int n_alive = 0;
#pragma unroll
            for (int w = 0; w < kSumWords; ++w) {
                int cnt = 0;
                unsigned long long mk[MW];
#pragma unroll
                for (int h = 0; h < MW; ++h) mk[h] = 0ull;
#pragma unroll
                for (int r = 0; r < NROW; ++r) {
                    const uint32_t c = transpose32(word_of(sv[r][w >> 2], w & 3), lane);
                    cnt += __popc(c);
                    mk[r >> 1] |= (unsigned long long)c << (32 * (r & 1));
                }
#pragma unroll
                for (int h = 0; h < MW; ++h) wmk[wi][w][h][lane] = mk[h];
                const uint32_t xw = __ballot_sync(0xffffffffu, cnt >= l);
                if (lane == 0) wlive[wi][w] = xw;
                n_alive += __popc(xw);
            }
            __syncwarp();
            // the next tile's summaries load while this tile is counted
            if (t + 1 < t1) load_summaries<NROW>(ix, b0, nbp, t + 1, sv);
            if (n_alive == 0) {
                if (lane == 0) st.clist_n[(int64_t)par * st.cln_par + qt] = 0;
                continue;
            }
            if (lane < kSumWords)
                st.bm_amask[((int64_t)par * st.cln_par + qt) * kSumWords + lane] = wlive[wi][lane];
            // this tile's bitmap numbers, one per lane and row
            int64_t bt[NROW];
#pragma unroll
            for (int r = 0; r < NROW; ++r) bt[r] = b0[r] >= 0 ? b0[r] + (int64_t)t * nbp[r] : -1;
            const int64_t pq = (int64_t)((level - 1) & 1) * st.cln_par + qt;
            const bool tile_prev = !first && st.clist_n[pq] > 0;
            int tile_n = 0;
            for (int base = 0; base < n_alive; base += 32) {
                // the (base + lane)-th live group of the tile
                const int kk = base + lane;
                int g = -1;
                {
                    int acc = 0;
#pragma unroll
                    for (int w = 0; w < kSumWords; ++w) {
                        const uint32_t xw = wlive[wi][w];
                        const int c = __popc(xw);
                        if (g < 0 && kk < acc + c) g = w * 32 + nth_set_bit(xw, kk - acc);
                        acc += c;
                    }
                }
                unsigned long long mk[MW];
#pragma unroll
                for (int h = 0; h < MW; ++h)
                    mk[h] = g >= 0 ? wmk[wi][g >> 5][h][g & 31] : 0ull;
                const bool has_prev =
                    g >= 0 && tile_prev &&
                    ((st.bm_amask[pq * kSumWords + (g >> 5)] >> (g & 31)) & 1u);
                const uint4 prev = has_prev ? st.cbits[(int64_t)((level - 1) & 1) * st.cb_par +
                                                       qt * kBmUint4 + g]
                                            : make_uint4(0, 0, 0, 0);
                Planes P;
#pragma unroll
                for (int kq = 0; kq < 7; ++kq)
#pragma unroll
                    for (int w = 0; w < 4; ++w) P.s[kq][w] = 0;
                int words = 0;
#pragma unroll
                for (int h = 0; h < MW; ++h) words += __popcll(mk[h]);
                for (int i0 = 0; i0 < m; i0 += 8) {
                    uint4 xv[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int i = i0 + u;
                        const int r = i >> 5;
                        int64_t bn = 0;
#pragma unroll
                        for (int rr = 0; rr < NROW; ++rr)
                            if (rr == r) bn = __shfl_sync(0xffffffffu, bt[rr], i & 31);
                        const bool on = i < m && ((mk[i >> 6] >> (i & 63)) & 1ull);
                        xv[u] = on ? __ldg(ix.bm + bn * kBmUint4 + g) : make_uint4(0, 0, 0, 0);
                    }
                    add8(P, xv);
                }
                uint4 cand = make_uint4(0, 0, 0, 0);
                int nc = 0;
                if (g >= 0) {
                    cand = candidates_of(P, l);
                    st.cbits[(int64_t)par * st.cb_par + qt * kBmUint4 + g] = cand;
                    nc = __popc(cand.x) + __popc(cand.y) + __popc(cand.z) + __popc(cand.w);
                    p_words += (unsigned long long)words;
                }
                // list positions: one reservation per warp
                int incl = nc;
#pragma unroll
                for (int off = 1; off < 32; off <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, incl, off);
                    if (lane >= off) incl += y;
                }
                const int tot = __shfl_sync(0xffffffffu, incl, 31);
                int pos0 = 0;
                if (lane == 0 && tot)
                    pos0 = atomicAdd(st.qbuf_n + (int64_t)par * st.qbn_par + q, tot);
                pos0 = __shfl_sync(0xffffffffu, pos0, 0);
                if (nc)
                    append_candidates(P, cand, prev,
                                      st.qbuf + (int64_t)par * st.qb_par + (int64_t)q * kQCap,
                                      pos0 + incl - nc, (int64_t)t * kTile + (int64_t)g * 128);
                tile_n += tot;
            }
            if (lane == 0) {
                st.clist_n[(int64_t)par * st.cln_par + qt] = tile_n;
                if (tile_n) atomicAdd(st.cross + q, tile_n);
            }
            p_items += 1;
            p_groups += (unsigned long long)n_alive;
        }
    }
    if (st.bm_prof) {
        p_words = __reduce_add_sync(0xffffffffu, (unsigned)p_words);
        if (lane == 0 && (p_items || p_words)) {
            atomicAdd(st.bm_prof + 0, p_items);
            atomicAdd(st.bm_prof + 1, p_groups);
            atomicAdd(st.bm_prof + 2, p_words);
        }
    }
}

// ---- the same level with the bitmaps staged by TMA
//
// One persistent CTA per SM walks the (query, tile) items of the batch,
// item k = blockIdx.x + j * gridDim.x (consecutive queries are in signature
// order, so the CTAs working at one time share most bitmaps in L2).  A
// producer warp streams stages of 8 bitmaps into a ring in shared memory: its
// lanes compute the 64 bitmap addresses of an item in parallel (bucket ids of
// the next item prefetched a step ahead), lane 0 issues one 4 KiB bulk copy
// per present bitmap and writes a small header per stage (item, which
// bitmaps are present, first / last stage of the item, end of work).  Eight
// consumer warps follow the stage stream: each adds a stage into its bit
// planes straight from shared memory and, at an item's last stage, writes the
// item's candidate bitmap, list and profile.  Consumers never wait on a
// global load for control flow.
constexpr int kRing = 6;
constexpr int kPerStage = 8;                       // bitmaps per stage
constexpr int kStageBytesBm = kPerStage * kTile / 8;  // 32 KiB
constexpr int TMA_CONSUMERS = BM_THREADS;          // 8 warps, one 16-byte word each
constexpr int TMA_THREADS = TMA_CONSUMERS + 32;    // + the producer warp
constexpr uint32_t kFirstStage = 1, kLastStage = 2, kFirstLevel = 4, kDone = 8;

struct StageHdr {
    int32_t q, t;
    uint32_t mask;   // which of the stage's bitmaps are present
    uint32_t flags;  // kFirstStage | kLastStage | kFirstLevel | kDone
};

struct TmaShared {
    uint64_t full[kRing];
    uint64_t empty[kRing];
    uint64_t group;                // consumer-only barrier (one arrival per warp)
    StageHdr hdr[kRing];
    int64_t pt[QW_MAX_M + 8];      // bitmap numbers of the current item (-1: empty)
    int64_t lbase[QW_MAX_M];       // per projection: bm_base + bm_lvl[min(level, J)]
    int32_t nbk[QW_MAX_M];         // per projection: buckets at this level (0: past J)
    int32_t pnb[QW_MAX_M];         // per projection: bitmaps per tile
    int base[2];                   // list position of the current item (alternating)
    int wsum[TMA_CONSUMERS / 32];
};

size_t tma_smem_bytes() { return sizeof(TmaShared) + 128 + (size_t)kRing * kStageBytesBm; }

// The consumer warps meet on an mbarrier (bounded wait) rather than a named
// barrier, so a warp that gave up on a wait cannot leave the others waiting.
__device__ __forceinline__ void group_sync(uint64_t *bar, uint32_t &ph, int *err, bool &stuck)
{
    __syncwarp();
    if ((threadIdx.x & 31) == 0) mbar_arrive(bar);
    mbar_wait(bar, ph & 1, err, stuck);
    ++ph;
}

// Exclusive prefix sum over the consumer threads (see block_exclusive_scan).
__device__ __forceinline__ int consumer_scan(int v, int *tmp, int *total, uint64_t *bar,
                                             uint32_t &ph, int *err, bool &stuck)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += y;
    }
    group_sync(bar, ph, err, stuck);  // tmp of the previous scan has been read
    if (lane == 31) tmp[warp] = incl;
    group_sync(bar, ph, err, stuck);
    int wbase = 0, tot = 0;
#pragma unroll
    for (int w = 0; w < TMA_CONSUMERS / 32; ++w) {
        int s = tmp[w];
        if (w < warp) wbase += s;
        tot += s;
    }
    *total = tot;
    return wbase + incl - v;
}

__global__ void __launch_bounds__(TMA_THREADS, 1) bm_level_tma_kernel(IndexView ix, int level,
                                                                      int64_t R, int l, int nb,
                                                                      QueryState st,
                                                                      const LoopCtl *ctl, int *err)
{
    extern __shared__ __align__(128) unsigned char smraw[];
    TmaShared &sh = *reinterpret_cast<TmaShared *>(smraw);
    unsigned char *ring = smraw + ((sizeof(TmaShared) + 127) / 128) * 128;
    if (ctl) {
        level = ctl->level;
        R = ctl->R;
    }
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int m = ix.m, nT = ix.nT;
    const int nst = (m + kPerStage - 1) / kPerStage;  // stages per item
    const int64_t items = (int64_t)nb * nT;
    if (tid == 0) {
        for (int k = 0; k < kRing; ++k) {
            mbar_init(&sh.full[k], 1);
            mbar_init(&sh.empty[k], TMA_CONSUMERS / 32);
        }
        mbar_init(&sh.group, TMA_CONSUMERS / 32);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int i = tid; i < m; i += TMA_THREADS) {
        const int J = ix.bm_J[i];
        const int L = level > J ? J : level;
        sh.lbase[i] = ix.bm_base[i] + ix.bm_lvl[i * kBmLevels + L];
        sh.nbk[i] = level > J ? 0 : (int32_t)((int64_t)ix.span[i] / R + 1);
        sh.pnb[i] = ix.bm_nb[i];
    }
    __syncthreads();
    bool stuck = false;
    if (warp == TMA_CONSUMERS / 32) {
        // ---- producer warp
        constexpr int kPL = (QW_MAX_M + 31) / 32;  // projections per lane
        uint32_t it = 0;
        int64_t k = blockIdx.x;
        int64_t gn[kPL];
        int act_n = 0, start_n = 0;
        auto prefetch = [&](int64_t kk) {
            if (kk >= items) return;
            const int qq = (int)(kk % nb);
            act_n = st.active[qq];
            start_n = st.start[qq];
#pragma unroll
            for (int u = 0; u < kPL; ++u) {
                const int i = lane + 32 * u;
                gn[u] = i < m ? st.g[(int64_t)qq * m + i] : 0;
            }
        };
        prefetch(k);
        for (; k < items && !stuck; k += gridDim.x) {
            // tile-major item order (one tile's bitmaps serve many queries in L2)
            const int q = (int)(k % nb), t = (int)(k / nb);
            int64_t g[kPL];
#pragma unroll
            for (int u = 0; u < kPL; ++u) g[u] = gn[u];
            const bool runs = act_n && level >= start_n;
            const bool first = level == start_n;
            prefetch(k + gridDim.x);  // in flight while this item is issued
            if (!runs) continue;
#pragma unroll
            for (int u = 0; u < kPL; ++u) {
                const int i = lane + 32 * u;
                if (i < m) {
                    const int64_t beta = floordiv64(g[u], R);
                    const int nbk = sh.nbk[i];
                    // past the last stored level one bucket (beta == 0) holds every id
                    const bool present = nbk == 0 ? beta == 0 : (beta >= 0 && beta < nbk);
                    sh.pt[i] = present ? sh.lbase[i] + (int64_t)t * sh.pnb[i] + (nbk ? beta : 0)
                                       : -1;
                }
            }
            __syncwarp();
            if (lane == 0) {
                for (int j = 0; j < nst && !stuck; ++j, ++it) {
                    const int slot = (int)(it % kRing);
                    if (it >= (uint32_t)kRing)
                        mbar_wait(&sh.empty[slot], ((it / kRing) - 1) & 1, err, stuck);
                    if (stuck) break;
                    uint32_t mask = 0;
#pragma unroll
                    for (int u = 0; u < kPerStage; ++u) {
                        const int i = j * kPerStage + u;
                        if (i < m && sh.pt[i] >= 0) mask |= 1u << u;
                    }
                    StageHdr &h = sh.hdr[slot];
                    h.q = q;
                    h.t = t;
                    h.mask = mask;
                    h.flags = (j == 0 ? kFirstStage : 0u) | (j == nst - 1 ? kLastStage : 0u) |
                              (first ? kFirstLevel : 0u);
                    mbar_arrive_expect_tx(&sh.full[slot], (uint32_t)__popc(mask) * (kTile / 8));
#pragma unroll
                    for (int u = 0; u < kPerStage; ++u)
                        if ((mask >> u) & 1u)
                            bulk_g2s(ring + (size_t)slot * kStageBytesBm + (size_t)u * (kTile / 8),
                                     ix.bm + sh.pt[j * kPerStage + u] * kBmUint4, kTile / 8,
                                     &sh.full[slot]);
                }
            }
            stuck = __shfl_sync(0xffffffffu, stuck, 0);
            __syncwarp();
        }
        if (lane == 0) {
            if (!stuck) {
                // end of work
                const int slot = (int)(it % kRing);
                if (it >= (uint32_t)kRing)
                    mbar_wait(&sh.empty[slot], ((it / kRing) - 1) & 1, err, stuck);
                if (!stuck) {
                    sh.hdr[slot].flags = kDone;
                    sh.hdr[slot].mask = 0;
                    mbar_arrive_expect_tx(&sh.full[slot], 0);
                    ++it;
                }
            }
            if (stuck) {
                // no bulk copy may still be writing shared memory at exit
                for (uint32_t d = 0; d < (uint32_t)kRing && d < it; ++d) {
                    const uint32_t jt = it - 1 - d;
                    bool again = false;
                    mbar_wait(&sh.full[jt % kRing], (jt / kRing) & 1, err, again);
                }
            }
        }
        return;
    }
    // ---- consumers: thread tid owns 16-byte word tid (128 ids) of every bitmap
    uint32_t it = 0, gph = 0;
    int par = 0;
    Planes P;
    uint4 prev = make_uint4(0, 0, 0, 0);
    for (;; ++it) {
        const int slot = (int)(it % kRing);
        mbar_wait(&sh.full[slot], (it / kRing) & 1, err, stuck);
        if (stuck) break;
        const StageHdr h = sh.hdr[slot];
        if (h.flags & kDone) break;
        const int64_t qt = (int64_t)h.q * nT + h.t;
        if (h.flags & kFirstStage) {
#pragma unroll
            for (int kk = 0; kk < 7; ++kk)
#pragma unroll
                for (int w = 0; w < 4; ++w) P.s[kk][w] = 0;
            prev = (h.flags & kFirstLevel)
                       ? make_uint4(0, 0, 0, 0)
                       : st.cbits[(int64_t)((level - 1) & 1) * st.cb_par + qt * kBmUint4 + tid];
        }
        const uint4 *stage = reinterpret_cast<const uint4 *>(ring + (size_t)slot * kStageBytesBm);
        uint4 x[kPerStage];
#pragma unroll
        for (int u = 0; u < kPerStage; ++u)
            x[u] = ((h.mask >> u) & 1u) ? stage[u * kBmUint4 + tid] : make_uint4(0, 0, 0, 0);
        __syncwarp();
        if (lane == 0) mbar_arrive(&sh.empty[slot]);
        add8(P, x);
        if (!(h.flags & kLastStage)) continue;
        // ---- the item's epilogue (consumers only: the producer does not take part)
        const uint4 cand = candidates_of(P, l);
        st.cbits[(int64_t)(level & 1) * st.cb_par + qt * kBmUint4 + tid] = cand;
        const int my_count = __popc(cand.x) + __popc(cand.y) + __popc(cand.z) + __popc(cand.w);
        int tot_count;
        const int pos = consumer_scan(my_count, sh.wsum, &tot_count, &sh.group, gph, err, stuck);
        if (tid == 0) {
            st.clist_n[(int64_t)(level & 1) * st.cln_par + qt] = tot_count;
            sh.base[par] = tot_count ? atomicAdd(st.qbuf_n + (int64_t)(level & 1) * st.qbn_par + h.q,
                                                 tot_count)
                                     : 0;
            if (tot_count) atomicAdd(st.cross + h.q, tot_count);
        }
        group_sync(&sh.group, gph, err, stuck);
        if (stuck) break;
        append_candidates(P, cand, prev,
                          st.qbuf + (int64_t)(level & 1) * st.qb_par + (int64_t)h.q * kQCap,
                          sh.base[par] + pos, (int64_t)h.t * kTile + tid * 128);
        par ^= 1;
    }
}

// Sort keys[0..n) ascending in shared memory (n padded to P2 with ~0).
__device__ __forceinline__ void smem_bitonic(uint64_t *keys, int n, int P2)
{
    for (int i = n + (int)threadIdx.x; i < P2; i += blockDim.x) keys[i] = ~0ull;
    __syncthreads();
    for (int kk = 2; kk <= P2; kk <<= 1) {
        for (int jj = kk >> 1; jj > 0; jj >>= 1) {
            for (int x = threadIdx.x; x < (P2 >> 1); x += blockDim.x) {
                const int a = 2 * x - (x & (jj - 1));
                const int c = a + jj;
                const bool up = (a & kk) == 0;
                if ((keys[a] > keys[c]) == up) {
                    const uint64_t tmp = keys[a];
                    keys[a] = keys[c];
                    keys[c] = tmp;
                }
            }
            __syncthreads();
        }
    }
}

// The k + v bound on the bitmap path, one block per query, from the list of
// its last level's candidates: the boundary count c* and how many ids at c*
// are kept follow from the counts exactly as on the level path (Section 3.1,
// readings R4/R5); candidates of the previous level and those above c* are
// kept, and of those at c* the ones with the smallest original ids (radix
// selection of the take-th smallest id of the tie class).  The kept list is
// written with its counts in no particular order, or in ascending original id
// when `sorted`, plus the per-query statistics.  A tie class longer than its
// list (kEqCap ids) is selected from the candidate list itself.  A query whose
// candidate list overflowed keeps nothing here and is marked (bm_ovf); the
// list rebuild below shortens its list and this selection runs again on it (a
// query whose rebuilt list would still overflow goes to the level path).
constexpr int SEL_THREADS = 256;
static_assert(kHistBins <= 256, "count histogram shares the radix histogram");

__global__ void __launch_bounds__(SEL_THREADS) bm_select_kernel(IndexView ix, int l, int cap,
                                                                QueryState st,
                                                                int64_t *__restrict__ stats_out,
                                                                bool sorted)
{
    extern __shared__ uint64_t keys[];
    __shared__ int hist[256];
    __shared__ int bc[4];
    __shared__ int s_np, s_nd, s_ne, s_nt, s_cstar, s_take, s_keep;
    const int q = blockIdx.x;
    const int m = ix.m;
    const int lane = threadIdx.x & 31;
    const uint32_t below = (1u << lane) - 1u;
    const int jf = st.levels[q] - 1;
    const int n = st.qbuf_n[(int64_t)(jf & 1) * st.qbn_par + q];
    const int nc = st.ncand[q];
    const uint64_t *E = st.qbuf + (int64_t)(jf & 1) * st.qb_par + (int64_t)q * kQCap;
    int32_t *cand = st.cand + (int64_t)q * cap;
    int32_t *col = st.cand_col + (int64_t)q * cap;
    int32_t *eq = st.eqbuf + (int64_t)q * kEqCap;
    // a rebuilt list (flag 4) holds only the kept entries and the tie class
    const bool ovf_list = n > kQCap || (n != nc && !(st.bm_ovf[q] & 4));
    const int nl = ovf_list ? 0 : n;
    if (threadIdx.x == 0) {
        s_np = 0;
        s_nd = 0;
        s_ne = 0;
        s_nt = 0;
    }
    for (int c = threadIdx.x; c < kHistBins; c += SEL_THREADS) hist[c] = 0;
    __syncthreads();
    // counts of the candidates not of the previous level, and how many are
    for (int j0 = 0; j0 < nl; j0 += SEL_THREADS) {
        const int j = j0 + threadIdx.x;
        const uint64_t e = j < nl ? E[j] : 0ull;
        const bool pf = j < nl && ((e >> 8) & 1u);
        const bool other = j < nl && !pf;
        const uint32_t bp = __ballot_sync(0xffffffffu, pf);
        if (lane == 0 && bp) atomicAdd(&s_np, __popc(bp));
        const uint32_t bin = other ? 1u + (uint32_t)(e & 0xffu) : 1024u + lane;
        const uint32_t peers = __match_any_sync(0xffffffffu, bin);
        if (other && lane == __ffs(peers) - 1) atomicAdd(&hist[bin], __popc(peers));
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int cstar = l - 1, take = 0;
        const int np = s_np;
        if (nc > cap) {
            const int need = cap - np;
            int acc = 0;
            for (int c = m; c >= l; --c) {
                const int hc = hist[1 + c];
                if (acc + hc >= need) {
                    cstar = c;
                    take = need - acc;
                    break;
                }
                acc += hc;
            }
        }
        int kept = np + take;
        for (int c = max(cstar + 1, l); c <= m; ++c) kept += hist[1 + c];
        s_cstar = cstar;
        s_take = take;
        s_keep = min(kept, cap);
    }
    __syncthreads();
    const int cstar = s_cstar, take = s_take, keep = s_keep;
    // kept outright, and the tie class at c* (original ids); one slot
    // reservation per warp
    const int32_t *perm = ix.perm;
    for (int j0 = 0; j0 < nl; j0 += SEL_THREADS) {
        const int j = j0 + threadIdx.x;
        const uint64_t e = j < nl ? E[j] : 0ull;
        const int c = (int)(e & 0xffu);
        const bool pf = (e >> 8) & 1u;
        const bool kp = j < nl && (pf || c > cstar);
        const bool ti = j < nl && !kp && c == cstar && take > 0;
        const uint32_t bk = __ballot_sync(0xffffffffu, kp);
        const uint32_t bt = __ballot_sync(0xffffffffu, ti);
        int baseK = 0, baseT = 0;
        if (lane == 0) {
            if (bk) baseK = atomicAdd(&s_nd, __popc(bk));
            if (bt) baseT = atomicAdd(&s_ne, __popc(bt));
        }
        baseK = __shfl_sync(0xffffffffu, baseK, 0);
        baseT = __shfl_sync(0xffffffffu, baseT, 0);
        if (kp || ti) {
            const int32_t orig = perm[e >> 32];
            if (kp) {
                const int d = baseK + __popc(bk & below);
                if (d < cap) {
                    cand[d] = orig;
                    col[d] = c;
                }
            } else {
                const int t = baseT + __popc(bt & below);
                if (t < kEqCap) eq[t] = orig;
            }
        }
    }
    __syncthreads();
    const int nd = s_nd, ne = s_ne;
    const bool ovf = ovf_list || nd + take != keep || take > ne;
    if (ovf) {
        if (threadIdx.x == 0) {
            atomicOr(st.bm_ovf + q, 1);
            st.nkeep[q] = 0;
        }
        for (int p = threadIdx.x; p < cap; p += SEL_THREADS) {
            cand[p] = -1;
            col[p] = 0;
        }
        return;
    }
    if (take > 0 && ne > kEqCap) {
        // a tie class larger than its list: select from the candidate list
        // itself (members: not of the previous level, count c*), keyed by
        // original id
        auto tie = [&](int j, uint32_t *u) {
            const uint64_t e = E[j];
            if (((e >> 8) & 1u) || (int)(e & 0xffu) != cstar) return false;
            *u = (uint32_t)perm[e >> 32];
            return true;
        };
        const uint32_t T =
            take < ne ? block_kth_smallest_if<SEL_THREADS>(nl, take, tie, hist, bc) : 0xffffffffu;
        for (int j0 = 0; j0 < nl; j0 += SEL_THREADS) {
            const int j = j0 + threadIdx.x;
            uint32_t id = 0u;
            const bool in = j < nl && tie(j, &id) && id <= T;
            const uint32_t b = __ballot_sync(0xffffffffu, in);
            int base = 0;
            if (lane == 0 && b) base = atomicAdd(&s_nt, __popc(b));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (in) {
                cand[nd + base + __popc(b & below)] = (int32_t)id;
                col[nd + base + __popc(b & below)] = cstar;
            }
        }
        __syncthreads();
    } else if (take > 0) {
        // the take smallest ids of the tie class: those <= its take-th smallest
        // (ids are distinct, so exactly take of them)
        const uint32_t T = take < ne ? block_kth_smallest<SEL_THREADS>(
                                           reinterpret_cast<const uint32_t *>(eq), ne, take, hist, bc)
                                     : 0xffffffffu;
        for (int j0 = 0; j0 < ne; j0 += SEL_THREADS) {
            const int j = j0 + threadIdx.x;
            const uint32_t id = j < ne ? (uint32_t)eq[j] : 0u;
            const bool in = j < ne && id <= T;
            const uint32_t b = __ballot_sync(0xffffffffu, in);
            int base = 0;
            if (lane == 0 && b) base = atomicAdd(&s_nt, __popc(b));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (in) {
                cand[nd + base + __popc(b & below)] = (int32_t)id;
                col[nd + base + __popc(b & below)] = cstar;
            }
        }
        __syncthreads();
    }
    if (sorted) {
        int P2 = 2;
        while (P2 < keep) P2 <<= 1;
        for (int i = threadIdx.x; i < keep; i += SEL_THREADS)
            keys[i] = ((uint64_t)(uint32_t)cand[i] << 32) | (uint32_t)col[i];
        smem_bitonic(keys, keep, P2);
        for (int i = threadIdx.x; i < keep; i += SEL_THREADS) {
            cand[i] = (int32_t)(keys[i] >> 32);
            col[i] = (int32_t)(keys[i] & 0xffffffffu);
        }
    }
    for (int p = keep + threadIdx.x; p < cap; p += SEL_THREADS) {
        cand[p] = -1;
        col[p] = 0;
    }
    if (threadIdx.x == 0) {
        st.nkeep[q] = keep;
        if (stats_out) {
            int64_t *so = stats_out + (int64_t)q * QW_NSTAT;
            so[0] = st.levels[q];
            so[1] = st.finalR[q];
            so[2] = nc;
            so[3] = keep;
            so[4] = st.term[q];
            so[5] = st.scan_last[q];
            so[6] = st.scan_full[q];
            so[7] = st.nprev[q];
        }
    }
}

// ---- a last level that overflows the candidate list
//
// The count kernels list every candidate of a level, up to kQCap per query.
// When one doubling of the radius sweeps whole clusters into a query's last
// level, that level can hold more.  Of them the k + v bound keeps only the
// previous level's candidates, every candidate whose count is above the
// boundary count c*, and the smallest original ids of the tie class at c*
// (Section 3.1, readings R4/R5).  The kernels below rebuild the list of such
// a query with only those entries, from the candidate words of its last level
// (still in place: a stopped query's tiles are not touched by later levels)
// and the level bitmaps, each read once:
//   rd_compact  lists the overflowing queries (slots) and their buckets;
//   rd_count    one thread per 128-id group holding candidates: the counts
//               from the m bitmap words of the last level, the previous
//               level's candidate word (at a learned first level: their
//               counts there, from that level's bitmaps), stored as seven bit
//               planes and the word (128 bytes per group); the histogram of
//               the counts of the candidates not of the previous level;
//   rd_plan 0   c* and how many ids at c* are kept, as the selection derives
//               them;
//   rd_scan     when the tie class at c* holds more than kRdTieList ids: walks
//               the original ids upward (data id -> internal id -> candidate
//               word, stored count, previous-level word) and lists the take
//               smallest tie members, so that the list stays short;
//   rd_emit     the other kept entries (and a short tie class) from the
//               stored planes, written as the count kernels write them;
//   rd_plan 2   the list lengths.
// The selection then runs on the rebuilt list as on any other, with the same
// result as from the whole list.  A query whose rebuilt list would still
// overflow keeps the level-path answer, and so do the slots beyond one
// store's worth (kRdStoreBytes).
constexpr int kRdTieList = 4096;   // larger tie classes are cut by the original-id walk
constexpr int kRdStoreWords = 8;  // uint4 per group: 7 count planes, previous-level word
constexpr int RD_THREADS = 256;
static_assert(RD_THREADS == kBmUint4, "one block covers the groups of one tile");

// The candidate word of group g at level L (zero where the level wrote none).
__device__ __forceinline__ uint4 rd_word(const QueryState &st, int L, int64_t qt, int g, bool tma)
{
    const int64_t pc = (int64_t)(L & 1) * st.cln_par + qt;
    if (st.clist_n[pc] == 0) return make_uint4(0, 0, 0, 0);
    if (!tma && !((st.bm_amask[pc * kSumWords + (g >> 5)] >> (g & 31)) & 1u))
        return make_uint4(0, 0, 0, 0);
    return st.cbits[(int64_t)(L & 1) * st.cb_par + qt * kBmUint4 + g];
}

// Count planes of group g of tile t from the bitmaps of one level: bq[i] is
// the bucket's bitmap in tile 0 (-1: no data), tile t adds t * bm_nb[i].
__device__ __forceinline__ void rd_planes(const IndexView &ix, const int64_t *bq, int t, int g,
                                          Planes &P)
{
    const int m = ix.m;
#pragma unroll
    for (int kk = 0; kk < 7; ++kk)
#pragma unroll
        for (int w = 0; w < 4; ++w) P.s[kk][w] = 0;
    for (int i0 = 0; i0 < m; i0 += 8) {
        uint4 x[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int i = i0 + u;
            const int64_t b = i < m ? bq[i] : -1;
            x[u] = b >= 0 ? __ldg(ix.bm + (b + (int64_t)t * ix.bm_nb[i]) * kBmUint4 + g)
                          : make_uint4(0, 0, 0, 0);
        }
        add8(P, x);
    }
}

// Bits of word w whose count equals c.
__device__ __forceinline__ uint32_t count_eq_planes(const Planes &P, int w, int c)
{
    uint32_t eq = 0xffffffffu;
#pragma unroll
    for (int k = 0; k < 7; ++k) eq &= ((c >> k) & 1) ? P.s[k][w] : ~P.s[k][w];
    return eq;
}

__global__ void rd_compact_kernel(IndexView ix, int cgrow, QueryState st, int nb)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nb) return;
    const int L = st.levels[q] - 1;
    if (L < 0 || st.qbuf_n[(int64_t)(L & 1) * st.qbn_par + q] <= kQCap) return;
    const int slot = atomicAdd(st.rd_ctl, 1);
    RdPlan p;
    memset(&p, 0, sizeof(p));
    p.q = q;
    p.mode = 1;
    p.prev_recount = (L - 1 < st.start[q] && L > 0) ? 1 : 0;
    st.rd_plan[slot] = p;
    int32_t *h = st.rd_hist + (int64_t)slot * kHistBins;
    for (int c = 0; c < kHistBins; ++c) h[c] = 0;
    const int64_t R = st.finalR[q];
    int64_t *bq = st.rd_bq + (int64_t)slot * 2 * QW_MAX_M;
    for (int i = 0; i < ix.m; ++i) {
        const int64_t gi = st.g[(int64_t)q * ix.m + i];
        bq[i] = bm_index(ix, i, 0, L, R, floordiv64(gi, R));
        bq[QW_MAX_M + i] =
            L > 0 ? bm_index(ix, i, 0, L - 1, R / cgrow, floordiv64(gi, R / cgrow)) : -1;
    }
}

// One block per (slot, tile) at a time, one thread per group.
__global__ void __launch_bounds__(RD_THREADS, 2) rd_count_kernel(IndexView ix, int l,
                                                                  QueryState st, bool tma, int s0,
                                                                  int wave)
{
    __shared__ int sh_hist[kHistBins];
    const int nslot = min(st.rd_ctl[0] - s0, wave);
    const int nT = ix.nT, g = threadIdx.x;
    for (int64_t it = blockIdx.x; it < (int64_t)max(nslot, 0) * nT; it += gridDim.x) {
        const int slot = s0 + (int)(it / nT), t = (int)(it % nT);
        const RdPlan pl = st.rd_plan[slot];
        const int q = pl.q, L = st.levels[q] - 1;
        const int64_t qt = (int64_t)q * nT + t;
        if (st.clist_n[(int64_t)(L & 1) * st.cln_par + qt] == 0) continue;  // block-uniform
        for (int c = threadIdx.x; c < kHistBins; c += RD_THREADS) sh_hist[c] = 0;
        __syncthreads();
        const uint4 cw = rd_word(st, L, qt, g, tma);
        int my_np = 0;
        if (cw.x | cw.y | cw.z | cw.w) {
            const int64_t *bq = st.rd_bq + (int64_t)slot * 2 * QW_MAX_M;
            Planes P;
            uint4 pw = make_uint4(0, 0, 0, 0);
            if (pl.prev_recount) {
                rd_planes(ix, bq + QW_MAX_M, t, g, P);
                pw = candidates_of(P, l);
            } else if (L > 0) {
                pw = rd_word(st, L - 1, qt, g, tma);
            }
            rd_planes(ix, bq, t, g, P);
            uint4 *store = st.rd_store +
                           ((int64_t)(slot - s0) * nT * kBmUint4 + (int64_t)t * kBmUint4 + g) *
                               kRdStoreWords;
#pragma unroll
            for (int k = 0; k < 7; ++k) store[k] = make_uint4(P.s[k][0], P.s[k][1], P.s[k][2], P.s[k][3]);
            store[7] = pw;
#pragma unroll
            for (int w = 0; w < 4; ++w) {
                my_np += __popc(word_of(cw, w) & word_of(pw, w));
                uint32_t x = word_of(cw, w) & ~word_of(pw, w);
                while (x) {
                    const int b = __ffs(x) - 1;
                    x &= x - 1;
                    atomicAdd(&sh_hist[count_of(P, w, b)], 1);
                }
            }
        }
        my_np = __reduce_add_sync(0xffffffffu, my_np);
        if ((threadIdx.x & 31) == 0 && my_np) atomicAdd(&st.rd_plan[slot].np, my_np);
        __syncthreads();
        int32_t *h = st.rd_hist + (int64_t)slot * kHistBins;
        for (int c = threadIdx.x; c < kHistBins; c += RD_THREADS)
            if (sh_hist[c]) atomicAdd(h + c, sh_hist[c]);
        __syncthreads();
    }
}

__global__ void rd_plan_kernel(int l, int m, int cap, int cgrow, QueryState st, int s0, int wave,
                               int stage)
{
    const int nslot = min(st.rd_ctl[0] - s0, wave);
    const int slot = s0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (slot >= s0 + nslot) return;
    RdPlan p = st.rd_plan[slot];
    const int q = p.q;
    const int L = st.levels[q] - 1;
    if (stage == 0) {
        if (!p.prev_recount) p.np = st.nprev[q];
        if (st.recount[q] && (st.finalR[q] / cgrow > st.top[q] || p.np >= cap)) {
            // a learned first level after the level where the plain path stops:
            // answered again from level 0
            atomicOr(st.bm_ovf + q, 2);
            p.mode = 0;
        } else {
            // histogram of counts -> the count c* at which the bound is reached
            const int32_t *h = st.rd_hist + (int64_t)slot * kHistBins;
            const int need = cap - p.np;
            int acc = 0, cstar = -1, take = 0;
            for (int c = m; c >= l; --c) {
                if (acc + h[c] >= need) {
                    cstar = c;
                    take = need - acc;
                    break;
                }
                acc += h[c];
            }
            if (cstar < 0) {
                p.mode = 0;  // cannot happen for a list that overflowed
            } else {
                p.cstar = cstar;
                p.take = take;
                // a short tie class is listed whole, a long one cut by rd_scan
                p.mode = h[cstar] <= kRdTieList ? 1 : 2;
            }
        }
    } else if (p.mode != 0) {
        // the rebuilt list (more than kQCap entries: the level path answers)
        st.qbuf_n[(int64_t)(L & 1) * st.qbn_par + q] = p.pos;
        st.bm_ovf[q] |= 4;
        if (st.recount[q]) {
            st.nprev[q] = p.np;
            st.recount[q] = 0;
        }
    }
    st.rd_plan[slot] = p;
}

// The stored planes of group g of tile t of a slot.
__device__ __forceinline__ void rd_stored(const QueryState &st, int slot, int nT, int t, int g,
                                          Planes &P, uint4 &pw)
{
    const uint4 *store = st.rd_store +
                         ((int64_t)slot * nT * kBmUint4 + (int64_t)t * kBmUint4 + g) * kRdStoreWords;
#pragma unroll
    for (int k = 0; k < 7; ++k) {
        const uint4 v = store[k];
        P.s[k][0] = v.x;
        P.s[k][1] = v.y;
        P.s[k][2] = v.z;
        P.s[k][3] = v.w;
    }
    pw = store[7];
}

// The kept entries of every rebuilt slot, one thread per group: previous-level
// candidates, counts above c*, and (a short tie class) the tie class.
__global__ void __launch_bounds__(RD_THREADS, 3) rd_emit_kernel(IndexView ix, QueryState st,
                                                                 bool tma, int wave)
{
    const int nslot = min(st.rd_ctl[0], wave);
    const int m = ix.m, nT = ix.nT, g = threadIdx.x;
    for (int64_t it = blockIdx.x; it < (int64_t)nslot * nT; it += gridDim.x) {
        const int slot = (int)(it / nT), t = (int)(it % nT);
        const RdPlan pl = st.rd_plan[slot];
        if (pl.mode == 0) continue;
        const int q = pl.q, L = st.levels[q] - 1;
        const int64_t qt = (int64_t)q * nT + t;
        const uint4 cw = rd_word(st, L, qt, g, tma);
        if (!(cw.x | cw.y | cw.z | cw.w)) continue;
        Planes P;
        uint4 pw;
        rd_stored(st, slot, nT, t, g, P, pw);
        uint4 keep;
        int my_n = 0;
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            const uint32_t c_w = word_of(cw, w), p_w = word_of(pw, w);
            const uint32_t oth = c_w & ~p_w;
            uint32_t kw = (c_w & p_w) | (pl.cstar < m ? count_ge_planes(P, w, pl.cstar + 1) & oth : 0u);
            if (pl.mode == 1) kw |= count_eq_planes(P, w, pl.cstar) & oth;
            if (w == 0) keep.x = kw;
            else if (w == 1) keep.y = kw;
            else if (w == 2) keep.z = kw;
            else keep.w = kw;
            my_n += __popc(kw);
        }
        if (my_n) {
            uint64_t *E = st.qbuf + (int64_t)(L & 1) * st.qb_par + (int64_t)q * kQCap;
            int pos = atomicAdd(&st.rd_plan[slot].pos, my_n);
#pragma unroll
            for (int w = 0; w < 4; ++w) {
                uint32_t x = word_of(keep, w);
                const uint32_t p_w = word_of(pw, w);
                while (x) {
                    const int b = __ffs(x) - 1;
                    x &= x - 1;
                    const int64_t iid = (int64_t)t * kTile + (int64_t)g * 128 + w * 32 + b;
                    if (pos < kQCap)
                        E[pos] = ((uint64_t)iid << 32) | ((uint64_t)((p_w >> b) & 1u) << 8) |
                                 (uint64_t)count_of(P, w, b);
                    ++pos;
                }
            }
        }
    }
}

// One block per slot with a long tie class: data ids 0, 1, 2, ... are tested
// kScanPer * 256 at a time (thread t takes ids o0 + u * 256 + t, so the loads
// of each u are coalesced and the kScanPer chains of dependent reads are in
// flight together; tie member: a candidate of the last level, not of the
// previous one, with count c*) until `take` members are found; those are the
// take smallest original ids of the tie class (reading R5), listed with count
// c*.  The walk reads about take * n / (tie class size) ids.
constexpr int kScanPer = 4;

__global__ void __launch_bounds__(RD_THREADS) rd_scan_kernel(IndexView ix, QueryState st,
                                                              bool tma, int wave)
{
    constexpr int NW = RD_THREADS / 32;
    __shared__ int s_wc[kScanPer][NW];
    __shared__ int s_base;
    const int nslot = min(st.rd_ctl[0], wave);
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    for (int slot = blockIdx.x; slot < nslot; slot += gridDim.x) {
        const RdPlan pl = st.rd_plan[slot];
        if (pl.mode != 2 || pl.take <= 0) continue;
        const int q = pl.q, L = st.levels[q] - 1;
        uint64_t *E = st.qbuf + (int64_t)(L & 1) * st.qb_par + (int64_t)q * kQCap;
        if (threadIdx.x == 0) s_base = atomicAdd(&st.rd_plan[slot].pos, pl.take);
        __syncthreads();
        const int base = s_base;
        int found = 0;
        for (int64_t o0 = 0; o0 < ix.n && found < pl.take; o0 += RD_THREADS * kScanPer) {
            int64_t iid[kScanPer];
#pragma unroll
            for (int u = 0; u < kScanPer; ++u) {
                const int64_t o = o0 + u * RD_THREADS + threadIdx.x;
                iid[u] = o < ix.n ? (int64_t)ix.inv[o] : -1;
            }
            uint4 cw[kScanPer];
#pragma unroll
            for (int u = 0; u < kScanPer; ++u) {
                const int64_t id = iid[u] >= 0 ? iid[u] : 0;
                const int t = (int)(id / kTile), g = (int)((id % kTile) >> 7);
                cw[u] = iid[u] >= 0 ? rd_word(st, L, (int64_t)q * ix.nT + t, g, tma)
                                    : make_uint4(0, 0, 0, 0);
            }
            bool tie[kScanPer];
#pragma unroll
            for (int u = 0; u < kScanPer; ++u) {
                tie[u] = false;
                const int64_t id = iid[u] >= 0 ? iid[u] : 0;
                const int t = (int)(id / kTile), g = (int)((id % kTile) >> 7), b = (int)(id & 127);
                if (iid[u] >= 0 && ((word_of(cw[u], b >> 5) >> (b & 31)) & 1u)) {
                    // the id's bit of each stored plane and of the previous
                    // level's word (word b / 32 of each 16-byte record)
                    const uint32_t *rec = reinterpret_cast<const uint32_t *>(
                        st.rd_store + ((int64_t)slot * ix.nT * kBmUint4 + (int64_t)t * kBmUint4 + g) *
                                          kRdStoreWords) + (b >> 5);
                    int cnt = 0;
#pragma unroll
                    for (int k = 0; k < 7; ++k) cnt |= (int)((rec[4 * k] >> (b & 31)) & 1u) << k;
                    tie[u] = !((rec[4 * 7] >> (b & 31)) & 1u) && cnt == pl.cstar;
                }
            }
            uint32_t bal[kScanPer];
#pragma unroll
            for (int u = 0; u < kScanPer; ++u) {
                bal[u] = __ballot_sync(0xffffffffu, tie[u]);
                if (lane == 0) s_wc[u][wi] = __popc(bal[u]);
            }
            __syncthreads();
            // ties before (u, this warp) in id order: all of the earlier u,
            // then the earlier warps of this u
            int total = 0;
#pragma unroll
            for (int u = 0; u < kScanPer; ++u) {
                int before = 0, tot_u = 0;
#pragma unroll
                for (int w = 0; w < NW; ++w) {
                    const int c = s_wc[u][w];
                    if (w < wi) before += c;
                    tot_u += c;
                }
                if (tie[u]) {
                    const int rank = found + total + before + __popc(bal[u] & lt);
                    if (rank < pl.take && base + rank < kQCap)
                        E[base + rank] = ((uint64_t)iid[u] << 32) | (uint64_t)pl.cstar;
                }
                total += tot_u;
            }
            found += total;
            __syncthreads();  // s_wc is rewritten next
        }
    }
}

// Learned starts on the bitmap path: a query that stopped at its first level
// L > 0 never counted level L - 1, whose candidates come first under the k + v
// bound (reading R5).  Those are exactly the final candidates whose level-(L-1)
// count reaches l (buckets nest, so C(L-1) is a subset of C(L)).  The count of
// a candidate is taken from its row of anchored bucket ids: on projection i it
// collides at radius R' = c^(L-1) when floor(h_i / R') == floor(g_i / R'), i.e.
// when h_i lies in [beta_i R', (beta_i + 1) R' - 1].  One block per query, one
// thread per candidate: the row is read in 16-byte pieces and compared with
// the bounds (packed like the row, in shared memory) 4, 2 or 1 ids per 32-bit
// word by SIMD compares.
// The plain path would have stopped earlier if |C(L-1)| >= k + v or if radius
// c^(L-1) already exceeded every useful radius of the query: such queries are
// marked for the level path.  A query's candidates are split over
// kRcSplits blocks (a long list would otherwise leave one block working
// alone); their counts add up in nprev, and a second kernel compares the sum
// with k + v.
constexpr int RC_THREADS = 128;
constexpr int kRcSplits = 8;
constexpr int kRcChunks = (QW_MAX_M * 4 + 15) / 16;  // 16-byte pieces of the widest row

// Ids of a 32-bit word within [lo, hi] (element-wise, inclusive).
template <typename T> __device__ __forceinline__ int in_range(uint32_t h, uint32_t lo, uint32_t hi);
template <> __device__ __forceinline__ int in_range<uint8_t>(uint32_t h, uint32_t lo, uint32_t hi)
{
    return __popc(__vcmpgeu4(h, lo) & __vcmpleu4(h, hi)) >> 3;
}
template <> __device__ __forceinline__ int in_range<uint16_t>(uint32_t h, uint32_t lo, uint32_t hi)
{
    return __popc(__vcmpgeu2(h, lo) & __vcmpleu2(h, hi)) >> 4;
}
template <> __device__ __forceinline__ int in_range<uint32_t>(uint32_t h, uint32_t lo, uint32_t hi)
{
    return (h >= lo && h <= hi) ? 1 : 0;
}

template <typename T>
__global__ void __launch_bounds__(RC_THREADS) bm_recount_kernel(IndexView ix, int l, int cap,
                                                                int cgrow, QueryState st)
{
    __shared__ uint4 blo[kRcChunks], bhi[kRcChunks];
    __shared__ int s_nprev;
    const int q = blockIdx.x;
    const int split = blockIdx.y, nsplit = gridDim.y;
    if (!st.recount[q]) return;
    const int m = ix.m;
    const int L = st.levels[q] - 1;
    const int64_t R = st.finalR[q] / cgrow;  // radius of level L - 1
    const int n = st.qbuf_n[(int64_t)(L & 1) * st.qbn_par + q];
    uint64_t *E = st.qbuf + (int64_t)(L & 1) * st.qb_par + (int64_t)q * kQCap;
    if (n > kQCap) return;  // the selection marks the query for the level path
    if (R > st.top[q]) {
        // the plain path stops at level L - 1 by radius: not this answer
        if (threadIdx.x == 0 && split == 0) atomicOr(st.bm_ovf + q, 2);
        return;
    }
    const int chunks = ix.hloc_stride / 16;
    // per projection, the ids of the level-(L-1) bucket in the width of the row
    // (an empty range as lo = max, hi = 0; padding never matches)
    const int64_t tmax = sizeof(T) == 4 ? (int64_t)INT32_MAX : ((int64_t)1 << (8 * sizeof(T))) - 1;
    T *lo_t = reinterpret_cast<T *>(blo), *hi_t = reinterpret_cast<T *>(bhi);
    for (int i = threadIdx.x; i < chunks * (16 / (int)sizeof(T)); i += RC_THREADS) {
        int64_t lo = tmax, hi = 0;
        if (i < m) {
            const int64_t beta = floordiv64(st.g[(int64_t)q * m + i], R);
            const int64_t a = beta * R, b = beta * R + R - 1;
            if (b >= 0 && a <= tmax) {
                lo = a > 0 ? a : 0;
                hi = b < tmax ? b : tmax;
            }
        }
        lo_t[i] = (T)lo;
        hi_t[i] = (T)hi;
    }
    if (threadIdx.x == 0) s_nprev = 0;
    __syncthreads();
    const char *H = static_cast<const char *>(ix.hloc);
    int mine = 0;
    for (int j = split * RC_THREADS + threadIdx.x; j < n; j += nsplit * RC_THREADS) {
        const uint64_t e = E[j];
        const uint4 *row = reinterpret_cast<const uint4 *>(H + (int64_t)(e >> 32) * ix.hloc_stride);
        int c = 0;
#pragma unroll 4
        for (int v = 0; v < chunks; ++v) {
            const uint4 h = __ldg(row + v);
            const uint4 a = blo[v], b = bhi[v];
            c += in_range<T>(h.x, a.x, b.x) + in_range<T>(h.y, a.y, b.y) +
                 in_range<T>(h.z, a.z, b.z) + in_range<T>(h.w, a.w, b.w);
        }
        if (c >= l) {
            E[j] = e | (1ull << 8);
            ++mine;
        }
    }
    mine = __reduce_add_sync(0xffffffffu, mine);
    if ((threadIdx.x & 31) == 0 && mine) atomicAdd(&s_nprev, mine);
    __syncthreads();
    // nprev of a query stopped at its first level starts at 0 (the decision
    // kernel set it from the empty count before that level)
    if (threadIdx.x == 0 && s_nprev) atomicAdd(st.nprev + q, s_nprev);
}

// After the split recount: a query whose |C(L-1)| reaches k + v would have
// stopped at level L - 1 on the plain path; it is marked for the level path.
__global__ void recount_decide_kernel(QueryState st, int nb, int cap, int cgrow)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nb || !st.recount[q]) return;
    const int L = st.levels[q] - 1;
    if (st.qbuf_n[(int64_t)(L & 1) * st.qbn_par + q] > kQCap) return;
    if (st.finalR[q] / cgrow > st.top[q]) return;
    if (st.nprev[q] >= cap) atomicOr(st.bm_ovf + q, 2);
}

template <typename T>
__global__ void hloc_kernel(const int32_t *__restrict__ Ht, const int32_t *__restrict__ perm,
                            const int32_t *__restrict__ o, int64_t n, int m, int stride,
                            char *__restrict__ out)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * m;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = e / m;
        const int i = (int)(e % m);
        reinterpret_cast<T *>(out + j * stride)[i] = (T)(Ht[(int64_t)i * n + perm[j]] - o[i]);
    }
}

// Workload indices of the batch's queries to answer again: list[0] those whose
// candidates overflowed the bitmap path's lists (flag 1: the level path), list
// [1] those whose learned first level was too late (flag 2 alone: the bitmap
// path from level 0); count[0], count[1] their numbers.
__global__ void bm_overflow_list_kernel(const QueryState st, int nb, const int32_t *order_perm,
                                        int64_t b0, int32_t *list0, int32_t *list1,
                                        int32_t *count)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nb) return;
    const int f = st.bm_ovf[q] & 3;
    if (!f) return;
    // a learned first level that was too late is answered again from level 0
    // on the bitmap path, whatever else happened to the query
    const int which = (f & 2) ? 1 : 0;
    const int pos = atomicAdd(count + which, 1);
    (which == 0 ? list0 : list1)[pos] = order_perm ? order_perm[b0 + q] : (int32_t)(b0 + q);
}

// Data objects per bid of every projection, then the exclusive prefix over
// bids: bid_prefix[off[i] + b] = objects with bid < b.
__global__ void bid_count_kernel(IndexView ix, int64_t *prefix, const int64_t *off)
{
    const int t = blockIdx.x, i = blockIdx.y;
    const int64_t dslot = (int64_t)i * ix.nT + t;
    const int32_t *ub = ix.dir_bid + ix.dir_start[dslot];
    const int32_t *uo = ix.dir_off + ix.dir_start[dslot];
    const int cnt = ix.dir_cnt[dslot];
    const int len = (int)min((int64_t)kTile, ix.n - (int64_t)t * kTile);
    for (int u = threadIdx.x; u < cnt; u += blockDim.x) {
        const int e1 = (u + 1 < cnt) ? uo[u + 1] : len;
        atomicAdd(reinterpret_cast<unsigned long long *>(prefix + off[i] + ub[u] + 1),
                  (unsigned long long)(e1 - uo[u]));
    }
}

__global__ void bid_scan_kernel(IndexView ix, int64_t *prefix, const int64_t *off)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ix.m) return;
    int64_t *P = prefix + off[i];
    int64_t acc = 0;
    for (int64_t b = 1; b <= (int64_t)ix.span[i] + 1; ++b) {
        acc += P[b];
        P[b] = acc;
    }
}

}  // namespace

qw_status launch_bitmap_build(const IndexView &ix, int c, int maxJ, const int32_t *Ht, uint4 *bm,
                              uint32_t *bm_sum, int64_t total_bitmaps, cudaStream_t s)
{
    const dim3 grid((unsigned)ix.nT, (unsigned)ix.m);
    bm_fill_level0_kernel<<<grid, BM_THREADS, 0, s>>>(ix, Ht, bm);
    QW_CUDA_TRY(cudaGetLastError());
    int64_t R = 1;
    for (int L = 1; L <= maxJ; ++L) {
        R *= c;
        bm_or_level_kernel<<<grid, BM_THREADS, 0, s>>>(ix, bm, L, R, c);
        QW_CUDA_TRY(cudaGetLastError());
    }
    const int64_t blocks = std::min<int64_t>(total_bitmaps, 152 * 64);
    bm_summary_kernel<<<(unsigned)std::max<int64_t>(blocks, 1), BM_THREADS, 0, s>>>(
        bm, total_bitmaps, bm_sum);
    QW_CUDA_TRY(cudaGetLastError());
    return QW_OK;
}

namespace {

// Run f(chunk, begin, end) over [0, n) in chunks of `chunk` on the host's
// cores.  Chunk boundaries do not depend on the thread count, so results
// combined per chunk in chunk order are deterministic.
template <class F>
void parallel_chunks(int64_t n, int64_t chunk, F &&f)
{
    const int64_t nc = (n + chunk - 1) / chunk;
    int64_t nt = (int64_t)std::max(1u, std::thread::hardware_concurrency());
    nt = std::min(nt, nc);
    if (nt <= 1) {
        for (int64_t c = 0; c < nc; ++c) f(c, c * chunk, std::min(n, (c + 1) * chunk));
        return;
    }
    std::atomic<int64_t> next(0);
    std::vector<std::thread> th;
    for (int64_t t = 0; t < nt; ++t)
        th.emplace_back([&] {
            for (;;) {
                const int64_t c = next.fetch_add(1);
                if (c >= nc) break;
                f(c, c * chunk, std::min(n, (c + 1) * chunk));
            }
        });
    for (auto &x : th) x.join();
}

struct TreeNode {
    int64_t lo, hi;
    int depth;
};

// Split perm[lo, hi) in two: two centroids seeded by the extremes along LSH
// projection depth mod m, refined by three rounds of two-means, then the
// points ordered by their side of the bisecting hyperplane and cut where the
// two-means boundary falls, rounded to a multiple of kGroupIds (so every
// 128-id group of the internal order stays inside one leaf).
void split_node(const float *X, int d, const float *A, int m, std::vector<int32_t> &perm,
                const TreeNode &nd, bool par, TreeNode *kids)
{
    const int64_t lo = nd.lo, len = nd.hi - nd.lo;
    const int64_t chunk = 4096;
    const int64_t nc = (len + chunk - 1) / chunk;
    auto each = [&](auto &&f) {
        if (par) {
            parallel_chunks(len, chunk, f);
        } else {
            for (int64_t c = 0; c < nc; ++c) f(c, c * chunk, std::min(len, (c + 1) * chunk));
        }
    };
    auto row = [&](int64_t j) { return X + (size_t)perm[(size_t)(lo + j)] * (size_t)d; };
    // seeds: smallest and largest projection on one LSH direction
    const float *a = A + (size_t)(nd.depth % m) * (size_t)d;
    std::vector<double> cmin(nc, HUGE_VAL), cmax(nc, -HUGE_VAL);
    std::vector<int64_t> amin(nc, 0), amax(nc, 0);
    each([&](int64_t c, int64_t b, int64_t e) {
        for (int64_t j = b; j < e; ++j) {
            const float *x = row(j);
            double t = 0.0;
            for (int k = 0; k < d; ++k) t += (double)a[k] * (double)x[k];
            if (t < cmin[c]) { cmin[c] = t; amin[c] = j; }
            if (t > cmax[c]) { cmax[c] = t; amax[c] = j; }
        }
    });
    int64_t jmin = amin[0], jmax = amax[0];
    double vmin = cmin[0], vmax = cmax[0];
    for (int64_t c = 1; c < nc; ++c) {
        if (cmin[c] < vmin) { vmin = cmin[c]; jmin = amin[c]; }
        if (cmax[c] > vmax) { vmax = cmax[c]; jmax = amax[c]; }
    }
    std::vector<double> c1(d), c2(d), v(d);
    for (int k = 0; k < d; ++k) {
        c1[k] = row(jmin)[k];
        c2[k] = row(jmax)[k];
    }
    double thr = 0.0;
    std::vector<double> part((size_t)nc * (2 * (size_t)d + 2));
    for (int it = 0; it < 4; ++it) {
        double n1 = 0.0, n2 = 0.0;
        double q1 = 0.0, q2 = 0.0;
        for (int k = 0; k < d; ++k) {
            v[k] = c2[k] - c1[k];
            q1 += c1[k] * c1[k];
            q2 += c2[k] * c2[k];
        }
        thr = 0.5 * (q2 - q1);
        if (it == 3) break;  // the last round only fixes the hyperplane
        std::fill(part.begin(), part.end(), 0.0);
        each([&](int64_t c, int64_t b, int64_t e) {
            double *ps = part.data() + (size_t)c * (2 * (size_t)d + 2);
            for (int64_t j = b; j < e; ++j) {
                const float *x = row(j);
                double t = 0.0;
                for (int k = 0; k < d; ++k) t += v[k] * (double)x[k];
                double *acc = t < thr ? ps : ps + d;
                for (int k = 0; k < d; ++k) acc[k] += (double)x[k];
                ps[2 * d + (t < thr ? 0 : 1)] += 1.0;
            }
        });
        std::vector<double> s1(d, 0.0), s2(d, 0.0);
        for (int64_t c = 0; c < nc; ++c) {
            const double *ps = part.data() + (size_t)c * (2 * (size_t)d + 2);
            for (int k = 0; k < d; ++k) {
                s1[k] += ps[k];
                s2[k] += ps[d + k];
            }
            n1 += ps[2 * d];
            n2 += ps[2 * d + 1];
        }
        if (n1 == 0.0 || n2 == 0.0) break;
        for (int k = 0; k < d; ++k) {
            c1[k] = s1[k] / n1;
            c2[k] = s2[k] / n2;
        }
    }
    // order by side of the hyperplane, cut at the boundary (aligned)
    std::vector<std::pair<double, int32_t>> key((size_t)len);
    std::vector<int64_t> below(nc, 0);
    each([&](int64_t c, int64_t b, int64_t e) {
        for (int64_t j = b; j < e; ++j) {
            const float *x = row(j);
            double t = -thr;
            for (int k = 0; k < d; ++k) t += v[k] * (double)x[k];
            key[(size_t)j] = {t, perm[(size_t)(lo + j)]};
            below[c] += t < 0.0 ? 1 : 0;
        }
    });
    int64_t k1 = 0;
    for (int64_t c = 0; c < nc; ++c) k1 += below[c];
    int64_t cut = (k1 + kGroupIds / 2) / kGroupIds * kGroupIds;
    cut = std::max<int64_t>(kGroupIds, std::min<int64_t>(cut, (len - 1) / kGroupIds * kGroupIds));
    std::nth_element(key.begin(), key.begin() + cut, key.end());
    for (int64_t j = 0; j < len; ++j) perm[(size_t)(lo + j)] = key[(size_t)j].second;
    kids[0] = {lo, lo + cut, nd.depth + 1};
    kids[1] = {lo + cut, nd.hi, nd.depth + 1};
}

}  // namespace

qw_status locality_order(const float *X, int64_t n, int d, const float *A, int m,
                         std::vector<int32_t> &perm)
{
    try {
        perm.resize((size_t)n);
        for (int64_t j = 0; j < n; ++j) perm[(size_t)j] = (int32_t)j;
        std::vector<TreeNode> cur;
        if (n > kGroupIds) cur.push_back({0, n, 0});
        const int64_t big = (int64_t)1 << 16;
        while (!cur.empty()) {
            std::vector<TreeNode> kids(2 * cur.size());
            // large nodes one at a time, each split on all cores ...
            std::vector<size_t> small;
            for (size_t u = 0; u < cur.size(); ++u) {
                if (cur[u].hi - cur[u].lo >= big) split_node(X, d, A, m, perm, cur[u], true, &kids[2 * u]);
                else small.push_back(u);
            }
            // ... small ones side by side (they touch disjoint ranges of perm)
            parallel_chunks((int64_t)small.size(), 1, [&](int64_t c, int64_t, int64_t) {
                const size_t u = small[(size_t)c];
                split_node(X, d, A, m, perm, cur[u], false, &kids[2 * u]);
            });
            std::vector<TreeNode> next;
            for (const TreeNode &k : kids)
                if (k.hi - k.lo > kGroupIds) next.push_back(k);
            cur.swap(next);
        }
    } catch (const std::bad_alloc &) {
        set_error("qw_build_index: out of host memory for the locality order");
        return QW_ERR_OOM;
    }
    return QW_OK;
}

qw_status launch_bid_prefix(const IndexView &ix, int64_t *prefix, const int64_t *off,
                            cudaStream_t s)
{
    bid_count_kernel<<<dim3((unsigned)ix.nT, (unsigned)ix.m), 128, 0, s>>>(ix, prefix, off);
    QW_CUDA_TRY(cudaGetLastError());
    bid_scan_kernel<<<(ix.m + 63) / 64, 64, 0, s>>>(ix, prefix, off);
    QW_CUDA_TRY(cudaGetLastError());
    return QW_OK;
}

ScanStats scan_stats_of(const IndexView &ix, int c)
{
    ScanStats ss;
    ss.prefix = ix.bid_prefix;
    ss.off = ix.prefix_off;
    ss.span = ix.span;
    ss.m = ix.m;
    ss.cgrow = c;
    return ss;
}

template <int TPW>
static void launch_filter_or_fused(const IndexView &ix, int nb, int level, int l, QueryState &st,
                                   const LoopCtl *ctl, bool fused, cudaStream_t s)
{
    const int64_t tasks = (int64_t)nb * ((ix.nT + TPW - 1) / TPW);
    const int blocks = (int)std::max<int64_t>(
        1, std::min<int64_t>((tasks + FL_WARPS - 1) / FL_WARPS, 152 * 16));
    if (fused) {
        if (ix.m <= 32)
            bm_fused_kernel<1, TPW><<<blocks, FL_WARPS * 32, 0, s>>>(ix, level, l, nb, st, ctl);
        else if (ix.m <= 64)
            bm_fused_kernel<2, TPW><<<blocks, FL_WARPS * 32, 0, s>>>(ix, level, l, nb, st, ctl);
        else
            bm_fused_kernel<4, TPW><<<blocks, FL_WARPS * 32, 0, s>>>(ix, level, l, nb, st, ctl);
    } else {
        if (ix.m <= 32)
            bm_filter_kernel<1, TPW><<<blocks, FL_WARPS * 32, 0, s>>>(ix, level, l, nb, st, ctl);
        else if (ix.m <= 64)
            bm_filter_kernel<2, TPW><<<blocks, FL_WARPS * 32, 0, s>>>(ix, level, l, nb, st, ctl);
        else
            bm_filter_kernel<4, TPW><<<blocks, FL_WARPS * 32, 0, s>>>(ix, level, l, nb, st, ctl);
    }
}

static void launch_filter_or_fused(const IndexView &ix, int nb, int level, int l, QueryState &st,
                                   const LoopCtl *ctl, bool fused, int tpw, cudaStream_t s)
{
    if (tpw == 4) launch_filter_or_fused<4>(ix, nb, level, l, st, ctl, fused, s);
    else if (tpw == 16) launch_filter_or_fused<16>(ix, nb, level, l, st, ctl, fused, s);
    else launch_filter_or_fused<8>(ix, nb, level, l, st, ctl, fused, s);
}

qw_status launch_bm_level(const IndexView &ix, int nb, int level, int64_t R, int64_t Rp, int l,
                          int cgrow, QueryState &st, int *err, int loads, cudaStream_t s,
                          const LoopCtl *ctl, int part, int tpw)
{
    (void)Rp;
    (void)cgrow;
    if (loads == QW_LOADS_FUSED) {
        if (part != 2) {
            const int64_t qi = (int64_t)nb * ix.m;
            bm_bucket_kernel<<<(unsigned)std::max<int64_t>(
                                   1, std::min<int64_t>((qi + 255) / 256, 152 * 8)),
                               256, 0, s>>>(ix, level, R, nb, st, ctl);
            QW_CUDA_TRY(cudaGetLastError());
        }
        if (part == 1) return QW_OK;
        launch_filter_or_fused(ix, nb, level, l, st, ctl, true, tpw, s);
        QW_CUDA_TRY(cudaGetLastError());
        return QW_OK;
    }
    if (loads == QW_LOADS_DIRECT) {
        // two passes: filter on the summaries, then count the live groups
        if (part != 2) {
            const int64_t qi = (int64_t)nb * ix.m;
            bm_bucket_kernel<<<(unsigned)std::max<int64_t>(
                                   1, std::min<int64_t>((qi + 255) / 256, 152 * 8)),
                               256, 0, s>>>(ix, level, R, nb, st, ctl);
            QW_CUDA_TRY(cudaGetLastError());
        }
        if (part == 1) return QW_OK;
        launch_filter_or_fused(ix, nb, level, l, st, ctl, false, tpw, s);
        QW_CUDA_TRY(cudaGetLastError());
        bm_count_kernel<<<152 * 8, 256, 0, s>>>(ix, level, l, st, ctl);
        QW_CUDA_TRY(cudaGetLastError());
        if (st.bm_prof) {
            bm_prof_kernel<<<1, 1, 0, s>>>(st);
            QW_CUDA_TRY(cudaGetLastError());
        }
        return QW_OK;
    }
    int dev = 0, n_sm = 0;
    QW_CUDA_TRY(cudaGetDevice(&dev));
    QW_CUDA_TRY(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
    const size_t smem = tma_smem_bytes();
    QW_CUDA_TRY(cudaFuncSetAttribute(bm_level_tma_kernel,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int64_t items = (int64_t)nb * ix.nT;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(n_sm, items));
    bm_level_tma_kernel<<<grid, TMA_THREADS, smem, s>>>(ix, level, R, l, nb, st, ctl, err);
    QW_CUDA_TRY(cudaGetLastError());
    return QW_OK;
}

qw_status launch_locality_copy(const float *X, const int32_t *perm, int64_t n, int d, float *Xloc,
                               int32_t *inv, cudaStream_t s)
{
    if (n == 0) return QW_OK;
    locality_copy_kernel<<<(unsigned)std::min<int64_t>(n, 152 * 64), 128, 0, s>>>(X, perm, n, d,
                                                                                 Xloc, inv);
    QW_CUDA_TRY(cudaGetLastError());
    return QW_OK;
}

qw_status launch_bm_recount(const IndexView &ix, int nb, int l, int cap, int cgrow, QueryState &st,
                            cudaStream_t s)
{
    if (nb == 0) return QW_OK;
    const dim3 grid((unsigned)nb, kRcSplits);
    if (ix.hloc_bytes == 1)
        bm_recount_kernel<uint8_t><<<grid, RC_THREADS, 0, s>>>(ix, l, cap, cgrow, st);
    else if (ix.hloc_bytes == 2)
        bm_recount_kernel<uint16_t><<<grid, RC_THREADS, 0, s>>>(ix, l, cap, cgrow, st);
    else
        bm_recount_kernel<uint32_t><<<grid, RC_THREADS, 0, s>>>(ix, l, cap, cgrow, st);
    QW_CUDA_TRY(cudaGetLastError());
    recount_decide_kernel<<<(nb + 255) / 256, 256, 0, s>>>(st, nb, cap, cgrow);
    QW_CUDA_TRY(cudaGetLastError());
    return QW_OK;
}

qw_status launch_hloc_build(const IndexView &ix, const int32_t *Ht, void *hloc, cudaStream_t s)
{
    if (ix.n == 0) return QW_OK;
    const unsigned blocks = (unsigned)std::min<int64_t>((ix.n * ix.m + 255) / 256, 152 * 32);
    char *out = static_cast<char *>(hloc);
    if (ix.hloc_bytes == 1)
        hloc_kernel<uint8_t><<<blocks, 256, 0, s>>>(Ht, ix.perm, ix.o, ix.n, ix.m, ix.hloc_stride, out);
    else if (ix.hloc_bytes == 2)
        hloc_kernel<uint16_t><<<blocks, 256, 0, s>>>(Ht, ix.perm, ix.o, ix.n, ix.m, ix.hloc_stride, out);
    else
        hloc_kernel<uint32_t><<<blocks, 256, 0, s>>>(Ht, ix.perm, ix.o, ix.n, ix.m, ix.hloc_stride, out);
    QW_CUDA_TRY(cudaGetLastError());
    return QW_OK;
}

qw_status launch_bm_collect(const IndexView &ix, int nb, int l, int cap, QueryState &st,
                            int64_t *stats_out, bool sorted, cudaStream_t s)
{
    int P2 = 2;
    while (P2 < cap) P2 <<= 1;
    const size_t smem = sorted ? (size_t)P2 * sizeof(uint64_t) : 0;
    QW_CUDA_TRY(cudaFuncSetAttribute(bm_select_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
    bm_select_kernel<<<nb, SEL_THREADS, smem, s>>>(ix, l, cap, st, stats_out, sorted);
    QW_CUDA_TRY(cudaGetLastError());
    return QW_OK;
}

int bm_reduce_wave(int nT)
{
    return (int)std::max<int64_t>(1, kRdStoreBytes / ((int64_t)nT * kBmUint4 * kRdStoreWords * 16));
}

qw_status launch_bm_reduce(const IndexView &ix, int nb, int l, int cap, int cgrow,
                           QueryState &st, bool tma, int wave_slots, cudaStream_t s)
{
    if (nb == 0) return QW_OK;
    QW_CUDA_TRY(cudaMemsetAsync(st.rd_ctl, 0, sizeof(int32_t), s));
    const unsigned qb = (unsigned)((nb + 127) / 128);
    rd_compact_kernel<<<qb, 128, 0, s>>>(ix, cgrow, st, nb);
    QW_CUDA_TRY(cudaGetLastError());
    // one store's worth of slots (wave_slots); queries past it keep the
    // level-path answer
    const unsigned grid = 152 * 6;
    const unsigned pb = (unsigned)((wave_slots + 127) / 128);
    rd_count_kernel<<<grid, RD_THREADS, 0, s>>>(ix, l, st, tma, 0, wave_slots);
    rd_plan_kernel<<<pb, 128, 0, s>>>(l, ix.m, cap, cgrow, st, 0, wave_slots, 0);
    rd_scan_kernel<<<152 * 4, RD_THREADS, 0, s>>>(ix, st, tma, wave_slots);
    rd_emit_kernel<<<grid, RD_THREADS, 0, s>>>(ix, st, tma, wave_slots);
    rd_plan_kernel<<<pb, 128, 0, s>>>(l, ix.m, cap, cgrow, st, 0, wave_slots, 2);
    QW_CUDA_TRY(cudaGetLastError());
    return QW_OK;
}

qw_status launch_bm_overflow_list(const QueryState &st, int nb, const int32_t *order_perm,
                                  int64_t b0, int32_t *list0, int32_t *list1, int32_t *count,
                                  cudaStream_t s)
{
    bm_overflow_list_kernel<<<(nb + 255) / 256, 256, 0, s>>>(st, nb, order_perm, b0, list0, list1,
                                                             count);
    QW_CUDA_TRY(cudaGetLastError());
    return QW_OK;
}

}  // namespace qw
