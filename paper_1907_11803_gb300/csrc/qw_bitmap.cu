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
// the m bitmaps B_i(beta_i) that contain it (Section 3.1).  The kernel loads
// those m bitmaps of a tile -- coalesced 16-byte loads, no atomics -- and adds
// them bit-sliced: a carry-save adder tree keeps, per group of 32 ids, the
// seven bit planes of their counts in registers.  Counts are recomputed from
// scratch at every level, so nothing is carried between levels except the
// candidate bitmap (count >= l) of the previous level, which orders the
// truncation to k + v candidates.  The results -- candidate sets, counts,
// statistics -- are those of the level path.
//
// Storage: per (projection, tile), sum over levels L of (span / c^L + 1)
// bitmaps, i.e. about (c / (c - 1)) * (span + 1) * 4 KiB.  A level-L bitmap is
// the OR of its c children at level L - 1; the finest level comes from the
// tile's sorted entries.
#include "qw_internal.cuh"
#include "qw_dir.cuh"
#include "qw_scan.cuh"
#include "qw_tma.cuh"

#include <algorithm>

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

// Level 0: one bitmap per bid present in the tile, from the tile's sorted
// entries.  Bitmaps of absent bids stay zero (the buffer is cleared first).
__global__ void __launch_bounds__(BM_THREADS) bm_fill_level0_kernel(IndexView ix, uint4 *bm)
{
    __shared__ __align__(16) uint32_t sb[kTile / 32];
    const int t = blockIdx.x, i = blockIdx.y;
    const int64_t dslot = (int64_t)i * ix.nT + t;
    const int32_t *ub = ix.dir_bid + ix.dir_start[dslot];
    const int32_t *uo = ix.dir_off + ix.dir_start[dslot];
    const int cnt = ix.dir_cnt[dslot];
    const int len = (int)min((int64_t)kTile, ix.n - (int64_t)t * kTile);
    const uint16_t *seg = ix.lid + dslot * kTile;
    uint4 *sb4 = reinterpret_cast<uint4 *>(sb);
    const int64_t blk = ix.bm_base[i] + (int64_t)t * ix.bm_nb[i] + ix.bm_lvl[i * kBmLevels + 0];
    sb4[threadIdx.x] = make_uint4(0, 0, 0, 0);
    __syncthreads();
    for (int u = 0; u < cnt; ++u) {
        const int e0 = uo[u], e1 = (u + 1 < cnt) ? uo[u + 1] : len;
        for (int e = e0 + threadIdx.x; e < e1; e += BM_THREADS) {
            const uint32_t id = seg[e];
            atomicOr(&sb[id >> 5], 1u << (id & 31));
        }
        __syncthreads();
        bm[(blk + ub[u]) * kBmUint4 + threadIdx.x] = sb4[threadIdx.x];
        sb4[threadIdx.x] = make_uint4(0, 0, 0, 0);
        __syncthreads();
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

// Bitmap of the level-`level` bucket beta of projection i in tile t, or null
// when the bucket holds no data (beta below zero or past the span).  Past the
// last stored level a single bucket (beta == 0) holds every id.
__device__ __forceinline__ const uint4 *bm_ptr(const IndexView &ix, int i, int t, int level,
                                               int64_t R, int64_t beta)
{
    const int J = ix.bm_J[i];
    int L = level;
    if (level > J) {
        if (beta != 0) return nullptr;
        L = J;
    } else if (beta < 0 || beta > (int64_t)ix.span[i] / R) {
        return nullptr;
    }
    const int64_t idx =
        ix.bm_base[i] + (int64_t)t * ix.bm_nb[i] + ix.bm_lvl[i * kBmLevels + L] + beta;
    return ix.bm + idx * kBmUint4;
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

// Counts of the 128 ids of this thread: the sum of the m bucket bitmaps bp[]
// (null = empty), padded with empty inputs to a multiple of 8.
__device__ __forceinline__ void count_planes(Planes &P, const uint4 *const *bp, int m8)
{
#pragma unroll
    for (int k = 0; k < 7; ++k)
#pragma unroll
        for (int w = 0; w < 4; ++w) P.s[k][w] = 0;
#pragma unroll 1
    for (int g = 0; g < m8; g += 8) {
        uint4 x[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const uint4 *p = bp[g + u];
            x[u] = p ? __ldg(p + threadIdx.x) : make_uint4(0, 0, 0, 0);
        }
        add8(P, x);
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

// Bucket bitmaps of the m projections for (query q, tile t) at one level
// (threads 0 .. m8 - 1 fill bp; entries m .. m8 - 1 are empty).
__device__ __forceinline__ void bucket_bitmaps(const IndexView &ix, const QueryState &st, int q,
                                               int t, int level, int64_t R, const uint4 **bp,
                                               int m8)
{
    const int m = ix.m;
    if (threadIdx.x < m) {
        const int i = threadIdx.x;
        bp[i] = bm_ptr(ix, i, t, level, R, floordiv64(st.g[(int64_t)q * m + i], R));
    } else if (threadIdx.x < m8) {
        bp[threadIdx.x] = nullptr;
    }
}

// Epilogue shared by both level kernels: the candidate bitmap of the thread's
// 128 ids, the previous level's, and the tile profile's counts by bin.
__device__ __forceinline__ uint4 candidates_of(const Planes &P, int l)
{
    uint4 cand;
    cand.x = count_ge_planes(P, 0, l);
    cand.y = count_ge_planes(P, 1, l);
    cand.z = count_ge_planes(P, 2, l);
    cand.w = count_ge_planes(P, 3, l);
    return cand;
}

// The tile profile's bins (candidates that were not candidates at the
// previous level, by count) and the candidate list entries of this thread's
// 128 ids, written in ascending id order from list position pos.
__device__ __forceinline__ void profile_and_list(const Planes &P, const uint4 &cand,
                                                 const uint4 &prev, int *hist, uint32_t *list,
                                                 int pos, int id_base)
{
#pragma unroll
    for (int w = 0; w < 4; ++w) {
        uint32_t x = word_of(cand, w);
        const uint32_t pw = word_of(prev, w);
        while (x) {
            const int b = __ffs(x) - 1;
            x &= x - 1;
            const int c = count_of(P, w, b);
            if (!((pw >> b) & 1u)) atomicAdd(&hist[1 + c], 1);
            if (pos < kListCap) list[pos] = ((uint32_t)c << 16) | (uint32_t)(id_base + w * 32 + b);
            ++pos;
        }
    }
}

// One level for one (tile, query), loads straight from global memory: counts
// of every id of the tile, the candidate bitmap (count >= l), and the tile's
// candidate profile (previous-level candidates; the others by count), as the
// level path produces it.
__global__ void __launch_bounds__(BM_THREADS, 3) bm_level_kernel(IndexView ix, int level,
                                                                 int64_t R, int l,
                                                                 QueryState st, const LoopCtl *ctl)
{
    __shared__ const uint4 *bp[QW_MAX_M + 8];
    __shared__ int hist[kHistBins];
    __shared__ int wsum[BM_THREADS / 32];
    const int t = blockIdx.x;
    const int q = blockIdx.y;
    if (!st.active[q]) return;
    if (ctl) {
        level = ctl->level;
        R = ctl->R;
    }
    const int qstart = st.start[q];
    if (level < qstart) return;
    const bool first = level == qstart;
    const int m8 = (ix.m + 7) & ~7;
    for (int c = threadIdx.x; c < kHistBins; c += BM_THREADS) hist[c] = 0;
    bucket_bitmaps(ix, st, q, t, level, R, bp, m8);
    __syncthreads();

    const int64_t slot = ((int64_t)q * ix.nT + t) * kBmUint4 + threadIdx.x;
    const uint4 prev = first ? make_uint4(0, 0, 0, 0)
                             : st.cbits[(int64_t)((level - 1) & 1) * st.cb_par + slot];
    Planes P;
    count_planes(P, bp, m8);
    const uint4 cand = candidates_of(P, l);
    st.cbits[(int64_t)(level & 1) * st.cb_par + slot] = cand;
    // prev-level candidates are candidates here too (ranges nest, counts grow)
    const int my_count = __popc(cand.x) + __popc(cand.y) + __popc(cand.z) + __popc(cand.w);
    const int my_prev = __popc(prev.x) + __popc(prev.y) + __popc(prev.z) + __popc(prev.w);
    int tot_count, tot_prev;
    const int pos = block_exclusive_scan<BM_THREADS>(my_count, wsum, &tot_count);
    block_exclusive_scan<BM_THREADS>(my_prev, wsum, &tot_prev);
    const int64_t qt = (int64_t)q * ix.nT + t;
    profile_and_list(P, cand, prev, hist, st.clist + (int64_t)(level & 1) * st.cl_par + qt * kListCap,
                     pos, threadIdx.x * 128);
    if (threadIdx.x == 0) {
        hist[0] += tot_prev;
        st.clist_n[(int64_t)(level & 1) * st.cln_par + qt] = tot_count;
    }
    __syncthreads();
    int *th = st.tile_hist + qt * kHistBins;
    for (int c = threadIdx.x; c < kHistBins; c += BM_THREADS) th[c] = hist[c];
    if (threadIdx.x == 0 && tot_count) atomicAdd(st.cross + q, tot_count);
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
    int hist[2][kHistBins];        // tile profile of the current item (alternating)
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
    for (int c = tid; c < 2 * kHistBins; c += TMA_THREADS) (&sh.hist[0][0])[c] = 0;
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
            const int qq = (int)(kk / nT);
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
            const int q = (int)(k / nT), t = (int)(k % nT);
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
        // ---- the item's epilogue
        const uint4 cand = candidates_of(P, l);
        st.cbits[(int64_t)(level & 1) * st.cb_par + qt * kBmUint4 + tid] = cand;
        const int my_count = __popc(cand.x) + __popc(cand.y) + __popc(cand.z) + __popc(cand.w);
        int my_prev = __popc(prev.x) + __popc(prev.y) + __popc(prev.z) + __popc(prev.w);
        // consumers only (the producer does not take part)
        int tot_count;
        const int pos = consumer_scan(my_count, sh.wsum, &tot_count, &sh.group, gph, err, stuck);
        profile_and_list(P, cand, prev, sh.hist[par],
                         st.clist + (int64_t)(level & 1) * st.cl_par + qt * kListCap, pos, tid * 128);
        my_prev = __reduce_add_sync(0xffffffffu, my_prev);
        if (lane == 0 && my_prev) atomicAdd(&sh.hist[par][0], my_prev);
        group_sync(&sh.group, gph, err, stuck);
        if (stuck) break;
        int *th = st.tile_hist + qt * kHistBins;
        for (int c = tid; c < kHistBins; c += TMA_CONSUMERS) {
            th[c] = sh.hist[par][c];
            sh.hist[par][c] = 0;
        }
        if (tid == 0) {
            st.clist_n[(int64_t)(level & 1) * st.cln_par + qt] = tot_count;
            if (tot_count) atomicAdd(st.cross + h.q, tot_count);
        }
        par ^= 1;
    }
}

// Emit the kept ids of one (tile, query) in ascending order at the tile's
// planned position (the plan comes from the tile profiles, as on the level
// path).  Ids and counts come from the final level's candidate list; a tile
// with more candidates than the list holds recounts its candidate groups.
__global__ void __launch_bounds__(BM_THREADS, 2) bm_emit_kernel(IndexView ix, int l, int cap,
                                                                QueryState st)
{
    __shared__ const uint4 *bp[QW_MAX_M + 8];
    __shared__ int scan_tmp[BM_THREADS / 32];
    const int t = blockIdx.x;
    const int q = blockIdx.y;
    const int nT = ix.nT;
    const int *plan = st.tile_plan + ((int64_t)q * nT + t) * 3;
    if (plan[2] == 0) return;
    const int out0 = plan[0];
    const int eq0 = plan[1];
    const int cstar = st.qplan[q * 2 + 0], take_eq = st.qplan[q * 2 + 1];
    const int jf = st.levels[q] - 1;
    const int64_t Rf = st.finalR[q];
    const int m8 = (ix.m + 7) & ~7;
    const int64_t qt = (int64_t)q * nT + t;
    const int64_t slot = qt * kBmUint4 + threadIdx.x;
    const bool has_prev = jf > st.start[q];
    const int nlist = st.clist_n[(int64_t)(jf & 1) * st.cln_par + qt];
    if (nlist <= kListCap) {
        // the level kernel listed the tile's candidates with their counts
        const uint32_t *L = st.clist + (int64_t)(jf & 1) * st.cl_par + qt * kListCap;
        const uint32_t *pw = reinterpret_cast<const uint32_t *>(
            st.cbits + (int64_t)((jf - 1) & 1) * st.cb_par + qt * kBmUint4);
        const int per = (nlist + BM_THREADS - 1) / BM_THREADS;
        const int j0 = min(nlist, (int)threadIdx.x * per), j1 = min(nlist, j0 + per);
        int n_eq = 0;
        if (cstar >= l)
            for (int j = j0; j < j1; ++j) {
                const uint32_t e = L[j], id = e & 0xffffu;
                const bool pf = has_prev && ((pw[id >> 5] >> (id & 31)) & 1u);
                n_eq += (!pf && (int)(e >> 16) == cstar) ? 1 : 0;
            }
        int eq_total;
        int r = eq0 + block_exclusive_scan<BM_THREADS>(n_eq, scan_tmp, &eq_total);
        int n_sel = 0;
        {
            int rr = r;
            for (int j = j0; j < j1; ++j) {
                const uint32_t e = L[j], id = e & 0xffffu;
                const int c = (int)(e >> 16);
                const bool pf = has_prev && ((pw[id >> 5] >> (id & 31)) & 1u);
                if (pf || c > cstar) ++n_sel;
                else if (c == cstar) { n_sel += (rr < take_eq) ? 1 : 0; ++rr; }
            }
        }
        int sel_total;
        int pos = out0 + block_exclusive_scan<BM_THREADS>(n_sel, scan_tmp, &sel_total);
        for (int j = j0; j < j1; ++j) {
            const uint32_t e = L[j], id = e & 0xffffu;
            const int c = (int)(e >> 16);
            const bool pf = has_prev && ((pw[id >> 5] >> (id & 31)) & 1u);
            bool sel;
            if (pf || c > cstar) sel = true;
            else if (c == cstar) { sel = r < take_eq; ++r; }
            else sel = false;
            if (!sel) continue;
            if (pos < cap) {
                st.cand[(int64_t)q * cap + pos] = (int32_t)((int64_t)t * kTile + id);
                st.cand_col[(int64_t)q * cap + pos] = c;
            }
            ++pos;
        }
        return;
    }
    // more candidates than the list holds: recount the groups that have some
    bucket_bitmaps(ix, st, q, t, jf, Rf, bp, m8);
    __syncthreads();
    const uint4 cand = st.cbits[(int64_t)(jf & 1) * st.cb_par + slot];
    const uint4 prev = has_prev ? st.cbits[(int64_t)((jf - 1) & 1) * st.cb_par + slot]
                                : make_uint4(0, 0, 0, 0);
    const bool mine = (cand.x | cand.y | cand.z | cand.w) != 0;
    Planes P;
    if (mine) count_planes(P, bp, m8);
    int n_eq = 0;
    if (mine && cstar >= l) {
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            uint32_t x = word_of(cand, w) & ~word_of(prev, w);
            while (x) {
                const int b = __ffs(x) - 1;
                x &= x - 1;
                n_eq += count_of(P, w, b) == cstar ? 1 : 0;
            }
        }
    }
    int eq_total;
    int r = eq0 + block_exclusive_scan<BM_THREADS>(n_eq, scan_tmp, &eq_total);
    int n_sel = 0;
    if (mine) {
        int rr = r;
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            uint32_t x = word_of(cand, w);
            const uint32_t pw = word_of(prev, w);
            while (x) {
                const int b = __ffs(x) - 1;
                x &= x - 1;
                const int c = count_of(P, w, b);
                if (((pw >> b) & 1u) || c > cstar) ++n_sel;
                else if (c == cstar) { n_sel += (rr < take_eq) ? 1 : 0; ++rr; }
            }
        }
    }
    int sel_total;
    int pos = out0 + block_exclusive_scan<BM_THREADS>(n_sel, scan_tmp, &sel_total);
    if (!mine) return;
    const int64_t id0 = (int64_t)t * kTile + (int64_t)threadIdx.x * 128;
#pragma unroll
    for (int w = 0; w < 4; ++w) {
        uint32_t x = word_of(cand, w);
        const uint32_t pw = word_of(prev, w);
        while (x) {
            const int b = __ffs(x) - 1;
            x &= x - 1;
            const int c = count_of(P, w, b);
            bool sel;
            if (((pw >> b) & 1u) || c > cstar) sel = true;
            else if (c == cstar) { sel = r < take_eq; ++r; }
            else sel = false;
            if (!sel) continue;
            if (pos < cap) {
                st.cand[(int64_t)q * cap + pos] = (int32_t)(id0 + w * 32 + b);
                st.cand_col[(int64_t)q * cap + pos] = c;
            }
            ++pos;
        }
    }
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

qw_status launch_bitmap_build(const IndexView &ix, int c, int maxJ, uint4 *bm, cudaStream_t s)
{
    const dim3 grid((unsigned)ix.nT, (unsigned)ix.m);
    bm_fill_level0_kernel<<<grid, BM_THREADS, 0, s>>>(ix, bm);
    QW_CUDA_TRY(cudaGetLastError());
    int64_t R = 1;
    for (int L = 1; L <= maxJ; ++L) {
        R *= c;
        bm_or_level_kernel<<<grid, BM_THREADS, 0, s>>>(ix, bm, L, R, c);
        QW_CUDA_TRY(cudaGetLastError());
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

qw_status launch_bm_level(const IndexView &ix, int nb, int level, int64_t R, int64_t Rp, int l,
                          int cgrow, QueryState &st, int *err, bool tma, cudaStream_t s,
                          const LoopCtl *ctl)
{
    (void)Rp;
    (void)cgrow;
    if (!tma) {
        bm_level_kernel<<<dim3((unsigned)ix.nT, (unsigned)nb), BM_THREADS, 0, s>>>(ix, level, R, l,
                                                                                  st, ctl);
        QW_CUDA_TRY(cudaGetLastError());
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

qw_status launch_bm_collect(const IndexView &ix, int nb, int l, int cap, QueryState &st,
                            int64_t *stats_out, cudaStream_t s)
{
    QW_TRY(launch_select_plan(ix, nb, l, cap, st, stats_out, s));
    bm_emit_kernel<<<dim3((unsigned)ix.nT, (unsigned)nb), BM_THREADS, 0, s>>>(ix, l, cap, st);
    QW_CUDA_TRY(cudaGetLastError());
    return QW_OK;
}

}  // namespace qw
