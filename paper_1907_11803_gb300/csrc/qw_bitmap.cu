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

// Bucket bitmaps of the m projections for (query q, tile t) at one level, and
// (when my_scan is given) the entries in the level's ranges, for the
// statistics; cgrow is c, used only for those.
__device__ __forceinline__ void bucket_bitmaps(const IndexView &ix, const QueryState &st, int q,
                                               int t, int level, int64_t R, int cgrow, bool first,
                                               const uint4 **bp, int m8,
                                               unsigned long long *my_scan)
{
    const int m = ix.m;
    if (my_scan) *my_scan = 0;
    if (threadIdx.x < m) {
        const int i = threadIdx.x;
        const int64_t gi = st.g[(int64_t)q * m + i];
        const int64_t beta = floordiv64(gi, R);
        bp[i] = bm_ptr(ix, i, t, level, R, beta);
        if (my_scan) {
            const int64_t sp1 = (int64_t)ix.span[i] + 1;
            const int64_t dslot = (int64_t)i * ix.nT + t;
            const int32_t *ub = ix.dir_bid + ix.dir_start[dslot];
            const int32_t *uo = ix.dir_off + ix.dir_start[dslot];
            const int cnt = ix.dir_cnt[dslot];
            const int len = (int)min((int64_t)kTile, ix.n - (int64_t)t * kTile);
            const int64_t lo = beta * R;
            const int64_t A = clamp64(lo, 0, sp1), B = clamp64(lo + R, 0, sp1);
            *my_scan = (unsigned long long)(dir_lower(ub, uo, cnt, len, B) -
                                            dir_lower(ub, uo, cnt, len, A));
            if (first && level > 0) {
                // entries in the ranges of the skipped levels, for the statistics
                unsigned long long skipped = 0;
                int64_t Rs = R;
                for (int L2 = level - 1; L2 >= 0; --L2) {
                    Rs /= cgrow;
                    const int64_t lo3 = floordiv64(gi, Rs) * Rs;
                    const int64_t A3 = clamp64(lo3, 0, sp1), B3 = clamp64(lo3 + Rs, 0, sp1);
                    skipped += (unsigned long long)(dir_lower(ub, uo, cnt, len, B3) -
                                                    dir_lower(ub, uo, cnt, len, A3));
                }
                if (skipped)
                    atomicAdd(reinterpret_cast<unsigned long long *>(st.scan_full + q), skipped);
            }
        }
    } else if (threadIdx.x < m8) {
        bp[threadIdx.x] = nullptr;
    }
}

// One level for one (tile, query): counts of every id of the tile, the
// candidate bitmap (count >= l), and the tile's candidate profile (previous-
// level candidates; the others by count), as the level path produces it.
__global__ void __launch_bounds__(BM_THREADS, 2) bm_level_kernel(IndexView ix, int level,
                                                                 int64_t R, int l, int cgrow,
                                                                 QueryState st, const LoopCtl *ctl)
{
    __shared__ const uint4 *bp[QW_MAX_M + 8];
    __shared__ int hist[kHistBins];
    __shared__ int wsum[BM_THREADS / 32];
    __shared__ unsigned long long red_scan;
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
    if (threadIdx.x == 0) red_scan = 0;
    unsigned long long my_scan;
    bucket_bitmaps(ix, st, q, t, level, R, cgrow, first, bp, m8, &my_scan);
    __syncthreads();
    if (my_scan) atomicAdd(&red_scan, my_scan);

    Planes P;
    count_planes(P, bp, m8);
    const int64_t slot = ((int64_t)q * ix.nT + t) * kBmUint4 + threadIdx.x;
    uint4 *cur = st.cbits + (int64_t)(level & 1) * st.cb_par;
    const uint4 prev = first ? make_uint4(0, 0, 0, 0)
                             : st.cbits[(int64_t)((level - 1) & 1) * st.cb_par + slot];
    uint4 cand;
    cand.x = count_ge_planes(P, 0, l);
    cand.y = count_ge_planes(P, 1, l);
    cand.z = count_ge_planes(P, 2, l);
    cand.w = count_ge_planes(P, 3, l);
    cur[slot] = cand;
    // prev-level candidates are candidates here too (ranges nest, counts grow)
    const int my_count = __popc(cand.x) + __popc(cand.y) + __popc(cand.z) + __popc(cand.w);
    const int my_prev = __popc(prev.x) + __popc(prev.y) + __popc(prev.z) + __popc(prev.w);
#pragma unroll
    for (int w = 0; w < 4; ++w) {
        uint32_t x = word_of(cand, w) & ~word_of(prev, w);
        while (x) {
            const int b = __ffs(x) - 1;
            x &= x - 1;
            atomicAdd(&hist[1 + count_of(P, w, b)], 1);
        }
    }
    int tot_count, tot_prev;
    block_exclusive_scan<BM_THREADS>(my_count, wsum, &tot_count);
    block_exclusive_scan<BM_THREADS>(my_prev, wsum, &tot_prev);
    if (threadIdx.x == 0) hist[0] += tot_prev;
    __syncthreads();
    int *th = st.tile_hist + ((int64_t)q * ix.nT + t) * kHistBins;
    for (int c = threadIdx.x; c < kHistBins; c += BM_THREADS) th[c] = hist[c];
    if (threadIdx.x == 0) {
        if (tot_count) atomicAdd(st.cross + q, tot_count);
        if (red_scan)
            atomicAdd(reinterpret_cast<unsigned long long *>(st.scan_level + q), red_scan);
    }
}

// Emit the kept ids of one (tile, query) in ascending order at the tile's
// planned position (the plan comes from the tile profiles, as on the level
// path).  Counts of the final level are recomputed for the 128-id groups that
// hold candidates.
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
    bucket_bitmaps(ix, st, q, t, jf, Rf, 2, false, bp, m8, nullptr);
    __syncthreads();
    const int64_t slot = ((int64_t)q * nT + t) * kBmUint4 + threadIdx.x;
    const uint4 cand = st.cbits[(int64_t)(jf & 1) * st.cb_par + slot];
    const uint4 prev = jf > st.start[q] ? st.cbits[(int64_t)((jf - 1) & 1) * st.cb_par + slot]
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

qw_status launch_bm_level(const IndexView &ix, int nb, int level, int64_t R, int64_t Rp, int l,
                          int cgrow, QueryState &st, cudaStream_t s, const LoopCtl *ctl)
{
    (void)Rp;
    bm_level_kernel<<<dim3((unsigned)ix.nT, (unsigned)nb), BM_THREADS, 0, s>>>(ix, level, R, l,
                                                                              cgrow, st, ctl);
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
