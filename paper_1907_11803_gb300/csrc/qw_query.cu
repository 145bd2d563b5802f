// qw_query.cu -- the query side of collision counting with virtual rehashing.
//
// For every query of a batch the host runs levels L = 0, 1, 2, ... with radius
// R = c^L (Section 2, C2LSH virtual rehashing).  At radius R the bucket of
// projection i is floor(bid / R); a data object collides with the query on
// projection i when its bid lies in [beta_i R, beta_i R + R - 1],
// beta_i = floor(g_i / R), g_i = h_i(q) - o_i.  Its collision count is the
// number of such projections, and it is a candidate when the count reaches
// the threshold l (Section 3.1).
//
// Ranges nest from one level to the next, so a level only scans the entries
// of the two new flanks of every projection's range and adds them to the
// running counts.  Counts live in one byte per (query, data id): 7 bits of
// count (m <= 127) and a flag bit meaning "was a candidate at the previous
// level", which orders the truncation to k + v candidates.
//
// One CTA owns one (index tile, query): it stages the tile's counters in
// shared memory, range-searches the tile's bucket directory for the flank
// boundaries of all m projections, increments the counters of every id in the
// flanks, counts the ids whose count reaches l, and writes the counters back.
#include "qw_internal.cuh"
#include "qw_count.cuh"
#include "qw_dir.cuh"
#include "qw_scan.cuh"

#include <algorithm>
#include <climits>

namespace qw {
namespace {

constexpr int LV_THREADS = 256;
constexpr int kWordsPerTile = kTile / 4;
constexpr int kUnroll = 4;

__global__ void query_setup_kernel(const int32_t *__restrict__ HQ, int nb, int m,
                                   const int32_t *__restrict__ o,
                                   const int32_t *__restrict__ span, QueryState st)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nb) return;
    int64_t top = 0;
    for (int i = 0; i < m; ++i) {
        int64_t g = (int64_t)HQ[(int64_t)q * m + i] - (int64_t)o[i];
        st.g[(int64_t)q * m + i] = g;
        top = max(top, max((int64_t)span[i], g));
        // with probes a query bucket id below the data collides once R > -g
        if (st.probes > 0) top = max(top, -g);
    }
    st.top[q] = top;
    st.active[q] = 1;
    st.ncand[q] = 0;
    st.nprev[q] = 0;
    st.cross[q] = 0;
    st.term[q] = 0;
    st.levels[q] = 0;
    st.finalR[q] = 0;
    st.scan_level[q] = 0;
    st.scan_last[q] = 0;
    st.scan_full[q] = 0;
    st.nkeep[q] = 0;
    st.start[q] = 0;
    st.fb[q] = 0;
    if (st.recount) st.recount[q] = 0;
    if (st.bm_ovf) st.bm_ovf[q] = 0;
    if (st.qbuf_n) {
        st.qbuf_n[q] = 0;
        st.qbuf_n[st.qbn_par + q] = 0;
    }
    atomicMax(st.max_top, (unsigned long long)top);
}

// Queries that stopped at a learned first level > 0 start over from level 0;
// fb_count[0] += their number, fb_count[1] += levels skipped by the others.
__global__ void fallback_kernel(int nb, QueryState st)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nb) return;
    if (!st.fb[q]) {
        if (st.start[q]) atomicAdd(st.fb_count + 1, (unsigned long long)st.start[q]);
        return;
    }
    st.fb[q] = 0;
    st.start[q] = 0;
    st.active[q] = 1;
    st.ncand[q] = 0;
    st.nprev[q] = 0;
    st.cross[q] = 0;
    st.term[q] = 0;
    st.levels[q] = 0;
    st.finalR[q] = 0;
    st.scan_level[q] = 0;
    st.scan_last[q] = 0;
    st.scan_full[q] = 0;
    if (st.qbuf_n) {
        st.qbuf_n[q] = 0;
        st.qbuf_n[st.qbn_par + q] = 0;
    }
    atomicAdd(st.fb_count, 1ull);
}

__global__ void __launch_bounds__(LV_THREADS) level_kernel(IndexView ix, int level, int64_t R,
                                                           int64_t Rp, int l, int cgrow,
                                                           QueryState st, int64_t words_per_query,
                                                           const LoopCtl *ctl)
{
    __shared__ __align__(16) uint32_t cnt_s[kWordsPerTile];
    __shared__ int64_t f_gc0[2 * QW_MAX_M];
    __shared__ int32_t f_cpref[2 * QW_MAX_M + 1];
    __shared__ uint8_t f_head[2 * QW_MAX_M], f_tail[2 * QW_MAX_M], f_tile[2 * QW_MAX_M];
    __shared__ int32_t wsum[LV_THREADS / 32];
    __shared__ int hist[kHistBins];
    __shared__ int32_t red_count;
    __shared__ unsigned long long red_scan;
    FlankSet fl{f_gc0, f_cpref, f_head, f_tail, f_tile};

    const int t = blockIdx.x;
    const int q = blockIdx.y;
    if (!st.active[q]) return;
    if (ctl) {
        level = ctl->level;
        R = ctl->R;
        Rp = ctl->Rp;
    }
    const int qstart = st.start[q];
    if (level < qstart) return;
    // the query's first level counts its whole range from zeroed counters
    const bool first = level == qstart;
    const int m = ix.m;
    const int64_t n = ix.n;
    const int64_t tbase = (int64_t)t * kTile;
    const int len = (int)min((int64_t)kTile, n - tbase);
    if (threadIdx.x == 0) {
        red_count = 0;
        red_scan = 0;
    }
    for (int c = threadIdx.x; c < kHistBins; c += LV_THREADS) hist[c] = 0;

    // 1. flank boundaries of every projection (one thread per projection)
    unsigned long long my_scan = 0;
    int my_c0 = 0, my_c1 = 0;
    if (ix.qkey) {
        // QALSH: the run of the tile's sorted projections inside this level's
        // interval p_i(q) +- qhalf R, and inside the previous level's; thread
        // 2i + j searches both ends of interval j of projection i (two binary
        // searches advancing together) and leaves (end << 32 | start) in
        // f_gc0[2i + j], which projection i's thread reads before it writes
        // its flanks there
        if (threadIdx.x < 2 * m && (threadIdx.x & 1) <= (first ? 0 : 1)) {
            const int i = threadIdx.x >> 1;
            const double h = __dmul_rn(ix.qhalf, (double)((threadIdx.x & 1) ? Rp : R));
            const double pq = __longlong_as_double((long long)st.g[(int64_t)q * m + i]);
            const double *kk = ix.qkey + (int64_t)i * ix.nT * kTile + tbase;
            int la = 0, ha = len, lb = 0, hb = len;
            while (la < ha || lb < hb) {
                if (la < ha) {
                    const int mid = (la + ha) >> 1;
                    if (__dsub_rn(kk[mid], pq) < -h) la = mid + 1; else ha = mid;
                }
                if (lb < hb) {
                    const int mid = (lb + hb) >> 1;
                    if (!(__dsub_rn(kk[mid], pq) > h)) lb = mid + 1; else hb = mid;
                }
            }
            f_gc0[threadIdx.x] = ((int64_t)lb << 32) | (int64_t)la;
        }
        __syncthreads();
        if (threadIdx.x < m) {
            const int i = threadIdx.x;
            const int64_t cur = f_gc0[2 * i];
            const int pA = (int)(cur & 0xffffffff), pB = (int)(cur >> 32);
            int s0 = pA, e0 = pB, s1 = 0, e1 = 0;
            if (!first) {
                // intervals nest from level to level: the two new flanks
                const int64_t prv = f_gc0[2 * i + 1];
                e0 = (int)(prv & 0xffffffff);
                s1 = (int)(prv >> 32);
                e1 = pB;
            }
            const int64_t ebase = (int64_t)i * ix.nT * kTile + tbase;
            flank_set(fl, 2 * i, ebase + s0, ebase + e0, 0, &my_c0);
            flank_set(fl, 2 * i + 1, ebase + s1, ebase + e1, 0, &my_c1);
            my_scan = (unsigned long long)(pB - pA);
        }
    } else if (threadIdx.x < m) {
        const int i = threadIdx.x;
        const int64_t gi = st.g[(int64_t)q * m + i];
        const int64_t sp1 = (int64_t)ix.span[i] + 1;
        const int64_t dslot = (int64_t)i * ix.nT + t;
        const int32_t *ub = ix.dir_bid + ix.dir_start[dslot];
        const int32_t *uo = ix.dir_off + ix.dir_start[dslot];
        const int cnt = ix.dir_cnt[dslot];
        // the level's bid range, widened to P buckets on each side with probes
        const int64_t P = st.probes;
        const int64_t lo = (floordiv64(gi, R) - P) * R;
        const int64_t A = clamp64(lo, 0, sp1), B = clamp64(lo + (2 * P + 1) * R, 0, sp1);
        const int pA = dir_lower(ub, uo, cnt, len, A);
        const int pB = dir_lower(ub, uo, cnt, len, B);
        int s0 = pA, e0 = pB, s1 = 0, e1 = 0;
        if (!first) {
            // ranges nest from level to level, so only the two new flanks are read
            const int64_t lo2 = (floordiv64(gi, Rp) - P) * Rp;
            const int64_t A2 = clamp64(lo2, 0, sp1), B2 = clamp64(lo2 + (2 * P + 1) * Rp, 0, sp1);
            if (A2 < B2) {
                e0 = dir_lower(ub, uo, cnt, len, A2);
                s1 = dir_lower(ub, uo, cnt, len, B2);
                e1 = pB;
            }
        } else if (level > 0) {
            // entries in the ranges of the skipped levels, for the statistics
            unsigned long long skipped = 0;
            int64_t Rs = R;
            for (int L2 = level - 1; L2 >= 0; --L2) {
                Rs /= cgrow;
                const int64_t lo3 = (floordiv64(gi, Rs) - P) * Rs;
                const int64_t A3 = clamp64(lo3, 0, sp1), B3 = clamp64(lo3 + (2 * P + 1) * Rs, 0, sp1);
                skipped += (unsigned long long)(dir_lower(ub, uo, cnt, len, B3) -
                                                dir_lower(ub, uo, cnt, len, A3));
            }
            if (skipped) atomicAdd(reinterpret_cast<unsigned long long *>(st.scan_full + q), skipped);
        }
        // the tile's slots start 16-byte aligned, so chunks are tile offsets / 8
        const int64_t ebase = (int64_t)i * ix.nT * kTile + tbase;
        flank_set(fl, 2 * i, ebase + s0, ebase + e0, 0, &my_c0);
        flank_set(fl, 2 * i + 1, ebase + s1, ebase + e1, 0, &my_c1);
        my_scan = (unsigned long long)(pB - pA);
    }
    {
        int total;
        const int excl = block_exclusive_scan<LV_THREADS>(my_c0 + my_c1, wsum, &total);
        if (threadIdx.x < m) {
            f_cpref[2 * threadIdx.x] = excl;
            f_cpref[2 * threadIdx.x + 1] = excl + my_c0;
        }
        if (threadIdx.x == 0) f_cpref[2 * m] = total;
    }
    if (my_scan) atomicAdd(&red_scan, my_scan);

    // 2. the tile's counters into shared memory; flag previous candidates
    uint4 *cg = reinterpret_cast<uint4 *>(st.counters + (int64_t)q * words_per_query +
                                          (int64_t)t * kWordsPerTile);
    uint4 *cs = reinterpret_cast<uint4 *>(cnt_s);
    const uint32_t lrep = (uint32_t)l * 0x01010101u;
    if (first) {
        for (int w4 = threadIdx.x; w4 < kWordsPerTile / 4; w4 += LV_THREADS)
            cs[w4] = make_uint4(0, 0, 0, 0);
    } else {
        for (int w4 = threadIdx.x; w4 < kWordsPerTile / 4; w4 += LV_THREADS) {
            uint4 x = cg[w4];
            x.x = flag_ge(x.x, lrep);
            x.y = flag_ge(x.y, lrep);
            x.z = flag_ge(x.z, lrep);
            x.w = flag_ge(x.w, lrep);
            cs[w4] = x;
        }
    }
    __syncthreads();

    // 3. count every id in the flanks: 8 ids per 16-byte load, kUnroll loads
    //    in flight per thread; the current flank's bounds stay in registers
    const int total = f_cpref[2 * m];
    const uint4 *lid4 = reinterpret_cast<const uint4 *>(ix.lid);
    int s = -1, c_lo = 0, c_hi = 0;
    int64_t g0 = 0;
    uint32_t head_mask = 0xffu, tail_mask = 0xffu;
    for (int e0 = threadIdx.x; e0 < total; e0 += LV_THREADS * kUnroll) {
        uint4 v[kUnroll];
        uint32_t mask[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const int e = e0 + u * LV_THREADS;
            mask[u] = 0;
            if (e < total) {
                if (e >= c_hi) {
                    do {
                        ++s;
                        c_hi = f_cpref[s + 1];
                    } while (e >= c_hi);
                    c_lo = f_cpref[s];
                    g0 = f_gc0[s];
                    head_mask = 0xffu << f_head[s];
                    tail_mask = 0xffu >> (8 - f_tail[s]);
                }
                v[u] = __ldg(lid4 + g0 + (e - c_lo));
                uint32_t mk = 0xffu;
                if (e == c_lo) mk &= head_mask;
                if (e == c_hi - 1) mk &= tail_mask;
                mask[u] = mk;
            }
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
            if (mask[u]) count_chunk(cnt_s, v[u], mask[u]);
    }
    __syncthreads();

    // 4. counters back to global memory, and this tile's candidate profile:
    //    previous-level candidates, and the other candidates by count
    int my_prev = 0, my_count = 0;
    for (int w4 = threadIdx.x; w4 < kWordsPerTile / 4; w4 += LV_THREADS) {
        const uint4 x = cs[w4];
        cg[w4] = x;
        const uint32_t wv[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const int c4 = count_ge(wv[h], lrep);
            if (!c4) continue;
            my_count += c4;
#pragma unroll
            for (int by = 0; by < 4; ++by) {
                const uint32_t b8 = (wv[h] >> (8 * by)) & 0xffu;
                if ((b8 & 0x7fu) < (uint32_t)l) continue;
                if (b8 & 0x80u) ++my_prev;
                else atomicAdd(&hist[1 + (b8 & 0x7fu)], 1);
            }
        }
    }
    my_prev = __reduce_add_sync(0xffffffffu, my_prev);
    my_count = __reduce_add_sync(0xffffffffu, my_count);
    if ((threadIdx.x & 31) == 0) {
        if (my_prev) atomicAdd(&hist[0], my_prev);
        if (my_count) atomicAdd(&red_count, my_count);
    }
    __syncthreads();
    int *th = st.tile_hist + ((int64_t)q * ix.nT + t) * kHistBins;
    for (int c = threadIdx.x; c < kHistBins; c += LV_THREADS) th[c] = hist[c];
    if (threadIdx.x == 0) {
        if (red_count) atomicAdd(st.cross + q, red_count);
        if (red_scan) atomicAdd(reinterpret_cast<unsigned long long *>(st.scan_level + q), red_scan);
    }
}

// Entries of projection i's data with bid in the level-R range of g.
__device__ __forceinline__ int64_t range_entries(const ScanStats &ss, int i, int64_t g, int64_t R)
{
    const int64_t sp1 = (int64_t)ss.span[i] + 1;
    const int64_t lo = floordiv64(g, R) * R;
    const int64_t A = clamp64(lo, 0, sp1), B = clamp64(lo + R, 0, sp1);
    const int64_t *P = ss.prefix + ss.off[i];
    return P[B] - P[A];
}

// One warp per query: the lanes add the entries-scanned statistics over the
// projections (bitmap path), lane 0 takes the decision.
__global__ void decide_kernel(int nb, int level, int64_t R, int cap, QueryState st,
                              LoopCtl *ctl, ScanStats ss)
{
    const int q = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (q >= nb || !st.active[q]) return;
    if (ctl) {
        level = ctl->level;
        R = ctl->R;
    }
    if (level < st.start[q]) {
        // not started yet: the device-driven loop must go on
        if (ctl && lane == 0) atomicAdd(&ctl->active, 1u);
        return;
    }
    const bool first = level == st.start[q];
    int64_t sl = 0, skipped = 0;
    if (ss.prefix) {
        // the same sums as the level kernel's, from the bid prefix counts: this
        // level's ranges, and at a learned first level > 0 the ranges of the
        // levels it skipped
        for (int i = lane; i < ss.m; i += 32) {
            const int64_t g = st.g[(int64_t)q * ss.m + i];
            sl += range_entries(ss, i, g, R);
            if (first && level > 0) {
                int64_t Rs = R;
                for (int L2 = level - 1; L2 >= 0; --L2) {
                    Rs /= ss.cgrow;
                    skipped += range_entries(ss, i, g, Rs);
                }
            }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            sl += __shfl_down_sync(0xffffffffu, sl, off);
            skipped += __shfl_down_sync(0xffffffffu, skipped, off);
        }
    }
    if (lane != 0) return;
    if (st.level_passes) atomicAdd(st.level_passes, 1ull);
    if (!ss.prefix) sl = st.scan_level[q];
    const int32_t before = st.ncand[q];  // |C_R| of the previous level
    const int32_t nc = st.cross[q];      // |C_R| of this level, summed over tiles
    st.cross[q] = 0;
    st.scan_full[q] += skipped;
    st.scan_level[q] = 0;
    st.scan_last[q] = sl;
    st.scan_full[q] += sl;
    st.levels[q] = level + 1;
    st.finalR[q] = R;
    const bool enough = nc >= cap;        // the k + v bound (Section 3.1)
    const bool past = R > st.top[q];      // no further level can change C_R
    if ((enough || past) && first && level > 0) {
        if (ss.recount_first) {
            // bitmap path: stop here; the previous level's candidates are
            // recounted from the bitmaps afterwards (and checked)
            st.recount[q] = 1;
        } else {
            // stopped at a learned first level: the previous level is unknown,
            // so the query is answered again from level 0
            st.fb[q] = 1;
            st.active[q] = 0;
            return;
        }
    }
    if (enough || past) {
        st.term[q] = enough ? 2 : 3;
        st.active[q] = 0;
        st.nprev[q] = before;
    } else {
        if (ctl) atomicAdd(&ctl->active, 1u);
        // the next level's candidate list starts empty (bitmap path)
        if (st.qbuf_n) st.qbuf_n[(int64_t)((level + 1) & 1) * st.qbn_par + q] = 0;
    }
    st.ncand[q] = nc;
}

// Graph mode: the level loop runs on the device.  The first pass starts at
// the smallest first level of the batch (0 unless every query has a learned
// start above it): levels below it would do no work.
__global__ void loop_min_start_kernel(LoopCtl *ctl, QueryState st, int nb)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    int s = q < nb ? st.start[q] : INT_MAX;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s = min(s, __shfl_down_sync(0xffffffffu, s, off));
    if ((threadIdx.x & 31) == 0 && s != INT_MAX) atomicMin(&ctl->min_start, s);
}

__global__ void loop_reset_kernel(LoopCtl *ctl)
{
    ctl->min_start = INT_MAX;
    ctl->active = 0;
}

__global__ void loop_init_kernel(LoopCtl *ctl, int cgrow)
{
    const int L = ctl->min_start == INT_MAX ? 0 : ctl->min_start;
    int64_t R = 1, Rp = 1;
    for (int j = 0; j < L; ++j) {
        Rp = R;
        R *= cgrow;
    }
    ctl->level = L;
    ctl->R = R;
    ctl->Rp = Rp;
    ctl->pass = 0;
    ctl->active = 0;
}

// After a level's decision: stop once R exceeds every query's last useful
// radius (after this level no query can still be active), else go to the
// next level.  Mirrors the host loop; level 63 would overflow R and is an
// error (flag 8).
__global__ void loop_ctl_kernel(LoopCtl *ctl, const unsigned long long *max_top, int cgrow,
                                cudaGraphConditionalHandle h, int *err)
{
    const int64_t R = ctl->R;
    // stop once R exceeds every useful radius, or no query is left to run
    bool more = (unsigned long long)R <= *max_top && ctl->active > 0;
    ctl->active = 0;
    ctl->iters += 1;
    if (more && ctl->level > 62) {
        atomicOr(err, 8);
        more = false;
    }
    if (more) {
        ctl->level += 1;
        ctl->Rp = R;
        ctl->R = R * cgrow;
    }
    cudaGraphSetConditional(h, more ? 1u : 0u);
}

// Learned start, graph mode: after the fallback kernel marked the queries that
// stopped at their learned first level, run the loop again from level 0 if
// there are any.
__global__ void second_pass_kernel(QueryState st, LoopCtl *ctl, cudaGraphConditionalHandle h)
{
    ctl->level = 0;
    ctl->R = 1;
    ctl->Rp = 1;
    ctl->pass = 1;
    ctl->active = 0;
    ctl->fb_total += st.fb_count[0];
    ctl->skipped_total += st.fb_count[1];
    cudaGraphSetConditional(h, st.fb_count[0] > 0 ? 1u : 0u);
}

constexpr int CL_THREADS = 256;
constexpr int CL_PER = 16;  // ids per thread per chunk (one 16-byte load)

// Plan the kept candidates of one query from the per-tile profiles of its
// last level: all ids with count >= l when there are at most k + v of them;
// otherwise the previous level's candidates, then by count descending, then by
// id ascending, up to k + v.  The boundary count c* splits the ids with count
// above it (all kept) from those equal to it (the first take_eq by id kept).
// Writes, per tile, where its kept ids start in the query's list and how many
// count-c* ids precede it; and the query's statistics.
__global__ void __launch_bounds__(CL_THREADS) select_plan_kernel(
    int nT, int m, int l, int cap, QueryState st, int64_t *__restrict__ stats_out)
{
    __shared__ int tot[kHistBins];
    __shared__ int s_cstar, s_take_eq;
    __shared__ int scan_tmp[CL_THREADS / 32];
    const int q = blockIdx.x;
    const int nc = st.ncand[q];
    const int np = st.nprev[q];
    const int *qh = st.tile_hist + (int64_t)q * nT * kHistBins;
    if (threadIdx.x == 0) {
        s_cstar = l - 1;
        s_take_eq = 0;
    }
    if (nc > cap) {
        for (int c = threadIdx.x; c < kHistBins; c += CL_THREADS) {
            int sum = 0;
            for (int t = 0; t < nT; ++t) sum += qh[(int64_t)t * kHistBins + c];
            tot[c] = sum;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            const int need = cap - np;
            int acc = 0;
            for (int c = m; c >= l; --c) {
                const int hc = tot[1 + c];
                if (acc + hc >= need) {
                    s_cstar = c;
                    s_take_eq = need - acc;
                    break;
                }
                acc += hc;
            }
        }
    }
    __syncthreads();
    const int cstar = s_cstar, take_eq = s_take_eq;
    // per tile: kept ids above c*, and ids at c*, then prefixes over tiles
    int eq_base = 0, out_base = 0;
    for (int t0 = 0; t0 < nT; t0 += CL_THREADS) {
        const int t = t0 + threadIdx.x;
        int above = 0, eq = 0;
        if (t < nT) {
            const int *th = qh + (int64_t)t * kHistBins;
            above = th[0];
            for (int c = max(cstar + 1, l); c <= m; ++c) above += th[1 + c];
            eq = (cstar >= l) ? th[1 + cstar] : 0;
        }
        int eq_tot;
        const int eq_ex = eq_base + block_exclusive_scan<CL_THREADS>(eq, scan_tmp, &eq_tot);
        const int kept = above + min(max(take_eq - eq_ex, 0), eq);
        int kept_tot;
        const int out_ex = out_base + block_exclusive_scan<CL_THREADS>(kept, scan_tmp, &kept_tot);
        if (t < nT) {
            st.tile_plan[((int64_t)q * nT + t) * 3 + 0] = out_ex;
            st.tile_plan[((int64_t)q * nT + t) * 3 + 1] = eq_ex;
            st.tile_plan[((int64_t)q * nT + t) * 3 + 2] = kept;
        }
        eq_base += eq_tot;
        out_base += kept_tot;
    }
    if (threadIdx.x == 0) {
        const int keep = min(out_base, cap);
        st.nkeep[q] = keep;
        st.qplan[q * 2 + 0] = cstar;
        st.qplan[q * 2 + 1] = take_eq;
        if (stats_out) {
            int64_t *so = stats_out + (int64_t)q * QW_NSTAT;
            so[0] = st.levels[q];
            so[1] = st.finalR[q];
            so[2] = nc;
            so[3] = keep;
            so[4] = st.term[q];
            so[5] = st.scan_last[q];
            so[6] = st.scan_full[q];
            so[7] = np;
        }
    }
    // pad the list (the emit kernel fills [0, keep))
    const int keep = min(out_base, cap);
    for (int p = keep + threadIdx.x; p < cap; p += CL_THREADS) {
        st.cand[(int64_t)q * cap + p] = -1;
        st.cand_col[(int64_t)q * cap + p] = 0;
    }
}

// Emit the kept ids of one (tile, query) in ascending order at the tile's
// planned position.  Each thread owns 128 consecutive ids of the tile, so one
// pair of block scans orders the whole tile.
constexpr int EM_PER = kTile / CL_THREADS;  // ids per thread

__global__ void __launch_bounds__(CL_THREADS) select_emit_kernel(
    int64_t n, int nT, int l, int cap, QueryState st, int64_t words_per_query)
{
    __shared__ int scan_tmp[CL_THREADS / 32];
    const int t = blockIdx.x;
    const int q = blockIdx.y;
    const int cstar = st.qplan[q * 2 + 0], take_eq = st.qplan[q * 2 + 1];
    const int *plan = st.tile_plan + ((int64_t)q * nT + t) * 3;
    if (plan[2] == 0) return;  // nothing kept in this tile: skip its counters
    const int out0 = plan[0];
    const int eq0 = plan[1];
    const int64_t tbase = (int64_t)t * kTile;
    // counters are allocated for whole tiles; ids past n hold zero
    const uint4 *cb = reinterpret_cast<const uint4 *>(
        reinterpret_cast<const uint8_t *>(st.counters + (int64_t)q * words_per_query) + tbase +
        (int64_t)threadIdx.x * EM_PER);
    const uint32_t lrep = (uint32_t)l * 0x01010101u;
    uint4 v[EM_PER / 16];
    bool mine = false;
#pragma unroll
    for (int u = 0; u < EM_PER / 16; ++u) {
        v[u] = cb[u];
        mine |= (count_ge(v[u].x, lrep) | count_ge(v[u].y, lrep) | count_ge(v[u].z, lrep) |
                 count_ge(v[u].w, lrep)) != 0;
    }
    // the few threads holding candidates walk their 32 words in a loop (kept
    // rolled: fully unrolled byte loops overflow the instruction cache)
    uint32_t words[EM_PER / 4];
    if (mine) {
#pragma unroll
        for (int u = 0; u < EM_PER / 16; ++u) {
            words[4 * u + 0] = v[u].x;
            words[4 * u + 1] = v[u].y;
            words[4 * u + 2] = v[u].z;
            words[4 * u + 3] = v[u].w;
        }
    }
    int n_eq = 0;
    if (mine && cstar >= l) {
#pragma unroll 1
        for (int wi = 0; wi < EM_PER / 4; ++wi) {
            const uint32_t x = words[wi];
            if (!count_ge(x, lrep)) continue;
            for (int by = 0; by < 4; ++by) {
                const uint32_t b8 = (x >> (8 * by)) & 0xffu;
                n_eq += ((b8 & 0x7fu) == (uint32_t)cstar && !(b8 & 0x80u)) ? 1 : 0;
            }
        }
    }
    int eq_total;
    int r = eq0 + block_exclusive_scan<CL_THREADS>(n_eq, scan_tmp, &eq_total);
    int n_sel = 0;
    if (mine) {
        int rr = r;
#pragma unroll 1
        for (int wi = 0; wi < EM_PER / 4; ++wi) {
            const uint32_t x = words[wi];
            if (!count_ge(x, lrep)) continue;
            for (int by = 0; by < 4; ++by) {
                const uint32_t b8 = (x >> (8 * by)) & 0xffu;
                const int c = (int)(b8 & 0x7fu);
                if (c < l) continue;
                if ((b8 & 0x80u) || c > cstar) ++n_sel;
                else if (c == cstar) { n_sel += (rr < take_eq) ? 1 : 0; ++rr; }
            }
        }
    }
    int sel_total;
    int pos = out0 + block_exclusive_scan<CL_THREADS>(n_sel, scan_tmp, &sel_total);
    if (!mine) return;
    const int64_t id0 = tbase + (int64_t)threadIdx.x * EM_PER;
#pragma unroll 1
    for (int wi = 0; wi < EM_PER / 4; ++wi) {
        const uint32_t x = words[wi];
        if (!count_ge(x, lrep)) continue;
        for (int by = 0; by < 4; ++by) {
            const uint32_t b8 = (x >> (8 * by)) & 0xffu;
            const int c = (int)(b8 & 0x7fu);
            if (c < l) continue;
            bool sel;
            if ((b8 & 0x80u) || c > cstar) sel = true;
            else if (c == cstar) { sel = r < take_eq; ++r; }
            else sel = false;
            if (!sel) continue;
            if (pos < cap) {
                st.cand[(int64_t)q * cap + pos] = (int32_t)(id0 + wi * 4 + by);
                st.cand_col[(int64_t)q * cap + pos] = c;
            }
            ++pos;
        }
    }
    (void)n;
}

__global__ void candidates_out_kernel(const int32_t *__restrict__ cand,
                                      const int32_t *__restrict__ cand_col, int64_t total,
                                      int64_t *__restrict__ ids_out, int32_t *__restrict__ col_out)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        ids_out[e] = (int64_t)cand[e];
        if (col_out) col_out[e] = cand_col[e];
    }
}

__global__ void sum_i32_kernel(const int32_t *__restrict__ v, int n, unsigned long long *out)
{
    unsigned long long acc = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) acc += v[i];
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0 && acc) atomicAdd(out, acc);
}

}  // namespace

qw_status launch_sum_i32(const int32_t *v, int n, unsigned long long *out, cudaStream_t s)
{
    sum_i32_kernel<<<std::min(152, (n + 255) / 256 + 1), 256, 0, s>>>(v, n, out);
    QW_CUDA_TRY(cudaGetLastError());
    return QW_OK;
}

qw_status launch_candidates_out(const QueryState &st, int nb, int cap, int64_t *cand_ids,
                                int32_t *cand_col, cudaStream_t s)
{
    const int64_t total = (int64_t)nb * cap;
    int64_t blocks = std::min<int64_t>((total + 255) / 256, 152 * 8);
    candidates_out_kernel<<<(unsigned)blocks, 256, 0, s>>>(st.cand, st.cand_col, total, cand_ids,
                                                           cand_col);
    QW_CUDA_TRY(cudaGetLastError());
    return QW_OK;
}

qw_status launch_query_setup(const IndexView &ix, const int32_t *HQ, int nb, QueryState &st,
                             cudaStream_t s)
{
    QW_CUDA_TRY(cudaMemsetAsync(st.max_top, 0, sizeof(unsigned long long), s));
    query_setup_kernel<<<(nb + 127) / 128, 128, 0, s>>>(HQ, nb, ix.m, ix.o, ix.span, st);
    QW_CUDA_TRY(cudaGetLastError());
    return QW_OK;
}

// A learned first level never lies past the query's own last useful level,
// the first L with c^L > top (there the radius rule stops the plain path, and
// the level loops run at least that far for every query of the batch); a
// later prediction would leave the query unstarted.
__global__ void clamp_start_kernel(QueryState st, int nb, int cgrow)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nb) return;
    int L = 0;
    for (int64_t R = 1; R <= st.top[q]; R *= cgrow) ++L;
    if (st.start[q] > L) st.start[q] = L;
}

qw_status launch_clamp_start(int nb, QueryState &st, int cgrow, cudaStream_t s)
{
    if (nb == 0) return QW_OK;
    clamp_start_kernel<<<(nb + 127) / 128, 128, 0, s>>>(st, nb, cgrow);
    QW_CUDA_TRY(cudaGetLastError());
    return QW_OK;
}

qw_status launch_level(const IndexView &ix, int nb, int level, int64_t R, int64_t Rp, int l,
                       int cgrow, QueryState &st, cudaStream_t s, const LoopCtl *ctl)
{
    const int64_t wpq = (int64_t)ix.nT * kWordsPerTile;
    level_kernel<<<dim3((unsigned)ix.nT, (unsigned)nb), LV_THREADS, 0, s>>>(ix, level, R, Rp, l,
                                                                           cgrow, st, wpq, ctl);
    QW_CUDA_TRY(cudaGetLastError());
    return QW_OK;
}

qw_status launch_loop_init(LoopCtl *ctl, const QueryState &st, int nb, int cgrow, cudaStream_t s)
{
    loop_reset_kernel<<<1, 1, 0, s>>>(ctl);
    QW_CUDA_TRY(cudaGetLastError());
    loop_min_start_kernel<<<(nb + 255) / 256, 256, 0, s>>>(ctl, st, nb);
    QW_CUDA_TRY(cudaGetLastError());
    loop_init_kernel<<<1, 1, 0, s>>>(ctl, cgrow);
    QW_CUDA_TRY(cudaGetLastError());
    return QW_OK;
}

qw_status launch_loop_ctl(LoopCtl *ctl, const unsigned long long *max_top, int cgrow,
                          cudaGraphConditionalHandle h, int *err, cudaStream_t s)
{
    loop_ctl_kernel<<<1, 1, 0, s>>>(ctl, max_top, cgrow, h, err);
    QW_CUDA_TRY(cudaGetLastError());
    return QW_OK;
}

qw_status launch_fallback_graph(int nb, QueryState &st, LoopCtl *ctl, cudaGraphConditionalHandle h,
                                cudaStream_t s)
{
    fallback_kernel<<<(nb + 127) / 128, 128, 0, s>>>(nb, st);
    QW_CUDA_TRY(cudaGetLastError());
    second_pass_kernel<<<1, 1, 0, s>>>(st, ctl, h);
    QW_CUDA_TRY(cudaGetLastError());
    return QW_OK;
}

qw_status launch_fallback(int nb, QueryState &st, cudaStream_t s)
{
    fallback_kernel<<<(nb + 127) / 128, 128, 0, s>>>(nb, st);
    QW_CUDA_TRY(cudaGetLastError());
    return QW_OK;
}

qw_status launch_decide(int nb, int level, int64_t R, int cap, QueryState &st, cudaStream_t s,
                        LoopCtl *ctl, const ScanStats &ss)
{
    decide_kernel<<<(unsigned)(((int64_t)nb * 32 + 127) / 128), 128, 0, s>>>(nb, level, R, cap, st,
                                                                            ctl, ss);
    QW_CUDA_TRY(cudaGetLastError());
    return QW_OK;
}

qw_status launch_select_plan(const IndexView &ix, int nb, int l, int cap, QueryState &st,
                             int64_t *stats_out, cudaStream_t s)
{
    select_plan_kernel<<<nb, CL_THREADS, 0, s>>>(ix.nT, ix.m, l, cap, st, stats_out);
    QW_CUDA_TRY(cudaGetLastError());
    return QW_OK;
}

qw_status launch_collect(const IndexView &ix, int nb, int l, int cap, QueryState &st,
                         int64_t *stats_out, cudaStream_t s)
{
    const int64_t wpq = (int64_t)ix.nT * kWordsPerTile;
    QW_TRY(launch_select_plan(ix, nb, l, cap, st, stats_out, s));
    select_emit_kernel<<<dim3((unsigned)ix.nT, (unsigned)nb), CL_THREADS, 0, s>>>(ix.n, ix.nT, l, cap,
                                                                                st, wpq);
    QW_CUDA_TRY(cudaGetLastError());
    return QW_OK;
}

}  // namespace qw
