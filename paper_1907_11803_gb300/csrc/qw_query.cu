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
#include "qw_scan.cuh"

#include <algorithm>

namespace qw {
namespace {

constexpr int LV_THREADS = 256;
constexpr int kWordsPerTile = kTile / 4;

__device__ __forceinline__ int64_t floordiv64(int64_t a, int64_t R)
{
    int64_t q = a / R;
    if ((a % R != 0) && (a < 0)) --q;
    return q;
}

__device__ __forceinline__ int64_t clamp64(int64_t x, int64_t lo, int64_t hi)
{
    return x < lo ? lo : (x > hi ? hi : x);
}

// Offset (inside the tile's entry segment) of the first entry with bid >= x.
// The directory of a tile holds its distinct bids ub[0..cnt) ascending and the
// offset uo[] of each bid's first entry.  When every bid between ub[0] and x is
// present the answer sits at slot x - ub[0]; otherwise binary search.
__device__ __forceinline__ int dir_lower(const int32_t *__restrict__ ub,
                                         const int32_t *__restrict__ uo, int cnt, int len,
                                         int64_t x)
{
    if (cnt == 0) return 0;
    const int32_t b0 = ub[0];
    if (x <= b0) return 0;
    const int64_t p = x - b0;
    if (p < cnt && ub[p] == x) return uo[p];
    int lo = 0, hi = cnt;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if ((int64_t)ub[mid] < x) lo = mid + 1; else hi = mid;
    }
    return lo < cnt ? uo[lo] : len;
}

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
    atomicMax(st.max_top, (unsigned long long)top);
}

__global__ void __launch_bounds__(LV_THREADS) level_kernel(IndexView ix, int level, int64_t R,
                                                           int64_t Rp, int l, QueryState st,
                                                           int64_t words_per_query)
{
    __shared__ __align__(16) uint32_t cnt_s[kWordsPerTile];
    __shared__ int64_t seg_base[2 * QW_MAX_M];
    __shared__ int32_t seg_pref[2 * QW_MAX_M + 1];
    __shared__ int32_t red_cross;
    __shared__ unsigned long long red_scan;

    const int t = blockIdx.x;
    const int q = blockIdx.y;
    if (!st.active[q]) return;
    const int m = ix.m;
    const int64_t n = ix.n;
    const int64_t tbase = (int64_t)t * kTile;
    const int len = (int)min((int64_t)kTile, n - tbase);
    if (threadIdx.x == 0) {
        red_cross = 0;
        red_scan = 0;
    }

    // 1. flank boundaries of every projection (one thread per projection)
    unsigned long long my_scan = 0;
    int my_len0 = 0, my_len1 = 0;
    if (threadIdx.x < m) {
        const int i = threadIdx.x;
        const int64_t gi = st.g[(int64_t)q * m + i];
        const int64_t sp1 = (int64_t)ix.span[i] + 1;
        const int64_t dslot = (int64_t)i * ix.nT + t;
        const int32_t *ub = ix.dir_bid + ix.dir_start[dslot];
        const int32_t *uo = ix.dir_off + ix.dir_start[dslot];
        const int cnt = ix.dir_cnt[dslot];
        const int64_t lo = floordiv64(gi, R) * R;
        const int64_t A = clamp64(lo, 0, sp1), B = clamp64(lo + R, 0, sp1);
        const int pA = dir_lower(ub, uo, cnt, len, A);
        const int pB = dir_lower(ub, uo, cnt, len, B);
        int s0 = pA, e0 = pB, s1 = 0, e1 = 0;
        if (level > 0) {
            const int64_t lo2 = floordiv64(gi, Rp) * Rp;
            const int64_t A2 = clamp64(lo2, 0, sp1), B2 = clamp64(lo2 + Rp, 0, sp1);
            if (A2 < B2) {
                e0 = dir_lower(ub, uo, cnt, len, A2);
                s1 = dir_lower(ub, uo, cnt, len, B2);
                e1 = pB;
            }
        }
        my_len0 = e0 - s0;
        my_len1 = e1 - s1;
        const int64_t ebase = (int64_t)i * n + tbase;
        seg_base[2 * i] = ebase + s0;
        seg_base[2 * i + 1] = ebase + s1;
        my_scan = (unsigned long long)(pB - pA);
    }
    // prefix over the 2m segment lengths (m <= 127 fits in the first 4 warps)
    {
        __shared__ int32_t wsum[LV_THREADS / 32];
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        int v = my_len0 + my_len1;
        int incl = v;
        for (int off = 1; off < 32; off <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += y;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        int wbase = 0;
        for (int w2 = 0; w2 < warp; ++w2) wbase += wsum[w2];
        const int excl = wbase + incl - v;
        if (threadIdx.x < m) {
            seg_pref[2 * threadIdx.x] = excl;
            seg_pref[2 * threadIdx.x + 1] = excl + my_len0;
        }
        if (threadIdx.x == m - 1) seg_pref[2 * m] = excl + v;
    }
    if (my_scan) atomicAdd(&red_scan, my_scan);

    // 2. the tile's counters into shared memory; flag previous candidates
    uint4 *cg = reinterpret_cast<uint4 *>(st.counters + (int64_t)q * words_per_query +
                                          (int64_t)t * kWordsPerTile);
    uint4 *cs = reinterpret_cast<uint4 *>(cnt_s);
    const uint32_t lrep = (uint32_t)l * 0x01010101u;
    if (level == 0) {
        for (int w4 = threadIdx.x; w4 < kWordsPerTile / 4; w4 += LV_THREADS)
            cs[w4] = make_uint4(0, 0, 0, 0);
    } else {
        for (int w4 = threadIdx.x; w4 < kWordsPerTile / 4; w4 += LV_THREADS) {
            uint4 x = cg[w4];
            x.x |= __vcmpgeu4(x.x & 0x7f7f7f7fu, lrep) & 0x80808080u;
            x.y |= __vcmpgeu4(x.y & 0x7f7f7f7fu, lrep) & 0x80808080u;
            x.z |= __vcmpgeu4(x.z & 0x7f7f7f7fu, lrep) & 0x80808080u;
            x.w |= __vcmpgeu4(x.w & 0x7f7f7f7fu, lrep) & 0x80808080u;
            cs[w4] = x;
        }
    }
    __syncthreads();

    // 3. count every id in the flanks
    const int total = seg_pref[2 * m];
    int my_cross = 0;
    int s = 0;
    const uint32_t lm1 = (uint32_t)(l - 1);
    for (int e = threadIdx.x; e < total; e += LV_THREADS) {
        while (e >= seg_pref[s + 1]) ++s;
        const uint32_t id = ix.lid[seg_base[s] + (e - seg_pref[s])];
        const uint32_t sh = (id & 3u) << 3;
        const uint32_t old = atomicAdd(&cnt_s[id >> 2], 1u << sh);
        my_cross += (((old >> sh) & 0x7fu) == lm1) ? 1 : 0;
    }
    my_cross = __reduce_add_sync(0xffffffffu, my_cross);
    if ((threadIdx.x & 31) == 0 && my_cross) atomicAdd(&red_cross, my_cross);
    __syncthreads();

    // 4. counters back to global memory
    for (int w4 = threadIdx.x; w4 < kWordsPerTile / 4; w4 += LV_THREADS) cg[w4] = cs[w4];
    if (threadIdx.x == 0) {
        if (red_cross) atomicAdd(st.cross + q, red_cross);
        if (red_scan) atomicAdd(reinterpret_cast<unsigned long long *>(st.scan_level + q), red_scan);
    }
}

__global__ void decide_kernel(int nb, int level, int64_t R, int cap, QueryState st)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nb || !st.active[q]) return;
    const int32_t before = st.ncand[q];
    const int32_t nc = before + st.cross[q];
    st.cross[q] = 0;
    const int64_t sl = st.scan_level[q];
    st.scan_level[q] = 0;
    st.scan_last[q] = sl;
    st.scan_full[q] += sl;
    st.levels[q] = level + 1;
    st.finalR[q] = R;
    const bool enough = nc >= cap;        // the k + v bound (Section 3.1)
    const bool past = R > st.top[q];      // no further level can change C_R
    if (enough || past) {
        st.term[q] = enough ? 2 : 3;
        st.active[q] = 0;
        st.nprev[q] = before;
    }
    st.ncand[q] = nc;
}

constexpr int CL_THREADS = 256;
constexpr int CL_PER = 16;  // ids per thread per chunk (one 16-byte load)

// Select the kept candidates of one query: all ids with count >= l when there
// are at most k + v of them; otherwise the previous level's candidates, then
// by count descending, then by id ascending, up to k + v.  Emits ids in
// ascending order with their counts, and the query's statistics.
__global__ void __launch_bounds__(CL_THREADS) collect_kernel(
    int64_t n, int m, int l, int cap, QueryState st, int64_t words_per_query,
    int64_t *__restrict__ stats_out)
{
    __shared__ int hist[128];
    __shared__ int s_cstar, s_take_eq;
    __shared__ int scan_tmp[CL_THREADS / 32];
    const int q = blockIdx.x;
    const int nc = st.ncand[q];
    const int np = st.nprev[q];
    const uint8_t *cb = reinterpret_cast<const uint8_t *>(st.counters + (int64_t)q * words_per_query);
    const int64_t n16 = (n + 15) / 16 * 16;  // counters are padded to whole tiles

    if (threadIdx.x < 128) hist[threadIdx.x] = 0;
    if (threadIdx.x == 0) {
        s_cstar = l - 1;
        s_take_eq = 0;
    }
    __syncthreads();
    if (nc > cap) {
        for (int64_t base = (int64_t)threadIdx.x * CL_PER; base < n16;
             base += (int64_t)CL_THREADS * CL_PER) {
            uint4 v4 = *reinterpret_cast<const uint4 *>(cb + base);
            const uint8_t *bytes = reinterpret_cast<const uint8_t *>(&v4);
#pragma unroll
            for (int u = 0; u < CL_PER; ++u) {
                int c = bytes[u] & 0x7f;
                if (c >= l && !(bytes[u] & 0x80)) atomicAdd(&hist[c], 1);
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            const int need = cap - np;
            int acc = 0;
            for (int c = m; c >= l; --c) {
                if (acc + hist[c] >= need) {
                    s_cstar = c;
                    s_take_eq = need - acc;
                    break;
                }
                acc += hist[c];
            }
        }
        __syncthreads();
    }
    const int cstar = s_cstar, take_eq = s_take_eq;
    int eq_base = 0, out_base = 0;
    for (int64_t chunk = 0; chunk < n16; chunk += (int64_t)CL_THREADS * CL_PER) {
        const int64_t base = chunk + (int64_t)threadIdx.x * CL_PER;
        uint4 v4 = make_uint4(0, 0, 0, 0);
        if (base < n16) v4 = *reinterpret_cast<const uint4 *>(cb + base);
        const uint8_t *bytes = reinterpret_cast<const uint8_t *>(&v4);
        int n_eq = 0;
#pragma unroll
        for (int u = 0; u < CL_PER; ++u) {
            int c = bytes[u] & 0x7f;
            n_eq += (c == cstar && !(bytes[u] & 0x80) && c >= l) ? 1 : 0;
        }
        int eq_total;
        int eq_excl = block_exclusive_scan<CL_THREADS>(n_eq, scan_tmp, &eq_total);
        int rank = eq_base + eq_excl;
        uint16_t selmask = 0;
        int n_sel = 0;
#pragma unroll
        for (int u = 0; u < CL_PER; ++u) {
            int c = bytes[u] & 0x7f;
            bool prev = bytes[u] & 0x80;
            bool sel = false;
            if (c >= l) {
                if (prev || c > cstar) sel = true;
                else if (c == cstar) { sel = rank < take_eq; ++rank; }
            }
            if (sel) { selmask |= (uint16_t)(1u << u); ++n_sel; }
        }
        int sel_total;
        int pos = out_base + block_exclusive_scan<CL_THREADS>(n_sel, scan_tmp, &sel_total);
#pragma unroll
        for (int u = 0; u < CL_PER; ++u) {
            if (selmask & (1u << u)) {
                if (pos < cap) {
                    st.cand[(int64_t)q * cap + pos] = (int32_t)(base + u);
                    st.cand_col[(int64_t)q * cap + pos] = bytes[u] & 0x7f;
                }
                ++pos;
            }
        }
        eq_base += eq_total;
        out_base += sel_total;
    }
    if (threadIdx.x == 0) {
        const int keep = min(out_base, cap);
        st.nkeep[q] = keep;
        for (int p = keep; p < cap; ++p) {
            st.cand[(int64_t)q * cap + p] = -1;
            st.cand_col[(int64_t)q * cap + p] = 0;
        }
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

}  // namespace

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

qw_status launch_level(const IndexView &ix, int nb, int level, int64_t R, int64_t Rp, int l,
                       QueryState &st, cudaStream_t s)
{
    const int64_t wpq = (int64_t)ix.nT * kWordsPerTile;
    level_kernel<<<dim3((unsigned)ix.nT, (unsigned)nb), LV_THREADS, 0, s>>>(ix, level, R, Rp, l,
                                                                           st, wpq);
    QW_CUDA_TRY(cudaGetLastError());
    return QW_OK;
}

qw_status launch_decide(int nb, int level, int64_t R, int cap, QueryState &st, cudaStream_t s)
{
    decide_kernel<<<(nb + 127) / 128, 128, 0, s>>>(nb, level, R, cap, st);
    QW_CUDA_TRY(cudaGetLastError());
    return QW_OK;
}

qw_status launch_collect(const IndexView &ix, int nb, int l, int cap, QueryState &st,
                         int64_t *stats_out, cudaStream_t s)
{
    const int64_t wpq = (int64_t)ix.nT * kWordsPerTile;
    collect_kernel<<<nb, CL_THREADS, 0, s>>>(ix.n, ix.m, l, cap, st, wpq, stats_out);
    QW_CUDA_TRY(cudaGetLastError());
    return QW_OK;
}

}  // namespace qw
