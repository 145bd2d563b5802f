// qw_rerank.cu -- exact distances on the kept candidates and the top-k
// (Section 3: c-k-ANN returns the k objects nearest to q among those found;
// Section 1.2: the candidates are read from storage to remove false
// positives).
//
// One CTA per query.  Each warp streams whole candidate rows with 16-byte
// loads and forms the FP32 squared distance (per-lane fused multiply-add
// chains, then a butterfly sum).  For that summation order the FP32 result
// differs from the exact value by at most rho times the value, with
//   rho = (ceil(d / 32) + 12) * 2^-24 * 1.02,
// (at most ceil(d / 32) + 3 chained additions per lane, 5 butterfly levels, 2
// roundings of the difference and square) -- and the FP64 reference differs
// from the exact value by far less than the slack in that constant.
// After sorting by (FP32 distance, id), two neighbours whose FP32 gap is not
// larger than the sum of their bounds may be out of order.  Every maximal run
// of such neighbours that reaches into the first k positions is recomputed in
// FP64 with the reference summation order (index order, no fused
// multiply-add), and the array is re-sorted on (FP64 value if recomputed,
// FP32 value otherwise, id).  The runs are separated from everything else by
// certain gaps, so the first k ids are exactly those of the FP64 order, ties
// broken by the smaller id.
// Only a prefix of the sorted order matters: the positions up to the end of
// the run holding position k - 1.  Its last value T is found without sorting
// (radix selection of the k-th smallest FP32 value, then the next larger
// value while the gap to it is uncertain), and only the candidates with FP32
// distance <= T are sorted; the other stages see exactly that prefix.
#include "qw_internal.cuh"
#include "qw_scan.cuh"
#include "qw_tc.cuh"

#include <cuda_bf16.h>
#include <math_constants.h>

namespace qw {
namespace {

constexpr int RR_THREADS = 256;
constexpr int RR_WARPS = RR_THREADS / 32;

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// Warp sums of R per-lane values a[0..R) (R a power of two <= 32) in
// 5 + R - 1 - log2 R shuffles: at each of the first log2 R steps a lane
// keeps half of its values and adds its partner's half of the others.  Lane
// l returns the sum of value l >> (5 - log2 R) (every value's sum is a tree
// of 5 additions over the lanes' partial sums, as in warp_sum).
// One halving step: lanes with `off` set keep value hi and receive their
// partner's hi; the others keep lo and receive the partner's lo.
__device__ __forceinline__ float fold_pair(float lo, float hi, bool up, int off)
{
    const float send = up ? lo : hi;
    return (up ? hi : lo) + __shfl_xor_sync(0xffffffffu, send, off);
}

template <int R>
__device__ __forceinline__ float rows_sum(const float (&a)[R], int lane)
{
    static_assert(R == 2 || R == 4 || R == 8, "rows per warp: 2, 4 or 8");
    float v;
    if constexpr (R == 2) {
        v = fold_pair(a[0], a[1], (lane & 16) != 0, 16);
    } else if constexpr (R == 4) {
        const bool u = (lane & 16) != 0;
        const float b0 = fold_pair(a[0], a[2], u, 16), b1 = fold_pair(a[1], a[3], u, 16);
        v = fold_pair(b0, b1, (lane & 8) != 0, 8);
    } else {
        const bool u = (lane & 16) != 0;
        const float b0 = fold_pair(a[0], a[4], u, 16), b1 = fold_pair(a[1], a[5], u, 16);
        const float b2 = fold_pair(a[2], a[6], u, 16), b3 = fold_pair(a[3], a[7], u, 16);
        const bool u2 = (lane & 8) != 0;
        const float c0 = fold_pair(b0, b2, u2, 8), c1 = fold_pair(b1, b3, u2, 8);
        v = fold_pair(c0, c1, (lane & 4) != 0, 4);
    }
#pragma unroll
    for (int off = 16 / R; off >= 1; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// Shared-memory arrays of one query's rerank (P2 entries each), and small
// scratch: scan_tmp (RR_WARPS ints), hist (256 ints), bc (4 ints).
struct RerankSmem {
    double *key;
    float *d32;
    float *outd;
    int32_t *sid;
    uint8_t *mark;
    int *scan_tmp;
    int *any_mark;
    int *hist;
    int *bc;
};

// Bitonic sort of P (a power of two) (key, id) pairs on (key, id), by the
// whole block, or by warp 0 alone when `one_warp` (the other warps skip it;
// the caller synchronises the block afterwards).
__device__ __forceinline__ void sort_pairs(float *kf, int32_t *id, int P, bool one_warp)
{
    const int step = one_warp ? 32 : RR_THREADS;
    if (one_warp && threadIdx.x >= 32) return;
    for (int kk = 2; kk <= P; kk <<= 1) {
        for (int jj = kk >> 1; jj > 0; jj >>= 1) {
            for (int x = threadIdx.x; x < (P >> 1); x += step) {
                const int a = 2 * x - (x & (jj - 1));
                const int c = a + jj;
                const bool up = (a & kk) == 0;
                const float ka = kf[a], kc = kf[c];
                const int32_t ia = id[a], ic = id[c];
                const bool gt = (ka > kc) || (ka == kc && ia > ic);
                if (gt == up) {
                    kf[a] = kc;
                    kf[c] = ka;
                    id[a] = ic;
                    id[c] = ia;
                }
            }
            if (one_warp) __syncwarp();
            else __syncthreads();
        }
    }
}

// Smallest of the n values above t, as bits (0xffffffff: none).  Block-wide.
__device__ uint32_t min_above(const float *v, int n, float t, int *bc)
{
    uint32_t mn = 0xffffffffu;
    for (int j = threadIdx.x; j < n; j += RR_THREADS)
        if (v[j] > t) mn = min(mn, __float_as_uint(v[j]));
    mn = __reduce_min_sync(0xffffffffu, mn);
    if (threadIdx.x == 0) bc[2] = (int)0xffffffffu;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) atomicMin(reinterpret_cast<unsigned int *>(bc + 2), mn);
    __syncthreads();
    const uint32_t r = (uint32_t)bc[2];
    __syncthreads();
    return r;
}

// Stages 1-6 for the nc candidates whose ids are in sm.sid[0..nc), using P2
// (a power of two >= nc) slots; writes the query's k results.
// row_of (optional): the row of data id `id` in X is row_of[id] (X in the
// bitmap path's locality order), else id.
template <int kRows>
__device__ void rerank_finish(const float *__restrict__ X, const int32_t *__restrict__ row_of,
                              int d, const float *__restrict__ qv,
                              int k, int P2, int nc, RerankSmem sm, int64_t *__restrict__ ids_q,
                              float *__restrict__ dists_q, bool vec)
{
    double *key = sm.key;
    float *d32 = sm.d32;
    float *outd = sm.outd;
    int32_t *sid = sm.sid;
    uint8_t *mark = sm.mark;
    int *scan_tmp = sm.scan_tmp;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) *sm.any_mark = 0;
    const double rho = (double)((d + 31) / 32 + 12) * 5.9604644775390625e-08 * 1.02;
    const float rhof = (float)(rho * (1.0 + 9.5367431640625e-07));

    // 0. the data row of every candidate (staged in `key`, free until stage 4)
    int32_t *rowi = reinterpret_cast<int32_t *>(key);
    for (int j = threadIdx.x; j < nc; j += RR_THREADS) rowi[j] = row_of ? row_of[sid[j]] : sid[j];
    __syncthreads();

    // 1. FP32 squared distances: a warp takes kRows candidate rows at a time,
    //    so each lane has kRows independent loads in flight; every row keeps
    //    its own per-lane chain and butterfly sum (the order rho covers)
    for (int j0 = warp * kRows; j0 < nc; j0 += RR_WARPS * kRows) {
        const float *xr[kRows];
        float acc[kRows];
#pragma unroll
        for (int u = 0; u < kRows; ++u) {
            const int j = j0 + u;
            xr[u] = j < nc ? X + (int64_t)rowi[j] * d : nullptr;
            acc[u] = 0.0f;
        }
        if (vec) {
            const float4 *q4 = reinterpret_cast<const float4 *>(qv);
            for (int c = lane; c < (d >> 2); c += 32) {
                const float4 b = __ldg(q4 + c);
                float4 a[kRows];
#pragma unroll
                for (int u = 0; u < kRows; ++u)
                    a[u] = xr[u] ? __ldg(reinterpret_cast<const float4 *>(xr[u]) + c)
                                 : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                for (int u = 0; u < kRows; ++u) {
                    const float t0 = a[u].x - b.x, t1 = a[u].y - b.y, t2 = a[u].z - b.z,
                                t3 = a[u].w - b.w;
                    acc[u] = fmaf(t0, t0, acc[u]);
                    acc[u] = fmaf(t1, t1, acc[u]);
                    acc[u] = fmaf(t2, t2, acc[u]);
                    acc[u] = fmaf(t3, t3, acc[u]);
                }
            }
        } else {
            for (int c = lane; c < d; c += 32) {
                const float qc = __ldg(qv + c);
#pragma unroll
                for (int u = 0; u < kRows; ++u) {
                    const float t0 = xr[u] ? __ldg(xr[u] + c) - qc : 0.0f;
                    acc[u] = fmaf(t0, t0, acc[u]);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < kRows; ++u) {
            const int j = j0 + u;
            const float sum = warp_sum(acc[u]);
            if (lane == 0 && j < nc) d32[j] = sum;
        }
    }
    __syncthreads();

    // 2. the prefix of the (FP32 distance, id) order that decides the result:
    //    T = the k-th smallest distance, extended while the gap to the next
    //    larger distance is uncertain (at most kExtend times, else the whole
    //    array is sorted); the candidates with distance <= T, sorted
    constexpr int kExtend = 16;
    bool whole = nc <= k;
    if (!whole) {
        // non-negative FP32 values are ordered like their bit patterns
        float T = __uint_as_float(block_kth_smallest<RR_THREADS>(
            reinterpret_cast<const uint32_t *>(d32), nc, k, sm.hist, sm.bc));
        whole = true;
        for (int it = 0; it < kExtend; ++it) {
            const uint32_t nb = min_above(d32, nc, T, sm.bc);
            const float b = __uint_as_float(nb);
            if (nb == 0xffffffffu || !((b - T) <= rhof * (T + b))) {
                whole = false;
                break;
            }
            T = b;
        }
        if (!whole) {
            // compact, in list order, into (outd, key as ids); sort; copy back
            float *db = outd;
            int32_t *ib = reinterpret_cast<int32_t *>(key);
            const int per0 = (nc + RR_THREADS - 1) / RR_THREADS;
            const int a0 = min(nc, (int)threadIdx.x * per0), a1 = min(nc, a0 + per0);
            int mine = 0;
            for (int j = a0; j < a1; ++j) mine += d32[j] <= T ? 1 : 0;
            int ns;
            int pos = block_exclusive_scan<RR_THREADS>(mine, sm.scan_tmp, &ns);
            for (int j = a0; j < a1; ++j)
                if (d32[j] <= T) {
                    db[pos] = d32[j];
                    ib[pos] = sid[j];
                    ++pos;
                }
            int P2s = 2;
            while (P2s < ns) P2s <<= 1;
            for (int j = ns + threadIdx.x; j < P2s; j += RR_THREADS) {
                db[j] = CUDART_INF_F;
                ib[j] = INT32_MAX;
            }
            __syncthreads();
            sort_pairs(db, ib, P2s, P2s <= 256);
            __syncthreads();
            for (int j = threadIdx.x; j < P2s; j += RR_THREADS) {
                d32[j] = db[j];
                sid[j] = ib[j];
            }
            __syncthreads();
            nc = ns;
            P2 = P2s;
        }
    }
    if (whole) {
        for (int j = nc + threadIdx.x; j < P2; j += RR_THREADS) {
            d32[j] = CUDART_INF_F;
            sid[j] = INT32_MAX;
        }
        __syncthreads();
        sort_pairs(d32, sid, P2, false);
    }

    // 3. runs of neighbours whose order FP32 cannot certify.  The test runs in
    //    FP32 with the bound raised by 2^-20: fl(b - a) and fl(rho (a + b)) are
    //    each within one rounding of the real values, so every pair the real
    //    test flags is flagged here
    const int per = (P2 + RR_THREADS - 1) / RR_THREADS;
    const int j0 = threadIdx.x * per;
    const int j1 = min(P2, j0 + per);
    auto gap_uncertain = [&](int j) -> bool {  // between j and j + 1
        if (j < 0 || j + 1 >= nc) return false;
        const float a = d32[j], b = d32[j + 1];
        return (b - a) <= rhof * (a + b);
    };
    int last_start = -1;
    for (int j = j0; j < j1; ++j)
        if (j == 0 || !gap_uncertain(j - 1)) last_start = j;
    int run_start = block_exclusive_max<RR_THREADS>(last_start, -1, scan_tmp);
    int nmark = 0;
    for (int j = j0; j < j1; ++j) {
        if (j == 0 || !gap_uncertain(j - 1)) run_start = j;
        bool mk = (j < nc) && (run_start < k) && (gap_uncertain(j - 1) || gap_uncertain(j));
        mark[j] = mk ? 1 : 0;
        nmark += mk ? 1 : 0;
    }
    if (nmark) atomicAdd(sm.any_mark, nmark);
    __syncthreads();

    // 4. FP64 recomputation of the marked runs, in the reference order
    for (int j = threadIdx.x; j < P2; j += RR_THREADS) {
        if (j < nc && mark[j]) {
            const float *x = X + (int64_t)(row_of ? row_of[sid[j]] : sid[j]) * d;
            double s = 0.0;
            for (int c = 0; c < d; ++c) {
                double t = __dsub_rn((double)x[c], (double)qv[c]);
                s = __dadd_rn(s, __dmul_rn(t, t));
            }
            key[j] = s;
            outd[j] = (float)sqrt(s);
        } else {
            key[j] = (j < nc) ? (double)d32[j] : CUDART_INF;
            outd[j] = (j < nc) ? sqrtf(d32[j]) : CUDART_INF_F;
        }
    }
    __syncthreads();

    // 5. re-sort every recomputed run on (FP64 value, id).  Runs are bounded by
    //    certain gaps, across which the FP64 values keep the FP32 order, so
    //    sorting each run in place equals re-sorting the whole array
    if (*sm.any_mark) {
        for (int j = threadIdx.x; j < nc; j += RR_THREADS) {
            if (!mark[j] || (j > 0 && mark[j - 1] && gap_uncertain(j - 1))) continue;
            int e = j + 1;
            while (e < nc && mark[e] && gap_uncertain(e - 1)) ++e;
            for (int a = j + 1; a < e; ++a) {  // insertion sort of [j, e)
                const double ka = key[a];
                const int32_t ia = sid[a];
                const float oa = outd[a];
                int b = a - 1;
                while (b >= j && (key[b] > ka || (key[b] == ka && sid[b] > ia))) {
                    key[b + 1] = key[b];
                    sid[b + 1] = sid[b];
                    outd[b + 1] = outd[b];
                    --b;
                }
                key[b + 1] = ka;
                sid[b + 1] = ia;
                outd[b + 1] = oa;
            }
        }
        __syncthreads();
    }

    // 6. the k nearest
    for (int j = threadIdx.x; j < k; j += RR_THREADS) {
        const bool have = j < nc;
        ids_q[j] = have ? (int64_t)sid[j] : -1;
        dists_q[j] = have ? outd[j] : CUDART_INF_F;
    }
}


__device__ __forceinline__ RerankSmem carve_rerank(unsigned char *base, int P2, int *scan_tmp,
                                                   int *any_mark, int *hist, int *bc)
{
    RerankSmem r;
    r.key = reinterpret_cast<double *>(base);
    r.d32 = reinterpret_cast<float *>(r.key + P2);
    r.outd = r.d32 + P2;
    r.sid = reinterpret_cast<int32_t *>(r.outd + P2);
    r.mark = reinterpret_cast<uint8_t *>(r.sid + P2);
    r.scan_tmp = scan_tmp;
    r.any_mark = any_mark;
    r.hist = hist;
    r.bc = bc;
    return r;
}

template <int kRows>
__global__ void __launch_bounds__(RR_THREADS) rerank_kernel(
    const float *__restrict__ X, const int32_t *__restrict__ row_of, int d,
    const float *__restrict__ Qb, int k, int cap, int P2,
    const int32_t *__restrict__ cand, const int32_t *__restrict__ nkeep,
    int64_t *__restrict__ ids_out, float *__restrict__ dists_out, bool vec)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ int scan_tmp[RR_WARPS];
    __shared__ int any_mark;
    __shared__ int hist[256];
    __shared__ int bc[4];
    RerankSmem sm = carve_rerank(smraw, P2, scan_tmp, &any_mark, hist, bc);
    const int q = blockIdx.x;
    const int nc = nkeep[q];
    const int32_t *cl = cand + (int64_t)q * cap;
    for (int j = threadIdx.x; j < nc; j += RR_THREADS) sm.sid[j] = cl[j];
    __syncthreads();
    rerank_finish<kRows>(X, row_of, d, Qb + (int64_t)q * d, k, P2, nc, sm, ids_out + (int64_t)q * k,
                  dists_out + (int64_t)q * k, vec);
}

// BF16 pre-filter.  Distances to every kept candidate are first bounded from
// the index's residual BF16 copy (half the bytes of the rows): row r of the
// rerank's row order is stored as r~ = bf16(r), r = fl32(x - C_g), C_g the
// mean of its 128-row group g = r / 128 rounded to BF16 (in the locality order
// the group is spatially compact, so |r| is about the group's spread).  With
// u' = q - C_g and w' = u' - r~ (both exact),
//   |w'|^2 = |q - C_g|^2 - 2 q.r~ + 2 C_g.r~ + |r~|^2,
// so the only per-candidate dot product is q.r~, over the BF16 row alone:
// FP32 FMA chains per lane and a butterfly sum (each BF16 value is exact in
// FP32), |P - q.r~| <= gam |q| |r~| with gam >= 1.02 (ceil(d / 32) + 8) 2^-24.
// C_g.r~ and |r~|^2 are per-row constants computed at build time in FP64 and
// rounded to FP32; S = |q - C_g|^2 is computed once per distinct group of the
// query's candidates (FP32 chains, relative error rho_s).  The computed
// a = ((S - 2P) + 2 C_g.r~) + |r~|^2 then satisfies
// | a - |w'|^2 | <= E2 = rho_s S + 2 gam |q| R~ + 2^-23 |C_g| R~ + 2^-24 |r~|^2
//                       + 3.03 2^-24 (S + 2|P| + 2|C_g.r~| + |r~|^2),
// with R~ = 1.004 R >= |r~| (R >= |r| is stored per row) and |C_g| <= |q| +
// |q - C_g|.  And | |q - x| - |w'| | <= |(x - C_g) - r| + |r - r~| <= 1.001
// (2^-24 + 2^-8) R = e.  Hence |q - x| lies in [max(0, W_lo - e), W_hi + e],
// W_lo / W_hi the square roots of max(0, a - E2) and a + E2; every bound is
// formed in FP32 with relative margins of 2^-18 or more that cover the
// rounding of the bound arithmetic itself (rsqrtf: 2 ulp).  A candidate whose
// lower bound exceeds the k-th smallest upper bound cannot be among the k
// nearest (the k candidates with the smallest upper bounds all lie within
// it); all others go through the exact FP32 + FP64 stages on the FP32 rows, so
// the result is the same as without the pre-filter.
__device__ __forceinline__ uint32_t group_slot(int32_t g, int P2)
{
    return ((uint32_t)g * 2654435761u) & (uint32_t)(P2 - 1);
}

// The candidates' distinct groups into the open-addressed table gkey (P2
// slots, -1 empty; at most nc <= P2 distinct groups, so an insertion ends
// within P2 probes); the insertion that takes a slot appends it to glist
// (*ngroups, zero on entry).  Then |q - C_g|^2 of each listed slot.
__device__ __forceinline__ void group_norms(const int32_t *rowi, int nc, int P2, int32_t *gkey,
                                            float *gS, int32_t *glist, int *ngroups,
                                            const __nv_bfloat16 *__restrict__ Cg,
                                            const float *__restrict__ qv, int d)
{
    // 16-byte loads of the query and of the group means when aligned
    const bool vec16 = (d % 8 == 0) && (((uintptr_t)qv | (uintptr_t)Cg) % 16 == 0);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int j = threadIdx.x; j < nc; j += RR_THREADS) {
        const int32_t g = rowi[j] >> 7;
        uint32_t h = group_slot(g, P2);
        for (int p = 0; p < P2; ++p) {
            const int32_t old = atomicCAS(&gkey[h], -1, g);
            if (old == -1) {
                glist[atomicAdd(ngroups, 1)] = (int32_t)h;
                break;
            }
            if (old == g) break;
            h = (h + 1) & (uint32_t)(P2 - 1);
        }
    }
    __syncthreads();
    // a warp takes kG listed groups at a time, their rows' loads in flight
    // together
    constexpr int kG = 8;
    const int G = *ngroups;
    for (int base = warp * kG; base < G; base += RR_WARPS * kG) {
        int32_t sl[kG];
        float acc[kG];
        const __nv_bfloat16 *cg[kG];
#pragma unroll
        for (int u = 0; u < kG; ++u) {
            sl[u] = base + u < G ? glist[base + u] : -1;
            acc[u] = 0.0f;
            cg[u] = Cg + (int64_t)(sl[u] >= 0 ? gkey[sl[u]] : 0) * d;
        }
        if (vec16) {
            for (int c = lane; c < (d >> 3); c += 32) {
                const float4 b0 = __ldg(reinterpret_cast<const float4 *>(qv) + 2 * c);
                const float4 b1 = __ldg(reinterpret_cast<const float4 *>(qv) + 2 * c + 1);
                const float qc[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
                uint4 raw[kG];
#pragma unroll
                for (int u = 0; u < kG; ++u)
                    raw[u] = sl[u] >= 0 ? __ldg(reinterpret_cast<const uint4 *>(cg[u]) + c)
                                        : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
                for (int u = 0; u < kG; ++u) {
                    const uint32_t wv[4] = {raw[u].x, raw[u].y, raw[u].z, raw[u].w};
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        const float gvv = __uint_as_float((e & 1) ? (wv[e >> 1] & 0xffff0000u)
                                                                  : (wv[e >> 1] << 16));
                        const float t = __fsub_rn(qc[e], gvv);
                        acc[u] = fmaf(t, t, acc[u]);
                    }
                }
            }
        } else {
            for (int c = lane; c < d; c += 32) {
                const float qc = __ldg(qv + c);
                float gv[kG];
#pragma unroll
                for (int u = 0; u < kG; ++u) gv[u] = sl[u] >= 0 ? __bfloat162float(cg[u][c]) : 0.0f;
#pragma unroll
                for (int u = 0; u < kG; ++u) {
                    const float t = __fsub_rn(qc, gv[u]);
                    acc[u] = fmaf(t, t, acc[u]);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < kG; ++u) {
            const float sum = warp_sum(acc[u]);
            if (lane == 0 && sl[u] >= 0) gS[sl[u]] = sum;
        }
    }
}

__device__ __forceinline__ float group_norm_of(const int32_t *gkey, const float *gS, int P2,
                                               int32_t g)
{
    uint32_t h = group_slot(g, P2);
    for (int p = 0; p < P2; ++p) {
        if (gkey[h] == g) return gS[h];
        h = (h + 1) & (uint32_t)(P2 - 1);
    }
    return 0.0f;  // not reached: every candidate's group was inserted
}

// Squared-distance bounds (lo2, hi2) of a candidate from P = q.r~ (above).
__device__ __forceinline__ void expanded_bounds(float P, float S, float2 cr, float R, float qn,
                                                float rho_s, float gam, float &lo2, float &hi2)
{
    const float a = __fadd_rn(__fadd_rn(__fsub_rn(S, 2.0f * P), 2.0f * cr.x), cr.y);
    const float Rt = R * 1.004f;
    const float Cn = qn + sqrtf(S) * 1.01f;
    const float absum = S + 2.0f * fabsf(P) + 2.0f * fabsf(cr.x) + cr.y;
    const float E2 = 1.01f * (rho_s * S + 2.0f * gam * qn * Rt + 0x1p-23f * Cn * Rt +
                              0x1p-24f * cr.y + 3.03f * 0x1p-24f * absum);
    const float tlo = fmaxf(a - E2, 0.0f) * (1.0f - 0x1p-20f);
    const float thi = (a + E2) * (1.0f + 0x1p-20f);
    const float wlo = tlo > 0.0f ? tlo * rsqrtf(tlo) : 0.0f;
    const float whi = thi > 0.0f ? thi * rsqrtf(thi) : 0.0f;
    const float e = 1.001f * 0x1.02p-8f * R;
    const float lo = fmaxf(wlo * (1.0f - 0x1p-18f) - e * (1.0f + 0x1p-18f), 0.0f);
    const float hi = (whi + e) * (1.0f + 0x1p-18f);
    lo2 = lo * lo * (1.0f - 0x1p-18f);
    hi2 = hi * hi * (1.0f + 0x1p-18f);
}

template <int kRows>
__global__ void __launch_bounds__(RR_THREADS) rerank_bf16_kernel(
    const float *__restrict__ Xr, const int32_t *__restrict__ row_of,
    const __nv_bfloat16 *__restrict__ Rb, const float *__restrict__ rnorm,
    const float2 *__restrict__ rcr, const __nv_bfloat16 *__restrict__ Cg, int d,
    const float *__restrict__ Qb, int k, int cap, int P2, const int32_t *__restrict__ cand,
    const int32_t *__restrict__ nkeep, int64_t *__restrict__ ids_out,
    float *__restrict__ dists_out, bool vec, bool vec8, bool vec16, float rho_s, float gam,
    unsigned long long *__restrict__ rows_fp32)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ int scan_tmp[RR_WARPS];
    __shared__ int any_mark;
    __shared__ int hist[256];
    __shared__ int bc[4];
    __shared__ float s_qq;
    __shared__ int s_ngroups;
    __shared__ int hist2[2048];
    RerankSmem sm = carve_rerank(smraw, P2, scan_tmp, &any_mark, hist, bc);
    int32_t *cid = reinterpret_cast<int32_t *>(sm.mark + P2 + 15 - ((P2 + 15) % 16));  // P2 ids
    int32_t *gkey = reinterpret_cast<int32_t *>(sm.key);  // P2 group slots (-1: empty)
    float *gS = reinterpret_cast<float *>(sm.key) + P2;    // |q - C_g|^2 per slot
    int32_t *rowi = sm.sid;                               // row of every candidate
    const int q = blockIdx.x;
    const int nc = nkeep[q];
    const float *qv = Qb + (int64_t)q * d;
    const int32_t *cl = cand + (int64_t)q * cap;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    // 0. ids, rows, empty group slots, |q|^2
    for (int j = threadIdx.x; j < nc; j += RR_THREADS) {
        const int32_t id = cl[j];
        cid[j] = id;
        rowi[j] = row_of ? row_of[id] : id;
    }
    for (int sl = threadIdx.x; sl < P2; sl += RR_THREADS) gkey[sl] = -1;
    if (threadIdx.x == 0) s_ngroups = 0;
    if (warp == 0) {
        float s = 0.0f;
        for (int c = lane; c < d; c += 32) s = fmaf(__ldg(qv + c), __ldg(qv + c), s);
        s = warp_sum(s);
        if (lane == 0) s_qq = s;
    }
    __syncthreads();
    // 1. |q - C_g|^2 per distinct group (the group list in d32, free until A)
    group_norms(rowi, nc, P2, gkey, gS, reinterpret_cast<int32_t *>(sm.d32), &s_ngroups, Cg, qv,
                d);
    __syncthreads();
    const float qn = sqrtf(s_qq) * 1.01f;  // >= |q|

    // A. q.r~ into d32.  A warp takes kRows candidates at a time (kRows
    //    independent row loads per lane in flight, 8 or 16 bytes each).
    //    The query's 16-byte chunks c = lane + 32 i (i < kQReg) stay in registers.
    //    (16-byte form: chunk c = lane + 32 i of 8 coordinates in qreg[2i],
    //    qreg[2i + 1])
    constexpr int kQReg = 4;
    const int nch4 = d >> 2;
    float4 qreg[kQReg];
#pragma unroll
    for (int i = 0; i < kQReg; ++i) {
        const int c = vec16 ? 2 * (lane + 32 * (i >> 1)) + (i & 1) : lane + 32 * i;
        qreg[i] = ((vec16 || vec8) && c < nch4) ? __ldg(reinterpret_cast<const float4 *>(qv) + c)
                                                : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    for (int j0 = warp * kRows; j0 < nc; j0 += RR_WARPS * kRows) {
        int64_t row[kRows];
        float acc[kRows];
#pragma unroll
        for (int u = 0; u < kRows; ++u) {
            const int j = j0 + u;
            row[u] = j < nc ? (int64_t)rowi[j] : -1;
            acc[u] = 0.0f;
        }
        if (vec16) {
            // d a multiple of 256: lane chunks c = lane + 32 i of 8 BF16 each
            const uint4 *r4[kRows];
#pragma unroll
            for (int u = 0; u < kRows; ++u)
                r4[u] = reinterpret_cast<const uint4 *>(Rb + (row[u] >= 0 ? row[u] : row[0]) * d);
            auto chunk8 = [&](int c, const float4 b0, const float4 b1) {
                uint4 raw[kRows];
#pragma unroll
                for (int u = 0; u < kRows; ++u) raw[u] = __ldg(r4[u] + c);
#pragma unroll
                for (int u = 0; u < kRows; ++u) {
                    acc[u] = fmaf(b0.x, __uint_as_float(raw[u].x << 16), acc[u]);
                    acc[u] = fmaf(b0.y, __uint_as_float(raw[u].x & 0xffff0000u), acc[u]);
                    acc[u] = fmaf(b0.z, __uint_as_float(raw[u].y << 16), acc[u]);
                    acc[u] = fmaf(b0.w, __uint_as_float(raw[u].y & 0xffff0000u), acc[u]);
                    acc[u] = fmaf(b1.x, __uint_as_float(raw[u].z << 16), acc[u]);
                    acc[u] = fmaf(b1.y, __uint_as_float(raw[u].z & 0xffff0000u), acc[u]);
                    acc[u] = fmaf(b1.z, __uint_as_float(raw[u].w << 16), acc[u]);
                    acc[u] = fmaf(b1.w, __uint_as_float(raw[u].w & 0xffff0000u), acc[u]);
                }
            };
            const int nch8 = d >> 3;
#pragma unroll
            for (int i = 0; i < kQReg / 2; ++i) {
                const int c = lane + 32 * i;
                if (c < nch8) chunk8(c, qreg[2 * i], qreg[2 * i + 1]);
            }
            for (int c = lane + 32 * (kQReg / 2); c < nch8; c += 32)
                chunk8(c, __ldg(reinterpret_cast<const float4 *>(qv) + 2 * c),
                       __ldg(reinterpret_cast<const float4 *>(qv) + 2 * c + 1));
        } else if (vec8) {
            const uint2 *r2[kRows];
#pragma unroll
            for (int u = 0; u < kRows; ++u)
                r2[u] = reinterpret_cast<const uint2 *>(Rb + (row[u] >= 0 ? row[u] : row[0]) * d);
            // one 16-byte chunk of the query against 4 BF16 of each row
            auto chunk = [&](int c, const float4 b) {
                uint2 raw[kRows];
#pragma unroll
                for (int u = 0; u < kRows; ++u) raw[u] = __ldg(r2[u] + c);
#pragma unroll
                for (int u = 0; u < kRows; ++u) {
                    acc[u] = fmaf(b.x, __uint_as_float(raw[u].x << 16), acc[u]);
                    acc[u] = fmaf(b.y, __uint_as_float(raw[u].x & 0xffff0000u), acc[u]);
                    acc[u] = fmaf(b.z, __uint_as_float(raw[u].y << 16), acc[u]);
                    acc[u] = fmaf(b.w, __uint_as_float(raw[u].y & 0xffff0000u), acc[u]);
                }
            };
#pragma unroll
            for (int i = 0; i < kQReg; ++i) {
                const int c = lane + 32 * i;
                if (c < nch4) chunk(c, qreg[i]);
            }
            for (int c = lane + 32 * kQReg; c < nch4; c += 32)
                chunk(c, __ldg(reinterpret_cast<const float4 *>(qv) + c));
        } else {
            for (int c = lane; c < d; c += 32) {
                const float qc = __ldg(qv + c);
#pragma unroll
                for (int u = 0; u < kRows; ++u)
                    if (row[u] >= 0) acc[u] = fmaf(qc, __bfloat162float(Rb[row[u] * d + c]), acc[u]);
            }
        }
        // lanes 32 / kRows * u ... hold row u's sum
        const float P = rows_sum<kRows>(acc, lane);
        const int jm = j0 + lane / (32 / kRows);
        if ((lane % (32 / kRows)) == 0 && jm < nc) sm.d32[jm] = P;
    }
    __syncthreads();
    // A2. the bounds, one candidate per thread (d32 <- lower, outd <- upper)
    for (int j = threadIdx.x; j < nc; j += RR_THREADS) {
        const int64_t row = rowi[j];
        const float S = group_norm_of(gkey, gS, P2, (int32_t)(row >> 7));
        float lo2, hi2;
        expanded_bounds(sm.d32[j], S, __ldg(rcr + row), __ldg(rnorm + row), qn, rho_s, gam,
                        lo2, hi2);
        sm.d32[j] = lo2;
        sm.outd[j] = hi2;
    }
    __syncthreads();
    // B. a bound uk >= the k-th smallest upper bound (non-negative: ordered like
    //    its bits; at most 2^-13 above it): every candidate among the k nearest
    //    has its lower bound <= uk
    float uk = CUDART_INF_F;
    if (nc > k)
        uk = __uint_as_float(block_kth_upper<RR_THREADS>(
            reinterpret_cast<const uint32_t *>(sm.outd), nc, k, hist2, sm.bc));
    // C. keep the candidates that could be among the k nearest, in list order
    //    (the rows array in sid is no longer read)
    const int per = (nc + RR_THREADS - 1) / RR_THREADS;
    const int j0 = min(nc, (int)threadIdx.x * per), j1 = min(nc, j0 + per);
    int mine = 0;
    for (int j = j0; j < j1; ++j) mine += (sm.d32[j] <= uk) ? 1 : 0;
    int ns;
    int pos = block_exclusive_scan<RR_THREADS>(mine, sm.scan_tmp, &ns);
    for (int j = j0; j < j1; ++j)
        if (sm.d32[j] <= uk) sm.sid[pos++] = cid[j];
    __syncthreads();
    if (rows_fp32 && threadIdx.x == 0) atomicAdd(rows_fp32, (unsigned long long)ns);
    int P2s = 2;
    while (P2s < ns) P2s <<= 1;
    rerank_finish<kRows>(Xr, row_of, d, qv, k, P2s, ns, sm, ids_out + (int64_t)q * k,
                  dists_out + (int64_t)q * k, vec);
}

// BF16 pre-filter on the tensor cores.  The same residual copy, expansion and
// bounds as rerank_bf16_kernel, but q.r~ is an MMA: a tile of 128 candidates'
// residual rows (A, M = 128, K = the dimension padded to 16) against the query
// split into BF16 hi and lo parts (B, N = 16, two columns used); the BF16
// products are exact in FP32, and the tensor cores accumulate in FP32 in
// tensor memory.  The dot product's coefficient gam becomes cP = 2^-16 (the
// split of q) + 1.02 (K - 1) 2^-22 (the tensor cores' FP32 additions, reading
// R15) + 2^-23.  A tensor-core wait that gives up marks every candidate of the
// query as a survivor (the result is still the exact one) and sets bit 32 of
// *err.
constexpr int TR_ROWS = 128;  // candidates per MMA (M)
constexpr int TR_N = 16;      // B rows: q_hi, q_lo, then zeros
constexpr int TR_KC = 64;     // coordinates per staged chunk of the A tile
constexpr int TR_STAGES = 4;  // chunks in flight

__global__ void __launch_bounds__(RR_THREADS) rerank_tc_kernel(
    const float *__restrict__ Xr, const int32_t *__restrict__ row_of,
    const __nv_bfloat16 *__restrict__ Rb, const float *__restrict__ rnorm,
    const float2 *__restrict__ rcr, const __nv_bfloat16 *__restrict__ Cg, int d,
    const float *__restrict__ Qb, int k, int cap, int P2, const int32_t *__restrict__ cand,
    const int32_t *__restrict__ nkeep, int64_t *__restrict__ ids_out,
    float *__restrict__ dists_out, bool vec, bool vec16, float rho_s, float cP,
    unsigned long long *__restrict__ rows_fp32, int *__restrict__ err)
{
    extern __shared__ __align__(128) unsigned char smraw[];
    __shared__ int scan_tmp[RR_WARPS];
    __shared__ int any_mark;
    __shared__ int hist[256];
    __shared__ int bc[4];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tbase_s;
    __shared__ int s_stuck;
    __shared__ int s_ngroups;
    __shared__ float s_qq;
    const int dk = (d + 15) & ~15;
    const int KC = dk < TR_KC ? dk : TR_KC;
    unsigned char *a_t = smraw;                         // TR_STAGES x TR_ROWS x KC BF16
    unsigned char *b_t = a_t + TR_STAGES * TR_ROWS * KC * 2;  // TR_N x dk BF16
    RerankSmem sm = carve_rerank(b_t + TR_N * dk * 2, P2, scan_tmp, &any_mark, hist, bc);
    int32_t *cid = reinterpret_cast<int32_t *>(sm.mark + P2 + 15 - ((P2 + 15) % 16));  // P2 ids
    int32_t *gkey = reinterpret_cast<int32_t *>(sm.key);  // P2 group slots (-1: empty)
    float *gS = reinterpret_cast<float *>(sm.key) + P2;    // |q - C_g|^2 per slot
    int32_t *rowi = sm.sid;                               // row of every candidate
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int q = blockIdx.x;
    const int nc = nkeep[q];
    const float *qv = Qb + (int64_t)q * d;
    const int32_t *cl = cand + (int64_t)q * cap;
    if (tid == 0) {
        s_stuck = 0;
        s_ngroups = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_smem(&bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 32;" ::"r"(
                         tc_smem(&tbase_s))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // 0. ids, rows, empty group slots, and B: the query split into BF16 hi
    //    (row 0) and lo (row 1); rows 2..15 and columns past d are zero
    for (int j = tid; j < nc; j += RR_THREADS) {
        const int32_t id = cl[j];
        cid[j] = id;
        rowi[j] = row_of ? row_of[id] : id;
    }
    for (int sl = tid; sl < P2; sl += RR_THREADS) gkey[sl] = -1;
    for (int e = tid; e < TR_N * dk; e += RR_THREADS) {
        const int r = e / dk, c = e % dk;
        float v = 0.0f;
        if (r < 2 && c < d) {
            const float x = __ldg(qv + c);
            const __nv_bfloat16 hi = __float2bfloat16_rn(x);
            v = r == 0 ? __bfloat162float(hi)
                       : __bfloat162float(__float2bfloat16_rn(x - __bfloat162float(hi)));
        }
        *reinterpret_cast<__nv_bfloat16 *>(b_t + tc_off(r, c, dk)) = __float2bfloat16_rn(v);
    }
    if (warp == 0) {
        float s = 0.0f;
        for (int c = lane; c < d; c += 32) s = fmaf(__ldg(qv + c), __ldg(qv + c), s);
        s = warp_sum(s);
        if (lane == 0) s_qq = s;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = tbase_s;
    // 1. |q - C_g|^2 per distinct group (the group list in d32, free until
    //    the tiles' bounds)
    group_norms(rowi, nc, P2, gkey, gS, reinterpret_cast<int32_t *>(sm.d32), &s_ngroups, Cg, qv,
                d);
    __syncthreads();
    // 2. tiles of TR_ROWS candidates, each in chunks of KC coordinates; the
    //    chunks of all tiles run through a TR_STAGES-deep cp.async pipeline
    //    (16-byte copies, rows past the candidates and coordinates past d
    //    zero-filled), and q . r~ accumulates in tensor memory (columns 0:
    //    hi, 1: lo).  A buffer is refilled only after the MMA that read it.
    const uint32_t idesc = tc_idesc_bf16(TR_ROWS, TR_N);
    const float qn = sqrtf(s_qq) * 1.01f;  // >= |q|
    const int cpt = (dk + KC - 1) / KC;    // chunks per tile
    const int n_tiles = (nc + TR_ROWS - 1) / TR_ROWS;
    const int n_chunks = n_tiles * cpt;
    auto issue = [&](int ci) {
        if (ci < n_chunks) {
            const int t0 = (ci / cpt) * TR_ROWS, k0 = (ci % cpt) * KC;
            const int kc = (dk - k0) < KC ? (dk - k0) : KC;
            const int per_row = kc >> 3;
            unsigned char *buf = a_t + (size_t)(ci % TR_STAGES) * TR_ROWS * KC * 2;
            for (int p = tid; p < TR_ROWS * per_row; p += RR_THREADS) {
                const int r = p / per_row, c8 = (p % per_row) * 8;
                const int j = t0 + r, c = k0 + c8;
                unsigned char *dst = buf + tc_off(r, c8, KC);
                if (vec16) {
                    // whole pieces inside the row are copied, the rest zero-filled
                    const bool in = j < nc && c + 8 <= d;
                    const __nv_bfloat16 *src = in ? Rb + (int64_t)rowi[j] * d + c : Rb;
                    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(tc_smem(dst)),
                                 "l"(src), "r"(in ? 16 : 0)
                                 : "memory");
                } else {
                    __align__(16) __nv_bfloat16 e8[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u)
                        e8[u] = (j < nc && c + u < d) ? Rb[(int64_t)rowi[j] * d + c + u]
                                                      : __float2bfloat16_rn(0.0f);
                    *reinterpret_cast<uint4 *>(dst) = *reinterpret_cast<const uint4 *>(e8);
                }
            }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    int mma_waited = -1;  // chunks whose MMA this thread has seen complete
    auto wait_mma = [&](int ci) {
        if (ci <= mma_waited) return;
        if (s_stuck == 0 && !tc_wait(&bar, (uint32_t)(ci & 1))) s_stuck = 1;
        mma_waited = ci;
    };
    for (int i = 0; i < TR_STAGES - 1; ++i) issue(i);
    for (int ci = 0; ci < n_chunks; ++ci) {
        // the next chunk's buffer held chunk ci - 1: its MMA must be done
        if (ci > 0) wait_mma(ci - 1);
        __syncthreads();
        issue(ci + TR_STAGES - 1);
        asm volatile("cp.async.wait_group %0;" ::"n"(TR_STAGES - 1) : "memory");
        tc_fence_async_smem();
        tc_fence_before();
        __syncthreads();
        const int k0 = (ci % cpt) * KC;
        const int kc = (dk - k0) < KC ? (dk - k0) : KC;
        if (tid == 0 && s_stuck == 0) {
            tc_fence_after();
            const unsigned char *buf = a_t + (size_t)(ci % TR_STAGES) * TR_ROWS * KC * 2;
            for (int s2 = 0; s2 < (kc >> 4); ++s2) {
                const uint32_t acc = (k0 | s2) != 0 ? 1u : 0u;
                const uint64_t da = tc_desc(buf + (uint32_t)(2 * s2) * 128, 128, KC * 16);
                const uint64_t db =
                    tc_desc(b_t + (uint32_t)((k0 >> 3) + 2 * s2) * 128, 128, dk * 16);
                tc_mma(tbase, da, db, idesc, acc);
            }
            tc_commit(&bar);
        }
        if (ci % cpt != cpt - 1) continue;
        // the tile's last chunk: bounds of its rows (warps 0-3 own lanes 0-127)
        wait_mma(ci);
        tc_fence_after();
        __syncthreads();
        const bool stuck = s_stuck != 0;
        const int t0 = (ci / cpt) * TR_ROWS;
        if (warp < 4) {
            float v[16];
            tc_ld16(tbase + ((uint32_t)(warp * 32) << 16), v);
            const int j = t0 + warp * 32 + lane;
            if (j < nc) {
                float lo2 = 0.0f, hi2 = CUDART_INF_F;
                if (!stuck) {
                    const int64_t row = rowi[j];
                    const float S = group_norm_of(gkey, gS, P2, (int32_t)(row >> 7));
                    expanded_bounds(__fadd_rn(v[0], v[1]), S, __ldg(rcr + row), __ldg(rnorm + row),
                                    qn, rho_s, cP, lo2, hi2);
                }
                sm.d32[j] = lo2;
                sm.outd[j] = hi2;
            }
        }
        tc_fence_before();
        __syncthreads();  // the accumulator is rewritten by the next tile
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();
    if (tid == 0 && s_stuck) atomicOr(err, 32);
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 32;" ::"r"(tbase) : "memory");
    }
    // 3. the k-th smallest upper bound; the candidates that could be among the
    //    k nearest go through the exact stages (the rows array is free now)
    float uk = CUDART_INF_F;
    if (nc > k)
        uk = __uint_as_float(block_kth_smallest<RR_THREADS>(
            reinterpret_cast<const uint32_t *>(sm.outd), nc, k, sm.hist, sm.bc));
    const int per = (nc + RR_THREADS - 1) / RR_THREADS;
    const int j0 = min(nc, tid * per), j1 = min(nc, j0 + per);
    int mine = 0;
    for (int j = j0; j < j1; ++j) mine += (sm.d32[j] <= uk) ? 1 : 0;
    int ns;
    int pos = block_exclusive_scan<RR_THREADS>(mine, sm.scan_tmp, &ns);
    for (int j = j0; j < j1; ++j)
        if (sm.d32[j] <= uk) sm.sid[pos++] = cid[j];
    __syncthreads();
    if (rows_fp32 && tid == 0) atomicAdd(rows_fp32, (unsigned long long)ns);
    int P2s = 2;
    while (P2s < ns) P2s <<= 1;
    rerank_finish<4>(Xr, row_of, d, qv, k, P2s, ns, sm, ids_out + (int64_t)q * k,
                     dists_out + (int64_t)q * k, vec);
}

}  // namespace

// Rows a warp takes at a time: 2, 4 (default) or 8.
#define QW_RERANK_ROWS_DISPATCH(rows, KERNEL, ...)                     \
    switch (rows) {                                                    \
    case 2: KERNEL<2>__VA_ARGS__; break;                               \
    case 8: KERNEL<8>__VA_ARGS__; break;                               \
    default: KERNEL<4>__VA_ARGS__; break;                              \
    }

qw_status launch_rerank_bf16(const IndexView &ix, const void *Rb, const float *rnorm,
                             const float2 *rcr, const void *C, const float *Qb, int nb, int k,
                             int cap, const QueryState &st, int64_t *ids_out, float *dists_out,
                             unsigned long long *rows_fp32, cudaStream_t s, int rows)
{
    if (nb == 0) return QW_OK;
    int P2 = 2;
    while (P2 < cap) P2 <<= 1;
    const size_t smem = (size_t)P2 * (sizeof(double) + 2 * sizeof(float) + sizeof(int32_t) + 1) +
                        16 + (size_t)P2 * sizeof(int32_t);
    const void *fn = rows == 2 ? (const void *)rerank_bf16_kernel<2>
                     : rows == 8 ? (const void *)rerank_bf16_kernel<8>
                                 : (const void *)rerank_bf16_kernel<4>;
    QW_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    // rows in the locality order when the index has them (the copy's order)
    const float *Xr = ix.Xloc ? ix.Xloc : ix.X;
    const int32_t *row_of = ix.Xloc ? ix.inv : nullptr;
    const int d = ix.d;
    const bool vec = (d % 4 == 0) && ((uintptr_t)Qb % 16 == 0) && ((uintptr_t)Xr % 16 == 0);
    const bool vec8 = (d % 4 == 0) && ((uintptr_t)Qb % 16 == 0) && ((uintptr_t)Rb % 8 == 0);
    const bool vec16 = (d % 256 == 0) && ((uintptr_t)Qb % 16 == 0) && ((uintptr_t)Rb % 16 == 0);
    // rho of the FP32 chains (the FP32 stage's bound, >= 1.02 (ceil(d / 32) +
    // 8) 2^-24 of the dot product's chains as well)
    const double rho = (double)((d + 31) / 32 + 12) * 5.9604644775390625e-08 * 1.02;
    const float rho_s = (float)(rho * 1.01);
    QW_RERANK_ROWS_DISPATCH(rows, rerank_bf16_kernel, <<<nb, RR_THREADS, smem, s>>>(
        Xr, row_of, reinterpret_cast<const __nv_bfloat16 *>(Rb), rnorm, rcr,
        reinterpret_cast<const __nv_bfloat16 *>(C), d, Qb, k, cap, P2, st.cand, st.nkeep,
        ids_out, dists_out, vec, vec8, vec16, rho_s, rho_s, rows_fp32))
    QW_CUDA_TRY(cudaGetLastError());
    return QW_OK;
}

qw_status launch_rerank_tc(const IndexView &ix, const void *Rb, const float *rnorm,
                           const float2 *rcr, const void *C, const float *Qb, int nb, int k,
                           int cap, const QueryState &st, int64_t *ids_out, float *dists_out,
                           unsigned long long *rows_fp32, int *err, cudaStream_t s)
{
    if (nb == 0) return QW_OK;
    int P2 = 2;
    while (P2 < cap) P2 <<= 1;
    const int d = ix.d;
    const int dk = (d + 15) & ~15;
    const int KC = dk < TR_KC ? dk : TR_KC;
    const size_t smem = (size_t)TR_STAGES * TR_ROWS * KC * 2 + (size_t)TR_N * dk * 2 +
                        (size_t)P2 * (sizeof(double) + 2 * sizeof(float) + sizeof(int32_t) + 1) +
                        16 + (size_t)P2 * sizeof(int32_t);
    if (smem + 2048 > 227 * 1024) {
        set_error("qw_run_workload: QW_RERANK_BF16_TC needs (k + v) and d small enough for its "
                  "shared-memory tiles");
        return QW_ERR_ARG;
    }
    QW_CUDA_TRY(cudaFuncSetAttribute(rerank_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
    const float *Xr = ix.Xloc ? ix.Xloc : ix.X;
    const int32_t *row_of = ix.Xloc ? ix.inv : nullptr;
    const bool vec = (d % 4 == 0) && ((uintptr_t)Qb % 16 == 0) && ((uintptr_t)Xr % 16 == 0);
    const bool vec16 = (d % 8 == 0) && ((uintptr_t)Rb % 16 == 0);
    // rho of the FP32 |q - C_g|^2 chains (as the FP32 stage's); the tensor-core
    // dot product's coefficient with K = d padded to 16 (reading R15)
    const double rho = (double)((d + 31) / 32 + 12) * 5.9604644775390625e-08 * 1.02;
    const double cP = 1.52587890625e-05 + 1.02 * (double)(dk - 1) * 2.384185791015625e-07 +
                      1.1920928955078125e-07;
    rerank_tc_kernel<<<nb, RR_THREADS, smem, s>>>(
        Xr, row_of, reinterpret_cast<const __nv_bfloat16 *>(Rb), rnorm, rcr,
        reinterpret_cast<const __nv_bfloat16 *>(C), d, Qb, k, cap, P2, st.cand, st.nkeep, ids_out,
        dists_out, vec, vec16, (float)(rho * 1.01), (float)(cP * 1.01), rows_fp32, err);
    QW_CUDA_TRY(cudaGetLastError());
    return QW_OK;
}

qw_status launch_rerank(const IndexView &ix, const float *Qb, int nb, int k, int cap,
                        const QueryState &st, int64_t *ids_out, float *dists_out,
                        cudaStream_t s, const float *Xrows, const int32_t *row_of, int rows)
{
    const float *X = Xrows ? Xrows : ix.X;
    int P2 = 2;
    while (P2 < cap) P2 <<= 1;
    const size_t smem = (size_t)P2 * (sizeof(double) + 2 * sizeof(float) + sizeof(int32_t) + 1);
    const void *fn = rows == 2 ? (const void *)rerank_kernel<2>
                     : rows == 8 ? (const void *)rerank_kernel<8> : (const void *)rerank_kernel<4>;
    QW_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    // 16-byte row loads need d % 4 == 0 and 16-byte aligned bases
    const bool vec = (ix.d % 4 == 0) && ((uintptr_t)Qb % 16 == 0) && ((uintptr_t)X % 16 == 0);
    QW_RERANK_ROWS_DISPATCH(rows, rerank_kernel, <<<nb, RR_THREADS, smem, s>>>(
        X, row_of, ix.d, Qb, k, cap, P2, st.cand, st.nkeep, ids_out, dists_out, vec))
    QW_CUDA_TRY(cudaGetLastError());
    return QW_OK;
}

}  // namespace qw
