// qw_cluster.cu -- the whole query loop of collision counting in one
// persistent, cluster-launched kernel.
//
// Same method as qw_query.cu (levels R = 1, c, c^2, ...; flanks of every
// projection's bucket range scanned incrementally; candidates = ids with at
// least l collisions; stop at |C_R| >= k + v or once R exceeds every bucket id;
// keep at most k + v), organised for GB300:
//   * one thread-block cluster of CS CTAs answers one query at a time; CTA r
//     owns index tiles [r * TPC, (r + 1) * TPC) and keeps their collision
//     counters in its shared memory for all levels of the query, so counters
//     never travel to HBM;
//   * after each level the CTAs add their new-candidate counts into CTA 0's
//     shared memory through distributed shared memory and meet at a cluster
//     barrier; every CTA reads the total and takes the same stop decision;
//   * clusters pull queries from a global work queue, so queries with many
//     levels do not hold up the rest (per-query work is very uneven).
// Selection under the k + v bound uses the same plan as the level-synchronous
// path: a histogram of collision counts gathered in CTA 0, the boundary count
// c*, and per-tile prefixes so each CTA writes its kept ids in id order.
#include "qw_internal.cuh"
#include "qw_count.cuh"
#include "qw_dir.cuh"
#include "qw_tma.cuh"
#include "qw_scan.cuh"

#include <cooperative_groups.h>

#include <algorithm>

namespace cg = cooperative_groups;

namespace qw {
namespace {

constexpr int CQ_THREADS = 512;
constexpr int kConsumers = CQ_THREADS - 32;  // warp 0 feeds, warps 1.. count
constexpr int kWordsPerTile = kTile / 4;
constexpr int kMaxCluster = 16;
constexpr int kMaxTPC = 6;
constexpr int kStages = 4;                     // ring of staged index entries
constexpr int kStageBytes = 8192;
constexpr int kCPS = kStageBytes / 16;         // 8-entry chunks per stage

struct ClusterShared {
    // used in every CTA
    int64_t g[QW_MAX_M];
    uint64_t full_bar[kStages];    // stage filled by the bulk copies
    uint64_t empty_bar[kStages];   // stage consumed by every counting warp
    int32_t wsum[CQ_THREADS / 32];
    int32_t hist_t[kMaxTPC][kHistBins];   // own tiles: [0] previous-level, [1 + c] others
    int32_t red_i;
    unsigned long long red_u;
    int64_t top;
    int32_t bcast[4];
    // meaningful in CTA 0 only (the cluster's meeting point)
    unsigned long long acc_cross[3];
    unsigned long long acc_scan[3];
    int32_t hist_all[kHistBins];
    int32_t tile_info[kMaxCluster * kMaxTPC][2];  // per tile: kept above c*, ids at c*
    int32_t next_q;
};

// Tiles whose (tile, projection) pairs are handled in one pass of the block.
__host__ __device__ inline int tiles_per_group(int tpc, int m)
{
    const int g = CQ_THREADS / m;
    return g < 1 ? 1 : (g < tpc ? g : tpc);
}

__host__ __device__ inline size_t cluster_smem_bytes(int tpc, int m)
{
    const size_t nseg = 2 * (size_t)tiles_per_group(tpc, m) * m;
    return (size_t)tpc * kTile + (size_t)kStages * kStageBytes + nseg * 8 + (nseg + 1) * 4 +
           3 * nseg + 16;
}

__global__ void __launch_bounds__(CQ_THREADS, 2) cluster_query_kernel(
    IndexView ix, const int32_t *__restrict__ HQ, int nq, int l, int cgrow, int cap, int tpc,
    QueryState st, int *__restrict__ queue, int64_t *__restrict__ stats_out, int *__restrict__ err)
{
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    extern __shared__ __align__(128) unsigned char dsm[];
    __shared__ ClusterShared sh;
    ClusterShared *sh0 = cluster.map_shared_rank(&sh, 0);
    const int G = tiles_per_group(tpc, ix.m);
    const int max_seg = 2 * G * ix.m;
    uint32_t *cnt_s = reinterpret_cast<uint32_t *>(dsm);                    // tpc * kWordsPerTile
    unsigned char *ring = dsm + (size_t)tpc * kTile;                          // kStages * kStageBytes
    FlankSet fl;
    fl.gc0 = reinterpret_cast<int64_t *>(ring + kStages * kStageBytes);
    fl.cpref = reinterpret_cast<int32_t *>(fl.gc0 + max_seg);                 // max_seg + 1
    fl.head = reinterpret_cast<uint8_t *>(fl.cpref + max_seg + 1);
    fl.tail = fl.head + max_seg;
    fl.tile = fl.tail + max_seg;
    bool stuck = false;
    uint32_t pipe = 0;  // stages issued so far (slot = pipe % kStages)

    const int m = ix.m;
    const int nT = ix.nT;
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const uint32_t lrep = (uint32_t)l * 0x01010101u;
    const int t_first = rank * tpc;
    const int my_tiles = max(0, min(tpc, nT - t_first));
    const unsigned char *lid_bytes = reinterpret_cast<const unsigned char *>(ix.lid);

    if (tid == 0) {
        for (int k = 0; k < kStages; ++k) {
            mbar_init(&sh.full_bar[k], 1);
            mbar_init(&sh.empty_bar[k], kConsumers / 32);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int w = tid; w < tpc * kWordsPerTile / 4; w += CQ_THREADS)
        reinterpret_cast<uint4 *>(cnt_s)[w] = make_uint4(0, 0, 0, 0);
    if (tid < 3) {
        sh.acc_cross[tid] = 0;
        sh.acc_scan[tid] = 0;
    }
    for (int c = tid; c < kHistBins; c += CQ_THREADS) sh.hist_all[c] = 0;
    cluster.sync();

    unsigned gl = 0;  // levels run by this cluster so far (accumulator slot = gl % 3)
    for (;;) {
        if (rank == 0 && tid == 0) sh.next_q = atomicAdd(queue, 1);
        cluster.sync();
        if (tid == 0) sh.bcast[0] = sh0->next_q;
        __syncthreads();
        const int q = sh.bcast[0];
        if (q >= nq) break;

        // query state: anchored bucket ids g_i and the radius beyond which no
        // level changes anything
        if (tid == 0) sh.top = 0;
        __syncthreads();
        if (tid < m) {
            const int64_t gi = (int64_t)HQ[(int64_t)q * m + tid] - (int64_t)ix.o[tid];
            sh.g[tid] = gi;
            const int64_t tv = max((int64_t)ix.span[tid], gi);
            atomicMax(reinterpret_cast<unsigned long long *>(&sh.top), (unsigned long long)tv);
        }
        __syncthreads();
        const int64_t top = sh.top;

        int32_t ncand = 0, nprev = 0, term = 0, levels = 0;
        int64_t R = 1, Rp = 1, scan_full = 0, scan_last = 0;
        for (int level = 0;; ++level) {
            // flag the previous level's candidates in the own counters
            if (level > 0) {
                for (int w = tid; w < my_tiles * kWordsPerTile; w += CQ_THREADS)
                    cnt_s[w] = flag_ge(cnt_s[w], lrep);
            }
            int my_cross = 0;
            unsigned long long my_scan = 0;
            for (int g0 = 0; g0 < my_tiles; g0 += G) {
                const int ng = min(G, my_tiles - g0);
                const int npairs = ng * m;
                // flanks of every (tile, projection) pair of the group
                int c0 = 0, c1 = 0;
                if (tid < npairs) {
                    const int ttl = tid / m, i = tid - ttl * m;
                    const int t = t_first + g0 + ttl;
                    const int64_t tbase = (int64_t)t * kTile;
                    const int len = (int)min((int64_t)kTile, ix.n - tbase);
                    const int64_t gi = sh.g[i];
                    const int64_t sp1 = (int64_t)ix.span[i] + 1;
                    const int64_t dslot = (int64_t)i * nT + t;
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
                    // the tile's slots start 16-byte aligned: chunks are tile offsets / 8
                    const int64_t ebase = (int64_t)i * nT * kTile + tbase;
                    flank_set(fl, 2 * tid, ebase + s0, ebase + e0, g0 + ttl, &c0);
                    flank_set(fl, 2 * tid + 1, ebase + s1, ebase + e1, g0 + ttl, &c1);
                    my_scan += (unsigned long long)(pB - pA);
                }
                int total;
                const int excl = block_exclusive_scan<CQ_THREADS>(c0 + c1, sh.wsum, &total);
                if (tid < npairs) {
                    fl.cpref[2 * tid] = excl;
                    fl.cpref[2 * tid + 1] = excl + c0;
                }
                if (tid == 0) fl.cpref[2 * npairs] = total;
                __syncthreads();
                const int nstages = (total + kCPS - 1) / kCPS;
                const int nseg = 2 * npairs;
                if (warp == 0) {
                    // producer: stage k holds chunks [k * kCPS, (k + 1) * kCPS) of the
                    // flattened flanks, one bulk copy per flank piece
                    if (lane == 0) {
                        int sg = 0;
                        for (int k = 0; k < nstages; ++k) {
                            const uint32_t it = pipe + (uint32_t)k;
                            const int slot = (int)(it % kStages);
                            if (it >= (uint32_t)kStages)
                                mbar_wait(&sh.empty_bar[slot], ((it / kStages) - 1) & 1, err, stuck);
                            const int cbeg = k * kCPS, cend = min(cbeg + kCPS, total);
                            mbar_arrive_expect_tx(&sh.full_bar[slot], (uint32_t)(cend - cbeg) * 16u);
                            while (fl.cpref[sg + 1] <= cbeg) ++sg;
                            for (int ss = sg; ss < nseg && fl.cpref[ss] < cend; ++ss) {
                                const int rb = max(fl.cpref[ss], cbeg);
                                const int re = min(fl.cpref[ss + 1], cend);
                                if (re <= rb) continue;
                                const int64_t gch = fl.gc0[ss] + (rb - fl.cpref[ss]);
                                bulk_g2s(ring + (size_t)slot * kStageBytes + (size_t)(rb - cbeg) * 16,
                                         lid_bytes + gch * 16, (uint32_t)(re - rb) * 16u,
                                         &sh.full_bar[slot]);
                            }
                        }
                    }
                    __syncwarp();
                } else {
                    // counters: every id of a staged chunk inside its flank
                    const int ctid = tid - 32;
                    int sg = 0;
                    for (int k = 0; k < nstages; ++k) {
                        const uint32_t it = pipe + (uint32_t)k;
                        const int slot = (int)(it % kStages);
                        mbar_wait(&sh.full_bar[slot], (it / kStages) & 1, err, stuck);
                        const int cbeg = k * kCPS, cend = min(cbeg + kCPS, total);
                        const uint4 *stage =
                            reinterpret_cast<const uint4 *>(ring + (size_t)slot * kStageBytes);
                        for (int cl = ctid; cl < cend - cbeg; cl += kConsumers) {
                            const int e = cbeg + cl;
                            while (e >= fl.cpref[sg + 1]) ++sg;
                            count_chunk(cnt_s + (size_t)fl.tile[sg] * kWordsPerTile, stage[cl],
                                        flank_mask(fl, sg, e));
                        }
                        __syncwarp();
                        if (lane == 0) mbar_arrive(&sh.empty_bar[slot]);
                    }
                }
                pipe += (uint32_t)nstages;
                __syncthreads();  // segment arrays are reused by the next group
            }
            // census: candidates among the own ids after this level
            for (int w = tid; w < my_tiles * kWordsPerTile; w += CQ_THREADS)
                my_cross += count_ge(cnt_s[w], lrep);
            // this CTA's share of the level, into CTA 0
            my_cross = __reduce_add_sync(0xffffffffu, my_cross);
            if (tid == 0) {
                sh.red_i = 0;
                sh.red_u = 0;
            }
            __syncthreads();
            if (lane == 0 && my_cross) atomicAdd(&sh.red_i, my_cross);
            if (my_scan) atomicAdd(&sh.red_u, my_scan);
            __syncthreads();
            const int slot = (int)(gl % 3);
            if (tid == 0) {
                if (sh.red_i) atomicAdd(&sh0->acc_cross[slot], (unsigned long long)sh.red_i);
                if (sh.red_u) atomicAdd(&sh0->acc_scan[slot], sh.red_u);
            }
            cluster.sync();
            if (tid == 0) {
                sh.bcast[1] = (int32_t)sh0->acc_cross[slot];
                const unsigned long long sc = sh0->acc_scan[slot];
                sh.red_u = sc;
                if (rank == 0) {
                    // a slot is reused two levels later, after another barrier
                    sh.acc_cross[(gl + 2) % 3] = 0;
                    sh.acc_scan[(gl + 2) % 3] = 0;
                }
            }
            __syncthreads();
            ++gl;
            const int32_t total_count = sh.bcast[1];  // |C_R| over the whole index
            const int64_t level_scan = (int64_t)sh.red_u;
            scan_full += level_scan;
            scan_last = level_scan;
            levels = level + 1;
            const int32_t before = ncand;
            ncand = total_count;
            const bool enough = ncand >= cap;
            const bool past = R > top;
            __syncthreads();
            if (enough || past) {
                term = enough ? 2 : 3;
                nprev = before;
                break;
            }
            Rp = R;
            R *= cgrow;
        }

        // ---- selection under the k + v bound
        for (int c = tid; c < kMaxTPC * kHistBins; c += CQ_THREADS) (&sh.hist_t[0][0])[c] = 0;
        __syncthreads();
        for (int tt = 0; tt < my_tiles; ++tt) {
            int my_prev = 0;
            const uint32_t *cnt_t = cnt_s + tt * kWordsPerTile;
            for (int w = tid; w < kWordsPerTile; w += CQ_THREADS) {
                const uint32_t x = cnt_t[w];
                if (!__vcmpgeu4(x & 0x7f7f7f7fu, lrep)) continue;
#pragma unroll
                for (int by = 0; by < 4; ++by) {
                    const uint32_t b8 = (x >> (8 * by)) & 0xffu;
                    if ((b8 & 0x7fu) < (uint32_t)l) continue;
                    if (b8 & 0x80u) ++my_prev;
                    else atomicAdd(&sh.hist_t[tt][1 + (b8 & 0x7fu)], 1);
                }
            }
            my_prev = __reduce_add_sync(0xffffffffu, my_prev);
            if (lane == 0 && my_prev) atomicAdd(&sh.hist_t[tt][0], my_prev);
        }
        __syncthreads();
        if (ncand > cap) {
            for (int c = tid; c < kHistBins; c += CQ_THREADS) {
                int sum = 0;
                for (int tt = 0; tt < my_tiles; ++tt) sum += sh.hist_t[tt][c];
                if (sum) atomicAdd(&sh0->hist_all[c], sum);
            }
        }
        cluster.sync();
        if (tid == 0) {
            int cstar = l - 1, take_eq = 0;
            if (ncand > cap) {
                const int need = cap - nprev;
                int acc = 0;
                for (int c = m; c >= l; --c) {
                    const int hc = sh0->hist_all[1 + c];
                    if (acc + hc >= need) {
                        cstar = c;
                        take_eq = need - acc;
                        break;
                    }
                    acc += hc;
                }
            }
            sh.bcast[2] = cstar;
            sh.bcast[3] = take_eq;
        }
        __syncthreads();
        const int cstar = sh.bcast[2], take_eq = sh.bcast[3];
        if (tid < my_tiles) {
            const int32_t *h = sh.hist_t[tid];
            int above = h[0];
            for (int c = max(cstar + 1, l); c <= m; ++c) above += h[1 + c];
            const int eq = (cstar >= l) ? h[1 + cstar] : 0;
            sh0->tile_info[t_first + tid][0] = above;
            sh0->tile_info[t_first + tid][1] = eq;
        }
        cluster.sync();
        // prefixes over the tiles before each own tile (tiles are in id order)
        __shared__ int32_t own_out[kMaxTPC], own_eq[kMaxTPC], s_keep;
        if (tid == 0) {
            int out = 0, eqb = 0;
            int keep_all = 0;
            for (int t = 0; t < nT; ++t) {
                const int above = sh0->tile_info[t][0], eq = sh0->tile_info[t][1];
                const int kept = above + min(max(take_eq - eqb, 0), eq);
                if (t >= t_first && t < t_first + my_tiles) {
                    own_out[t - t_first] = out;
                    own_eq[t - t_first] = eqb;
                }
                out += kept;
                eqb += eq;
                keep_all = out;
            }
            s_keep = min(keep_all, cap);
        }
        __syncthreads();
        const int keep = s_keep;
        for (int tt = 0; tt < my_tiles; ++tt) {
            const int t = t_first + tt;
            const int64_t tbase = (int64_t)t * kTile;
            const int len = (int)min((int64_t)kTile, ix.n - tbase);
            const uint8_t *cb = reinterpret_cast<const uint8_t *>(cnt_s + tt * kWordsPerTile);
            int rank_eq = own_eq[tt];
            int out_base = own_out[tt];
            if (sh.hist_t[tt][0] == 0) {
                bool any = false;
                for (int c = max(cstar, l); c <= m && !any; ++c) any = sh.hist_t[tt][1 + c] != 0;
                if (!any) continue;
            }
            for (int chunk = 0; chunk < len; chunk += CQ_THREADS * 16) {
                const int base = chunk + tid * 16;
                uint4 v4 = make_uint4(0, 0, 0, 0);
                if (base < len) v4 = *reinterpret_cast<const uint4 *>(cb + base);
                const uint8_t *bytes = reinterpret_cast<const uint8_t *>(&v4);
                int n_eq = 0;
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    const int c = bytes[u] & 0x7f;
                    n_eq += (c == cstar && c >= l && !(bytes[u] & 0x80)) ? 1 : 0;
                }
                int eq_total;
                int r = rank_eq + block_exclusive_scan<CQ_THREADS>(n_eq, sh.wsum, &eq_total);
                uint16_t selmask = 0;
                int n_sel = 0;
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    const int c = bytes[u] & 0x7f;
                    bool sel = false;
                    if (c >= l) {
                        if ((bytes[u] & 0x80) || c > cstar) sel = true;
                        else if (c == cstar) { sel = r < take_eq; ++r; }
                    }
                    if (sel) { selmask |= (uint16_t)(1u << u); ++n_sel; }
                }
                int sel_total;
                int pos = out_base + block_exclusive_scan<CQ_THREADS>(n_sel, sh.wsum, &sel_total);
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    if (selmask & (1u << u)) {
                        if (pos < cap) {
                            st.cand[(int64_t)q * cap + pos] = (int32_t)(tbase + base + u);
                            st.cand_col[(int64_t)q * cap + pos] = bytes[u] & 0x7f;
                        }
                        ++pos;
                    }
                }
                rank_eq += eq_total;
                out_base += sel_total;
            }
        }
        if (rank == 0) {
            for (int p = keep + tid; p < cap; p += CQ_THREADS) {
                st.cand[(int64_t)q * cap + p] = -1;
                st.cand_col[(int64_t)q * cap + p] = 0;
            }
            if (tid == 0) {
                st.nkeep[q] = keep;
                if (stats_out) {
                    int64_t *so = stats_out + (int64_t)q * QW_NSTAT;
                    so[0] = levels;
                    so[1] = R;
                    so[2] = ncand;
                    so[3] = keep;
                    so[4] = term;
                    so[5] = scan_last;
                    so[6] = scan_full;
                    so[7] = nprev;
                }
            }
            for (int c = tid; c < kHistBins; c += CQ_THREADS) sh.hist_all[c] = 0;
        }
        // clear the own counters for the next query
        for (int w = tid; w < tpc * kWordsPerTile / 4; w += CQ_THREADS)
            reinterpret_cast<uint4 *>(cnt_s)[w] = make_uint4(0, 0, 0, 0);
        __syncthreads();
    }
    // no bulk copy may still be writing this CTA's shared memory at exit
    if (tid == 0 && stuck) {
        for (uint32_t k = 0; k < (uint32_t)kStages && k < pipe; ++k) {
            const uint32_t it = pipe - 1 - k;
            bool again = false;
            mbar_wait(&sh.full_bar[it % kStages], (it / kStages) & 1, err, again);
        }
    }
    // no CTA may leave while others can still address its shared memory
    cluster.sync();
}

}  // namespace

static cudaLaunchConfig_t cluster_config(int cluster_size, int tpc, int m, cudaStream_t s,
                                         cudaLaunchAttribute *attr)
{
    cudaLaunchConfig_t cfg = {};
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cluster_size;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(CQ_THREADS, 1, 1);
    cfg.dynamicSmemBytes = cluster_smem_bytes(tpc, m);
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cfg.gridDim = dim3(cluster_size, 1, 1);
    return cfg;
}

// Most clusters of this shape resident at once on the current device (0 if
// the shape cannot be launched).
static int cluster_capacity(int cluster_size, int tpc, int m)
{
    const int smem = (int)cluster_smem_bytes(tpc, m);
    if (cudaFuncSetAttribute(cluster_query_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             smem) != cudaSuccess) {
        (void)cudaGetLastError();
        return 0;
    }
    if (cluster_size > 8 &&
        cudaFuncSetAttribute(cluster_query_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed,
                             1) != cudaSuccess) {
        (void)cudaGetLastError();
        return 0;
    }
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = cluster_config(cluster_size, tpc, m, 0, attr);
    int active = 0;
    if (cudaOccupancyMaxActiveClusters(&active, (void *)cluster_query_kernel, &cfg) != cudaSuccess) {
        (void)cudaGetLastError();
        return 0;
    }
    return active;
}

bool cluster_path_fits(const IndexView &ix, int *cluster_size, int *tiles_per_cta)
{
    for (int cap_cs : {kMaxCluster, 8}) {
        const int cs = std::min(cap_cs, ix.nT);
        const int tpc = (ix.nT + cs - 1) / cs;
        if (tpc > kMaxTPC) continue;
        if (cluster_capacity(cs, tpc, ix.m) < 1) continue;
        *cluster_size = cs;
        *tiles_per_cta = tpc;
        return true;
    }
    return false;
}

qw_status launch_cluster_query(const IndexView &ix, const int32_t *HQ, int nq, int l, int c,
                               int cap, int cluster_size, int tpc, int max_clusters,
                               QueryState &st, int *queue, int64_t *stats_out, int *err,
                               cudaStream_t s, int *clusters_used)
{
    const int active = cluster_capacity(cluster_size, tpc, ix.m);
    if (active < 1) {
        set_error("cluster launch does not fit on this device");
        return QW_ERR_CUDA;
    }
    int nclusters = std::min(active, std::max(1, nq));
    if (max_clusters > 0) nclusters = std::min(nclusters, max_clusters);
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = cluster_config(cluster_size, tpc, ix.m, s, attr);
    cfg.gridDim = dim3((unsigned)(nclusters * cluster_size), 1, 1);
    QW_CUDA_TRY(cudaMemsetAsync(queue, 0, sizeof(int), s));
    QW_CUDA_TRY(cudaLaunchKernelEx(&cfg, cluster_query_kernel, ix, HQ, nq, l, c, cap, tpc, st, queue,
                                   stats_out, err));
    if (clusters_used) *clusters_used = nclusters;
    return QW_OK;
}

}  // namespace qw
