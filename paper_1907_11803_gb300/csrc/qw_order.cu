// qw_order.cu -- workload ordering: answer queries that fall into the same
// region of the projected space together.
//
// qwLSH's premise (Section 1.2, Section 4) is that queries of a workload are
// near each other and share index files and data objects, so a cache split
// between them pays off.  On GB300 the shared resource is L2: queries that
// hit the same bucket ranges at the same time read the same index entries.
// The queries of a workload are sorted by a coarse signature -- the quantised
// anchored bucket ids of their first four projections, 16 quanta of each
// projection's span -- with a counting sort, processed in that order, and
// their results scattered back to the caller's order.  Results do not depend
// on the order; only the index reuse does.
#include "qw_internal.cuh"

#include <algorithm>

namespace qw {
namespace {

constexpr int kKeyBins = 1 << 16;

__global__ void order_key_kernel(const int32_t *__restrict__ HQ, int64_t nq, int m,
                                 const int32_t *__restrict__ o, const int32_t *__restrict__ span,
                                 uint32_t *__restrict__ keys, int32_t *__restrict__ hist)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nq) return;
    uint32_t key = 0;
    const int np = m < 4 ? m : 4;
    for (int i = 0; i < np; ++i) {
        const int64_t g = (int64_t)HQ[q * m + i] - (int64_t)o[i];
        const int64_t quantum = ((int64_t)span[i] + 16) / 16;  // >= 1
        int64_t z = g < 0 ? 0 : g / quantum;
        z = z > 15 ? 15 : z;
        key = (key << 4) | (uint32_t)z;
    }
    key <<= 4 * (4 - np);
    keys[q] = key;
    atomicAdd(hist + key, 1);
}

// Exclusive scan of kKeyBins counts in one block.
__global__ void __launch_bounds__(1024) order_scan_kernel(int32_t *__restrict__ hist)
{
    __shared__ int32_t wsum[32];
    constexpr int per = kKeyBins / 1024;
    const int t = threadIdx.x;
    int local[per];
    int sum = 0;
#pragma unroll
    for (int j = 0; j < per; ++j) {
        local[j] = hist[t * per + j];
        sum += local[j];
    }
    const int lane = t & 31, warp = t >> 5;
    int incl = sum;
    for (int off = 1; off < 32; off <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += y;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int v = wsum[lane];
        int wi = v;
        for (int off = 1; off < 32; off <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, wi, off);
            if (lane >= off) wi += y;
        }
        wsum[lane] = wi - v;
    }
    __syncthreads();
    int run = wsum[warp] + incl - sum;
#pragma unroll
    for (int j = 0; j < per; ++j) {
        hist[t * per + j] = run;
        run += local[j];
    }
}

__global__ void order_scatter_kernel(const uint32_t *__restrict__ keys, int64_t nq,
                                     int32_t *__restrict__ next, int32_t *__restrict__ perm)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nq) return;
    const int pos = atomicAdd(next + keys[q], 1);
    perm[pos] = (int32_t)q;
}

__global__ void gather_kernel(const float *__restrict__ Q, const int32_t *__restrict__ HQ,
                              const int32_t *__restrict__ perm, int64_t b0, int nb, int d, int m,
                              float *__restrict__ Qb, int32_t *__restrict__ HQb)
{
    const int slot = blockIdx.x;
    if (slot >= nb) return;
    const int64_t q = perm[b0 + slot];
    for (int j = threadIdx.x; j < d; j += blockDim.x) Qb[(int64_t)slot * d + j] = Q[q * d + j];
    for (int i = threadIdx.x; i < m; i += blockDim.x) HQb[(int64_t)slot * m + i] = HQ[q * m + i];
}

__global__ void scatter_kernel(const int32_t *__restrict__ perm, int64_t b0, int nb, int k, int cap,
                               const int64_t *__restrict__ ids_b, const float *__restrict__ dists_b,
                               const int64_t *__restrict__ stats_b,
                               const int64_t *__restrict__ cids_b,
                               const int32_t *__restrict__ ccol_b, int64_t *__restrict__ ids,
                               float *__restrict__ dists, int64_t *__restrict__ stats,
                               int64_t *__restrict__ cids, int32_t *__restrict__ ccol)
{
    const int slot = blockIdx.x;
    if (slot >= nb) return;
    const int64_t q = perm[b0 + slot];
    if (ids_b) {
        for (int j = threadIdx.x; j < k; j += blockDim.x) {
            ids[q * k + j] = ids_b[(int64_t)slot * k + j];
            dists[q * k + j] = dists_b[(int64_t)slot * k + j];
        }
    }
    if (stats_b)
        for (int j = threadIdx.x; j < QW_NSTAT; j += blockDim.x)
            stats[q * QW_NSTAT + j] = stats_b[(int64_t)slot * QW_NSTAT + j];
    if (cids_b) {
        for (int j = threadIdx.x; j < cap; j += blockDim.x) {
            cids[q * cap + j] = cids_b[(int64_t)slot * cap + j];
            if (ccol_b) ccol[q * cap + j] = ccol_b[(int64_t)slot * cap + j];
        }
    }
}

}  // namespace

size_t order_hist_ints() { return kKeyBins; }

qw_status launch_order(const int32_t *HQ, int64_t nq, const IndexView &ix, uint32_t *keys,
                       int32_t *hist, int32_t *perm, cudaStream_t s)
{
    if (nq == 0) return QW_OK;
    QW_CUDA_TRY(cudaMemsetAsync(hist, 0, kKeyBins * sizeof(int32_t), s));
    const unsigned blocks = (unsigned)((nq + 255) / 256);
    order_key_kernel<<<blocks, 256, 0, s>>>(HQ, nq, ix.m, ix.o, ix.span, keys, hist);
    QW_CUDA_TRY(cudaGetLastError());
    order_scan_kernel<<<1, 1024, 0, s>>>(hist);
    QW_CUDA_TRY(cudaGetLastError());
    order_scatter_kernel<<<blocks, 256, 0, s>>>(keys, nq, hist, perm);
    QW_CUDA_TRY(cudaGetLastError());
    return QW_OK;
}

qw_status launch_gather(const float *Q, const int32_t *HQ, const int32_t *perm, int64_t b0, int nb,
                        int d, int m, float *Qb, int32_t *HQb, cudaStream_t s)
{
    if (nb == 0) return QW_OK;
    gather_kernel<<<nb, 128, 0, s>>>(Q, HQ, perm, b0, nb, d, m, Qb, HQb);
    QW_CUDA_TRY(cudaGetLastError());
    return QW_OK;
}

qw_status launch_scatter(const int32_t *perm, int64_t b0, int nb, int k, int cap,
                         const int64_t *ids_b, const float *dists_b, const int64_t *stats_b,
                         const int64_t *cids_b, const int32_t *ccol_b, int64_t *ids, float *dists,
                         int64_t *stats, int64_t *cids, int32_t *ccol, cudaStream_t s)
{
    if (nb == 0) return QW_OK;
    scatter_kernel<<<nb, 128, 0, s>>>(perm, b0, nb, k, cap, ids_b, dists_b, stats_b, cids_b, ccol_b,
                                      ids, dists, stats, cids, ccol);
    QW_CUDA_TRY(cudaGetLastError());
    return QW_OK;
}

}  // namespace qw
