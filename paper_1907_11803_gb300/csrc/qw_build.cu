// qw_build.cu -- building the sorted bucket arrays (Section 2: QALSH keeps one
// sorted search structure per hash function and range-searches it; here the
// structure is a flat sorted array with a directory instead of a B-tree).
//
// Layout, per projection i (all device memory):
//   lid[i * nT * kTile + t * kTile + p]
//                    16-bit id within its tile (id = t * kTile + lid); every
//                    tile owns kTile slots (the last one is padded), entries
//                    of a tile sorted by (bid, id);
//   dir_bid / dir_off at dir_start[i * nT + t]: the distinct bucket ids of
//                    tile t and the offset of the first entry of each, so a
//                    bucket-id range maps to an entry range by two searches.
// bid = h - o_i with o_i = min over the data of h_i, so bid >= 0.
#include "qw_internal.cuh"

namespace qw {
namespace {

constexpr int MM_THREADS = 256;

__global__ void minmax_kernel(const int32_t *__restrict__ Ht, int64_t n, int32_t *hmin,
                              int32_t *hmax)
{
    const int i = blockIdx.y;
    const int32_t *col = Ht + (int64_t)i * n;
    int32_t lo = INT32_MAX, hi = INT32_MIN;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        int32_t h = col[j];
        lo = min(lo, h);
        hi = max(hi, h);
    }
    lo = __reduce_min_sync(0xffffffffu, lo);
    hi = __reduce_max_sync(0xffffffffu, hi);
    if ((threadIdx.x & 31) == 0) {
        atomicMin(hmin + i, lo);
        atomicMax(hmax + i, hi);
    }
}

constexpr int SORT_THREADS = 1024;

__device__ __forceinline__ bool pair_greater(int32_t b0, uint16_t l0, int32_t b1, uint16_t l1)
{
    return (b0 > b1) || (b0 == b1 && l0 > l1);
}

// One CTA sorts one (tile, projection) pair of up to kTile entries in shared
// memory with a bitonic network on the unique key (bid, lid), then writes the
// 16-bit ids and the tile's bucket directory.
__global__ void __launch_bounds__(SORT_THREADS) tile_sort_kernel(
    const int32_t *__restrict__ Ht, int64_t n, const int32_t *__restrict__ o,
    uint16_t *__restrict__ lid_out, int32_t *__restrict__ dir_bid, int32_t *__restrict__ dir_off,
    const int64_t *__restrict__ dir_start, int32_t *__restrict__ dir_cnt, int nT)
{
    extern __shared__ __align__(16) unsigned char smem[];
    int32_t *sb = reinterpret_cast<int32_t *>(smem);               // kTile
    uint16_t *sl = reinterpret_cast<uint16_t *>(sb + kTile);       // kTile
    __shared__ int32_t warp_sums[SORT_THREADS / 32];
    __shared__ int32_t carry;

    const int t = blockIdx.x;
    const int i = blockIdx.y;
    const int64_t base = (int64_t)t * kTile;
    const int len = (int)min((int64_t)kTile, n - base);
    int P = 1;
    while (P < len) P <<= 1;
    const int32_t oi = o[i];
    const int32_t *col = Ht + (int64_t)i * n + base;
    for (int j = threadIdx.x; j < P; j += SORT_THREADS) {
        if (j < len) {
            sb[j] = col[j] - oi;
            sl[j] = (uint16_t)j;
        } else {
            sb[j] = INT32_MAX;
            sl[j] = 0xffff;
        }
    }
    __syncthreads();
    for (int k = 2; k <= P; k <<= 1) {
        for (int jj = k >> 1; jj > 0; jj >>= 1) {
            for (int x = threadIdx.x; x < (P >> 1); x += SORT_THREADS) {
                int a = 2 * x - (x & (jj - 1));
                int c = a + jj;
                bool up = (a & k) == 0;
                int32_t ba = sb[a], bc = sb[c];
                uint16_t la = sl[a], lc = sl[c];
                if (pair_greater(ba, la, bc, lc) == up) {
                    sb[a] = bc; sb[c] = ba;
                    sl[a] = lc; sl[c] = la;
                }
            }
            __syncthreads();
        }
    }
    uint16_t *lo = lid_out + (int64_t)i * nT * kTile + base;
    for (int j = threadIdx.x; j < len; j += SORT_THREADS) lo[j] = sl[j];

    // Directory: each thread owns a contiguous run of entries; a block scan
    // of the number of bucket starts gives each start its directory slot.
    const int per = (len + SORT_THREADS - 1) / SORT_THREADS;
    const int j0 = threadIdx.x * per;
    const int j1 = min(len, j0 + per);
    int cnt = 0;
    for (int j = j0; j < j1; ++j) cnt += (j == 0 || sb[j] != sb[j - 1]) ? 1 : 0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = cnt;
    for (int off = 1; off < 32; off <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += y;
    }
    if (lane == 31) warp_sums[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int ws = warp_sums[lane];
        int wi = ws;
        for (int off = 1; off < 32; off <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, wi, off);
            if (lane >= off) wi += y;
        }
        warp_sums[lane] = wi - ws;
        if (lane == 31) carry = wi;
    }
    __syncthreads();
    int slot = warp_sums[warp] + incl - cnt;
    const int64_t ds = dir_start[(int64_t)i * nT + t];
    for (int j = j0; j < j1; ++j) {
        if (j == 0 || sb[j] != sb[j - 1]) {
            dir_bid[ds + slot] = sb[j];
            dir_off[ds + slot] = j;
            ++slot;
        }
    }
    if (threadIdx.x == 0) dir_cnt[(int64_t)i * nT + t] = carry;
}

// Expand the index into per-entry (bid, id) for inspection.
__global__ void export_kernel(const uint16_t *__restrict__ lid, const int32_t *__restrict__ dir_bid,
                              const int32_t *__restrict__ dir_off,
                              const int64_t *__restrict__ dir_start,
                              const int32_t *__restrict__ dir_cnt, int64_t n, int nT,
                              int32_t *__restrict__ entry_bid, int32_t *__restrict__ entry_id)
{
    const int t = blockIdx.x;
    const int i = blockIdx.y;
    const int64_t base = (int64_t)t * kTile;
    const int len = (int)min((int64_t)kTile, n - base);
    const int32_t *ub = dir_bid + dir_start[(int64_t)i * nT + t];
    const int32_t *uo = dir_off + dir_start[(int64_t)i * nT + t];
    const int cnt = dir_cnt[(int64_t)i * nT + t];
    const uint16_t *tl = lid + (int64_t)i * nT * kTile + base;
    for (int p = threadIdx.x; p < len; p += blockDim.x) {
        // last directory slot whose offset is <= p
        int lo = 0, hi = cnt - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (uo[mid] <= p) lo = mid; else hi = mid - 1;
        }
        int64_t e = (int64_t)i * n + base + p;
        if (entry_bid) entry_bid[e] = ub[lo];
        if (entry_id) entry_id[e] = (int32_t)(base + tl[p]);
    }
}

}  // namespace

qw_status launch_minmax(const int32_t *Ht, int64_t n, int m, int32_t *hmin, int32_t *hmax,
                        cudaStream_t s)
{
    int64_t blocks = (n + MM_THREADS - 1) / MM_THREADS;
    if (blocks > 64) blocks = 64;
    minmax_kernel<<<dim3((unsigned)blocks, (unsigned)m), MM_THREADS, 0, s>>>(Ht, n, hmin, hmax);
    QW_CUDA_TRY(cudaGetLastError());
    return QW_OK;
}

qw_status launch_tile_sort(const int32_t *Ht, int64_t n, int m, int nT, const int32_t *o,
                           uint16_t *lid, int32_t *dir_bid, int32_t *dir_off,
                           const int64_t *dir_start, int32_t *dir_cnt, cudaStream_t s)
{
    const size_t smem = (size_t)kTile * (sizeof(int32_t) + sizeof(uint16_t));
    QW_CUDA_TRY(cudaFuncSetAttribute(tile_sort_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
    tile_sort_kernel<<<dim3((unsigned)nT, (unsigned)m), SORT_THREADS, smem, s>>>(
        Ht, n, o, lid, dir_bid, dir_off, dir_start, dir_cnt, nT);
    QW_CUDA_TRY(cudaGetLastError());
    return QW_OK;
}

qw_status launch_export(const uint16_t *lid, const int32_t *dir_bid, const int32_t *dir_off,
                        const int64_t *dir_start, const int32_t *dir_cnt, int64_t n, int m,
                        int nT, int32_t *entry_bid, int32_t *entry_id, cudaStream_t s)
{
    export_kernel<<<dim3((unsigned)nT, (unsigned)m), 256, 0, s>>>(
        lid, dir_bid, dir_off, dir_start, dir_cnt, n, nT, entry_bid, entry_id);
    QW_CUDA_TRY(cudaGetLastError());
    return QW_OK;
}

}  // namespace qw
