// qw_build.cu -- building the sorted bucket arrays (Section 2: QALSH keeps one
// sorted search structure per hash function and range-searches it; here the
// structure is a flat sorted array with a directory instead of a B-tree).
//
// Layout, per projection i (all device memory):
//   lid[i * nT * kTile + t * kTile + p]
//                    16-bit id within its tile (id = t * kTile + lid); every
//                    tile owns kTile slots (the last one is padded), entries
//                    of a tile grouped by bid in ascending order;
//   dir_bid / dir_off at dir_start[i * nT + t]: the distinct bucket ids of
//                    tile t and the offset of the first entry of each, so a
//                    bucket-id range maps to an entry range by two searches.
// bid = h - o_i with o_i = min over the data of h_i, so bid >= 0.
//
// Inside one bucket the ids form a set; their order is free.  It is chosen
// for the counting kernels, which add one to a shared-memory byte counter per
// id (4 counters per 32-bit word, word w in bank w mod 32): the ids of a
// bucket are laid out in groups of up to 8 ids of the same bank, the groups
// cycling through the banks.  A warp then reads 32 consecutive 8-id chunks
// whose ids fall in (mostly) different banks, instead of 32 random banks.
#include "qw_internal.cuh"
#include "qw_scan.cuh"

#include <cuda_bf16.h>

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

__device__ __forceinline__ uint32_t lid_bank(uint16_t lid) { return ((uint32_t)lid >> 2) & 31u; }

// In-place bitonic sort of P (a power of two) entries of (sb, sl, sg) in
// shared memory, ascending by the strict total order `greater`.
template <class Greater>
__device__ __forceinline__ void bitonic_sort(int P, int32_t *sb, uint16_t *sl, uint8_t *sg,
                                             Greater greater)
{
    for (int k = 2; k <= P; k <<= 1) {
        for (int jj = k >> 1; jj > 0; jj >>= 1) {
            for (int x = threadIdx.x; x < (P >> 1); x += SORT_THREADS) {
                const int a = 2 * x - (x & (jj - 1));
                const int c = a + jj;
                const bool up = (a & k) == 0;
                if (greater(a, c) == up) {
                    const int32_t tb = sb[a]; sb[a] = sb[c]; sb[c] = tb;
                    const uint16_t tl = sl[a]; sl[a] = sl[c]; sl[c] = tl;
                    const uint8_t tg = sg[a]; sg[a] = sg[c]; sg[c] = tg;
                }
            }
            __syncthreads();
        }
    }
}

// One CTA orders one (tile, projection) pair of up to kTile entries in shared
// memory: by bucket id, and inside a bucket in bank-interleaved groups (see
// the file comment); then writes the 16-bit ids and the tile's directory.
__global__ void __launch_bounds__(SORT_THREADS) tile_sort_kernel(
    const int32_t *__restrict__ Ht, int64_t n, const int32_t *__restrict__ o,
    uint16_t *__restrict__ lid_out, int32_t *__restrict__ dir_bid, int32_t *__restrict__ dir_off,
    const int64_t *__restrict__ dir_start, int32_t *__restrict__ dir_cnt, int nT)
{
    extern __shared__ __align__(16) unsigned char smem[];
    int32_t *sb = reinterpret_cast<int32_t *>(smem);               // kTile bucket ids
    uint16_t *sl = reinterpret_cast<uint16_t *>(sb + kTile);       // kTile in-tile ids
    uint8_t *sg = reinterpret_cast<uint8_t *>(sl + kTile);         // kTile group numbers
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
            sb[j] = INT32_MAX;  // sorts after every bucket id
            sl[j] = 0xffff;
        }
        sg[j] = 0;
    }
    __syncthreads();
    // 1. by (bid, bank, id): the ids of one bank inside a bucket become a run
    bitonic_sort(P, sb, sl, sg, [&](int a, int c) {
        if (sb[a] != sb[c]) return sb[a] > sb[c];
        const uint32_t ka = lid_bank(sl[a]), kc = lid_bank(sl[c]);
        if (ka != kc) return ka > kc;
        return sl[a] > sl[c];
    });
    // 2. group number = rank inside the (bid, bank) run / 8
    {
        const int per = P / SORT_THREADS > 0 ? P / SORT_THREADS : 1;
        const int j0 = min(P, (int)threadIdx.x * per), j1 = min(P, j0 + per);
        auto run_start = [&](int j) {
            return j == 0 || sb[j] != sb[j - 1] || lid_bank(sl[j]) != lid_bank(sl[j - 1]);
        };
        int last = -1;
        for (int j = j0; j < j1; ++j)
            if (run_start(j)) last = j;
        int start = block_exclusive_max<SORT_THREADS>(last, -1, warp_sums);
        for (int j = j0; j < j1; ++j) {
            if (run_start(j)) start = j;
            sg[j] = (uint8_t)((j - start) >> 3);  // a bank holds <= 1024 ids of a tile
        }
        __syncthreads();
    }
    // 3. by (bid, group, bank, id): groups of one bank, cycling the banks
    bitonic_sort(P, sb, sl, sg, [&](int a, int c) {
        if (sb[a] != sb[c]) return sb[a] > sb[c];
        if (sg[a] != sg[c]) return sg[a] > sg[c];
        const uint32_t ka = lid_bank(sl[a]), kc = lid_bank(sl[c]);
        if (ka != kc) return ka > kc;
        return sl[a] > sl[c];
    });
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

// Residual BF16 copy of the data, for the BF16 pre-filter of the rerank.
// Rows are taken in the index's row order (the locality order when the index
// has bitmaps: 128 consecutive rows are then spatially compact) and grouped
// by 128.  C[g] is the mean of group g (FP64 sums) rounded to BF16; row r is
// stored as Rb[r] = bf16(fl32(x_r - C[r / 128])), with rnorm[r] an upper bound
// of the Euclidean norm of the FP32 residual fl32(x_r - C[r / 128]).  Within a
// group the residuals are about the group's spread, far smaller than the rows
// themselves, so the BF16 rounding error (2^-8 of the residual) is small.  The
// mean itself is any fixed vector for the error bound, so it is kept in BF16
// (exact in FP32) to halve what the pre-filter reads.
__global__ void group_centroid_kernel(const float *__restrict__ Xs, int64_t n, int d,
                                      __nv_bfloat16 *__restrict__ C)
{
    const int64_t g = blockIdx.x;
    const int64_t r0 = g * 128, r1 = min(n, r0 + 128);
    for (int c = threadIdx.x; c < d; c += blockDim.x) {
        double s = 0.0;
        for (int64_t r = r0; r < r1; ++r) s += (double)Xs[r * d + c];
        C[g * d + c] = __double2bfloat16(s / (double)(r1 - r0));
    }
}

// Per row r: the BF16 residual r~ to its group mean, a bound R >= |r| of the
// FP32 residual's norm, and (for the pre-filter's expanded distance) C_g . r~
// and |r~|^2, summed in FP64 and rounded to FP32 (relative error 2^-24).
__global__ void shadow_residual_kernel(const float *__restrict__ Xs, int64_t n, int d,
                                       const __nv_bfloat16 *__restrict__ C,
                                       __nv_bfloat16 *__restrict__ Rb, float *__restrict__ rnorm,
                                       float2 *__restrict__ rcr)
{
    const int64_t r = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= n) return;
    const float *x = Xs + r * d;
    const __nv_bfloat16 *cg = C + (r >> 7) * d;
    double s = 0.0, cr = 0.0, rr = 0.0;
    for (int j = lane; j < d; j += 32) {
        const float v = __fsub_rn(x[j], __bfloat162float(cg[j]));
        const __nv_bfloat16 vb = __float2bfloat16_rn(v);
        Rb[r * d + j] = vb;
        s += (double)v * (double)v;
        const double rb = (double)__bfloat162float(vb);
        cr += (double)__bfloat162float(cg[j]) * rb;
        rr += rb * rb;
    }
    for (int off = 16; off > 0; off >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, off);
        cr += __shfl_xor_sync(0xffffffffu, cr, off);
        rr += __shfl_xor_sync(0xffffffffu, rr, off);
    }
    if (lane == 0) {
        rnorm[r] = __double2float_ru(sqrt(s) * (1.0 + 1e-12));
        if (rcr) rcr[r] = make_float2(__double2float_rn(cr), __double2float_rn(rr));
    }
}

}  // namespace

qw_status launch_shadow_bf16(const float *Xs, int64_t n, int d, void *Rb, float *rnorm,
                             void *C, cudaStream_t s, float2 *rcr)
{
    const int64_t groups = (n + 127) / 128;
    __nv_bfloat16 *Cb = reinterpret_cast<__nv_bfloat16 *>(C);
    group_centroid_kernel<<<(unsigned)groups, 128, 0, s>>>(Xs, n, d, Cb);
    QW_CUDA_TRY(cudaGetLastError());
    const int64_t blocks = (n + 7) / 8;
    shadow_residual_kernel<<<(unsigned)blocks, 256, 0, s>>>(
        Xs, n, d, Cb, reinterpret_cast<__nv_bfloat16 *>(Rb), rnorm, rcr);
    QW_CUDA_TRY(cudaGetLastError());
    return QW_OK;
}

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
    const size_t smem = (size_t)kTile * (sizeof(int32_t) + sizeof(uint16_t) + sizeof(uint8_t));
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
