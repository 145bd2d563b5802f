// qw_scan.cuh -- block-wide scans used by the query kernels.
#pragma once

namespace qw {

// Exclusive prefix sum of one int per thread over a block of NT threads.
// tmp: NT / 32 ints of shared memory.  *total receives the block sum.  Safe to
// call repeatedly with the same tmp (it synchronises before reusing it).
template <int NT>
__device__ __forceinline__ int block_exclusive_scan(int v, int *tmp, int *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += y;
    }
    __syncthreads();
    if (lane == 31) tmp[warp] = incl;
    __syncthreads();
    int wbase = 0, tot = 0;
#pragma unroll
    for (int w = 0; w < NT / 32; ++w) {
        int s = tmp[w];
        if (w < warp) wbase += s;
        tot += s;
    }
    *total = tot;
    return wbase + incl - v;
}

// Exclusive running maximum of one int per thread (identity `lowest`).
template <int NT>
__device__ __forceinline__ int block_exclusive_max(int v, int lowest, int *tmp)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl = max(incl, y);
    }
    int excl = __shfl_up_sync(0xffffffffu, incl, 1);
    if (lane == 0) excl = lowest;
    __syncthreads();
    if (lane == 31) tmp[warp] = incl;
    __syncthreads();
    int wbase = lowest;
#pragma unroll
    for (int w = 0; w < NT / 32; ++w)
        if (w < warp) wbase = max(wbase, tmp[w]);
    return max(wbase, excl);
}

// The kk-th smallest (1-based, 1 <= kk <= n) of n unsigned 32-bit keys, by
// radix selection, 8 bits a pass (most keys share their leading bits, so a
// warp adds one count per distinct bin).  Block-wide over NT threads; v may be
// shared or global memory written before the call's first barrier.  hist: 256
// ints and bc: 2 ints of shared memory.  Returns the key in every thread.
// block_kth_smallest_if: the same over the keys of the members of a set
// given by `get(j, &key)` (true: element j < n is a member, with that key);
// kk counts members only.
template <int NT, class Get>
__device__ uint32_t block_kth_smallest_if(int n, int kk, Get get, int *hist, int *bc)
{
    const int lane = threadIdx.x & 31;
    uint32_t prefix = 0, mask = 0;
    for (int shift = 24; shift >= 0; shift -= 8) {
        for (int i = threadIdx.x; i < 256; i += NT) hist[i] = 0;
        __syncthreads();
        for (int j0 = 0; j0 < n; j0 += NT) {
            const int j = j0 + threadIdx.x;
            uint32_t u = 0u;
            const bool member = j < n && get(j, &u);
            const bool in = member && (u & mask) == prefix;
            const uint32_t bin = in ? (u >> shift) & 255u : 256u + lane;
            const uint32_t peers = __match_any_sync(0xffffffffu, bin);
            if (in && lane == __ffs(peers) - 1) atomicAdd(&hist[bin], __popc(peers));
        }
        __syncthreads();
        if (threadIdx.x < 32) {
            // the bin holding the kk-th: lane sums 8 bins, warp scan, then the
            // lane whose range holds kk walks its bins
            int c[8], sl = 0;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                c[u] = hist[lane * 8 + u];
                sl += c[u];
            }
            int incl = sl;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, off);
                if (lane >= off) incl += y;
            }
            const int excl = incl - sl;
            if (excl < kk && kk <= incl) {
                int cum = excl;
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    if (cum < kk && kk <= cum + c[u]) {
                        bc[0] = lane * 8 + u;
                        bc[1] = kk - cum;
                    }
                    cum += c[u];
                }
            }
        }
        __syncthreads();
        prefix |= (uint32_t)bc[0] << shift;
        mask |= 255u << shift;
        kk = bc[1];
        __syncthreads();
    }
    return prefix;
}

template <int NT>
__device__ uint32_t block_kth_smallest(const uint32_t *v, int n, int kk, int *hist, int *bc)
{
    return block_kth_smallest_if<NT>(
        n, kk,
        [v](int j, uint32_t *u) {
            *u = v[j];
            return true;
        },
        hist, bc);
}

// An upper bound U of the kk-th smallest (1-based, 1 <= kk <= n) of n
// unsigned 32-bit keys with at least kk keys <= U: two radix passes of 11 bits
// (bits 31..21, then 20..10), U = the found prefix with bits 9..0 set.  For
// non-negative floats (ordered like their bits) U exceeds the kk-th smallest
// by less than 2^-13 of it.  Block-wide over NT threads; hist: 2048 ints and
// bc: 2 ints of shared memory.  Returns U in every thread.
template <int NT>
__device__ uint32_t block_kth_upper(const uint32_t *v, int n, int kk, int *hist, int *bc)
{
    const int lane = threadIdx.x & 31;
    uint32_t prefix = 0, mask = 0;
    for (int shift = 21; shift >= 10; shift -= 11) {
        for (int i = threadIdx.x; i < 2048; i += NT) hist[i] = 0;
        __syncthreads();
        for (int j0 = 0; j0 < n; j0 += NT) {
            const int j = j0 + threadIdx.x;
            const uint32_t u = j < n ? v[j] : 0u;
            const bool in = j < n && (u & mask) == prefix;
            const uint32_t bin = in ? (u >> shift) & 2047u : 2048u + lane;
            const uint32_t peers = __match_any_sync(0xffffffffu, bin);
            if (in && lane == __ffs(peers) - 1) atomicAdd(&hist[bin], __popc(peers));
        }
        __syncthreads();
        if (threadIdx.x < 32) {
            // lane sums 64 bins, warp scan, then the lane holding kk walks them
            int sl = 0;
            for (int u = 0; u < 64; ++u) sl += hist[lane * 64 + u];
            int incl = sl;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, off);
                if (lane >= off) incl += y;
            }
            const int excl = incl - sl;
            if (excl < kk && kk <= incl) {
                int cum = excl;
                for (int u = 0; u < 64; ++u) {
                    const int c = hist[lane * 64 + u];
                    if (cum < kk && kk <= cum + c) {
                        bc[0] = lane * 64 + u;
                        bc[1] = kk - cum;
                    }
                    cum += c;
                }
            }
        }
        __syncthreads();
        prefix |= (uint32_t)bc[0] << shift;
        mask |= 2047u << shift;
        kk = bc[1];
        __syncthreads();
    }
    return prefix | 1023u;
}

}  // namespace qw
