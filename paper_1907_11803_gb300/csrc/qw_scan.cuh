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

}  // namespace qw
