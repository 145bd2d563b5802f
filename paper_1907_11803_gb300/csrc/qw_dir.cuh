// qw_dir.cuh -- integer helpers of the bucket-range search (virtual
// rehashing, Section 2), shared by the query kernels.
#pragma once

#include <stdint.h>

namespace qw {

// floor(a / R) for R > 0 (C division truncates toward zero).
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

}  // namespace qw
