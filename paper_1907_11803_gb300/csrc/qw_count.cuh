// qw_count.cuh -- the inner loop of collision counting, shared by the level
// path (qw_query.cu) and the cluster path (qw_cluster.cu).
//
// A flank is a run of index entries [lo, hi) of one (tile, projection): the
// 16-bit in-tile ids of the data objects whose bucket id entered the query's
// range at this level.  Runs are read in 16-byte chunks of 8 ids; a flank
// covers chunks [lo / 8, ceil(hi / 8)), its first chunk skips lo % 8 ids and
// its last keeps ((hi - 1) % 8) + 1.  Every id adds one to its byte counter
// (4 counters per 32-bit word of shared memory).
#pragma once

#include "qw_internal.cuh"

namespace qw {

// Flank descriptors of one pass, in shared memory.
struct FlankSet {
    int64_t *gc0;    // first chunk (index into the id array in 16-byte units)
    int32_t *cpref;  // exclusive prefix of chunk counts over the flanks (n + 1)
    uint8_t *head;   // ids to skip in the first chunk
    uint8_t *tail;   // ids to keep in the last chunk (1..8)
    uint8_t *tile;   // which counter tile the flank increments
};

__device__ __forceinline__ void flank_set(FlankSet &f, int s, int64_t lo, int64_t hi, int tile,
                                          int *nchunks)
{
    f.gc0[s] = lo >> 3;
    f.head[s] = (uint8_t)(lo & 7);
    f.tail[s] = (uint8_t)(((hi - 1) & 7) + 1);
    f.tile[s] = (uint8_t)tile;
    *nchunks = (hi > lo) ? (int)(((hi + 7) >> 3) - (lo >> 3)) : 0;
}

// Mask of the ids of chunk e (in the flattened chunk space) that lie in
// flank s.
__device__ __forceinline__ uint32_t flank_mask(const FlankSet &f, int s, int e)
{
    uint32_t mask = 0xffu;
    if (e == f.cpref[s]) mask &= 0xffu << f.head[s];
    if (e == f.cpref[s + 1] - 1) mask &= 0xffu >> (8 - f.tail[s]);
    return mask;
}

// Add one to the byte counter of every id of chunk v selected by mask.
__device__ __forceinline__ void count_chunk(uint32_t *cnt, const uint4 v, uint32_t mask)
{
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
    if (mask == 0xffu) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const uint32_t id = (j & 1) ? (w[j >> 1] >> 16) : (w[j >> 1] & 0xffffu);
            atomicAdd(&cnt[id >> 2], 1u << ((id << 3) & 24u));
        }
    } else {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            if (!(mask & (1u << j))) continue;
            const uint32_t id = (j & 1) ? (w[j >> 1] >> 16) : (w[j >> 1] & 0xffffu);
            atomicAdd(&cnt[id >> 2], 1u << ((id << 3) & 24u));
        }
    }
}

// Number of the 4 byte counters of x whose count (low 7 bits) is >= l;
// lrep = l replicated in every byte.
__device__ __forceinline__ int count_ge(uint32_t x, uint32_t lrep)
{
    return __popc(__vcmpgeu4(x & 0x7f7f7f7fu, lrep)) >> 3;
}

// Same with the "candidate at the previous level" flag (bit 7) set for those.
__device__ __forceinline__ uint32_t flag_ge(uint32_t x, uint32_t lrep)
{
    return x | (__vcmpgeu4(x & 0x7f7f7f7fu, lrep) & 0x80808080u);
}

}  // namespace qw
