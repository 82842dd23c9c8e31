// Warp-aggregated counter updates: the lanes of a warp that add 1 to the same
// counter are grouped (__match_any_sync on the counter's address) and one
// lane per group issues a single atomic for the whole group.  On inputs
// sorted by the counter's key most of a warp shares one counter, so this
// turns 32 contended atomics into one.
#pragma once

#include <cstdint>

namespace hpa {

// Every lane of the warp must call this (ctr may be null for lanes with
// nothing to add).  Returns the counter's old value plus the lane's rank
// among the lanes of its group -- a unique slot when the counter is a cursor
// (the order within a group follows the lanes).
__device__ __forceinline__ uint32_t warp_agg_inc(uint32_t* ctr) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t peers = __match_any_sync(0xffffffffu, (unsigned long long)ctr);
    const uint32_t leader = __ffs(peers) - 1;
    uint32_t old = 0;
    if (lane == leader && ctr) old = atomicAdd(ctr, (uint32_t)__popc(peers));
    old = __shfl_sync(0xffffffffu, old, leader);
    return old + __popc(peers & ((1u << lane) - 1u));
}

}  // namespace hpa
