// Device scratch words shared by the persistent kernels.
#pragma once

#include "epsm_tile.cuh"

namespace epsm {

// Scratch counters shared by every launch of a context: a tile ticket (the
// order in which tiles are claimed, which makes the look-back wait only on
// tiles already claimed by running blocks), a "done" counter (the last block
// to finish resets both for the next launch), the error word and a count slot.
struct DevMisc {
    uint64_t count;    // count slot for the synchronous entry points
    uint32_t ticket;   // next work unit to claim
    uint32_t done;     // blocks that have finished
    uint32_t err;      // device error bits
    uint32_t barrier;  // arrivals at the streaming kernel's grid barrier
    uint32_t ticket2;  // next emit range to claim (batched emission kernel)
    uint32_t done2;    // emission blocks that have finished
};

__device__ __forceinline__ uint32_t claim_tile(DevMisc *misc) { return atomicAdd(&misc->ticket, 1u); }

// Called once per block, by the thread that claimed the block's tiles, after
// its last (failing) claim: the last block to get here resets the counters.
__device__ __forceinline__ void finish_claims(DevMisc *misc) {
    __threadfence();
    uint32_t d = atomicAdd(&misc->done, 1u);
    if (d == gridDim.x - 1u) {
        misc->ticket = 0u;
        misc->done = 0u;
        misc->barrier = 0u;
        __threadfence();
    }
}

__device__ __forceinline__ void finish_block(DevMisc *misc) {
    if (threadIdx.x == 0) finish_claims(misc);
}

}  // namespace epsm
