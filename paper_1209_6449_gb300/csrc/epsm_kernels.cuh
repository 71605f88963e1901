// Kernels: single-search scan and batched persistent scan.
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

// ---------------------------------------------------------------------------
// batched search: many (text, pattern) pairs in one persistent launch
// ---------------------------------------------------------------------------

struct BatchPair {
    SearchJob job;
    uint64_t tile0;    // first global tile of the pair
    uint32_t variant;  // V_* (DIRECT uses mp = m)
    uint32_t pad;
};

struct BatchParams {
    const BatchPair *pairs;  // device, npairs entries, ascending tile0
    uint32_t npairs;
    uint64_t ntiles;         // total tiles over all pairs
    TileOut out;
    uint64_t *offsets;       // device, npairs + 1: pair output offsets and total
    DevMisc *misc;
};

// Index of the pair that owns global tile g (pairs with no tiles are skipped
// because their tile0 equals the next pair's).
__device__ __forceinline__ uint32_t find_pair(const BatchPair *pairs, uint32_t npairs, uint64_t g) {
    uint32_t lo = 0, hi = npairs - 1u;
    while (lo < hi) {
        uint32_t mid = (lo + hi + 1u) >> 1;
        if (pairs[mid].tile0 <= g) lo = mid; else hi = mid - 1u;
    }
    return lo;
}

template <int U>
__global__ void __launch_bounds__(kThreads) batch_kernel(const __grid_constant__ BatchParams prm) {
    __shared__ TileSmem sm;
    __shared__ BatchPair cur;
    __shared__ uint32_t cur_pair;
    __shared__ uint32_t table_pair;
    if (threadIdx.x == 0) {
        sm.next_tile = claim_tile(prm.misc);
        cur_pair = 0xFFFFFFFFu;
        table_pair = 0xFFFFFFFFu;
    }
    __syncthreads();
    uint32_t tile = sm.next_tile;
    while (tile < prm.ntiles) {
        if (threadIdx.x == 0) {
            uint32_t p = find_pair(prm.pairs, prm.npairs, tile);
            if (p != cur_pair) {
                cur = prm.pairs[p];
                cur_pair = p;
            }
        }
        __syncthreads();
        const uint32_t p = cur_pair;
        const SearchJob &J = cur.job;
        const uint64_t lt = tile - cur.tile0;
        uint64_t *first_out = lt == 0 ? prm.offsets + p : nullptr;
        uint64_t *count_out = (uint64_t)tile + 1u == prm.ntiles ? prm.offsets + prm.npairs : nullptr;
        const BcastWords B(J.pat);
        switch (cur.variant) {
            case V_DIRECT:
                switch (J.pat.m) {
                    case 1: scan_tile<V_DIRECT, U, 1>(J, lt, tile, B, sm, prm.out, count_out, first_out, 0); break;
                    case 2: scan_tile<V_DIRECT, U, 2>(J, lt, tile, B, sm, prm.out, count_out, first_out, 0); break;
                    case 3: scan_tile<V_DIRECT, U, 3>(J, lt, tile, B, sm, prm.out, count_out, first_out, 0); break;
                    default: scan_tile<V_DIRECT, U, 4>(J, lt, tile, B, sm, prm.out, count_out, first_out, 0); break;
                }
                break;
            case V_PREFIX4:
                scan_tile<V_PREFIX4, U, 4>(J, lt, tile, B, sm, prm.out, count_out, first_out, 0);
                break;
            case V_PREFIX8:
                scan_tile<V_PREFIX8, U, 8>(J, lt, tile, B, sm, prm.out, count_out, first_out, 0);
                break;
            default:
                if (table_pair != p) {  // block-uniform: rebuild table L only when the pair changes
                    build_block_table(J.pat, sm.table, sm.pblk);
                    if (threadIdx.x == 0) table_pair = p;
                }
                scan_tile<V_BLOCK8, U, 8>(J, lt, tile, B, sm, prm.out, count_out, first_out, 0);
                break;
        }
        if (threadIdx.x == 0) sm.next_tile = claim_tile(prm.misc);
        __syncthreads();
        tile = sm.next_tile;
    }
    finish_block(prm.misc);
}

}  // namespace epsm
