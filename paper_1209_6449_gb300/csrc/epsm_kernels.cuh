// Device scratch words shared by the persistent kernels.
#pragma once

#include "epsm_tile.cuh"

namespace epsm {

// Scratch words of a context, shared by its launches: the filter kernels'
// stage ticket and "done" counter (the last block to finish resets both for
// the next launch), the emission kernels' range ticket and "done" counter,
// the error word, and a count slot for the synchronous entry points.
struct DevMisc {
    uint64_t count;    // count slot for the synchronous entry points
    uint32_t ticket;   // next stage to claim (filter kernels)
    uint32_t done;     // filter blocks that have finished
    uint32_t err;      // device error bits
    uint32_t probe;    // never set: the flag the wait probe waits for
    uint32_t ticket2;  // next emit range to claim (emission kernels)
    uint32_t done2;    // emission blocks that have finished
};

}  // namespace epsm
