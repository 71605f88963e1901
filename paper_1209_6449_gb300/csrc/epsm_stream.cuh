// Streaming scan: filter pass, one cross-block prefix, emit pass — in one
// cooperative persistent launch (up to two blocks per SM, all co-resident).
//
// The text is cut into 16 KiB stages (1024 chunks of 16 bytes) and each stage
// into 8 segments of 128 chunks (2 KiB), one per consumer warp.  Block b owns a
// contiguous run of stages, so positions found by block b all precede those
// of block b+1, and inside a block the stages are handled in order.
//
// Phase 1 (no waiting on other blocks).  A producer warp streams the block's
// stages through a ring of shared-memory buffers with 1-D bulk copies
// (cp.async.bulk, completion on an mbarrier), keeping up to kStages x 16 KiB of
// reads in flight.  Each consumer warp runs the variant's filter and verify
// (chunk_hits) on its segment of the staged stage, writes the segment's hit
// count, and, only if the segment has hits, its 128 16-bit chunk masks to
// scratch memory.
// Phase 2.  The block publishes its total; one warp sums the totals of all
// earlier blocks (decoupled look-back over at most #SM words, one round).
// Phase 3.  Consumer warps prefix-sum the segment counts of the block in
// order and emit the positions of every segment with hits: offsets of the
// segment's hits are staged in shared memory in output order, then written as
// consecutive 8-byte positions (coalesced stores).
//
// Every wait is bounded in time; on expiry the error word gets kErrTimeout and
// the waiting warp gives up, so the kernel always ends.  The producer waits,
// again bounded, for its last bulk copies before the block can end.
#pragma once

#include "epsm_kernels.cuh"

namespace epsm {
namespace stream {

constexpr int kConsumerWarps = 8;
constexpr int kThreadsStream = (kConsumerWarps + 1) * 32;  // + producer warp
constexpr int kStageChunks = kConsumerWarps * 128;          // 1024 chunks = 16 KiB
constexpr uint64_t kStageBytes = (uint64_t)kStageChunks * 16u;
constexpr int kStageBuf = (int)kStageBytes + 128;           // + halo chunk, 128-B aligned
constexpr int kStages = 6;                                  // ring depth (96 KiB in flight per block)
constexpr int kSegChunks = 128;                             // chunks per segment (2 KiB)
constexpr uint64_t kWaitNs = 2000000000ull;
constexpr int kConsumerBarrier = 1;                         // named barrier of consumer warps
constexpr int kMaxBlocksPerSm = 2;

struct alignas(128) StreamSmem {
    uint8_t buf[kStages][kStageBuf];
    uint64_t full[kStages];
    uint64_t empty[kStages];
    uint32_t pblk[16];
    uint8_t table[kHashSlots];
    uint16_t emit_stage[kConsumerWarps][32 * 16];  // per-warp staging of hit offsets
    uint32_t warp_total[kConsumerWarps];
    uint32_t scan_tmp[kConsumerWarps];
    uint64_t cta_excl;
    uint64_t cta_total;
};

// ---------------------------------------------------------------------------
// mbarrier / bulk-copy primitives
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_tx(uint64_t *bar, uint32_t tx) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(tx)
                 : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0u;
}

// Bounded wait for the phase with the given parity; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    if (mbar_test(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    while (!mbar_test(bar, parity)) {
        if (globaltimer_ns() - t0 > kWaitNs) return false;
    }
    return true;
}

// Whole-warp bounded wait; true only if every lane saw the phase complete.
__device__ __forceinline__ bool warp_wait(uint64_t *bar, uint32_t parity) {
    const bool ok = mbar_wait(bar, parity);
    return __all_sync(kFull, ok) != 0;
}

__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes,
                                          uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ void consumer_sync() {
    asm volatile("bar.sync %0, %1;" ::"n"(kConsumerBarrier), "n"(kConsumerWarps * 32) : "memory");
}

struct StreamParams {
    SearchJob job;
    uint64_t *positions;   // device output
    uint64_t capacity;
    uint64_t *count_out;   // device: receives the total
    uint32_t *seg_count;   // scratch: hits per segment
    uint16_t *seg_mask;    // scratch: 128 chunk masks per segment with hits
    uint64_t *cta_status;  // scratch: one status word per block (kStatusStride apart)
    uint32_t *err;
    uint64_t nstages;      // 16 KiB stages of the text
    uint64_t chunk_full0;  // first chunk lying fully inside [delta, lim)
    uint64_t chunk_full1;  // one past the last such chunk
    uint32_t tag;          // call tag of the status words
    int emit;              // 0: count only
};

__device__ __forceinline__ uint4 staged_chunk(const StreamParams &P, const uint8_t *buf,
                                              uint64_t c0, uint64_t c) {
    if (c >= P.chunk_full0 && c < P.chunk_full1)
        return *reinterpret_cast<const uint4 *>(buf + (c - c0) * 16u);
    return load_chunk(P.job, c);
}

__device__ __forceinline__ void block_range(uint64_t n, uint64_t *a, uint64_t *b) {
    *a = n * blockIdx.x / gridDim.x;
    *b = n * (blockIdx.x + 1) / gridDim.x;
}

// ---------------------------------------------------------------------------
// phase 1 roles
// ---------------------------------------------------------------------------

__device__ __forceinline__ void producer(const StreamParams &P, StreamSmem &S, uint64_t st0,
                                         uint64_t st1) {
    const SearchJob &J = P.job;
    uint32_t issued = 0;
    bool failed = false;
    for (uint64_t st = st0; st < st1; ++st) {
        const int s = issued % kStages;
        const uint32_t n = issued / kStages;
        if (n > 0 && !mbar_wait(&S.empty[s], (n - 1) & 1)) { failed = true; break; }
        const uint64_t c0 = st * kStageChunks;
        const uint64_t a = c0 > P.chunk_full0 ? c0 : P.chunk_full0;
        uint64_t b = c0 + kStageChunks + 1u;  // + halo chunk
        if (b > P.chunk_full1) b = P.chunk_full1;
        if (a < b) {
            const uint32_t bytes = (uint32_t)((b - a) * 16u);
            mbar_arrive_tx(&S.full[s], bytes);
            bulk_load(S.buf[s] + (a - c0) * 16u, J.base + a * 16u, bytes, &S.full[s]);
        } else {
            mbar_arrive(&S.full[s]);
        }
        ++issued;
    }
    if (failed) atomicOr(P.err, kErrTimeout);
    // Leave no copy in flight: wait (bounded) for the last issued stages.
    const uint32_t lo = issued > (uint32_t)kStages ? issued - kStages : 0u;
    for (uint32_t i = lo; i < issued; ++i) mbar_wait(&S.full[i % kStages], (i / kStages) & 1);
}

// A chunk read through the ragged-end path (its stage is not entirely inside
// the text): out of line, to keep the hot loop small.
__device__ __noinline__ uint4 edge_chunk(const StreamParams &P, const uint8_t *buf, uint64_t c0,
                                         uint64_t c) {
    return staged_chunk(P, buf, c0, c);
}

template <int V, int MP>
__device__ __forceinline__ uint32_t filter_stages(const StreamParams &P, StreamSmem &S, uint64_t st0,
                                                  uint64_t st1, int w, int lane, bool *ok) {
    constexpr int OFF = (V == V_BLOCK8) ? -7 : 0;
    const SearchJob &J = P.job;
    const BcastWords B(J.pat);
    uint32_t total = 0u;
    uint32_t i = 0;
    const uint32_t lane_off = (uint32_t)(w * kSegChunks + lane) * 16u;  // byte offset in a stage
    for (uint64_t st = st0; st < st1; ++st, ++i) {
        const int s = i % kStages;
        if (!warp_wait(&S.full[s], (i / kStages) & 1)) { *ok = false; break; }
        const uint64_t c0 = st * kStageChunks;
        const uint8_t *buf = S.buf[s];
        // stage entirely inside the text (all but the first and last stages):
        // 32-bit shared-memory offsets, no per-chunk bounds checks
        const bool inside = c0 >= P.chunk_full0 && c0 + kStageChunks + 1u <= P.chunk_full1;
        uint4 ch[4];
        uint4 halo = make_uint4(0u, 0u, 0u, 0u);
        if (inside) {
#pragma unroll
            for (int u = 0; u < 4; ++u)
                ch[u] = *reinterpret_cast<const uint4 *>(buf + lane_off + 512u * u);
            if (V != V_BLOCK8 && lane == 0)
                halo = *reinterpret_cast<const uint4 *>(buf + lane_off + 2048u);
        } else {
            const uint64_t cw = c0 + (uint64_t)w * kSegChunks;
#pragma unroll
            for (int u = 0; u < 4; ++u) ch[u] = edge_chunk(P, buf, c0, cw + 32u * u + lane);
            if (V != V_BLOCK8 && lane == 0) halo = edge_chunk(P, buf, c0, cw + kSegChunks);
        }
        const int64_t sp0 = (int64_t)((c0 + (uint64_t)w * kSegChunks) * 16u) + OFF;
        const bool interior = sp0 >= (int64_t)J.delta &&
                              sp0 + (int64_t)(kSegChunks * 16) - 1 <= J.pmax;
        uint32_t h[4];
        uint32_t cnt = 0u;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint4 cur = ch[u];
            const uint4 nsrc = (lane == 0) ? (u + 1 < 4 ? ch[u + 1 < 4 ? u + 1 : u] : halo) : cur;
            const int64_t p0 = sp0 + (int64_t)((32 * u + lane) * 16);
            uint32_t hh = chunk_hits<V, MP>(J, cur, nsrc, p0, B, S.table, S.pblk, lane);
            if (!interior) hh &= range_mask((int64_t)J.delta - p0, J.pmax - p0);
            h[u] = hh;
            cnt += __popc(hh);
        }
        // the stage buffer is no longer needed: release it to the producer
        __syncwarp();
        if (lane == 0) mbar_arrive(&S.empty[s]);
        const uint32_t wc = warp_sum(cnt);
        const uint64_t seg = st * kConsumerWarps + (uint64_t)w;
        if (lane == 0) P.seg_count[seg] = wc;
        if (wc != 0u && P.emit) {
            uint16_t *mk = P.seg_mask + seg * kSegChunks;
#pragma unroll
            for (int u = 0; u < 4; ++u) mk[u * 32 + lane] = (uint16_t)h[u];
        }
        total += wc;
    }
    return total;
}

// Emit the positions of one segment (a whole warp): bit b of the mask of
// chunk c is the start 16*c + OFF + b.
template <int OFF>
__device__ __forceinline__ void emit_segment(const StreamParams &P, uint64_t seg, uint64_t idx0,
                                             uint16_t *stage, int lane) {
    const SearchJob &J = P.job;
    const uint16_t *mk = P.seg_mask + seg * kSegChunks;
    uint32_t run = 0u;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const uint32_t h = mk[u * 32 + lane];
        const uint32_t c = __popc(h);
        if (!__any_sync(kFull, c != 0u)) continue;
        const uint32_t inc = warp_incl_scan(c, lane);
        const uint32_t T = __shfl_sync(kFull, inc, 31);
        uint32_t k = inc - c;
        uint32_t hh = h;
        while (hh) {
            const uint32_t b = (uint32_t)(__ffs(hh) - 1);
            hh &= hh - 1u;
            stage[k++] = (uint16_t)(lane * 16 + b);
        }
        __syncwarp();
        const int64_t s0 = (int64_t)((seg * kSegChunks + 32u * u) * 16u) + OFF - (int64_t)J.delta;
        const uint64_t base = idx0 + run;
        if (lane == 0 && base + T > P.capacity) atomicOr(P.err, kErrCapacity);
        for (uint32_t q = lane; q < T; q += 32u) {
            const uint64_t idx = base + q;
            if (idx < P.capacity) P.positions[idx] = (uint64_t)(s0 + stage[q]);
        }
        __syncwarp();
        run += T;
    }
}

// Phase 3 for the consumer warps: block-ordered prefix of the segment counts
// in batches of 256 segments, and emission of the segments with hits.
template <int OFF>
__device__ __forceinline__ void emit_block(const StreamParams &P, StreamSmem &S, uint64_t st0,
                                           uint64_t st1, int w, int lane) {
    const int t = w * 32 + lane;
    const uint64_t seg0 = st0 * kConsumerWarps, seg1 = st1 * kConsumerWarps;
    uint64_t base = S.cta_excl;
    for (uint64_t sb = seg0; sb < seg1; sb += kConsumerWarps * 32) {
        const uint64_t seg = sb + (uint64_t)t;
        const uint32_t c = seg < seg1 ? P.seg_count[seg] : 0u;
        const uint32_t inc = warp_incl_scan(c, lane);
        if (lane == 31) S.scan_tmp[w] = inc;
        consumer_sync();
        uint32_t wbase = 0u, btotal = 0u;
#pragma unroll
        for (int k = 0; k < kConsumerWarps; ++k) {
            const uint32_t v = S.scan_tmp[k];
            if (k < w) wbase += v;
            btotal += v;
        }
        consumer_sync();
        const uint64_t excl = base + wbase + inc - c;
        uint32_t todo = __ballot_sync(kFull, c != 0u);
        while (todo) {
            const int j = __ffs(todo) - 1;
            todo &= todo - 1u;
            const uint64_t sj = sb + (uint64_t)w * 32u + (uint64_t)j;
            const uint64_t ej = __shfl_sync(kFull, excl, j);
            emit_segment<OFF>(P, sj, ej, S.emit_stage[w], lane);
        }
        base += btotal;
    }
}

// Sum of the totals of blocks 0..blockIdx.x-1 (one warp).  Every block is
// resident (cooperative launch), so each waits only for blocks that run.
__device__ __forceinline__ uint64_t blocks_before(const StreamParams &P, uint64_t mine, int lane,
                                                  bool *ok) {
    uint64_t *st = P.cta_status;
    if (lane == 0)
        st_relaxed_u64(st + (uint64_t)blockIdx.x * kStatusStride,
                       pack_status(P.tag, kFlagAgg, mine));
    uint64_t sum = 0;
    const uint64_t t0 = globaltimer_ns();
    for (uint32_t base = 0; base < blockIdx.x; base += 32) {
        const uint32_t b = base + lane;
        uint64_t v = 0;
        if (b < blockIdx.x) {
            for (;;) {
                const uint64_t s = ld_relaxed_u64(st + (uint64_t)b * kStatusStride);
                if ((uint32_t)(s >> kTagShift) == P.tag) { v = s & kValMask; break; }
                if (globaltimer_ns() - t0 > kWaitNs) { *ok = false; break; }
                __nanosleep(64);
            }
        }
        sum += warp_sum64(v);
    }
    *ok = __all_sync(kFull, *ok) != 0;
    return sum;
}

}  // namespace stream

template <int V, int MP>
__global__ void __launch_bounds__(stream::kThreadsStream, stream::kMaxBlocksPerSm)
    stream_kernel(const __grid_constant__ stream::StreamParams P) {
    using namespace stream;
    constexpr int OFF = (V == V_BLOCK8) ? -7 : 0;
    extern __shared__ __align__(128) uint8_t smem_raw[];
    StreamSmem &S = *reinterpret_cast<StreamSmem *>(smem_raw);
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&S.full[s], 1);
            mbar_init(&S.empty[s], kConsumerWarps);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // S1: pattern preprocessing (block fingerprint table, Section 3.4)
    if (V == V_BLOCK8) build_block_table(P.job.pat, S.table, S.pblk);
    __syncthreads();

    uint64_t st0, st1;
    block_range(P.nstages, &st0, &st1);

    // phase 1: stream and filter
    bool ok = true;
    if (warp == kConsumerWarps) {
        if (lane == 0) producer(P, S, st0, st1);
    } else {
        const uint32_t total = filter_stages<V, MP>(P, S, st0, st1, warp, lane, &ok);
        if (lane == 0) S.warp_total[warp] = total;
        if (!ok && lane == 0) atomicOr(P.err, kErrTimeout);
    }
    __syncthreads();

    // phase 2: block total and the totals of all earlier blocks
    if (warp == 0) {
        uint64_t mine = 0;
        for (int k = 0; k < kConsumerWarps; ++k) mine += S.warp_total[k];
        bool bok = true;
        const uint64_t before = blocks_before(P, mine, lane, &bok);
        if (lane == 0) {
            if (!bok) atomicOr(P.err, kErrTimeout);
            S.cta_excl = before;
            S.cta_total = mine;
            if (blockIdx.x + 1 == gridDim.x) *P.count_out = before + mine;
        }
    }
    __syncthreads();

    // phase 3: ordered emit
    if (P.emit && warp < kConsumerWarps && S.cta_total != 0ull)
        emit_block<OFF>(P, S, st0, st1, warp, lane);
}

}  // namespace epsm
