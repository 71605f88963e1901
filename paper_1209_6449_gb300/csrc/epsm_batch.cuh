// Batched search: many (text, pattern) pairs of uneven n and m in one
// cooperative persistent launch, on the streaming design of epsm_stream.cuh.
//
// The stages of all pairs form one numbering (pair-major).  Phase 1 claims
// stages dynamically; the producer finds each stage's pair (binary search over
// the pairs' first stages, with a cache of the last pair), streams it from that
// pair's text, and the consumers run that pair's variant (a runtime switch per
// stage) with its pattern words and, for the block variant, its fingerprint
// table from global memory (built beforehand by build_tables_kernel, the
// pattern preprocessing step).  After the grid barrier every block emits its
// contiguous range of stages in order, which also yields each pair's output
// offset: the exclusive prefix at the pair's first segment.
//
// The sizes of a batch (number of pairs, number of stages) are read from a
// device header, not from kernel parameters, so one captured CUDA graph serves
// every batch that fits its capacity.
#pragma once

#include "epsm_stream.cuh"

namespace epsm {
namespace batch {

using namespace stream;

constexpr uint32_t kNoTable = 0xFFFFFFFFu;
constexpr int kTableBytes = kHashSlots + 16 * 4;  // fingerprint slots + pattern blocks

struct JobDesc {
    SearchJob job;
    uint64_t stage0;       // first global stage of the pair
    uint64_t nstages;      // > 0 (pairs without stages are left out on the host)
    uint64_t chunk_full0;  // first chunk fully inside the pair's text
    uint64_t chunk_full1;
    uint32_t variant;      // V_*; V_DIRECT uses mp = m
    uint32_t table;        // index of its fingerprint table (block variant), else kNoTable
    uint32_t pair;         // index of the pair in the caller's arrays
    int32_t off;           // start offset of a chunk's bit 0 (-7 for the block variant)
};

struct Header {
    uint32_t njobs;
    uint32_t ntables;
    uint64_t nstages;       // stages over all jobs
    uint64_t range_stages;  // stages per emit range
    uint64_t capacity;      // positions available
    uint64_t *positions;    // output pool (device)
    uint32_t emit;          // 0: count only
    uint32_t pad;
};

struct BatchParams {
    const Header *hdr;
    const JobDesc *jobs;    // njobs, ascending stage0
    uint8_t *tables;        // ntables x kTableBytes
    uint64_t *offsets;      // indexed by job: exclusive prefix at its first segment; [njobs] = total
    uint32_t *seg_count;
    uint16_t *seg_mask;
    unsigned long long *range_total;
    uint32_t *err;
    DevMisc *misc;
};

struct alignas(128) BatchSmem {
    StreamSmem s;
    uint32_t stage_job[kStages];
    uint64_t batch_excl[kConsumerWarps * 32];
};

// Pattern preprocessing (Section 3.4, table L) for every block-variant job:
// one thread block per table.
__global__ void build_tables_kernel(const BatchParams P) {
    const Header H = *P.hdr;
    for (uint32_t j = blockIdx.x; j < H.njobs; j += gridDim.x) {
        const JobDesc &D = P.jobs[j];
        if (D.table == kNoTable) continue;
        uint8_t *tb = P.tables + (uint64_t)D.table * kTableBytes;
        uint32_t *tw = reinterpret_cast<uint32_t *>(tb);
        for (int i = threadIdx.x; i < kHashSlots / 4; i += blockDim.x) tw[i] = 0u;
        __syncthreads();
        if (threadIdx.x < 8) {
            const int q = threadIdx.x >> 2;
            const uint32_t sh = 8u * (uint32_t)(threadIdx.x & 3);
            const uint32_t lo = __funnelshift_r(D.job.pat.w[q], D.job.pat.w[q + 1], sh);
            const uint32_t hi = __funnelshift_r(D.job.pat.w[q + 1], D.job.pat.w[q + 2], sh);
            uint32_t *pb = reinterpret_cast<uint32_t *>(tb + kHashSlots);
            pb[2 * threadIdx.x] = lo;
            pb[2 * threadIdx.x + 1] = hi;
            tb[block_hash(lo, hi)] = 1;
        }
        __syncthreads();
    }
}

// The job owning global stage st: the last job with stage0 <= st.
__device__ __forceinline__ uint32_t find_job(const JobDesc *jobs, uint32_t njobs, uint64_t st,
                                             uint32_t hint) {
    if (hint < njobs && jobs[hint].stage0 <= st && st < jobs[hint].stage0 + jobs[hint].nstages)
        return hint;
    uint32_t lo = 0, hi = njobs - 1u;
    while (lo < hi) {
        const uint32_t mid = (lo + hi + 1u) >> 1;
        if (jobs[mid].stage0 <= st) lo = mid; else hi = mid - 1u;
    }
    return lo;
}

__device__ __forceinline__ void producer(const BatchParams &P, const Header &H, BatchSmem &B) {
    StreamSmem &S = B.s;
    uint32_t issued = 0;
    bool failed = false;
    uint32_t hint = 0;
    uint64_t claim = atomicAdd(&P.misc->ticket, kClaim);
    for (;;) {
        if (claim >= H.nstages) {
            const int s = issued % kStages;
            const uint32_t n = issued / kStages;
            if (n > 0 && !mbar_wait(&S.empty[s], (n - 1) & 1)) { failed = true; break; }
            S.stage_id[s] = kEndStage;
            mbar_arrive(&S.full[s]);
            ++issued;
            break;
        }
        const uint64_t next = atomicAdd(&P.misc->ticket, kClaim);
        const uint64_t last = claim + kClaim < H.nstages ? claim + kClaim : H.nstages;
        for (uint64_t st = claim; st < last; ++st) {
            const int s = issued % kStages;
            const uint32_t n = issued / kStages;
            if (n > 0 && !mbar_wait(&S.empty[s], (n - 1) & 1)) { failed = true; break; }
            hint = find_job(P.jobs, H.njobs, st, hint);
            const JobDesc &D = P.jobs[hint];
            S.stage_id[s] = st;
            B.stage_job[s] = hint;
            const uint64_t c0 = (st - D.stage0) * kStageChunks;
            const uint64_t a = c0 > D.chunk_full0 ? c0 : D.chunk_full0;
            uint64_t b = c0 + kStageChunks + 1u;  // + halo chunk
            if (b > D.chunk_full1) b = D.chunk_full1;
            if (a < b) {
                const uint32_t bytes = (uint32_t)((b - a) * 16u);
                mbar_arrive_tx(&S.full[s], bytes);
                bulk_load(S.buf[s] + (a - c0) * 16u, D.job.base + a * 16u, bytes, &S.full[s]);
            } else {
                mbar_arrive(&S.full[s]);
            }
            ++issued;
        }
        if (failed) break;
        claim = next;
    }
    if (failed) atomicOr(P.err, kErrTimeout);
    const uint32_t lo = issued > (uint32_t)kStages ? issued - kStages : 0u;
    for (uint32_t i = lo; i < issued; ++i) mbar_wait(&S.full[i % kStages], (i / kStages) & 1);
}

template <int V, int MP>
__device__ __forceinline__ uint32_t job_stage_hits(const BatchParams &P, const JobDesc &D,
                                                   const uint8_t *buf, uint64_t c0, int w,
                                                   int lane, uint32_t (&h)[4]) {
    const BcastWords Bw(D.job.pat);
    const uint8_t *tb = D.table == kNoTable ? nullptr : P.tables + (uint64_t)D.table * kTableBytes;
    const uint32_t *pb = tb ? reinterpret_cast<const uint32_t *>(tb + kHashSlots) : nullptr;
    return stage_hits<V, MP>(D.job, D.chunk_full0, D.chunk_full1, Bw, tb, pb, buf, c0, w, lane, h);
}

__device__ __forceinline__ void consumer(const BatchParams &P, const Header &H, BatchSmem &B, int w,
                                         int lane, bool *ok) {
    StreamSmem &S = B.s;
    int s = 0;
    uint32_t phase = 0;
    for (;;) {
        if (!warp_wait(&S.full[s], phase)) { *ok = false; break; }
        const uint64_t st = S.stage_id[s];
        if (st == kEndStage) break;
        const JobDesc &D = P.jobs[B.stage_job[s]];
        const uint64_t c0 = (st - D.stage0) * kStageChunks;
        const uint8_t *buf = S.buf[s];
        uint32_t h[4] = {0u, 0u, 0u, 0u};
        uint32_t cnt = 0u;
        switch (D.variant) {
            case V_DIRECT:
                switch (D.job.pat.m) {
                    case 1: cnt = job_stage_hits<V_DIRECT, 1>(P, D, buf, c0, w, lane, h); break;
                    case 2: cnt = job_stage_hits<V_DIRECT, 2>(P, D, buf, c0, w, lane, h); break;
                    case 3: cnt = job_stage_hits<V_DIRECT, 3>(P, D, buf, c0, w, lane, h); break;
                    default: cnt = job_stage_hits<V_DIRECT, 4>(P, D, buf, c0, w, lane, h); break;
                }
                break;
            case V_PREFIX4: cnt = job_stage_hits<V_PREFIX4, 4>(P, D, buf, c0, w, lane, h); break;
            case V_PREFIX8: cnt = job_stage_hits<V_PREFIX8, 8>(P, D, buf, c0, w, lane, h); break;
            default: cnt = job_stage_hits<V_BLOCK8, 8>(P, D, buf, c0, w, lane, h); break;
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&S.empty[s]);
        if (++s == kStages) { s = 0; phase ^= 1u; }
        store_segment(P.seg_count, P.seg_mask, P.range_total, H.range_stages, st,
                      st * kConsumerWarps + (uint64_t)w, cnt, h, H.emit != 0, lane);
    }
}

// First job whose first stage is >= st (njobs if none).
__device__ __forceinline__ uint32_t first_job_from(const JobDesc *jobs, uint32_t njobs, uint64_t st) {
    uint32_t lo = 0, hi = njobs;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (jobs[mid].stage0 < st) lo = mid + 1u; else hi = mid;
    }
    return lo;
}

// Phase 3 for the consumer warps: ordered prefix over the range's segments in
// batches of 256, job output offsets at the jobs' first segments, and the
// emission of every segment with hits.
__device__ __forceinline__ void emit_range(const BatchParams &P, const Header &H, BatchSmem &B,
                                           uint64_t st0, uint64_t st1, uint64_t cta_excl, int w,
                                           int lane) {
    StreamSmem &S = B.s;
    const int t = w * 32 + lane;
    const uint64_t seg0 = st0 * kConsumerWarps, seg1 = st1 * kConsumerWarps;
    uint64_t base = cta_excl;
    uint32_t jcur = first_job_from(P.jobs, H.njobs, st0);     // next job start to record
    uint32_t wj = jcur > 0 ? jcur - 1u : 0u;                  // job of the warp's segments
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
        const uint64_t excl = base + wbase + inc - c;
        B.batch_excl[t] = excl;
        consumer_sync();
        // output offsets of the jobs starting in this batch
        if (t == 0) {
            const uint64_t bst1 = (sb + kConsumerWarps * 32) / kConsumerWarps;
            while (jcur < H.njobs && P.jobs[jcur].stage0 < bst1 && P.jobs[jcur].stage0 < st1) {
                const uint64_t fs = P.jobs[jcur].stage0 * kConsumerWarps;
                P.offsets[jcur] = B.batch_excl[fs - sb];
                ++jcur;
            }
        }
        const uint32_t todo = __ballot_sync(kFull, c != 0u);
        if (todo && H.emit) {
            emit_list(todo, sb + (uint64_t)w * 32u, excl, P.seg_mask, lane,
                      [&](uint64_t sj, uint64_t ej, uint2 packed) {
                          const uint64_t stg = sj / kConsumerWarps;
                          while (wj + 1u < H.njobs && P.jobs[wj + 1u].stage0 <= stg) ++wj;
                          const JobDesc &D = P.jobs[wj];
                          const int64_t s0 = (int64_t)(((stg - D.stage0) * kStageChunks +
                                                        (sj % kConsumerWarps) * kSegChunks) * 16u) +
                                             D.off - (int64_t)D.job.delta;
                          emit_segment(H.positions, H.capacity, P.err, s0, ej, packed,
                                       S.emit_stage[w], lane);
                      });
        }
        base += btotal;
        consumer_sync();  // batch_excl is rewritten by the next batch
    }
}

}  // namespace batch

__global__ void __launch_bounds__(stream::kThreadsStream, stream::kMaxBlocksPerSm)
    batch_stream_kernel(const __grid_constant__ batch::BatchParams P) {
    using namespace batch;
    extern __shared__ __align__(128) uint8_t smem_raw[];
    BatchSmem &B = *reinterpret_cast<BatchSmem *>(smem_raw);
    StreamSmem &S = B.s;
    const Header H = *P.hdr;
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&S.full[s], 1);
            mbar_init(&S.empty[s], kConsumerWarps);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    bool ok = true;
    if (H.njobs > 0) {
        if (warp == kConsumerWarps) {
            if (lane == 0) producer(P, H, B);
        } else {
            consumer(P, H, B, warp, lane, &ok);
            if (!ok && lane == 0) atomicOr(P.err, kErrTimeout);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && !grid_barrier(P.misc)) atomicOr(P.err, kErrTimeout);
    __syncthreads();

    const uint64_t st0 = (uint64_t)blockIdx.x * H.range_stages;
    const uint64_t st1 = st0 + H.range_stages < H.nstages ? st0 + H.range_stages : H.nstages;
    if (warp == 0) {
        uint64_t before = 0, all = 0;
        for (uint32_t b = lane; b < gridDim.x; b += 32) {
            const uint64_t v = ld_relaxed_u64(reinterpret_cast<const uint64_t *>(P.range_total) + b);
            all += v;
            if (b < blockIdx.x) before += v;
        }
        before = warp_sum64(before);
        all = warp_sum64(all);
        if (lane == 0) {
            S.cta_excl = before;
            if (blockIdx.x + 1 == gridDim.x) P.offsets[H.njobs] = all;
        }
    }
    __syncthreads();
    if (warp < kConsumerWarps && st0 < st1 && H.njobs > 0)
        emit_range(P, H, B, st0, st1, S.cta_excl, warp, lane);
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const uint32_t d = atomicAdd(&P.misc->done, 1u);
        if (d == gridDim.x - 1u) {
            for (uint32_t b = 0; b < gridDim.x; ++b) P.range_total[b] = 0ull;
            P.misc->ticket = 0u;
            P.misc->done = 0u;
            P.misc->barrier = 0u;
            __threadfence();
        }
    }
}

}  // namespace epsm
