// Streaming scan of one search: a filter kernel and an emission kernel.
//
// The text is cut into 16 KiB stages (1024 chunks of 16 bytes) and each stage
// into 8 segments of 128 chunks (2 KiB), one per consumer warp.
//
// stream_kernel (persistent, two blocks per SM; no ordering, no waiting on
// other blocks).  A producer warp claims stages in batches from a global
// ticket (the next claim is requested while the current batch is issued) and
// streams them through a ring of shared-memory buffers with 1-D bulk copies
// (cp.async.bulk, completion on an mbarrier), keeping up to kStages x 16 KiB
// of reads in flight per block.  Each consumer warp runs the variant's filter
// and verify (chunk_hits) on its segment of each staged stage and writes the
// segment's hit count, adds it to its emit range's total, and, only if it has
// hits, writes its 128 16-bit chunk masks to scratch.  Dynamic claiming keeps
// every SM busy until the text is exhausted.
//
// stream_emit_kernel (as many blocks as fit, launched after it when positions
// are wanted).  Each block takes the exclusive prefix of the range totals
// (256 slices, one block scan), then claims emit ranges dynamically: a batch
// of 256 segment counts at a time, one block scan, and each warp expands its
// segments with hits into positions (masks loaded ahead; hit offsets staged
// in shared memory in output order, then written as consecutive 8-byte
// positions).  Dense ranges take longer than sparse ones; dynamic claiming
// balances them.
//
// Every wait is bounded in time; on expiry the error word gets kErrTimeout and
// the waiting warp gives up, so the kernels always end.  The producer waits,
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
// Launch shapes of the filter kernel: ring depth (16 KiB stages in flight per
// block) and resident blocks per SM, whose shared memory must fit an SM.  A
// search's shape comes from the tuning table (shape 1 by default).
template <int SH> struct Shape;
template <> struct Shape<0> { static constexpr int stages = 6, blocks = 2; };  // 99 KiB x 2
template <> struct Shape<1> { static constexpr int stages = 4, blocks = 3; };  // 66 KiB x 3
constexpr int kShapes = 2;
constexpr int kDefaultShape = 1;
constexpr int kSegChunks = 128;                             // chunks per segment (2 KiB)
constexpr uint64_t kWaitNs = 2000000000ull;
constexpr int kConsumerBarrier = 1;                         // named barrier of consumer warps
constexpr uint64_t kMaxBlocks = 512;                        // grid bound (range totals, status words)

constexpr uint32_t kClaim = 2;                              // stages per claim

// A segment's count word: its hits in the low 16 bits (at most 2048) and, when
// its hits are stored as chunk records, the number of records in the high 16
// bits (0: stored as the 128 chunk masks).  A record is chunk << 16 | mask for
// a chunk with hits, in chunk order; segments with at most kRecMax chunks with
// hits use records (4 bytes per such chunk instead of 256 bytes of masks).
constexpr uint32_t kCountMask = 0xFFFFu;
constexpr uint32_t kRecMax = 32;
// Records pay off where chunks with hits carry several each (runs) or where
// there are few; a segment of scattered single hits expands faster from masks.
__device__ __forceinline__ bool use_records(uint32_t hits, uint32_t nz) {
    return nz <= kRecMax && (nz <= 8u || hits >= 2u * nz);
}
constexpr int kAdaptDense = 2;   // probe: steps of 4 with a block match somewhere => dense text
constexpr uint64_t kEndStage = ~0ull;

template <int NS>
struct alignas(128) StreamSmem {
    static constexpr int kStages = NS;
    uint8_t buf[kStages][kStageBuf];
    uint64_t stage_id[kStages];  // global stage held by each ring slot (kEndStage: done)
    alignas(16) uint32_t wcnt[kStages][kConsumerWarps];  // per slot: the segments' hit counts
    uint32_t votes;              // adaptive variant: consumer warps whose probe found dense text
    uint64_t full[kStages];
    uint64_t empty[kStages];
    uint32_t pblk[32];
    uint32_t table[kTableWords];  // block fingerprint bit table
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

// try_wait with a suspend-time hint: a waiting thread sleeps until the phase
// completes (or the hint elapses) instead of spinning, so waiting consumer
// warps do not take issue slots from the producer.
constexpr uint32_t kSuspendHintNs = 20000u;

__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity), "r"(kSuspendHintNs)
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
    uint32_t *err;
    DevMisc *misc;         // claim ticket, done counter, grid-barrier counter
    unsigned long long *range_total;  // scratch: hits per emit range (zero between calls)
    uint64_t range_stages; // stages per emit range
    uint32_t nranges;      // emit ranges (claimed dynamically by the emission kernel)
    int32_t off;           // start of bit 0 of a chunk relative to it (-7: block variant)
    uint64_t nstages;      // 16 KiB stages of the text
    uint64_t chunk_full0;  // first chunk lying fully inside [delta, lim)
    uint64_t chunk_full1;  // one past the last such chunk
    int emit;              // 0: count only
    const uint8_t *tail;   // long pattern (m > 32, block variant): its bytes past the first 32
    uint32_t mtail;        // their number (0: none)
    uint64_t *cursor;      // device word: output index of the first position (null: 0); the
                           // emission kernel advances it by the count (searches chained
                           // into one buffer)
};

// Chunk c of job J as staged in `buf` (the stage's first chunk is c0), or read
// from global memory when it is not fully inside the text (ragged ends).
__device__ __forceinline__ uint4 staged_chunk(const SearchJob &J, uint64_t cf0, uint64_t cf1,
                                              const uint8_t *buf, uint64_t c0, uint64_t c) {
    if (c >= cf0 && c < cf1) return *reinterpret_cast<const uint4 *>(buf + (c - c0) * 16u);
    return load_chunk(J, c);
}

// ---------------------------------------------------------------------------
// phase 1 roles
// ---------------------------------------------------------------------------

template <typename SMEM>
__device__ __forceinline__ void issue_stage(const StreamParams &P, SMEM &S, int s,
                                            uint64_t st) {
    const SearchJob &J = P.job;
    S.stage_id[s] = st;
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
}

// Producer (one thread): claims batches of kClaim stages and issues them; the
// claim of the next batch is requested before the current batch is issued so
// that its latency overlaps the copies.  When a claim comes back past the end
// of the text, the next ring slot is marked kEndStage.
// Publishes the counts of the stage a ring slot held, once its consumers
// released it: the eight segment counts as two 16-byte stores, and the stage
// total added to its range total.
template <typename SMEM>
__device__ __forceinline__ void flush_slot(const StreamParams &P, SMEM &S, int s) {
    const uint64_t st = S.stage_id[s];
    const uint4 a = *reinterpret_cast<const uint4 *>(&S.wcnt[s][0]);
    const uint4 b = *reinterpret_cast<const uint4 *>(&S.wcnt[s][4]);
    uint4 *dst = reinterpret_cast<uint4 *>(P.seg_count + st * kConsumerWarps);
    dst[0] = a;
    dst[1] = b;
    const uint32_t tot = ((a.x & kCountMask) + (a.y & kCountMask) + (a.z & kCountMask) +
                          (a.w & kCountMask)) +
                         ((b.x & kCountMask) + (b.y & kCountMask) + (b.z & kCountMask) +
                          (b.w & kCountMask));
    if (tot) atomicAdd(&P.range_total[st / P.range_stages], (unsigned long long)tot);
}

template <typename SMEM>
__device__ __forceinline__ void producer(const StreamParams &P, SMEM &S) {
    constexpr int kStages = SMEM::kStages;
    static_assert(kConsumerWarps == 8, "flush_slot publishes eight counts");
    uint32_t issued = 0;
    uint32_t pend = 0;  // bit s: slot s holds a stage whose counts are not yet published
    bool failed = false;
    uint64_t claim = atomicAdd(&P.misc->ticket, kClaim);
    for (;;) {
        if (claim >= P.nstages) {
            const int s = issued % kStages;
            const uint32_t n = issued / kStages;
            if (n > 0 && !mbar_wait(&S.empty[s], (n - 1) & 1)) { failed = true; break; }
            if (pend >> s & 1u) { flush_slot(P, S, s); pend &= ~(1u << s); }
            S.stage_id[s] = kEndStage;
            mbar_arrive(&S.full[s]);
            ++issued;
            break;
        }
        const uint64_t next = atomicAdd(&P.misc->ticket, kClaim);
        const uint64_t last = claim + kClaim < P.nstages ? claim + kClaim : P.nstages;
        for (uint64_t st = claim; st < last; ++st) {
            const int s = issued % kStages;
            const uint32_t n = issued / kStages;
            if (n > 0 && !mbar_wait(&S.empty[s], (n - 1) & 1)) { failed = true; break; }
            if (pend >> s & 1u) { flush_slot(P, S, s); pend &= ~(1u << s); }
            issue_stage(P, S, s, st);
            if (P.emit) pend |= 1u << s;
            ++issued;
        }
        if (failed) break;
        claim = next;
    }
    if (failed) atomicOr(P.err, kErrTimeout);
    // Leave no copy in flight: wait (bounded) for the last issued stages.
    const uint32_t lo = issued > (uint32_t)kStages ? issued - kStages : 0u;
    for (uint32_t i = lo; i < issued; ++i) mbar_wait(&S.full[i % kStages], (i / kStages) & 1);
    // Publish the counts of the stages still held: wait (bounded) until their
    // consumers released them.
    if (!failed) {
        for (uint32_t i = lo; i < issued; ++i) {
            const int s = (int)(i % kStages);
            if (!(pend >> s & 1u)) continue;
            if (!mbar_wait(&S.empty[s], (i / kStages) & 1)) { atomicOr(P.err, kErrTimeout); break; }
            flush_slot(P, S, s);
            pend &= ~(1u << s);
        }
    }
}

// A chunk read through the ragged-end path (its stage is not entirely inside
// the text): out of line, to keep the hot loop small.
__device__ __noinline__ uint4 edge_chunk(const SearchJob &J, uint64_t cf0, uint64_t cf1,
                                         const uint8_t *buf, uint64_t c0, uint64_t c) {
    return staged_chunk(J, cf0, cf1, buf, c0, c);
}

// The four chunks lane l holds for segment w of a staged stage (chunks 32u + l
// of the segment), and for lane 0 the halo chunk after the segment.
__device__ __forceinline__ void load_segment(const SearchJob &J, uint64_t cf0, uint64_t cf1,
                                             const uint8_t *buf, uint64_t c0, int w, int lane,
                                             bool want_halo, uint4 (&ch)[4], uint4 &halo) {
    const uint32_t lane_off = (uint32_t)(w * kSegChunks + lane) * 16u;  // byte offset in a stage
    // stage entirely inside the text (all but the first and last stages):
    // 32-bit shared-memory offsets, no per-chunk bounds checks
    const bool inside = c0 >= cf0 && c0 + kStageChunks + 1u <= cf1;
    halo = make_uint4(0u, 0u, 0u, 0u);
    if (inside) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
            ch[u] = *reinterpret_cast<const uint4 *>(buf + lane_off + 512u * u);
        if (want_halo && lane == 0) halo = *reinterpret_cast<const uint4 *>(buf + lane_off + 2048u);
    } else {
        const uint64_t cw = c0 + (uint64_t)w * kSegChunks;
#pragma unroll
        for (int u = 0; u < 4; ++u) ch[u] = edge_chunk(J, cf0, cf1, buf, c0, cw + 32u * u + lane);
        if (want_halo && lane == 0) halo = edge_chunk(J, cf0, cf1, buf, c0, cw + kSegChunks);
    }
}

// Filter and verify one consumer warp's segment of a staged stage of job J:
// the stage holds the job's chunks c0 .. c0+1024 (+ halo); lane l takes chunks
// 32u + l of segment w.  Writes the four 16-bit hit masks to h and returns the
// lane's hit count.
//   PROBE (4-byte block variant only): first decide from the segment whether
//   the text is dense in block matches (`dense`), and if so filter it with
//   the prefix filter instead.
// The hits of one warp's segment, given its loaded chunks (lane l: chunks
// 32u + l; lane 0 also the halo chunk after the segment).
template <int V, int MP>
__device__ __forceinline__ uint32_t segment_hits(const SearchJob &J, const uint4 (&ch)[4], const uint4 halo,
                                                 int64_t sp0, bool interior, const BcastWords &B,
                                                 const uint32_t *table, const uint32_t *pblk,
                                                 const StagedText &T, int lane, uint32_t (&h)[4]) {
    uint32_t cnt = 0u;
    if constexpr (V == V_CODE2) {
        // 2-bit code filter (Section 3.3's filter-then-verify, with the first
        // min(m, 8) bytes of the window in the filter at two bits each): the
        // code words of the four steps and of the halo, the next lane's by a
        // shuffle; then, for all 16 starts of a chunk at once, the code
        // stream shifted by j chars is XORed with the code of p_j replicated
        // 16 times and ORed into acc, so a start survives iff its 2-bit field
        // of acc stays zero.  Survivors are checked on the bytes in registers.
        uint32_t C[4], Cn[4], acc[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) C[u] = code2_of(ch[u]);
        const uint32_t Ch = code2_of(halo);
        const int src = (lane + 1) & 31;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint32_t cs = (lane == 0) ? (u + 1 < 4 ? C[u + 1 < 4 ? u + 1 : u] : Ch) : C[u];
            Cn[u] = __shfl_sync(kFull, cs, src);
            acc[u] = 0u;
        }
        const Pattern &pat = J.pat;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            if ((uint32_t)j < pat.m) {
#pragma unroll
                for (int u = 0; u < 4; ++u) acc[u] |= __funnelshift_r(C[u], Cn[u], 2 * j) ^ B.r2[j];
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            // (soundness build: every start is a candidate)
            const uint32_t z = kSoundness ? 0x55555555u : ~(acc[u] | (acc[u] >> 1)) & 0x55555555u;
            uint32_t hh = 0u;
            if (__any_sync(kFull, z != 0u)) {
                const uint4 nsrc = (lane == 0) ? (u + 1 < 4 ? ch[u + 1 < 4 ? u + 1 : u] : halo) : ch[u];
                const uint32_t n0 = __shfl_sync(kFull, nsrc.x, src);
                const uint32_t n1 = __shfl_sync(kFull, nsrc.y, src);
                const uint32_t n2 = __shfl_sync(kFull, nsrc.z, src);
                const uint32_t n3 = __shfl_sync(kFull, nsrc.w, src);
                const uint32_t cand = z ? even_bits(z) : 0u;
                if constexpr (MP == kMpRun) {
                    // one byte repeated (a kernel of its own): the chunk's
                    // starts decided at once from the byte-equality masks of
                    // the chunk and the next (that one from the next lane)
                    const uint32_t bb = bcast_byte(pat.w[0], 0);
                    const uint32_t e_own = eq_mask16(ch[u], bb);
                    const uint32_t e_next = __shfl_sync(kFull, lane == 0 ? eq_mask16(nsrc, bb) : e_own, src);
                    hh = cand ? runs_of(((uint64_t)e_next << 16) | e_own, pat.m) & cand : 0u;
                } else if (__any_sync(kFull, __popc(cand) > 3)) {
                    // many candidates somewhere in the warp (a run of one
                    // byte): all 16 starts checked at once on the bytes
                    hh = cand ? exact_chunk_regs(pat, ch[u], n0, n1, n2, n3) & cand : 0u;
                } else if (cand) {
                    hh = verify_cands_regs(pat, ch[u], n0, n1, n2, n3, cand);
                }
            }
            const int64_t p0 = sp0 + (int64_t)((32 * u + lane) * 16);
            if (!interior) hh &= range_mask((int64_t)J.delta - p0, J.pmax - p0);
            h[u] = hh;
            cnt += __popc(hh);
        }
    } else {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint4 cur = ch[u];
            const uint4 nsrc = (lane == 0) ? (u + 1 < 4 ? ch[u + 1 < 4 ? u + 1 : u] : halo) : cur;
            const int64_t p0 = sp0 + (int64_t)((32 * u + lane) * 16);
            uint32_t hh = chunk_hits<V, MP>(J, cur, nsrc, p0, B, table, pblk, lane, T);
            if (!interior) hh &= range_mask((int64_t)J.delta - p0, J.pmax - p0);
            h[u] = hh;
            cnt += __popc(hh);
        }
    }
    return cnt;
}

// Filter and verify one consumer warp's segment of a staged stage of job J:
// the stage holds the job's chunks c0 .. c0+1024 (+ halo); lane l takes chunks
// 32u + l of segment w.  Writes the four 16-bit hit masks to h and returns the
// lane's hit count.
//   V_ADAPT (PROBE only): a probe of the segment decides whether the text
//   makes 4-byte block matches of the pattern frequent (small alphabets:
//   most steps of the block or prefix filter would take the candidate path;
//   *dense_out), and the segment is filtered with the 2-bit code filter if
//   so, else with the 4-byte block filter (m >= 7) or the prefix filter.
template <int V, int MP, bool PROBE = false>
__device__ __forceinline__ uint32_t stage_hits(const SearchJob &J, uint64_t cf0, uint64_t cf1,
                                               const BcastWords &B, const uint32_t *table,
                                               const uint32_t *pblk, const uint8_t *buf,
                                               uint64_t c0, int w, int lane, uint32_t (&h)[4],
                                               bool *dense_out = nullptr, const uint8_t *tail = nullptr,
                                               uint32_t mtail = 0u) {
    constexpr int OFF = (V == V_BLOCK8) ? -7 : (V == V_BLOCK8S) ? -15 : 0;
    uint4 ch[4];
    uint4 halo;
    load_segment(J, cf0, cf1, buf, c0, w, lane, V != V_BLOCK8 && V != V_BLOCK8S, ch, halo);
    StagedText T;
    T.buf = buf;
    T.sbase = (int64_t)(c0 * 16u);
    T.span = (uint32_t)((kStageChunks + 1) * 16);
    T.inside = (c0 >= cf0 && c0 + kStageChunks + 1u <= cf1) ? 1u : 0u;
    T.tail = tail;
    T.mtail = mtail;
    const int64_t sp0 = (int64_t)((c0 + (uint64_t)w * kSegChunks) * 16u) + OFF;
    const bool interior = sp0 >= (int64_t)J.delta && sp0 + (int64_t)(kSegChunks * 16) - 1 <= J.pmax;
    if constexpr (V == V_ADAPT) {
        static_assert(PROBE, "the adaptive variant always probes");
        uint32_t q0, q1, q2, q3;
        pattern_blocks4(J.pat, q0, q1, q2, q3);
        int steps = 0;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint4 ns = (lane == 0) ? (u + 1 < 4 ? ch[u + 1 < 4 ? u + 1 : u] : halo) : ch[u];
            const uint32_t n0 = __shfl_sync(kFull, ns.x, (lane + 1) & 31);
            steps += __any_sync(kFull, block4_any(ch[u], n0, q0, q1, q2, q3)) ? 1 : 0;
        }
        const bool dense = steps >= kAdaptDense;
        *dense_out = dense;
        if (dense) return segment_hits<V_CODE2, 4>(J, ch, halo, sp0, interior, B, table, pblk, T, lane, h);
        if (J.pat.m >= 7u) return segment_hits<V_BLOCK4, 4>(J, ch, halo, sp0, interior, B, table, pblk, T, lane, h);
        return segment_hits<V_PREFIX4, 4>(J, ch, halo, sp0, interior, B, table, pblk, T, lane, h);
    } else {
        return segment_hits<V, MP>(J, ch, halo, sp0, interior, B, table, pblk, T, lane, h);
    }
}

// Per-segment results of the filter: the count always; the 128 chunk masks,
// in chunk order, only if the segment has hits (lane l writes chunks 32u + l).
// The count goes to the ring slot's shared-memory row; the producer publishes
// the stage's counts and its range total when it recycles the slot
// (flush_slot).
__device__ __forceinline__ void store_segment(const StreamParams &P, uint32_t *wslot, uint64_t seg,
                                              uint32_t cnt, const uint32_t (&h)[4], int lane,
                                              uint64_t &acc) {
    if (!__any_sync(kFull, cnt != 0u)) {
        if (P.emit && lane == 0) *wslot = 0u;
        return;
    }
    const uint32_t wc = warp_sum(cnt);
    if (!P.emit) {  // count only: the warp adds its total once, at the end
        acc += wc;
        return;
    }
    uint32_t bal[4], nz = 0u;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        bal[u] = __ballot_sync(kFull, h[u] != 0u);
        nz += __popc(bal[u]);
    }
    if (use_records(wc, nz)) {
        // chunk records in chunk order (chunk 32u + lane)
        uint32_t *rec = reinterpret_cast<uint32_t *>(P.seg_mask + seg * kSegChunks);
        const uint32_t below = (1u << lane) - 1u;
        uint32_t off = 0u;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (h[u]) rec[off + __popc(bal[u] & below)] = ((uint32_t)(32 * u + lane) << 16) | h[u];
            off += __popc(bal[u]);
        }
        if (lane == 0) *wslot = wc | (nz << 16);
    } else {
        uint16_t *m = P.seg_mask + seg * kSegChunks;
#pragma unroll
        for (int u = 0; u < 4; ++u) m[32 * u + lane] = (uint16_t)h[u];
        if (lane == 0) *wslot = wc;
    }
}

// One segment of the warp's ring: wait for the next stage, filter the warp's
// segment of it, release the buffer and store the results.  Returns false at
// the end of the stream (or when a wait gave up, with *ok cleared).
template <int V, int MP, bool PROBE, typename SMEM>
__device__ __forceinline__ bool one_segment(const StreamParams &P, SMEM &S, const BcastWords &B,
                                            int &s, uint32_t &phase, int w, int lane, bool *ok,
                                            uint64_t &acc, bool *dense) {
    if (!warp_wait(&S.full[s], phase)) { *ok = false; return false; }
    const uint64_t st = S.stage_id[s];
    if (st == kEndStage) return false;
    uint32_t h[4];
    const uint32_t cnt = stage_hits<V, MP, PROBE>(P.job, P.chunk_full0, P.chunk_full1, B, S.table,
                                                  S.pblk, S.buf[s], st * kStageChunks, w, lane, h,
                                                  dense, P.tail, P.mtail);
    store_segment(P, &S.wcnt[s][w], st * kConsumerWarps + (uint64_t)w, cnt, h, lane, acc);
    // the stage buffer is no longer needed: release it to the producer
    __syncwarp();
    if (lane == 0) mbar_arrive(&S.empty[s]);
    if (++s == SMEM::kStages) { s = 0; phase ^= 1u; }
    return true;
}

template <int V, int MP, typename SMEM>
__device__ __forceinline__ void filter_stages(const StreamParams &P, SMEM &S, int w, int lane,
                                              bool *ok) {
    const BcastWords B(P.job.pat);
    int s = 0;
    uint32_t phase = 0;
    uint64_t acc = 0;
    if constexpr (V == V_ADAPT) {
        // The consumer warps probe their first segments (one stage of the
        // text) and the block takes the majority: the code filter for the
        // block's whole run where the text is dense in block matches, else
        // the 4-byte block filter (m >= 7) or the prefix filter.  One mode
        // per block keeps each loop as tight as the plain variant's.
        bool dense = false;
        const bool more = one_segment<V_ADAPT, 4, true>(P, S, B, s, phase, w, lane, ok, acc, &dense);
        if (lane == 0 && dense) atomicAdd(&S.votes, 1u);
        consumer_sync();  // every consumer warp gets here, whatever its first segment did
        if (more) {
            if (S.votes * 2u >= (uint32_t)kConsumerWarps) {
                while (one_segment<V_CODE2, 4, false>(P, S, B, s, phase, w, lane, ok, acc, nullptr)) {
                }
            } else if (P.job.pat.m >= 7u) {
                while (one_segment<V_BLOCK4, 4, false>(P, S, B, s, phase, w, lane, ok, acc, nullptr)) {
                }
            } else {
                while (one_segment<V_PREFIX4, 4, false>(P, S, B, s, phase, w, lane, ok, acc, nullptr)) {
                }
            }
        }
    } else {
        while (one_segment<V, MP, false>(P, S, B, s, phase, w, lane, ok, acc, nullptr)) {
        }
    }
    if (!P.emit && lane == 0 && acc) atomicAdd(&P.range_total[blockIdx.x % P.nranges], (unsigned long long)acc);
}

// Emit the positions of one segment (a whole warp), given its 128 chunk masks
// in chunk order: lane l holds chunks 4l .. 4l+3 as one 64-bit word (`packed`,
// low half first), whose bit j is the start 64l + j of the segment.  One warp
// scan of the lanes' counts places every hit.  A segment with few hits has
// each lane store its own positions; otherwise the hits are staged in shared
// memory as offsets inside the segment, in output order, and written as
// consecutive 8-byte positions, 512 at a time (one window unless the
// segment is dense).
//   s0: the start (user coordinates) of bit 0 of the segment's first chunk.
constexpr uint32_t kEmitWindow = 512;
constexpr uint32_t kEmitDirect = 64;  // segments with at most this many hits skip the staging
__device__ __forceinline__ void emit_segment(uint64_t *positions, uint64_t capacity, uint32_t *err,
                                             int64_t s0, uint64_t idx0, uint2 packed,
                                             uint16_t *stage, int lane) {
    uint32_t lo = packed.x, hi = packed.y;  // starts 64l .. 64l+31, 64l+32 .. 64l+63
    const uint32_t c = (uint32_t)(__popc(lo) + __popc(hi));
    const uint32_t inc = warp_incl_scan(c, lane);
    const uint32_t total = __shfl_sync(kFull, inc, 31);
    // the whole segment fits in the output: no per-store bound check
    const bool fits = idx0 + total <= capacity;
    if (lane == 0 && !fits) set_err(err, kErrCapacity);
    const uint32_t pos0 = (uint32_t)lane * 64u;
    uint64_t *dst = positions + idx0;  // (unsigned arithmetic: s0 may be negative,
    const uint64_t base = (uint64_t)s0; //  every emitted position is not)
    uint32_t k = inc - c;  // the lane's first output index inside the segment
    if (total <= kEmitDirect) {
        // few hits: each lane writes its own (at most a few) positions
        while (lo) {
            const uint32_t b = (uint32_t)(__ffs(lo) - 1);
            lo &= lo - 1u;
            if (fits || idx0 + k < capacity) dst[k] = base + pos0 + b;
            ++k;
        }
        while (hi) {
            const uint32_t b = (uint32_t)(__ffs(hi) - 1);
            hi &= hi - 1u;
            if (fits || idx0 + k < capacity) dst[k] = base + pos0 + 32u + b;
            ++k;
        }
        return;
    }
    if (total <= kEmitWindow) {
        // the common dense case: one staging window
        while (lo) {
            const uint32_t b = (uint32_t)(__ffs(lo) - 1);
            lo &= lo - 1u;
            stage[k++] = (uint16_t)(pos0 + b);
        }
        while (hi) {
            const uint32_t b = (uint32_t)(__ffs(hi) - 1);
            hi &= hi - 1u;
            stage[k++] = (uint16_t)(pos0 + 32u + b);
        }
        __syncwarp();
        if (fits) {
            for (uint32_t q = lane; q < total; q += 32u) dst[q] = base + stage[q];
        } else {
            for (uint32_t q = lane; q < total; q += 32u)
                if (idx0 + q < capacity) dst[q] = base + stage[q];
        }
        __syncwarp();
        return;
    }
    // very dense (more than one window): 64-bit mask, window by window
    uint64_t mk = ((uint64_t)hi << 32) | (uint64_t)lo;
    for (uint32_t w0 = 0; w0 < total; w0 += kEmitWindow) {
        const uint32_t w1 = w0 + kEmitWindow;
        while (mk != 0ull && k < w1) {
            const uint32_t b = (uint32_t)(__ffsll((long long)mk) - 1);
            mk &= mk - 1ull;
            stage[k - w0] = (uint16_t)(pos0 + b);
            ++k;
        }
        __syncwarp();
        const uint32_t nw = total - w0 < kEmitWindow ? total - w0 : kEmitWindow;
        for (uint32_t q = lane; q < nw; q += 32u) {
            const uint64_t idx = idx0 + w0 + q;
            if (idx < capacity) positions[idx] = base + stage[q];
        }
        __syncwarp();
    }
}

__device__ __forceinline__ uint2 load_masks(const uint16_t *seg_mask, uint64_t seg, int lane) {
    return reinterpret_cast<const uint2 *>(seg_mask + seg * kSegChunks)[lane];
}

// Emits the segments of a warp's batch listed in `todo` (bit j: segment
// first + j has hits; lane j holds its exclusive output offset in `excl`).  The
// masks of up to kEmitAhead segments are loaded together before they are
// emitted, so the L2 latency of the mask loads is paid once per group.
#ifndef EPSM_EMIT_AHEAD
#define EPSM_EMIT_AHEAD 4
#endif
constexpr int kEmitAhead = EPSM_EMIT_AHEAD;

template <typename EmitFn>
__device__ __forceinline__ void emit_list(uint32_t todo, uint64_t first, uint64_t excl,
                                          const uint16_t *seg_mask, int lane, EmitFn &&emit) {
    while (todo) {
        int js[kEmitAhead];
        uint2 mk[kEmitAhead];
#pragma unroll
        for (int k = 0; k < kEmitAhead; ++k) {
            js[k] = -1;
            if (todo) {
                js[k] = __ffs(todo) - 1;
                todo &= todo - 1u;
                mk[k] = load_masks(seg_mask, first + (uint64_t)js[k], lane);
            }
        }
        // one copy of the emit code (not unrolled): it is large
#pragma unroll 1
        for (int k = 0; k < kEmitAhead; ++k) {
            int jk = js[0];
            uint2 mkk = mk[0];
#pragma unroll
            for (int q = 1; q < kEmitAhead; ++q)
                if (q == k) { jk = js[q]; mkk = mk[q]; }
            if (jk < 0) break;
            emit(first + (uint64_t)jk, __shfl_sync(kFull, excl, jk), mkk);
        }
    }
}

// Phase 3 for the consumer warps: block-ordered prefix of the segment counts
// in batches of 256 segments, and emission of the segments with hits.  Each
// warp walks its segments with hits and loads the next one's masks before it
// emits the current one, so mask loads overlap the stores.
// Shared memory of the emission kernel (one block: 8 warps).
constexpr int kEmitWarps = 8;
constexpr int kEmitThreads = kEmitWarps * 32;
struct alignas(16) StreamEmitSmem {
    uint16_t emit_stage[kEmitWarps][32 * 16];  // per-warp staging of hit offsets
    uint32_t scan_tmp[2][kEmitWarps];            // per batch, alternating (one barrier a batch)
    uint64_t scan64[kEmitWarps];
    uint64_t slice_pre[kEmitThreads];          // exclusive prefix of the slices' range totals
    uint64_t range_base;
    uint32_t claim;
};

// Emission of the record-format segments among a warp's 32 consecutive
// segments (lane j: segment first + j, its count word and its output offset
// excl).  The records are expanded in passes: a pass takes consecutive
// segments whose records fit in the 32 lanes (and no mask-format segment with
// hits among them, so that the pass's positions are one output range); lane r
// takes record r, a segmented warp scan of the records' hit counts places its
// hits, which go to shared memory as offsets from the pass's first segment,
// and the warp writes the pass's positions as consecutive 8-byte stores.
__device__ __forceinline__ void emit_records(const StreamParams &P, uint64_t first, uint32_t word,
                                             uint64_t excl, int64_t seg_pos0, uint16_t *stage,
                                             int lane) {
    const uint32_t c = word & kCountMask;
    const uint32_t R = c ? (word >> 16) : 0u;  // records (0: none, or the mask format)
    const uint32_t balR = __ballot_sync(kFull, R != 0u);
    if (balR == 0u) return;
    const uint32_t balM = __ballot_sync(kFull, c != 0u && R == 0u);
    const uint32_t inclR = warp_incl_scan(R, lane);
    const uint32_t exclR = inclR - R;
    const uint64_t cincl = excl + c;  // output offset past this segment
    uint32_t j0 = (uint32_t)(__ffs(balR) - 1);
    for (;;) {
        const uint32_t B = __shfl_sync(kFull, exclR, (int)j0);
        uint32_t j1 = (uint32_t)__popc(__ballot_sync(kFull, inclR <= B + 32u));  // > j0
        const uint32_t mafter = balM & ~((2u << j0) - 1u);
        if (mafter) j1 = min(j1, (uint32_t)(__ffs(mafter) - 1));
        const uint32_t TR = __shfl_sync(kFull, inclR, (int)(j1 - 1u)) - B;
        const uint64_t E0 = __shfl_sync(kFull, excl, (int)j0);
        const uint64_t E1 = __shfl_sync(kFull, cincl, (int)(j1 - 1u));
        const uint32_t T = (uint32_t)(E1 - E0);  // hits of the pass, at most 32 x 16
        // record g = B + lane: its segment j (lanes whose inclusive count <= g)
        const uint32_t g = B + (uint32_t)lane;
        uint32_t j = 0u;
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
            const uint32_t v = __shfl_sync(kFull, inclR, (int)(j + (uint32_t)d - 1u));
            if (v <= g) j += (uint32_t)d;
        }
        const bool act = (uint32_t)lane < TR;
        j = act ? j : j0;
        const uint32_t ej = __shfl_sync(kFull, exclR, (int)j);
        const uint64_t oj = __shfl_sync(kFull, excl, (int)j);
        uint32_t rec = 0u;
        if (act)
            rec = reinterpret_cast<const uint32_t *>(P.seg_mask + (first + j) * kSegChunks)[g - ej];
        uint32_t mk = rec & 0xFFFFu;
        const uint32_t cnt = __popc(mk);
        const uint32_t incl = warp_incl_scan(cnt, lane);
        const uint32_t f = ej - B;  // the segment's first lane in this pass
        const uint32_t pre = __shfl_sync(kFull, incl, (int)(f > 0u ? f - 1u : 0u));
        uint32_t k = (uint32_t)(oj - E0) + incl - cnt - (f > 0u ? pre : 0u);
        const uint32_t off = (j - j0) * (uint32_t)(kSegChunks * 16) + (rec >> 16) * 16u;
        while (mk) {
            const uint32_t b = (uint32_t)(__ffs(mk) - 1);
            mk &= mk - 1u;
            stage[k++] = (uint16_t)(off + b);
        }
        __syncwarp();
        const bool fits = E0 + T <= P.capacity;
        if (lane == 0 && !fits) set_err(P.err, kErrCapacity);
        const uint64_t base = (uint64_t)((int64_t)((first + j0) * kSegChunks * 16u) + seg_pos0);
        uint64_t *dst = P.positions + E0;
        if (fits) {
            for (uint32_t q = (uint32_t)lane; q < T; q += 32u) dst[q] = base + stage[q];
        } else {
            for (uint32_t q = (uint32_t)lane; q < T; q += 32u)
                if (E0 + q < P.capacity) dst[q] = base + stage[q];
        }
        __syncwarp();
        if (j1 >= 32u) break;
        const uint32_t rest = balR & ~((1u << j1) - 1u);
        if (rest == 0u) break;
        j0 = (uint32_t)(__ffs(rest) - 1);
    }
}

// Ordered emission of the stages [st0, st1) from output offset base0:
// batches of 256 segments, a block scan of their counts, and each warp emits
// its segments with hits: those stored as masks one at a time (their masks
// loaded ahead, see emit_list), those stored as chunk records in passes
// (emit_records).
__device__ __forceinline__ void emit_stages(const StreamParams &P, StreamEmitSmem &S, uint64_t st0,
                                            uint64_t st1, uint64_t base0, int w, int lane) {
    const int t = w * 32 + lane;
    const uint64_t seg0 = st0 * kConsumerWarps, seg1 = st1 * kConsumerWarps;
    uint64_t base = base0;
    const int64_t seg_pos0 = (int64_t)P.off - (int64_t)P.job.delta;
    // the next batch's count words are loaded while this one is emitted
    uint32_t word_next = seg0 + (uint64_t)t < seg1 ? P.seg_count[seg0 + (uint64_t)t] : 0u;
    uint32_t par = 0u;
    for (uint64_t sb = seg0; sb < seg1; sb += kEmitThreads) {
        const uint32_t word = word_next;
        const uint64_t segn = sb + kEmitThreads + (uint64_t)t;
        word_next = segn < seg1 ? P.seg_count[segn] : 0u;
        const uint32_t c = word & kCountMask;
        const uint32_t inc = warp_incl_scan(c, lane);
        // (a warp writes this parity's row again two batches later, after
        // every warp has passed the next batch's barrier, so after its reads)
        if (lane == 31) S.scan_tmp[par][w] = inc;
        __syncthreads();
        uint32_t wbase = 0u, btotal = 0u;
#pragma unroll
        for (int k = 0; k < kEmitWarps; ++k) {
            const uint32_t v = S.scan_tmp[par][k];
            if (k < w) wbase += v;
            btotal += v;
        }
        par ^= 1u;
        const uint64_t excl = base + wbase + inc - c;
        const uint64_t first = sb + (uint64_t)w * 32u;
        const uint32_t todo = __ballot_sync(kFull, c != 0u && (word >> 16) == 0u);
        emit_list(todo, first, excl, P.seg_mask, lane,
                  [&](uint64_t sj, uint64_t ej, uint2 packed) {
                      const int64_t s0 = (int64_t)(sj * kSegChunks * 16u) + seg_pos0;
                      emit_segment(P.positions, P.capacity, P.err, s0, ej, packed,
                                   S.emit_stage[w], lane);
                  });
        emit_records(P, first, word, excl, seg_pos0, S.emit_stage[w], lane);
        base += btotal;
    }
}

// The last block of the filter kernel resets the claim counters; when only
// the count is wanted it also sums the range totals into count_out and
// clears them (otherwise the emission kernel does both).
__device__ __forceinline__ void finish_stream(const StreamParams &P) {
    __threadfence();
    const uint32_t d = atomicAdd(&P.misc->done, 1u);
    if (d == gridDim.x - 1u) {
        if (!P.emit) {
            uint64_t all = 0;
            for (uint32_t r = 0; r < P.nranges; ++r) {
                all += ld_relaxed_u64(reinterpret_cast<const uint64_t *>(P.range_total) + r);
                P.range_total[r] = 0ull;
            }
            *P.count_out = all;
        }
        P.misc->ticket = 0u;
        P.misc->done = 0u;
        __threadfence();
    }
}

}  // namespace stream

template <int V, int MP, int SH>
__global__ void __launch_bounds__(stream::kThreadsStream, stream::Shape<SH>::blocks)
    stream_kernel(const __grid_constant__ stream::StreamParams P) {
    using namespace stream;
    using SMEM = StreamSmem<Shape<SH>::stages>;
    constexpr int kStages = SMEM::kStages;
    extern __shared__ __align__(128) uint8_t smem_raw[];
    SMEM &S = *reinterpret_cast<SMEM *>(smem_raw);
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&S.full[s], 1);
            mbar_init(&S.empty[s], kConsumerWarps);
        }
        S.votes = 0u;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // S1: pattern preprocessing (block fingerprint table, Section 3.4)
    if (V == V_BLOCK8) build_block_table(P.job.pat, S.table, S.pblk, 8);
    if (V == V_BLOCK8S) build_block_table(P.job.pat, S.table, S.pblk, 16);
    // the previous kernel of the stream (a search's emission, or whatever
    // wrote the text) has finished before any global memory is touched
    grid_dep_wait();
    grid_dep_launch();
    __syncthreads();

    // phase 1: stream and filter (stages claimed dynamically)
    bool ok = true;
    if (warp == kConsumerWarps) {
        if (lane == 0) producer(P, S);
    } else {
        filter_stages<V, MP>(P, S, warp, lane, &ok);
        if (!ok && lane == 0) atomicOr(P.err, kErrTimeout);
    }
    __syncthreads();
    if (threadIdx.x == 0) finish_stream(P);
}

// Emission of a single search (after stream_kernel, when positions are
// wanted): each block takes the exclusive prefix of the range totals in 256
// slices, then claims ranges dynamically and emits them in order; block 0
// writes the total, and the last block clears the range totals and the claim
// counters for the next search.
// Emission blocks resident per SM that the register budget is set for (a
// build-time tuning knob).
#ifndef EPSM_EMIT_MIN_BLOCKS
#define EPSM_EMIT_MIN_BLOCKS 4
#endif
__global__ void __launch_bounds__(stream::kEmitThreads, EPSM_EMIT_MIN_BLOCKS)
    stream_emit_kernel(const __grid_constant__ stream::StreamParams P) {
    using namespace stream;
    __shared__ StreamEmitSmem S;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    grid_dep_wait();  // the filter kernel's counts and masks are complete
    grid_dep_launch();
    const uint32_t nr = P.nranges;
    const uint32_t per = (nr + kEmitThreads - 1) / kEmitThreads;
    const uint64_t *rt = reinterpret_cast<const uint64_t *>(P.range_total);
    // (read by every block before the last one to finish advances it)
    const uint64_t cbase = P.cursor ? *P.cursor : 0ull;
    uint64_t all = 0;
    {
        const uint32_t r0 = (uint32_t)t * per, r1 = r0 + per < nr ? r0 + per : nr;
        uint64_t sum = 0;
#pragma unroll 8
        for (uint32_t r = r0; r < r1; ++r) sum += rt[r];
        uint64_t inc = sum;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint64_t v = __shfl_up_sync(kFull, inc, d);
            if (lane >= d) inc += v;
        }
        if (lane == 31) S.scan64[warp] = inc;
        __syncthreads();
        uint64_t before = 0;
#pragma unroll
        for (int k = 0; k < kEmitWarps; ++k) {
            const uint64_t v = S.scan64[k];
            if (k < warp) before += v;
            all += v;
        }
        S.slice_pre[t] = before + inc - sum;
        if (t == 0 && blockIdx.x == 0) *P.count_out = all;
        __syncthreads();
    }
    for (;;) {
        if (t == 0) S.claim = atomicAdd(&P.misc->ticket2, 1u);
        __syncthreads();
        const uint32_t r = S.claim;
        if (r >= nr) break;
        if (warp == 0) {
            const uint32_t sl = r / per;
            uint64_t part = 0;
            for (uint32_t q = sl * per + (uint32_t)lane; q < r; q += 32) part += rt[q];
            part = warp_sum64(part);
            if (lane == 0) S.range_base = cbase + S.slice_pre[sl] + part;
        }
        __syncthreads();
        const uint64_t st0 = (uint64_t)r * P.range_stages;
        const uint64_t st1 = st0 + P.range_stages < P.nstages ? st0 + P.range_stages : P.nstages;
        if (st0 < st1 && rt[r] != 0ull) emit_stages(P, S, st0, st1, S.range_base, warp, lane);
        __syncthreads();
    }
    // the last block to finish clears the range totals and the counters
    if (t == 0) {
        __threadfence();
        S.claim = atomicAdd(&P.misc->done2, 1u) == gridDim.x - 1u ? 1u : 0u;
    }
    __syncthreads();
    if (S.claim) {
        for (uint32_t r = (uint32_t)t; r < nr; r += kEmitThreads) P.range_total[r] = 0ull;
        if (t == 0) {
            P.misc->ticket2 = 0u;
            P.misc->done2 = 0u;
            if (P.cursor) *P.cursor = cbase + all;
        }
        __threadfence();
    }
}

}  // namespace epsm
