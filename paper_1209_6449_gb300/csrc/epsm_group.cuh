// Batched search with shared text passes: many (text, pattern) pairs in one
// persistent launch, where all pairs on the same text form a group
// whose stages are loaded once and searched for every pattern of the group.
//
// Shared filter.  The patterns of a group with m >= 5 share one exact-match
// hash table of pattern windows, a multi-pattern form of the block
// fingerprint of Section 3.4.  A pattern of length m contributes the windows
// p[j..j+W) for j = 0..K-1, with width W = 4 (m <= 10) or 8 (m >= 11) and
// stride K the largest power of two <= m - W + 1 (at most 4 for W = 4, 8 for
// W = 8).  Every occurrence at s contains exactly one text window that starts
// at a multiple of K in [s, s+K), at j = that start - s, so looking up the
// text windows at the multiples of K finds each occurrence exactly once.  A
// lane holding chunk c (starts 16c .. 16c+15) looks up the windows at 16c + q
// for q = 0 .. < 16, q a multiple of the group's smallest stride of that
// width, and accepts an entry (i, j, K) when K divides q; the start q - j
// falls in its own chunk or, for q = 0, in the chunk before (the segment's
// last chunk also looks up q = 16, for its own starts).
// The table lives in shared memory: 4096 head slots, each 0 or a 16-bit tag
// of the window's hash plus the index of its first entry (for a slot shared
// by several entries, the OR of their tags), and the entries {window,
// pattern, j, K, next}.  A window whose slot is empty or whose tag has a bit
// outside the slot's is rejected with one shared load; the chains of the
// others are compared exactly after the chunk's lookups and a window match is
// checked in full (from the staged bytes where they cover it).
//
// Confirmed hits go to a per-warp list; each pattern's segment count and masks
// are then written in the layout of the single search (one segment numbering
// per pattern, chunk bit i <-> start 16c + i), so the ordered emit, the range
// totals and the pair offsets are those of the single search.  A pattern whose
// hits do not fit in the list is redone alone on that segment with a prefix
// filter (dense hits).  Patterns with m <= 4 and patterns alone on their text
// run their own single-search variant on the staged bytes.
//
// Two kernels.  group_kernel (persistent, two blocks per SM): claim group
// stages dynamically and stream them through a ring of stage buffers; for
// every pattern segment write its hit count (added to its emit range's total)
// and its hits (offset list or chunk masks) into a pool.  group_emit_kernel
// (as many blocks as fit): each block takes the prefix of the range totals,
// then claims emit ranges dynamically and writes their positions in order.
// Every wait is bounded in time.
#pragma once

#include "epsm_stream.cuh"

namespace epsm {
namespace group {

using namespace stream;

constexpr int kRing = 3;                 // stages in flight per block
constexpr int kGroupBlocksPerSm = 2;     // resident blocks per SM the registers are set for
constexpr int kSlotBits = 12;
constexpr int kSlots = 1 << kSlotBits;   // head slots of the shared table
constexpr int kMaxEnt = 1536;            // window entries per group
constexpr int kMaxShared = 256;          // shared-filter patterns per group
constexpr int kIndivMax = 64;            // single-variant patterns per group
constexpr int kHitCap = 256;             // confirmed hits per warp and stage
constexpr uint32_t kNone = 0xFFFFFFFFu;
constexpr uint32_t kEndChain = 0x7FFu;  // (entry indices have 11 bits)
constexpr uint32_t kW8Min = 11;          // patterns this long use 8-byte windows
constexpr int kRangesPerBlock = 32;      // emit ranges per block (dealt round-robin)
constexpr uint32_t kPoolChunk = 4096;    // pool entries a warp reserves at a time (>= 2048)
constexpr uint32_t kMaskMin = 128;       // segments with this many hits store chunk masks
constexpr uint32_t kMaskFlag = 0x80000000u;  // seg_off: the segment's pool entry holds masks

struct alignas(16) JobDesc {
    SearchJob job;         // text view and pattern
    uint64_t stage0;       // first stage of the pair in the per-pattern numbering
    uint64_t nstages;      // > 0
    uint32_t variant;      // single-search variant (individual patterns)
    uint32_t table;        // block-variant table (kNone if unused)
    uint32_t pair;         // index in the caller's arrays
    int32_t off;           // start offset of bit 0 of a chunk (-7 for the block variant)
    uint32_t kstride;      // shared patterns: window stride K (0: individual pattern)
    uint32_t ent0;         // shared patterns: index of its first table entry
};

struct alignas(16) GroupDesc {
    SearchJob text;        // text view (pattern unused)
    uint64_t chunk_full0, chunk_full1;
    uint64_t gstage0;      // first stage of the group in the group numbering
    uint64_t nstages;      // max over the group's patterns
    uint32_t job0;         // group_jobs[job0 ..]: shared patterns, then individual ones
    uint32_t nshared;
    uint32_t nindiv;
    uint32_t nent;         // table entries
    uint32_t cfg;          // k8 | k4 << 8: smallest stride of the 8- and 4-byte windows (0: none)
    uint32_t comb;         // index of its table (kNone for a group of one pattern)
};
static_assert(sizeof(JobDesc) % 16 == 0 && sizeof(GroupDesc) % 16 == 0, "copied as uint4");

struct Header {
    const GroupDesc *groups;          // ascending gstage0 (in the uploaded staging, after the jobs)
    const uint32_t *group_jobs;      // job indices per group
    uint32_t ngroups;
    uint32_t njobs;
    uint64_t gstages;       // stages over all groups (claimed in phase 1)
    uint64_t jstages;       // stages over all patterns (emitted in phase 3)
    uint64_t range_stages;  // pattern stages per emit range
    uint32_t nranges;       // emit ranges (at most kRangesPerBlock x grid)
    uint32_t pad2;
    uint64_t pool_cap;      // hit-list pool entries
    uint64_t capacity;
    uint64_t *positions;
    uint32_t emit;
    uint32_t pad;
};

// The shared table of one group (built in global memory, copied to shared
// memory when a block starts on the group).  An entry is {window's first 4
// bytes, meta}: meta = next | j << 11 | log2 K << 14 | w4 << 16 | i << 17.  An
// 8-byte window is compared on its first 4 bytes after its 16-bit tag matched;
// the full check decides.
struct SharedTable {
    uint32_t head[kSlots];           // 0, or (OR of its entries' tags) << 16 | (entry + 1)
    uint2 ent[kMaxEnt];
    uint64_t stage0[kMaxShared];     // per-pattern stage numbering
    uint32_t nst[kMaxShared];
    uint32_t m[kMaxShared];
    // the group's short patterns (direct compare)
    uint64_t istage0[kIndivMax];
    int64_t ipmax[kIndivMax];
    uint32_t iw0[kIndivMax];
    uint32_t im[kIndivMax];
    uint32_t inst[kIndivMax];
    uint32_t ipad[kIndivMax];
};
static_assert(sizeof(SharedTable) % 16 == 0, "copied as uint4");

// A group's table and its patterns' words (read from global memory only by
// the full check of a candidate).
struct GroupTables {
    SharedTable t;
    uint32_t pw[kMaxShared][8];
    uint32_t sig[kSlots];            // (table build) per slot: OR of its entries' tags
};

struct Params {
    const Header *hdr;
    const JobDesc *jobs;
    GroupTables *comb;           // one per group of more than one pattern
    uint8_t *tables;             // block-variant tables of individual patterns (kTableBytes each:
                                 // the fingerprint bit table, then the 8 pattern blocks)
    uint64_t *offsets;           // per job: exclusive prefix at its first segment; [njobs] = total
    uint32_t *seg_count;         // per pattern segment: hits
    uint32_t *seg_off;           // per pattern segment with hits: its list in pool
    uint16_t *pool;              // hit lists: offsets in the segment, ascending
    uint32_t *pool_ctr;          // entries handed out (zeroed by the table kernel)
    unsigned long long *range_total;  // per emit range (zeroed by the table kernel)
    uint32_t *err;
    DevMisc *misc;
};

constexpr int kTableBytes = kTableWords * 4 + 16 * 4;

// What a warp needs to check a candidate in full.
struct VCtx {
    const uint8_t *tbase;  // text base (16-byte aligned)
    const uint8_t *buf;    // the staged stage
    int64_t delta;         // first internal byte of the text
    int64_t lim;           // first internal byte past the text
    int64_t sbase;         // internal byte of buf[0]
    const uint32_t *gpw;   // the group's pattern words (global)
    uint32_t inside;       // the whole stage buffer holds text bytes
    uint32_t pad;
};

struct alignas(128) Smem {
    uint8_t buf[kRing][kStageBuf];
    SharedTable tab;                             // table of the current group
    uint64_t stage_id[kRing];
    uint32_t stage_group[kRing];
    GroupDesc sgroup[kRing];                     // the stage's group, copied by the producer
    JobDesc sjob[kRing];                         // and its pattern when it has only one
    uint64_t full[kRing];
    uint64_t empty[kRing];
    uint64_t tab_free;                           // mbarrier: every warp is done with the old table
    uint64_t tab_ready;                          // mbarrier: every warp has copied its share
    uint32_t hits[kConsumerWarps][kHitCap];      // pattern << 11 | chunk << 4 | bit
    uint32_t nhits[kConsumerWarps];
    uint16_t hitcnt[kConsumerWarps][kMaxShared];
    uint32_t ovf[kConsumerWarps][kMaxShared / 32];  // patterns whose hits did not fit
    VCtx vc[kConsumerWarps];
    alignas(16) uint16_t stage16[kConsumerWarps][32 * 16];  // one step's hit offsets, before the pool store;
                                                 // also a shared pattern's 128 chunk masks
    uint32_t pcur[kConsumerWarps];               // warp's pool chunk: next entry
    uint32_t pend[kConsumerWarps];               //   and its end
};

// Shared memory of the emission kernel (one block: kEmitWarps = 8 warps, as
// the single search's emission kernel).
constexpr int kEmitSlices = kEmitThreads;  // the range totals are summed in this many slices
struct alignas(16) EmitSmem {
    uint32_t spre[kEmitWarps][32 * 8];   // [lane * 8 + k]: hits before segment k of the lane's
                                         // stage, in lists | all << 16
    uint32_t soff[kEmitWarps][32 * 8];   // its pool entry (kNone: none)
    alignas(16) uint16_t estage[kEmitWarps][32 * 16];  // staging of a mask segment's offsets
    uint32_t scan_tmp[kEmitWarps];
    uint64_t batch_excl[kEmitThreads];
    uint64_t slice_pre[kEmitSlices];     // exclusive prefix of the slices' range totals
    uint64_t range_base;                 // output offset of the claimed range
    uint32_t claim;
};

// Window hashes: the head slot is the top 12 bits, the tag bits 4..19 (never 0).
__device__ __forceinline__ uint32_t hash8(uint32_t lo, uint32_t hi) {
    return lo * 0x9E3779B1u + hi * 0x85EBCA77u;
}

__device__ __forceinline__ uint32_t hash4(uint32_t lo) { return lo * 0x2545F491u + 0x6A09E667u; }

__device__ __forceinline__ uint32_t slot_of(uint32_t x) { return x >> (32 - kSlotBits); }

__device__ __forceinline__ uint32_t tag_of(uint32_t x) { return ((x >> 4) & 0xFFFFu) | 1u; }

// A slot's head keeps the OR of its entries' tags (the one tag when it holds
// one entry); a window passes when its tag's bits are all among them, so a
// window that merely shares a crowded slot mostly skips the chain walk (one
// AND and one compare, as for a single tag).
__device__ __forceinline__ bool slot_passes(uint32_t v, uint32_t x) {
    const uint32_t t = tag_of(x);
    return v != 0u && ((v >> 16) & t) == t;
}

// ---------------------------------------------------------------------------
// pattern preprocessing (a kernel): block-variant tables of individual
// patterns and the groups' shared tables
// ---------------------------------------------------------------------------

__global__ void build_group_tables_kernel(const Params P) {
    const Header H = *P.hdr;
    for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < H.nranges; r += gridDim.x * blockDim.x)
        P.range_total[r] = 0ull;
    if (blockIdx.x == 0 && threadIdx.x == 0) *P.pool_ctr = 0u;
    // segment counts start at zero: phase 1 writes only segments with hits
    {
        uint4 *sc = reinterpret_cast<uint4 *>(P.seg_count);  // 8 counts (two uint4) per stage
        const uint64_t nv = H.jstages * (kConsumerWarps / 4);
        for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nv;
             i += (uint64_t)gridDim.x * blockDim.x)
            sc[i] = make_uint4(0u, 0u, 0u, 0u);
    }
    // block-variant tables, one block per job
    for (uint32_t j = blockIdx.x; j < H.njobs; j += gridDim.x) {
        const JobDesc &D = P.jobs[j];
        if (D.table == kNone) continue;
        uint8_t *tb = P.tables + (uint64_t)D.table * kTableBytes;
        uint32_t *tw = reinterpret_cast<uint32_t *>(tb);
        for (int i = threadIdx.x; i < kTableWords; i += blockDim.x) tw[i] = 0u;
        __syncthreads();
        if (threadIdx.x < 8) {
            const int q = threadIdx.x >> 2;
            const uint32_t sh = 8u * (uint32_t)(threadIdx.x & 3);
            const uint32_t lo = __funnelshift_r(D.job.pat.w[q], D.job.pat.w[q + 1], sh);
            const uint32_t hi = __funnelshift_r(D.job.pat.w[q + 1], D.job.pat.w[q + 2], sh);
            uint32_t *pb = tw + kTableWords;
            pb[2 * threadIdx.x] = lo;
            pb[2 * threadIdx.x + 1] = hi;
            const uint32_t h = block_hash(lo, hi, D.job.pat.kbits);
            atomicOr(&tw[h >> 5], 1u << (h & 31u));
        }
        __syncthreads();
    }
    // shared tables, one block per group
    for (uint32_t g = blockIdx.x; g < H.ngroups; g += gridDim.x) {
        const GroupDesc &G = H.groups[g];
        if (G.comb == kNone) continue;
        SharedTable &T = P.comb[G.comb].t;  // (groups of more than one pattern)
        uint32_t (*tpw)[8] = P.comb[G.comb].pw;
        uint32_t *sig = P.comb[G.comb].sig;
        for (int i = threadIdx.x; i < kSlots; i += blockDim.x) {
            T.head[i] = 0u;
            sig[i] = 0u;
        }
        for (uint32_t i = threadIdx.x; i < G.nshared; i += blockDim.x) {
            const JobDesc &D = P.jobs[H.group_jobs[G.job0 + i]];
#pragma unroll
            for (int k = 0; k < 8; ++k) tpw[i][k] = D.job.pat.w[k];
            T.stage0[i] = D.stage0;
            T.nst[i] = (uint32_t)D.nstages;
            T.m[i] = D.job.pat.m;
        }
        for (uint32_t i = threadIdx.x; i < G.nindiv; i += blockDim.x) {
            const JobDesc &D = P.jobs[H.group_jobs[G.job0 + G.nshared + i]];
            T.istage0[i] = D.stage0;
            T.ipmax[i] = D.job.pmax;
            T.iw0[i] = D.job.pat.w[0];
            T.im[i] = D.job.pat.m;
            T.inst[i] = (uint32_t)D.nstages;
        }
        __syncthreads();
        // entries: (pattern i, j) for j < K_i; insertion pushes on the slot's chain
        for (uint32_t k = threadIdx.x; k < G.nshared * 8u; k += blockDim.x) {
            const uint32_t i = k >> 3, j = k & 7u;
            const JobDesc &D = P.jobs[H.group_jobs[G.job0 + i]];
            if (j >= D.kstride) continue;
            const Pattern &pt = D.job.pat;
            const uint32_t q = j >> 2, sh = 8u * (j & 3u);
            const uint32_t lo = __funnelshift_r(pt.w[q], pt.w[q + 1], sh);
            const bool w4 = pt.m < kW8Min;
            const uint32_t hi = w4 ? 0u : __funnelshift_r(pt.w[q + 1], pt.w[q + 2], sh);
            const uint32_t x = w4 ? hash4(lo) : hash8(lo, hi);
            const uint32_t lk = (uint32_t)(__ffs((int)D.kstride) - 1);
            const uint32_t e = D.ent0 + j;
            const uint32_t old = atomicExch(&T.head[slot_of(x)], (tag_of(x) << 16) | (e + 1u));
            atomicOr(&sig[slot_of(x)], tag_of(x));
            const uint32_t next = old ? (old & 0xFFFFu) - 1u : kEndChain;
            T.ent[e] = make_uint2(lo, next | (j << 11) | (lk << 14) | ((w4 ? 1u : 0u) << 16) | (i << 17));
        }
        __syncthreads();
        // a slot holding a chain of several entries gets the OR of their tags
        for (int i = threadIdx.x; i < kSlots; i += blockDim.x) {
            const uint32_t v = T.head[i];
            if (v) T.head[i] = (sig[i] << 16) | (v & 0xFFFFu);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// phase 1
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint32_t find_group(const GroupDesc *groups, uint32_t ng, uint64_t st,
                                               uint32_t hint) {
    if (hint < ng && groups[hint].gstage0 <= st && st < groups[hint].gstage0 + groups[hint].nstages)
        return hint;
    uint32_t lo = 0, hi = ng - 1u;
    while (lo < hi) {
        const uint32_t mid = (lo + hi + 1u) >> 1;
        if (groups[mid].gstage0 <= st) lo = mid; else hi = mid - 1u;
    }
    return lo;
}

__device__ __forceinline__ void producer(const Params &P, const Header &H, Smem &S) {
    uint32_t issued = 0;
    bool failed = false;
    uint32_t hint = 0;
    uint64_t claim = atomicAdd(&P.misc->ticket, kClaim);
    for (;;) {
        if (claim >= H.gstages) {
            const int s = issued % kRing;
            const uint32_t n = issued / kRing;
            if (n > 0 && !mbar_wait(&S.empty[s], (n - 1) & 1)) { failed = true; break; }
            S.stage_id[s] = kEndStage;
            mbar_arrive(&S.full[s]);
            ++issued;
            break;
        }
        const uint64_t next = atomicAdd(&P.misc->ticket, kClaim);
        const uint64_t last = claim + kClaim < H.gstages ? claim + kClaim : H.gstages;
        for (uint64_t st = claim; st < last; ++st) {
            const int s = issued % kRing;
            const uint32_t n = issued / kRing;
            if (n > 0 && !mbar_wait(&S.empty[s], (n - 1) & 1)) { failed = true; break; }
            const uint32_t prev = hint;
            hint = find_group(H.groups, H.ngroups, st, hint);
            const GroupDesc &G = H.groups[hint];
            S.stage_id[s] = st;
            S.stage_group[s] = hint;
            // the consumers read the stage's descriptors from shared memory
            // (copied again only when the group changes)
            const int sp = (s + kRing - 1) % kRing;
            if (issued == 0 || hint != prev || S.stage_group[sp] != hint) {
                const uint4 *gs = reinterpret_cast<const uint4 *>(&G);
                uint4 *gd = reinterpret_cast<uint4 *>(&S.sgroup[s]);
                for (int k = 0; k < (int)(sizeof(GroupDesc) / 16); ++k) gd[k] = gs[k];
                if (G.nshared == 0u && G.nindiv == 1u) {
                    const uint4 *js = reinterpret_cast<const uint4 *>(&P.jobs[H.group_jobs[G.job0]]);
                    uint4 *jd = reinterpret_cast<uint4 *>(&S.sjob[s]);
                    for (int k = 0; k < (int)(sizeof(JobDesc) / 16); ++k) jd[k] = js[k];
                }
            } else {
                S.sgroup[s] = S.sgroup[sp];
                S.sjob[s] = S.sjob[sp];
            }
            const uint64_t c0 = (st - G.gstage0) * kStageChunks;
            const uint64_t a = c0 > G.chunk_full0 ? c0 : G.chunk_full0;
            uint64_t b = c0 + kStageChunks + 1u;
            if (b > G.chunk_full1) b = G.chunk_full1;
            if (a < b) {
                const uint32_t bytes = (uint32_t)((b - a) * 16u);
                mbar_arrive_tx(&S.full[s], bytes);
                bulk_load(S.buf[s] + (a - c0) * 16u, G.text.base + a * 16u, bytes, &S.full[s]);
            } else {
                mbar_arrive(&S.full[s]);
            }
            ++issued;
        }
        if (failed) break;
        claim = next;
    }
    if (failed) atomicOr(P.err, kErrTimeout);
    const uint32_t lo = issued > (uint32_t)kRing ? issued - kRing : 0u;
    for (uint32_t i = lo; i < issued; ++i) mbar_wait(&S.full[i % kRing], (i / kRing) & 1);
}

// Pool entries for one segment: the warp's current chunk, or a new one
// (lane 0; kNone when the pool is exhausted).  align: 1, or 4 for masks.
__device__ __forceinline__ uint32_t pool_take(const Params &P, const Header &H, Smem &S, int w,
                                              uint32_t n, uint32_t align) {
    uint32_t cur = (S.pcur[w] + align - 1u) & ~(align - 1u);
    if (cur + n > S.pend[w]) {
        const uint32_t b = atomicAdd(P.pool_ctr, kPoolChunk);
        cur = b;
        S.pend[w] = (uint64_t)b + kPoolChunk <= H.pool_cap ? b + kPoolChunk : b;
    }
    if (cur + n > S.pend[w]) {
        S.pcur[w] = cur;
        set_err(P.err, kErrCapacity);
        return kNone;
    }
    S.pcur[w] = cur + n;
    return cur;
}

// The sorted offset list of a segment with few hits (a whole warp): per
// step u, a warp scan of the lanes' counts, the offsets put in order in
// shared memory, then stored with consecutive lanes on consecutive entries.
// Out of line and compact (a rolled loop): it runs for sparse segments only.
__device__ __noinline__ void store_short_list(const Params &P, const Header &H, Smem &S, uint64_t st,
                                              uint64_t seg, uint32_t h0, uint32_t h1, uint32_t h2,
                                              uint32_t h3, uint32_t total, int w, int lane) {
    uint32_t base = 0u;
    if (lane == 0) {
        P.seg_count[seg] = total;
        atomicAdd(&P.range_total[st / H.range_stages], (unsigned long long)total);
        base = pool_take(P, H, S, w, total, 1u);
        P.seg_off[seg] = base;
    }
    base = __shfl_sync(kFull, base, 0);
    if (base == kNone) return;
    uint16_t *stg = S.stage16[w];
#pragma unroll 1
    for (uint32_t u = 0; u < 4u; ++u) {
        uint32_t hh = u == 0u ? h0 : (u == 1u ? h1 : (u == 2u ? h2 : h3));
        const uint32_t c = __popc(hh);
        const uint32_t inc = warp_incl_scan(c, lane);
        const uint32_t T = __shfl_sync(kFull, inc, 31);
        if (T == 0u) continue;
        uint32_t k = inc - c;
        while (hh) {
            const uint32_t b = (uint32_t)(__ffs(hh) - 1);
            hh &= hh - 1u;
            stg[k++] = (uint16_t)((32u * u + (uint32_t)lane) * 16u + b);
        }
        __syncwarp();
        for (uint32_t q = (uint32_t)lane; q < T; q += 32u) P.pool[base + q] = stg[q];
        __syncwarp();
        base += T;
    }
}

// Phase-1 result of one pattern segment (a whole warp; lane l holds the hit
// masks of chunks 32u + l): the count, added to its emit range's total, and,
// when positions are wanted, in the warp's current pool chunk either its 128
// chunk masks in chunk order (at least kMaskMin hits) or the sorted list of
// its hit offsets (chunk * 16 + bit).
__device__ __forceinline__ void store_list(const Params &P, const Header &H, Smem &S, uint64_t st,
                                           uint64_t seg, uint32_t h0, uint32_t h1, uint32_t h2,
                                           uint32_t h3, int w, int lane) {
    // segments without hits keep the zero count the table kernel wrote
    const uint32_t cnt = __popc(h0) + __popc(h1) + __popc(h2) + __popc(h3);
    if (!__any_sync(kFull, cnt != 0u)) return;
    const uint32_t total = warp_sum(cnt);
    if (H.emit && total < kMaskMin) {
        store_short_list(P, H, S, st, seg, h0, h1, h2, h3, total, w, lane);
        return;
    }
    uint32_t base = 0u;
    if (lane == 0) {
        P.seg_count[seg] = total;
        atomicAdd(&P.range_total[st / H.range_stages], (unsigned long long)total);
        if (H.emit) {
            base = pool_take(P, H, S, w, kSegChunks, 4u);
            P.seg_off[seg] = base == kNone ? kNone : (base | kMaskFlag);
        }
    }
    if (!H.emit) return;
    base = __shfl_sync(kFull, base, 0);
    if (base == kNone) return;
    // the 128 chunk masks in chunk order (lane l holds chunks 32u + l)
    uint16_t *m = P.pool + base;
    m[lane] = (uint16_t)h0;
    m[32 + lane] = (uint16_t)h1;
    m[64 + lane] = (uint16_t)h2;
    m[96 + lane] = (uint16_t)h3;
}

// Single-search variant of one individual pattern on the staged stage, stored
// as its segment.
__device__ __noinline__ void plain_job(const Params &P, const Header &H, Smem &S, const JobDesc &D,
                                       const uint8_t *buf, uint64_t ls, int w, int lane) {
    const uint64_t c0 = ls * kStageChunks;
    const BcastWords Bw(D.job.pat);
    const uint32_t *tb = D.table == kNone
                             ? nullptr
                             : reinterpret_cast<const uint32_t *>(P.tables + (uint64_t)D.table * kTableBytes);
    const uint32_t *pb = tb ? tb + kTableWords : nullptr;
    const uint64_t cf0 = (D.job.delta + 15u) / 16u, cf1 = D.job.lim / 16u;
    uint32_t h[4] = {0u, 0u, 0u, 0u};
    bool dense = false;  // the adaptive variant probes every segment here
    switch (D.variant) {  // (store_list counts the hits from the masks)
        case V_DIRECT: stage_hits<V_DIRECT, 0>(D.job, cf0, cf1, Bw, tb, pb, buf, c0, w, lane, h); break;
        case V_PREFIX4: stage_hits<V_PREFIX4, 4>(D.job, cf0, cf1, Bw, tb, pb, buf, c0, w, lane, h); break;
        case V_PREFIX8: stage_hits<V_PREFIX8, 8>(D.job, cf0, cf1, Bw, tb, pb, buf, c0, w, lane, h); break;
        case V_BLOCK4: stage_hits<V_BLOCK4, 4>(D.job, cf0, cf1, Bw, tb, pb, buf, c0, w, lane, h); break;
        case V_ADAPT: stage_hits<V_ADAPT, 4, true>(D.job, cf0, cf1, Bw, tb, pb, buf, c0, w, lane, h, &dense); break;
        case V_CODE2: stage_hits<V_CODE2, 4>(D.job, cf0, cf1, Bw, tb, pb, buf, c0, w, lane, h); break;
        default: stage_hits<V_BLOCK8, 8>(D.job, cf0, cf1, Bw, tb, pb, buf, c0, w, lane, h); break;
    }
    const uint64_t st = D.stage0 + ls;
    store_list(P, H, S, st, st * kConsumerWarps + (uint64_t)w, h[0], h[1], h[2], h[3], w, lane);
}

// t[P..P+m) == p (pattern words pw), read from the staged bytes when the stage
// buffer covers them, else from global memory.
__device__ __forceinline__ bool verify_at(const uint32_t *pw, uint32_t m, int64_t P, const VCtx &V) {
    const int64_t o = P - V.sbase;
    const uint32_t nw = (m + 3u) >> 2;
    if (V.inside && o >= 0 && o + (int64_t)m <= (int64_t)(kStageBytes + 16u)) {
        const uint32_t *W = reinterpret_cast<const uint32_t *>(V.buf);
        const uint32_t a = (uint32_t)o >> 2, sh = ((uint32_t)o & 3u) * 8u;
        uint32_t cur = W[a];
        for (uint32_t i = 0; i < nw; ++i) {
            const uint32_t nxt = W[a + i + 1u];
            if ((__funnelshift_r(cur, nxt, sh) ^ pw[i]) & word_mask(m, i)) return false;
            cur = nxt;
        }
        return true;
    }
    SearchJob T;
    T.base = V.tbase;
    T.delta = (uint64_t)V.delta;
    T.lim = (uint64_t)V.lim;
    const uint64_t a = (uint64_t)P >> 2;
    const uint32_t sh = ((uint32_t)P & 3u) * 8u;
    uint32_t cur = load_word(T, a);
    for (uint32_t i = 0; i < nw; ++i) {
        const uint32_t nxt = load_word(T, a + i + 1u);
        if ((__funnelshift_r(cur, nxt, sh) ^ pw[i]) & word_mask(m, i)) return false;
        cur = nxt;
    }
    return true;
}

// Appends a confirmed hit of shared pattern i at (chunk, bit) to the warp's
// list; a pattern whose hit does not fit is marked for the dense path.
__device__ __forceinline__ void push_hit(Smem &S, int w, uint32_t i, uint32_t chunk, uint32_t bit) {
    const uint32_t k = atomicAdd(&S.nhits[w], 1u);
    if (k >= (uint32_t)kHitCap) {
        atomicOr(&S.ovf[w][i >> 5], 1u << (i & 31u));
        return;
    }
    S.hits[w][k] = (i << 11) | (chunk << 4) | bit;
    atomicAdd(reinterpret_cast<unsigned int *>(&S.hitcnt[w][0]) + (i >> 1), (i & 1u) ? 0x10000u : 1u);
}

// Word k (0..5) of a chunk and the first two words of the next one.
__device__ __forceinline__ uint32_t pick_word(uint4 c, uint32_t n0, uint32_t n1, uint32_t k) {
    uint32_t r = n1;
    r = k == 4u ? n0 : r;
    r = k == 3u ? c.w : r;
    r = k == 2u ? c.z : r;
    r = k == 1u ? c.y : r;
    r = k == 0u ? c.x : r;
    return r;
}

// The windows whose head slot may hold them (bit q of need8 / need4 for the
// 8- / 4-byte window at 16c + q): walk each slot's chain, compare exactly, and
// check the matches in full.  Out of line: it runs for few lanes.
__device__ __noinline__ void walk_chains(Smem &S, int w, uint4 cur, uint32_t n0, uint32_t n1,
                                         uint32_t need8, uint32_t need4, int64_t p0, uint32_t chunk) {
    const VCtx &V = S.vc[w];
    for (uint32_t pass = 0; pass < 2; ++pass) {
        uint32_t need = pass ? need4 : need8;
        const uint32_t w4 = pass;
        while (need) {
            const uint32_t q = (uint32_t)(__ffs(need) - 1);
            need &= need - 1u;
            const uint32_t k = q >> 2, sh = 8u * (q & 3u);
            const uint32_t r0 = pick_word(cur, n0, n1, k), r1 = pick_word(cur, n0, n1, k + 1u);
            const uint32_t lo = __funnelshift_r(r0, r1, sh);
            const uint32_t hi = w4 ? 0u : __funnelshift_r(r1, k + 2u <= 5u ? pick_word(cur, n0, n1, k + 2u) : 0u, sh);
            const uint32_t x = w4 ? hash4(lo) : hash8(lo, hi);
            uint32_t e = (S.tab.head[slot_of(x)] & 0xFFFFu) - 1u;
            (void)hi;  // an 8-byte window is told apart by its tag; the full check decides
            for (int guard = 0; guard < kMaxEnt && e < (uint32_t)kMaxEnt; ++guard) {
                const uint2 E = S.tab.ent[e];
                const uint32_t meta = E.y;
                const uint32_t i = meta >> 17, j = (meta >> 11) & 7u, K = 1u << ((meta >> 14) & 3u);
                // start 16c + q - j: in this chunk, or (q = 0) in the one
                // before, when that one is in the warp's segment
                const int b = (int)q - (int)j;
                if (((meta >> 16) & 1u) == w4 && E.x == lo && (q & (K - 1u)) == 0u && b <= 15 &&
                    (b >= 0 || chunk > 0u)) {
                    const int64_t Pp = p0 + (int64_t)b;
                    const uint32_t m = S.tab.m[i];
                    if (Pp >= V.delta && Pp <= V.lim - (int64_t)m && verify_at(V.gpw + 8u * i, m, Pp, V))
                        push_hit(S, w, i, b >= 0 ? chunk : chunk - 1u, (uint32_t)(b & 15));
                }
                const uint32_t next = meta & kEndChain;
                if (next == kEndChain) break;
                e = next;
            }
        }
    }
}

// Lookups of one chunk: 8-byte windows at q = 0, K8, 2 K8, .. < 16 and 4-byte
// windows at q = 0, K4, .. < 16 (K = 0: no window of that width); a window at
// 16c + q holds the starts 16c + q - j (j < K), so the window at q = 0 also
// serves the chunk before, and only the segment's last chunk (`last`) looks
// up the window at q = 16, the next segment's first.  A window passes when
// its head slot is non-empty and holds all of its tag's bits; the chains of
// the passing windows are walked afterwards.
template <int K8, int K4>
__device__ __forceinline__ void filter_chunk(Smem &S, int w, uint4 cur, uint32_t n0, uint32_t n1,
                                             int64_t p0, uint32_t chunk, bool last) {
    const uint32_t R[6] = {cur.x, cur.y, cur.z, cur.w, n0, n1};
    const uint32_t *head = S.tab.head;
    uint32_t need8 = 0u, need4 = 0u;
#pragma unroll
    for (int q = 0; q <= 16; ++q) {
        if (q == 16 && !last) break;
        const int k = q >> 2, j = q & 3;
        const uint32_t lo = j ? __funnelshift_r(R[k], R[k + 1], 8 * j) : R[k];
        if constexpr (K8 != 0) {
            if (q % K8 == 0) {
                const uint32_t hi = q == 16 ? R[5] : (j ? __funnelshift_r(R[k + 1], R[k + 2 < 6 ? k + 2 : 5], 8 * j) : R[k + 1]);
                const uint32_t x = hash8(lo, hi);
                if (slot_passes(head[slot_of(x)], x)) need8 |= 1u << q;
            }
        }
        if constexpr (K4 != 0) {
            if (q % K4 == 0) {
                const uint32_t x = hash4(lo);
                if (slot_passes(head[slot_of(x)], x)) need4 |= 1u << q;
            }
        }
    }
    if (need8 | need4) walk_chains(S, w, cur, n0, n1, need8, need4, p0, chunk);
}

// Dense path: shared pattern i alone on the warp's segment, with its prefix
// (4 or 8 bytes) compared at every start and candidates checked in full.
__device__ __noinline__ void pattern_pass(const Params &P, const Header &H, const GroupDesc &G,
                                          Smem &S, uint32_t i, uint64_t ls, int w, int lane) {
    const VCtx &V = S.vc[w];
    const uint32_t *pw = V.gpw + 8u * i;
    const uint32_t m = S.tab.m[i];
    const uint64_t c0 = ls * kStageChunks;
    uint4 ch[4];
    uint4 halo;
    load_segment(G.text, G.chunk_full0, G.chunk_full1, V.buf, c0, w, lane, true, ch, halo);
    uint32_t b[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) b[k] = bcast_byte(pw[k >> 2], k & 3);
    const int64_t sp0 = (int64_t)((c0 + (uint64_t)w * kSegChunks) * 16u);
    const int64_t pmax = V.lim - (int64_t)m;
    const int src = (lane + 1) & 31;
    uint32_t h[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const uint4 cur = ch[u];
        const uint4 nsrc = (lane == 0) ? (u + 1 < 4 ? ch[u + 1 < 4 ? u + 1 : u] : halo) : cur;
        const uint32_t n0 = __shfl_sync(kFull, nsrc.x, src);
        const uint32_t n1 = __shfl_sync(kFull, nsrc.y, src);
        const uint32_t R[6] = {cur.x, cur.y, cur.z, cur.w, n0, n1};
        uint32_t cand = 0u;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            uint32_t X = window_mismatch<4>(0u, R[k], R[k + 1], b[0], b[1], b[2], b[3]);
            if (m >= 8u) X = window_mismatch<4>(X, R[k + 1], R[k + 2], b[4], b[5], b[6], b[7]);
            cand |= nibble_of(zero_bytes(X)) << (4 * k);
        }
        const int64_t p0 = sp0 + (int64_t)((32 * u + lane) * 16);
        cand &= range_mask(V.delta - p0, pmax - p0);
        uint32_t hh = 0u;
        while (cand) {
            const int bit = __ffs(cand) - 1;
            cand &= cand - 1u;
            if (verify_at(pw, m, p0 + bit, V)) hh |= 1u << bit;
        }
        h[u] = hh;
    }
    const uint64_t st = S.tab.stage0[i] + ls;
    store_list(P, H, S, st, st * kConsumerWarps + (uint64_t)w, h[0], h[1], h[2], h[3], w, lane);
}

// Writes the segment of every shared pattern: count 0 for patterns without
// hits, masks from the hit list for the others, the dense path for patterns
// whose hits did not fit.
__device__ __forceinline__ void finish_shared(const Params &P, const Header &H, const GroupDesc &G,
                                              Smem &S, uint64_t ls, int w, int lane) {
    const uint32_t nS = G.nshared;
    const uint32_t nh = S.nhits[w] < (uint32_t)kHitCap ? S.nhits[w] : (uint32_t)kHitCap;
    uint32_t *mbuf = reinterpret_cast<uint32_t *>(S.stage16[w]);  // 128 chunk masks
    for (uint32_t i0 = 0; i0 < nS; i0 += 32) {
        const uint32_t i = i0 + (uint32_t)lane;
        const bool valid = i < nS && ls < S.tab.nst[i < nS ? i : 0];
        const bool over = valid && ((S.ovf[w][i >> 5] >> (i & 31u)) & 1u);
        const uint32_t hc = valid ? S.hitcnt[w][i] : 0u;
        uint32_t todo = __ballot_sync(kFull, valid && !over && hc != 0u);
        while (todo) {
            const uint32_t ii = i0 + (uint32_t)(__ffs(todo) - 1);
            todo &= todo - 1u;
#pragma unroll
            for (int u = 0; u < 4; ++u) mbuf[u * 32 + lane] = 0u;
            __syncwarp();
            for (uint32_t k = lane; k < nh; k += 32) {
                const uint32_t e = S.hits[w][k];
                if ((e >> 11) == ii) atomicOr(&mbuf[(e >> 4) & 127u], 1u << (e & 15u));
            }
            __syncwarp();
            uint32_t h[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                h[u] = mbuf[u * 32 + lane];
            }
            __syncwarp();
            const uint64_t st = S.tab.stage0[ii] + ls;
            store_list(P, H, S, st, st * kConsumerWarps + (uint64_t)w, h[0], h[1], h[2], h[3], w, lane);
        }
        uint32_t dense = __ballot_sync(kFull, over);
        while (dense) {
            const uint32_t ii = i0 + (uint32_t)(__ffs(dense) - 1);
            dense &= dense - 1u;
            pattern_pass(P, H, G, S, ii, ls, w, lane);
        }
    }
}

// Shared filter of one group on one staged stage (a whole consumer warp).
template <int K8, int K4>
__device__ __noinline__ void shared_filter(const Params &P, const Header &H, const GroupDesc &G,
                                           Smem &S, const uint8_t *buf, uint64_t ls, int w, int lane) {
    const uint64_t c0 = ls * kStageChunks;
    if (lane == 0) {
        S.nhits[w] = 0u;
        VCtx &V = S.vc[w];
        V.tbase = G.text.base;
        V.buf = buf;
        V.delta = (int64_t)G.text.delta;
        V.lim = (int64_t)G.text.lim;
        V.sbase = (int64_t)(c0 * 16u);
        V.inside = (c0 >= G.chunk_full0 && c0 + kStageChunks + 1u <= G.chunk_full1) ? 1u : 0u;
        V.gpw = &P.comb[G.comb].pw[0][0];
    }
    if (lane < kMaxShared / 32) S.ovf[w][lane] = 0u;
    for (uint32_t i = lane; i < (G.nshared + 1u) / 2u; i += 32)
        reinterpret_cast<uint32_t *>(&S.hitcnt[w][0])[i] = 0u;
    __syncwarp();
    uint4 ch[4];
    uint4 halo;
    load_segment(G.text, G.chunk_full0, G.chunk_full1, buf, c0, w, lane, true, ch, halo);
    const int64_t sp0 = (int64_t)((c0 + (uint64_t)w * kSegChunks) * 16u);
    const int src = (lane + 1) & 31;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const uint4 cur = ch[u];
        const uint4 nsrc = (lane == 0) ? (u + 1 < 4 ? ch[u + 1 < 4 ? u + 1 : u] : halo) : cur;
        const uint32_t n0 = __shfl_sync(kFull, nsrc.x, src);
        const uint32_t n1 = __shfl_sync(kFull, nsrc.y, src);
        filter_chunk<K8, K4>(S, w, cur, n0, n1, sp0 + (int64_t)((32 * u + lane) * 16),
                             (uint32_t)(32 * u + lane), u == 3 && lane == 31);
    }
    __syncwarp();
    finish_shared(P, H, G, S, ls, w, lane);
}

// Shared filter dispatch on the group's smallest strides.
__device__ __forceinline__ void shared_filter_any(const Params &P, const Header &H, const GroupDesc &G,
                                                  Smem &S, const uint8_t *buf, uint64_t ls, int w,
                                                  int lane) {
    const uint32_t k8 = G.cfg & 0xFFu, k4 = (G.cfg >> 8) & 0xFFu;
    switch (k8 * 16u + k4) {
        case 0x02: shared_filter<0, 2>(P, H, G, S, buf, ls, w, lane); break;
        case 0x04: shared_filter<0, 4>(P, H, G, S, buf, ls, w, lane); break;
        case 0x40: shared_filter<4, 0>(P, H, G, S, buf, ls, w, lane); break;
        case 0x42: shared_filter<4, 2>(P, H, G, S, buf, ls, w, lane); break;
        case 0x44: shared_filter<4, 4>(P, H, G, S, buf, ls, w, lane); break;
        case 0x80: shared_filter<8, 0>(P, H, G, S, buf, ls, w, lane); break;
        case 0x82: shared_filter<8, 2>(P, H, G, S, buf, ls, w, lane); break;
        default: shared_filter<8, 4>(P, H, G, S, buf, ls, w, lane); break;
    }
}

// The group's short patterns (m <= 4) on one staged stage: the packed window
// compare of Section 3.2 for each of them on the segment loaded once.
__device__ __noinline__ void direct_jobs(const Params &P, const Header &H, const GroupDesc &G,
                                         Smem &S, const uint8_t *buf, uint64_t ls, int w, int lane) {
    const uint64_t c0 = ls * kStageChunks;
    uint4 ch[4];
    uint4 halo;
    load_segment(G.text, G.chunk_full0, G.chunk_full1, buf, c0, w, lane, true, ch, halo);
    const int src = (lane + 1) & 31;
    uint32_t nx[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const uint4 nsrc = (lane == 0) ? (u + 1 < 4 ? ch[u + 1 < 4 ? u + 1 : u] : halo) : ch[u];
        nx[u] = __shfl_sync(kFull, nsrc.x, src);
    }
    const int64_t sp0 = (int64_t)((c0 + (uint64_t)w * kSegChunks) * 16u);
    const int64_t delta = (int64_t)G.text.delta;
    for (uint32_t i = 0; i < G.nindiv; ++i) {
        if (ls >= S.tab.inst[i]) continue;
        const uint32_t m = S.tab.im[i], p0w = S.tab.iw0[i];
        const uint32_t b0 = bcast_byte(p0w, 0), b1 = bcast_byte(p0w, 1);
        const uint32_t b2 = bcast_byte(p0w, 2), b3 = bcast_byte(p0w, 3);
        const uint32_t mk1 = m <= 1u ? 0u : 0xFFFFFFFFu, mk2 = m <= 2u ? 0u : 0xFFFFFFFFu;
        const uint32_t mk3 = m <= 3u ? 0u : 0xFFFFFFFFu;
        const int64_t pmax = S.tab.ipmax[i];
        const bool interior = sp0 >= delta && sp0 + (int64_t)(kSegChunks * 16) - 1 <= pmax;
        uint32_t h[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint32_t R[5] = {ch[u].x, ch[u].y, ch[u].z, ch[u].w, nx[u]};
            uint32_t hh = 0u;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const uint32_t X = (R[k] ^ b0) | ((__funnelshift_r(R[k], R[k + 1], 8) ^ b1) & mk1) |
                                   ((__funnelshift_r(R[k], R[k + 1], 16) ^ b2) & mk2) |
                                   ((__funnelshift_r(R[k], R[k + 1], 24) ^ b3) & mk3);
                hh |= nibble_of(zero_bytes(X)) << (4 * k);
            }
            if (!interior) {
                const int64_t p0 = sp0 + (int64_t)((32 * u + lane) * 16);
                hh &= range_mask(delta - p0, pmax - p0);
            }
            h[u] = hh;
        }
        const uint64_t st = S.tab.istage0[i] + ls;
        store_list(P, H, S, st, st * kConsumerWarps + (uint64_t)w, h[0], h[1], h[2], h[3], w, lane);
    }
}

__device__ __forceinline__ void consumer(const Params &P, const Header &H, Smem &S, int w, int lane,
                                         bool *ok) {
    int s = 0;
    uint32_t phase = 0;
    const int t = w * 32 + lane;
    uint32_t tab_group = kNone;  // group whose table this warp last loaded
    uint32_t tab_loads = 0;      // table loads so far (mbarrier phase parity)
    for (;;) {
        if (!warp_wait(&S.full[s], phase)) { *ok = false; break; }
        const uint64_t st = S.stage_id[s];
        if (st == kEndStage) break;
        const uint32_t g = S.stage_group[s];
        const GroupDesc &G = S.sgroup[s];
        const uint64_t ls = st - G.gstage0;
        const uint8_t *buf = S.buf[s];
        // load the group's table: every consumer warp reaches this stage;
        // bounded mbarrier waits (not a block barrier) so that a warp that
        // gave up cannot hold the others forever
        if (G.comb != kNone && tab_group != g) {
            if (lane == 0) mbar_arrive(&S.tab_free);
            if (!warp_wait(&S.tab_free, tab_loads & 1u)) { *ok = false; break; }
            const uint4 *src = reinterpret_cast<const uint4 *>(&P.comb[G.comb].t);
            uint4 *dst = reinterpret_cast<uint4 *>(&S.tab);
            for (int i = t; i < (int)(sizeof(SharedTable) / 16); i += kConsumerWarps * 32) dst[i] = src[i];
            __syncwarp();
            if (lane == 0) mbar_arrive(&S.tab_ready);
            if (!warp_wait(&S.tab_ready, tab_loads & 1u)) { *ok = false; break; }
            ++tab_loads;
            tab_group = g;
        }
        // individual patterns: a pattern alone on its text runs its own
        // variant; the short patterns of a shared text run together
        if (G.nindiv == 1u && G.nshared == 0u) {
            const JobDesc &D = S.sjob[s];
            if (ls < D.nstages) plain_job(P, H, S, D, buf, ls, w, lane);
        } else if (G.nindiv) {
            direct_jobs(P, H, G, S, buf, ls, w, lane);
        }
        if (G.nshared) shared_filter_any(P, H, G, S, buf, ls, w, lane);
        __syncwarp();
        if (lane == 0) mbar_arrive(&S.empty[s]);
        if (++s == kRing) { s = 0; phase ^= 1u; }
    }
}

// ---------------------------------------------------------------------------
// phase 3 (per-pattern segment numbering, as the plain batched launch)
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint32_t first_job_from(const JobDesc *jobs, uint32_t njobs, uint64_t st) {
    uint32_t lo = 0, hi = njobs;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (jobs[mid].stage0 < st) lo = mid + 1u; else hi = mid;
    }
    return lo;
}

// Emission of the pattern stages [st0, st1) with output offset base0, in
// batches of 256 stages (one per consumer thread: its 8 segment counts, one
// block scan of the stage totals; the next batch's counts are loaded before
// this one is processed).  Each warp then copies the hit lists of its 32
// stages as one flat sequence: lane q takes hits q, q + 32, .. of it, finds
// the stage (binary search over the warp's inclusive totals) and the segment
// (the stage's 8 prefix counts, in shared memory), and writes segment start +
// offset; consecutive lanes store consecutive positions and the pool loads of
// many stages overlap.  The per-warp phase-1 buffers hold the stages' segment
// prefixes and list offsets here.
__device__ __forceinline__ void emit_range(const Params &P, const Header &H, EmitSmem &S, uint64_t st0,
                                           uint64_t st1, uint64_t base0, int w, int lane) {
    const int t = w * 32 + lane;
    uint64_t base = base0;
    uint32_t jcur = first_job_from(P.jobs, H.njobs, st0);
    uint32_t wj = jcur > 0 ? jcur - 1u : 0u;
    const uint4 *sc = reinterpret_cast<const uint4 *>(P.seg_count);
    uint32_t *spre = S.spre[w];
    uint32_t *soff = S.soff[w];
    uint16_t *estage = S.estage[w];
    uint4 na = make_uint4(0u, 0u, 0u, 0u), nb = na;
    if (st0 + (uint64_t)t < st1) {
        na = sc[2 * (st0 + (uint64_t)t)];
        nb = sc[2 * (st0 + (uint64_t)t) + 1];
    }
    for (uint64_t sb = st0; sb < st1; sb += kEmitThreads) {
        const uint64_t stg = sb + (uint64_t)t;
        const uint4 ca = na, cb = nb;
        const uint64_t nx = stg + kEmitThreads;
        na = nb = make_uint4(0u, 0u, 0u, 0u);  // past the range: no stage
        if (nx < st1) {
            na = sc[2 * nx];
            nb = sc[2 * nx + 1];
        }
        const uint32_t c = ca.x + ca.y + ca.z + ca.w + cb.x + cb.y + cb.z + cb.w;
        const uint32_t inc = warp_incl_scan(c, lane);
        if (lane == 31) S.scan_tmp[w] = inc;
        __syncthreads();
        uint32_t wbase = 0u, btotal = 0u;
#pragma unroll
        for (int k = 0; k < kEmitWarps; ++k) {
            const uint32_t v = S.scan_tmp[k];
            if (k < w) wbase += v;
            btotal += v;
        }
        const uint64_t excl = base + wbase + inc - c;
        S.batch_excl[t] = excl;
        __syncthreads();
        if (t == 0) {
            const uint64_t bst1 = sb + kEmitThreads;
            while (jcur < H.njobs && P.jobs[jcur].stage0 < bst1 && P.jobs[jcur].stage0 < st1) {
                P.offsets[jcur] = S.batch_excl[P.jobs[jcur].stage0 - sb];
                ++jcur;
            }
        }
        const uint32_t wtotal = __shfl_sync(kFull, inc, 31);
        if (H.emit && wtotal != 0u) {
            // this lane's stage: start, and per segment k its list offset and
            // the numbers of hits before it in the stage (all / in lists)
            int64_t s0 = 0;
            uint32_t lcount = 0u;    // hits of the stage held in lists
            uint32_t mbits = 0u;     // segments held as masks
            if (c != 0u) {
                while (wj + 1u < H.njobs && P.jobs[wj + 1u].stage0 <= stg) ++wj;
                const JobDesc &D = P.jobs[wj];
                s0 = (int64_t)((stg - D.stage0) * (uint64_t)kStageBytes) + D.off - (int64_t)D.job.delta;
                const uint4 oa = reinterpret_cast<const uint4 *>(P.seg_off)[2 * stg];
                const uint4 ob = reinterpret_cast<const uint4 *>(P.seg_off)[2 * stg + 1];
                const uint32_t cs[8] = {ca.x, ca.y, ca.z, ca.w, cb.x, cb.y, cb.z, cb.w};
                const uint32_t os[8] = {oa.x, oa.y, oa.z, oa.w, ob.x, ob.y, ob.z, ob.w};
                uint32_t all = 0u;
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const uint32_t o = cs[k] ? os[k] : kNone;
                    const bool mk = o != kNone && (o & kMaskFlag);
                    spre[lane * 8 + k] = lcount | (all << 16);
                    soff[lane * 8 + k] = o;
                    if (mk) mbits |= 1u << k;
                    else if (o != kNone) lcount += cs[k];  // (kNone: no pool room, not emitted)
                    all += cs[k];
                }
            }
            __syncwarp();
            const uint64_t wexcl = __shfl_sync(kFull, excl, 0);
            if (lane == 0 && wexcl + wtotal > H.capacity) set_err(P.err, kErrCapacity);
            const uint16_t *__restrict__ pool = P.pool;
            uint64_t *__restrict__ out = H.positions;
            // segments held as masks: expanded a segment at a time (staged in
            // the table's shared memory, which phase 3 no longer needs)
            uint32_t todo = __ballot_sync(kFull, mbits != 0u);
            while (todo) {
                const int j = __ffs(todo) - 1;
                todo &= todo - 1u;
                uint32_t mb = __shfl_sync(kFull, mbits, j);
                const uint64_t ej = __shfl_sync(kFull, excl, j);
                const int64_t sj = __shfl_sync(kFull, s0, j);
                while (mb) {
                    // the masks of up to four segments are loaded together
                    uint32_t ks[4];
                    uint2 pk4[4];
                    int nk = 0;
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        ks[r] = 8u;
                        if (mb) {
                            ks[r] = (uint32_t)(__ffs(mb) - 1);
                            mb &= mb - 1u;
                            const uint32_t o = soff[j * 8 + ks[r]] & ~kMaskFlag;
                            pk4[r] = reinterpret_cast<const uint2 *>(pool + o)[lane];
                            nk = r + 1;
                        }
                    }
#pragma unroll 1
                    for (int r = 0; r < nk; ++r) {
                        uint32_t k = ks[0];
                        uint2 packed = pk4[0];
#pragma unroll
                        for (int q = 1; q < 4; ++q)
                            if (q == r) {
                                k = ks[q];
                                packed = pk4[q];
                            }
                        const uint32_t pk = spre[j * 8 + k] >> 16;
                        emit_segment(out, H.capacity, P.err, sj + (int64_t)(k * (uint32_t)(kSegChunks * 16)),
                                     ej + pk, packed, estage, lane);
                    }
                }
            }
            // hits held in lists: one flat sequence across the warp, lane q
            // taking hits q, q + 32, ..
            const uint32_t incs = warp_incl_scan(lcount, lane);
            const uint32_t stotal = __shfl_sync(kFull, incs, 31);
            for (uint32_t q0 = 0; q0 < stotal; q0 += 32u) {
                const uint32_t q = q0 + (uint32_t)lane;
                uint32_t j = 0u;
#pragma unroll
                for (int d = 16; d > 0; d >>= 1) {
                    const uint32_t v = __shfl_sync(kFull, incs, (int)(j + (uint32_t)d - 1u));
                    if (v <= q) j += (uint32_t)d;
                }
                j = j < 31u ? j : 31u;
                const uint32_t ij = __shfl_sync(kFull, incs, (int)j);
                const uint32_t cj = __shfl_sync(kFull, lcount, (int)j);
                const uint64_t ej = __shfl_sync(kFull, excl, (int)j);
                const int64_t sj = __shfl_sync(kFull, s0, (int)j);
                if (q < stotal) {
                    const uint32_t within = q - (ij - cj);  // among the stage's list hits
                    const uint32_t *pr = spre + j * 8u;
                    uint32_t k = 0u, pv = pr[0];
#pragma unroll
                    for (int kk = 1; kk < 8; ++kk) {
                        const uint32_t v = pr[kk];
                        // a later list segment that starts at or before `within`
                        // (mask segments and empty ones do not advance the list count)
                        if ((v & 0xFFFFu) <= within && soff[j * 8u + kk] != kNone &&
                            !(soff[j * 8u + kk] & kMaskFlag)) {
                            k = (uint32_t)kk;
                            pv = v;
                        }
                    }
                    const uint32_t ok_ = soff[j * 8u + k];
                    const uint32_t inlist = within - (pv & 0xFFFFu);
                    const uint64_t idx = ej + (pv >> 16) + inlist;
                    if (ok_ != kNone && idx < H.capacity)
                        out[idx] = (uint64_t)(sj + (int64_t)(k * (uint32_t)(kSegChunks * 16)) +
                                              (int64_t)pool[ok_ + inlist]);
                }
            }
            __syncwarp();
        }
        base += btotal;
        __syncthreads();
    }
}

}  // namespace group

__global__ void __launch_bounds__(stream::kThreadsStream, group::kGroupBlocksPerSm)
    group_kernel(const __grid_constant__ group::Params P) {
    using namespace group;
    extern __shared__ __align__(128) uint8_t smem_raw[];
    Smem &S = *reinterpret_cast<Smem *>(smem_raw);
    const Header H = *P.hdr;
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kRing; ++s) {
            mbar_init(&S.full[s], 1);
            mbar_init(&S.empty[s], kConsumerWarps);
        }
        mbar_init(&S.tab_free, kConsumerWarps);
        mbar_init(&S.tab_ready, kConsumerWarps);
        for (int k = 0; k < kConsumerWarps; ++k) S.pcur[k] = S.pend[k] = 0u;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    bool ok = true;
    if (H.ngroups > 0) {
        if (warp == kConsumerWarps) {
            if (lane == 0) producer(P, H, S);
        } else {
            consumer(P, H, S, warp, lane, &ok);
            if (!ok && lane == 0) atomicOr(P.err, kErrTimeout);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const uint32_t d = atomicAdd(&P.misc->done, 1u);
        if (d == gridDim.x - 1u) {
            P.misc->ticket = 0u;
            P.misc->done = 0u;
            __threadfence();
        }
    }
}

// Emission of a batched search (after group_kernel): the pattern stages are
// cut into ranges whose hit totals group_kernel accumulated; blocks claim
// ranges dynamically (dense ranges take longer than sparse ones), and each
// block first takes the exclusive prefix of all range totals in 256 slices
// (one per thread, one block scan) so that a claimed range's output offset is
// its slice's prefix plus the totals before it in the slice.
__global__ void __launch_bounds__(stream::kEmitThreads, 4)
    group_emit_kernel(const __grid_constant__ group::Params P) {
    using namespace group;
    __shared__ EmitSmem S;
    const Header H = *P.hdr;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const uint32_t nr = H.nranges;
    const uint32_t per = (nr + kEmitSlices - 1) / kEmitSlices;
    const uint64_t *rt = reinterpret_cast<const uint64_t *>(P.range_total);
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
        if (lane == 31) S.batch_excl[warp] = inc;
        __syncthreads();
        uint64_t before = 0, all = 0;
#pragma unroll
        for (int k = 0; k < kEmitWarps; ++k) {
            const uint64_t v = S.batch_excl[k];
            if (k < warp) before += v;
            all += v;
        }
        S.slice_pre[t] = before + inc - sum;
        if (t == 0 && blockIdx.x == 0) P.offsets[H.njobs] = all;
        __syncthreads();
    }
    for (;;) {
        if (t == 0) S.claim = atomicAdd(&P.misc->ticket2, 1u);
        __syncthreads();
        const uint32_t r = S.claim;
        if (r >= nr || H.njobs == 0) break;
        if (warp == 0) {
            // output offset of range r: its slice's prefix + the totals before r
            const uint32_t sl = r / per;
            uint64_t part = 0;
            for (uint32_t q = sl * per + (uint32_t)lane; q < r; q += 32) part += rt[q];
            part = warp_sum64(part);
            if (lane == 0) S.range_base = S.slice_pre[sl] + part;
        }
        __syncthreads();
        const uint64_t st0 = (uint64_t)r * H.range_stages;
        const uint64_t st1 = st0 + H.range_stages < H.jstages ? st0 + H.range_stages : H.jstages;
        if (st0 < st1 && rt[r] != 0ull) {
            emit_range(P, H, S, st0, st1, S.range_base, warp, lane);
        } else if (st0 < st1 && t == 0) {
            // no hits in the range: the jobs starting in it begin at its base
            for (uint32_t j = first_job_from(P.jobs, H.njobs, st0); j < H.njobs && P.jobs[j].stage0 < st1; ++j)
                P.offsets[j] = S.range_base;
        }
        __syncthreads();
    }
    if (t == 0) {
        __threadfence();
        const uint32_t d = atomicAdd(&P.misc->done2, 1u);
        if (d == gridDim.x - 1u) {
            P.misc->ticket2 = 0u;
            P.misc->done2 = 0u;
            __threadfence();
        }
    }
}

}  // namespace epsm
